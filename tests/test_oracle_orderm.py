"""Pins for the response of any order m (oracle.sp2.sp2_pt(order=m)).

Each order o's S^(o) is the lambda^o Taylor coefficient of the SP2 sequence
of H + lambda H1 (Sec. III A, Eq. (S_n detailed)); the converged values are
the Taylor coefficients P_o of theta(mu - H - lambda H1).  The pins come from
routes that share nothing with the recursion by order: plain SP2 on the
block upper-triangular matrix of Sec. III B, a symbolic derivative of the
2x2 projector, finite differences of the second-order sum over states, and
the idempotency, commutation and trace identities order by order.
"""

import numpy as np
import pytest

import oracle
from oracle.sos import response2_sos
from paper_2203_09621_gb300.workloads import make_workload, sym_gauss


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def order4():
    inst = make_workload(1)
    r = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ, order=4)
    return inst, r


def test_lower_orders_unchanged(order4):
    inst, r = order4
    r1 = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ)
    r2 = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ, order=2)
    assert r.converged and len(r.Pk) == 4
    np.testing.assert_array_equal(r.P, r1.P)
    np.testing.assert_array_equal(r.Pk[0], r1.P1)
    np.testing.assert_array_equal(r.Pk[1], r2.P2)
    assert r.dk_layer[0] == r1.d1_layer and r.dk_layer[1] == r2.d2_layer


def test_block_matrix_all_orders(order4):
    """Plain SP2 on the 5n x 5n matrix with H on the diagonal and H1 above it
    carries P_o in the block (0, o) of its first block row (Sec. III B)."""
    inst, r = order4
    n, m = inst.n, 4
    Hb = np.zeros(((m + 1) * n, (m + 1) * n))
    for b in range(m + 1):
        Hb[b * n:(b + 1) * n, b * n:(b + 1) * n] = inst.H
        if b < m:
            Hb[b * n:(b + 1) * n, (b + 1) * n:(b + 2) * n] = inst.H1[0]
    e1, eN = r.bounds
    for o in range(1, m + 1):
        S = (eN * np.eye((m + 1) * n) - Hb) / (eN - e1)
        for s in r.sigma[: r.dk_layer[o - 1][0] - 1]:
            S = S @ S if s == 1 else 2 * S - S @ S
        assert rel(S[:n, o * n:(o + 1) * n], r.Pk[o - 1][0]) < 1e-9, o


def test_identities_by_order(order4):
    """Order o of D^2 = D, [H + lambda H1, D] = 0 and Tr D = n_occ."""
    inst, r = order4
    H, H1 = inst.H, inst.H1[0]
    Pk = [r.P] + [p[0] for p in r.Pk]
    for o in range(1, 5):
        sq = sum(Pk[a] @ Pk[o - a] for a in range(o + 1))
        scale = np.linalg.norm(Pk[o])
        assert np.linalg.norm(sq - Pk[o]) < 1e-9 * scale, o
        comm = H @ Pk[o] - Pk[o] @ H + H1 @ Pk[o - 1] - Pk[o - 1] @ H1
        assert np.linalg.norm(comm) < 1e-8 * scale * np.linalg.norm(H), o
        assert abs(np.trace(Pk[o])) < 1e-11 * max(scale, 1.0), o


def test_third_order_finite_differences_of_sos():
    """P_3 = (d/dh) P_2(H + h H1) / 3 at h = 0, with P_2 by sum over states."""
    inst = make_workload(1)
    r = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ, order=3)
    D2 = lambda t: response2_sos(inst.H + t * inst.H1[0], inst.H1[0], inst.n_occ)
    errs = [rel((D2(h) - D2(-h)) / (6 * h), r.Pk[2][0]) for h in (0.02, 0.01, 0.005)]
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0   # O(h^2)
    assert errs[2] < 1e-3


def test_two_level_symbolic_third_derivative():
    sp = pytest.importorskip("sympy")
    lam = sp.symbols("lam", real=True)
    rng = np.random.default_rng(23)
    for trial in range(3):
        a, b = sorted(rng.uniform(-2, 2, 2))
        th = rng.uniform(0, np.pi)
        c, s = np.cos(th), np.sin(th)
        R = np.array([[c, -s], [s, c]])
        H = R @ np.diag([a, b]) @ R.T
        H1 = sym_gauss(2, 500 + trial)
        M = sp.Matrix(2, 2, lambda i, j: sp.Float(H[i, j], 30) + lam * sp.Float(H1[i, j], 30))
        tr = M[0, 0] + M[1, 1]
        d = sp.sqrt(((M[0, 0] - M[1, 1]) / 2) ** 2 + M[0, 1] ** 2)
        e_hi, e_lo = tr / 2 + d, tr / 2 - d
        Plow = (e_hi * sp.eye(2) - M) / (e_hi - e_lo)
        r = oracle.sp2_pt(H, H1, 1, order=3)
        assert r.converged
        for o in (1, 2, 3):
            want = np.array((sp.diff(Plow, lam, o) / sp.factorial(o)).subs(lam, 0).evalf(20),
                            dtype=float)
            np.testing.assert_allclose(r.Pk[o - 1][0], want, atol=1e-9 * max(1, np.abs(want).max()))


def test_trivial_occupations_all_orders():
    inst = make_workload(1)
    for n_occ in (0, inst.n):
        r = oracle.sp2_pt(inst.H, inst.H1, n_occ, order=3)
        assert r.layers == 0 and len(r.Pk) == 3
        assert all(not p.any() for p in r.Pk)


def test_directions_are_independent():
    """Each direction's terms depend on its own H1 only: a run with the
    stack [H1_a, H1_b] gives direction a's terms of a run with H1_a alone
    (the shared S0 recursion is the same, and a converged term stays
    frozen while the other direction runs on), so a mix-up of directions'
    slots would show."""
    inst = make_workload(3, n=96, k=2)
    both = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ, order=3)
    for j in range(2):
        alone = oracle.sp2_pt(inst.H, inst.H1[j:j + 1], inst.n_occ, order=3)
        for o in range(3):
            assert both.dk_layer[o][j] == alone.dk_layer[o][0]
            np.testing.assert_array_equal(both.Pk[o][j], alone.Pk[o][0])
