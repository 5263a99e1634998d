"""Pins for the second-order response oracles (oracle.sos.response2_*,
oracle.sp2.sp2_pt(order=2))."""

import numpy as np
import pytest

import oracle
from oracle.sos import response2_sos
from paper_2203_09621_gb300.workloads import make_workload, sym_gauss


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_two_level_order2_golden(golden):
    g = golden("two_level_order2.json")
    H, H1 = np.array(g["H"]), np.array(g["H1"])
    np.testing.assert_allclose(response2_sos(H, H1, g["n_occ"]), g["P2"], atol=1e-15)
    r = oracle.sp2_pt(H, H1, g["n_occ"], order=2)
    assert r.converged
    np.testing.assert_allclose(r.P2[0], g["P2"], atol=1e-15)


def test_two_level_symbolic_second_derivative():
    sp = pytest.importorskip("sympy")
    lam = sp.symbols("lam", real=True)
    rng = np.random.default_rng(17)
    for trial in range(3):
        a, b = sorted(rng.uniform(-2, 2, 2))
        th = rng.uniform(0, np.pi)
        c, s = np.cos(th), np.sin(th)
        R = np.array([[c, -s], [s, c]])
        H = R @ np.diag([a, b]) @ R.T
        H1 = sym_gauss(2, 300 + trial)
        M = sp.Matrix(2, 2, lambda i, j: sp.Float(H[i, j], 30) + lam * sp.Float(H1[i, j], 30))
        tr = M[0, 0] + M[1, 1]
        d = sp.sqrt(((M[0, 0] - M[1, 1]) / 2) ** 2 + M[0, 1] ** 2)
        e_hi, e_lo = tr / 2 + d, tr / 2 - d
        Plow = (e_hi * sp.eye(2) - M) / (e_hi - e_lo)
        want = np.array((sp.diff(Plow, lam, 2) / 2).subs(lam, 0).evalf(20), dtype=float)
        np.testing.assert_allclose(response2_sos(H, H1, 1), want, atol=1e-11)
        r = oracle.sp2_pt(H, H1, 1, order=2)
        np.testing.assert_allclose(r.P2[0], want, atol=1e-9)


@pytest.fixture(scope="module")
def plain128():
    inst = make_workload(1)
    D2 = response2_sos(inst.H, inst.H1[0], inst.n_occ)
    r = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ, order=2)
    return inst, D2, r


def test_sp2_order2_agrees_with_sos(plain128):
    inst, D2, r = plain128
    assert r.converged and rel(r.P2[0], D2) < 1e-12


def test_second_finite_differences(plain128):
    inst, D2, r = plain128
    D = lambda t: oracle.density_matrix(inst.H + t * inst.H1[0], inst.n_occ)
    D0 = D(0.0)
    errs = []
    for h in (0.04, 0.02, 0.01):
        errs.append(rel((D(h) - 2 * D0 + D(-h)) / (2 * h * h), D2))
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0   # O(h^2)


def test_order2_identities(plain128):
    """Blocks (1,3) of D^2 = D and HD = DH for the 3n x 3n block matrices (Sec. III B)."""
    inst, D2, r = plain128
    P, P1 = r.P, r.P1[0]
    H, H1 = inst.H, inst.H1[0]
    assert np.linalg.norm(P @ D2 + P1 @ P1 + D2 @ P - D2) < 1e-10 * np.linalg.norm(D2)
    assert np.linalg.norm(H @ D2 - D2 @ H + H1 @ P1 - P1 @ H1) < 1e-9 * np.linalg.norm(D2)
    assert abs(np.trace(D2)) < 1e-12


def test_block_matrix_order2(plain128):
    inst, D2, r = plain128
    n = inst.n
    Z = np.zeros((n, n))
    Hb = np.block([[inst.H, inst.H1[0], Z], [Z, inst.H, inst.H1[0]], [Z, Z, inst.H]])
    e1, eN = r.bounds
    S = (eN * np.eye(3 * n) - Hb) / (eN - e1)
    for s in r.sigma[: r.d2_layer[0] - 1]:
        S = S @ S if s == 1 else 2 * S - S @ S
    assert rel(S[:n, 2 * n:], r.P2[0]) < 1e-10
