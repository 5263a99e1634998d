"""Pins for the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, an invariant, a second
route to the same quantity (finite differences, the block-matrix form of
Sec. III B, symbolic differentiation) or a hand-computed fixture; none of
them re-types the formula of the function it checks.
"""

import numpy as np
import pytest

import oracle
from oracle.sos import response_columns
from paper_2203_09621_gb300.workloads import make_workload, make_instance, sym_gauss


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# --------------------------------------------------------------------------
# Gershgorin bounds (Sec. II B)

def test_gershgorin_golden_3x3(golden):
    g = golden("gershgorin_3x3.json")
    lo, hi = oracle.gershgorin_bounds(np.array(g["H"]))
    assert (lo, hi) == tuple(g["bounds"])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gershgorin_contains_spectrum(seed):
    H = sym_gauss(37, seed)
    lo, hi = oracle.gershgorin_bounds(H)
    ev = np.linalg.eigvalsh(H)
    assert lo <= ev[0] and ev[-1] <= hi


def test_gershgorin_diagonal_is_exact():
    d = np.array([3.0, -2.5, 0.25, 7.0])
    assert oracle.gershgorin_bounds(np.diag(d)) == (-2.5, 7.0)


# --------------------------------------------------------------------------
# Two-level system: closed form (golden) and symbolic derivative

def test_two_level_golden_both_oracles(golden):
    g = golden("two_level.json")
    H, H1, n_occ = np.array(g["H"]), np.array(g["H1"]), g["n_occ"]
    P, P1 = oracle.response_sos(H, H1, n_occ)
    np.testing.assert_allclose(P, g["P"], atol=1e-15)
    np.testing.assert_allclose(P1, g["P1"], atol=1e-15)
    r = oracle.sp2_pt(H, H1, n_occ)
    assert r.converged
    assert r.bounds == tuple(g["bounds"])
    assert r.d0_layer == g["d0_layer"]
    np.testing.assert_allclose(r.P, g["P"], atol=1e-15)
    np.testing.assert_allclose(r.P1[0], g["P1"], atol=1e-15)


def test_two_level_symbolic_derivative():
    """d/dlambda of the closed-form 2x2 projector, differentiated by sympy."""
    sp = pytest.importorskip("sympy")
    lam = sp.symbols("lam", real=True)
    rng = np.random.default_rng(7)
    for trial in range(4):
        a, b = sorted(rng.uniform(-2, 2, 2))
        th = rng.uniform(0, np.pi)
        c, s = np.cos(th), np.sin(th)
        R = np.array([[c, -s], [s, c]])
        H = R @ np.diag([a, b]) @ R.T
        H1 = sym_gauss(2, 100 + trial)
        M = sp.Matrix(2, 2, lambda i, j: sp.Float(H[i, j], 30) + lam * sp.Float(H1[i, j], 30))
        tr = M[0, 0] + M[1, 1]
        d = sp.sqrt(((M[0, 0] - M[1, 1]) / 2) ** 2 + M[0, 1] ** 2)
        e_hi = tr / 2 + d
        e_lo = tr / 2 - d
        # projector on the lower eigenvalue of a 2x2 symmetric matrix
        Plow = (e_hi * sp.eye(2) - M) / (e_hi - e_lo)
        dP = sp.diff(Plow, lam).subs(lam, 0)
        want_P = np.array(Plow.subs(lam, 0).evalf(20), dtype=float)
        want_P1 = np.array(dP.evalf(20), dtype=float)
        P, P1 = oracle.response_sos(H, H1, 1)
        np.testing.assert_allclose(P, want_P, atol=1e-13)
        np.testing.assert_allclose(P1, want_P1, atol=1e-12)
        r = oracle.sp2_pt(H, H1, 1)
        assert r.converged
        np.testing.assert_allclose(r.P, want_P, atol=1e-12)
        np.testing.assert_allclose(r.P1[0], want_P1, atol=1e-10)


# --------------------------------------------------------------------------
# Invariants on the n = 128 workload (blocks of D^2 = D and HD = DH, Sec. III B)

@pytest.fixture(scope="module")
def plain128():
    inst = make_workload(1)
    P, P1 = oracle.response_sos(inst.H, inst.H1[0], inst.n_occ)
    r = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ)
    return inst, P, P1, r


@pytest.mark.parametrize("which", ["sos", "sp2"])
def test_invariants(plain128, which):
    inst, P, P1, r = plain128
    H, H1 = inst.H, inst.H1[0]
    if which == "sp2":
        P, P1 = r.P, r.P1[0]
    tol = 1e-12 if which == "sos" else 1e-11
    assert np.linalg.norm(P @ P - P) < tol * 10
    assert abs(np.trace(P) - inst.n_occ) < tol * 100
    assert np.linalg.norm(H @ P - P @ H) < tol * 100
    assert abs(np.trace(P1)) < tol * 10
    assert np.linalg.norm(P @ P1 + P1 @ P - P1) < tol * 10 * np.linalg.norm(P1)
    assert np.linalg.norm(H @ P1 - P1 @ H + H1 @ P - P @ H1) < tol * 100 * np.linalg.norm(P1)
    # eigenbasis: occupied-occupied and virtual-virtual blocks of P1 vanish (Sec. IV A)
    _, V = np.linalg.eigh(H)
    Y = V.T @ P1 @ V
    o = inst.n_occ
    assert np.abs(Y[:o, :o]).max() < 1e-11 and np.abs(Y[o:, o:]).max() < 1e-11


def test_two_oracles_agree(plain128):
    inst, P, P1, r = plain128
    assert r.converged
    assert rel(r.P, P) < 1e-12
    assert rel(r.P1[0], P1) < 1e-12


@pytest.mark.parametrize("cfg", [2, 3])
def test_two_oracles_agree_n256(cfg):
    inst = make_workload(cfg, n=256)
    P, P1 = oracle.response_sos(inst.H, inst.H1, inst.n_occ)
    r = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ)
    assert r.converged
    assert rel(r.P, P) < 1e-12
    for j in range(inst.k):
        assert rel(r.P1[j], P1[j]) < 1e-11


def test_known_eigs_match_eigh(plain128):
    inst, P, P1, r = plain128
    P_b, P1_b = oracle.response_from_eigs(inst.eps, inst.Q, inst.H1[0], inst.n_occ)
    assert rel(P_b, P) < 1e-12 and rel(P1_b, P1) < 1e-11
    # the projector from the known eigenvectors: eigh route, and its invariants
    P_c = oracle.density_from_eigs(inst.eps, inst.Q, inst.n_occ)
    assert rel(P_c, P) < 1e-12
    assert abs(np.trace(P_c) - inst.n_occ) < 1e-10
    assert np.linalg.norm(P_c @ P_c - P_c) < 1e-12 * np.linalg.norm(P_c)
    # every column of P1 from the occupied-virtual block equals the full transform
    np.testing.assert_allclose(response_columns(inst.eps, inst.Q, inst.H1[0], inst.n_occ,
                                                np.arange(inst.n)), P1_b, atol=1e-13)
    cols = [0, 5, 77, 127]
    np.testing.assert_allclose(response_columns(inst.eps, inst.Q, inst.H1[0], inst.n_occ, cols),
                               P1[:, cols], atol=1e-13)


# --------------------------------------------------------------------------
# Finite differences of the density matrix (Eq. (FnD_2), Eq. (FnD_4))

def test_finite_differences(plain128):
    inst, P, P1, r = plain128
    H, H1, o = inst.H, inst.H1[0], inst.n_occ
    D = lambda lam: oracle.density_matrix(H + lam * H1, o)
    errs2, errs4 = [], []
    for h in (0.08, 0.04, 0.02):
        fd2 = (D(h) - D(-h)) / (2 * h)
        fd4 = (-D(2 * h) + 8 * D(h) - 8 * D(-h) + D(-2 * h)) / (12 * h)
        errs2.append(rel(fd2, P1))
        errs4.append(rel(fd4, P1))
    # second order: halving h divides the error by ~4; fourth order by ~16
    assert 3.0 < errs2[0] / errs2[1] < 5.0 and 3.0 < errs2[1] / errs2[2] < 5.0
    assert errs4[0] / errs4[1] > 10.0
    assert errs4[-1] < errs2[-1] and errs2[-1] < 1e-2


# --------------------------------------------------------------------------
# Block upper-triangular form (Sec. III B): plain SP2 of [[H, H1], [0, H]]

def _plain_sp2_fixed(M, bounds, sigmas):
    """Plain SP2 of a (non-symmetric) matrix with a given branch sequence."""
    e1, eN = bounds
    S = (eN * np.eye(M.shape[0]) - M) / (eN - e1)
    for s in sigmas:
        S = S @ S if s == 1 else 2 * S - S @ S
    return S


def test_block_matrix_form(plain128):
    inst, P, P1, r = plain128
    n = inst.n
    Hb = np.block([[inst.H, inst.H1[0]], [np.zeros((n, n)), inst.H]])
    # layers that updated S1: all layers before the one whose Alg. 3 test fired
    sig = r.sigma[: r.d1_layer[0] - 1]
    Sb = _plain_sp2_fixed(Hb, r.bounds, sig)
    assert rel(Sb[:n, n:], r.P1[0]) < 1e-10
    assert rel(Sb[:n, :n], r.P) < 1e-10
    assert np.abs(Sb[n:, :n]).max() == 0.0


# --------------------------------------------------------------------------
# Edge cases

@pytest.mark.parametrize("n_occ", [0, 16])
def test_trivial_occupations(n_occ):
    H = sym_gauss(16, 3)
    H1 = sym_gauss(16, 4, 0.01)
    r = oracle.sp2_pt(H, H1, n_occ)
    P, P1 = oracle.response_sos(H, H1, n_occ)
    want = np.zeros((16, 16)) if n_occ == 0 else np.eye(16)
    np.testing.assert_allclose(r.P, want, atol=0)
    np.testing.assert_allclose(P, want, atol=1e-13)
    assert np.abs(r.P1).max() == 0.0 and np.abs(P1).max() < 1e-15
    assert r.layers == 0


def test_degenerate_homo_lumo_raises():
    H = np.diag([-1.0, 0.5, 0.5, 2.0])
    with pytest.raises(ValueError):
        oracle.response_sos(H, np.eye(4), 2)


def test_layer_cap_reports_not_converged():
    inst = make_workload(1)
    r = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ, max_layers=5)
    assert not r.converged and r.layers == 5


def test_d1_stops_two_layers_after_d0(plain128):
    # Sec. IV A: the criterion fires a few layers after D^(0) has converged,
    # never before one sigma-flip pair has been applied.
    inst, P, P1, r = plain128
    assert r.d1_layer[0] >= r.d0_layer + 2
    assert r.layers == max(r.d1_layer)
    # after D^(0) converges the branches alternate (the sigma flip of Alg. 1)
    tail = r.sigma[r.d0_layer:]
    assert all(tail[i] == -tail[i - 1] for i in range(1, len(tail)))


# --------------------------------------------------------------------------
# Adjoint of the S_0 recursion (L = Tr[G P])

def test_adjoint_matches_response_and_fd():
    inst = make_instance("adj", 64, 32, (-2.0, -0.3), (0.3, 2.0), seed=11)
    G = sym_gauss(64, 12)
    r = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ)
    sig_d0 = r.sigma[: r.d0_layer - 1]
    dLdH = oracle.sp2_adjoint(inst.H, G, inst.n_occ, sig_d0, r.bounds)
    # Daleckii-Krein derivative is self-adjoint: dL/dH = P1(H1 := G)
    _, P1G = oracle.response_sos(inst.H, G, inst.n_occ)
    assert rel(dLdH, P1G) < 1e-10
    # directional check with central differences of Tr[G P(H + t E)]
    E = sym_gauss(64, 13)
    L = lambda t: np.sum(G * oracle.density_matrix(inst.H + t * E, inst.n_occ))
    h = 1e-4
    fd = (L(h) - L(-h)) / (2 * h)
    assert abs(fd - np.sum(dLdH * E)) < 1e-6 * max(1.0, abs(fd))


# --------------------------------------------------------------------------
# Stopping rules (Alg. 2 second clause, Alg. 3 / Eq. (ConvCrit)): a
# hand-worked diagonal case whose values are exact dyadic rationals

def stopping_fixture(g):
    from fractions import Fraction
    H = np.diag(np.array(g["H_diag"]))
    n = H.shape[0]
    H1 = np.zeros((n, n))
    for i, j in g["H1_offdiag"]["pairs"]:
        H1[i, j] = H1[j, i] = g["H1_offdiag"]["value"]
    return H, H1, Fraction


def test_stopping_rules_golden(golden):
    g = golden("stopping_rules_dyadic.json")
    H, H1, Fraction = stopping_fixture(g)
    r = oracle.sp2_pt(H, H1, g["n_occ"], c_pt=g["c_pt"], c_d0=g["c_d0"], max_layers=30)
    assert r.bounds == tuple(g["bounds"])
    assert r.converged
    # Alg. 2: branch sequence, exact idempotency errors, the second clause at layer 4
    assert r.d0_layer == g["d0_layer"]
    assert r.sigma == g["sigma"]
    want_iderr = [float(Fraction(s)) for s in g["iderr"]]
    assert r.iderr == want_iderr          # exact: every value is a short dyadic rational
    assert r.iderr[-1] > 0.0              # fired by the second clause, not by IdErr <= 0
    assert r.froerr0 == pytest.approx(float(Fraction(g["froerr0_sq"])) ** 0.5, rel=1e-14)
    # Alg. 3: FroErr^(1) history from the D^(0) layer on and the layer where it fires
    for layer, want in g["froerr1"].items():
        assert r.froerr1[0][int(layer) - 1] == pytest.approx(want, rel=1e-10)
    assert all(np.isnan(r.froerr1[0][m - 1]) for m in range(1, g["d0_layer"]))
    assert r.d1_layer == [g["d1_layer"]]
    assert r.layers == g["d1_layer"]


@pytest.mark.parametrize("variant", range(3))
def test_stopping_rules_golden_variants(golden, variant):
    g = golden("stopping_rules_dyadic.json")
    v = g["variants"][variant]
    H, H1, _ = stopping_fixture(g)
    r = oracle.sp2_pt(H, H1, g["n_occ"], c_pt=v["c_pt"], c_d0=v["c_d0"], max_layers=30)
    assert r.d0_layer == v["d0_layer"]
    if "d1_layer" in v:
        assert r.converged == v["converged"]
        assert r.d1_layer == [v["d1_layer"]]
        if not v["converged"]:
            assert r.layers == 30


def test_stopping_rule_constants_default_to_the_paper():
    import inspect
    sig = inspect.signature(oracle.sp2_pt)
    assert sig.parameters["c_pt"].default == 9.0    # Eq. (ConvCrit), Alg. 3
    assert sig.parameters["c_d0"].default == 4.5    # Alg. 2
