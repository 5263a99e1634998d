"""The oracle's pins catch plausible mistakes (mutation check, CPU only).

Each case plants one mistake in a copy of an oracle module (a dropped
term, a wrong sign, a wrong index, a transposed or one-sided product, a
wrong branch rule), loads the copy as a separate module, and checks that at
least one pin that does not use the mutated formula itself fails on it.

SP2 recursion (oracle/sp2.py):
  * agreement with the sum-over-states response (a different route to the
    same limit), first and second order;
  * the order-by-order identities of the converged terms (idempotency,
    commutation, trace);
  * plain SP2 on the block upper-triangular matrix of Sec. III B.
Sum over states (oracle/sos.py), first and second order:
  * the 2x2 closed form (tests/golden/two_level.json);
  * central finite differences of the eigendecomposition projector;
  * the identities of the first- and second-order blocks of D^2 = D and
    [H + lambda H1, D] = 0.
Adjoint (oracle/sp2.py, sp2_adjoint): the self-adjoint Daleckii-Krein
derivative (the forward response with H1 := G, by sum over states) and
central differences of Tr[G P(H + t E)].
Gershgorin bounds (oracle/gershgorin.py): the hand-computed 3x3 fixture
and containment of the spectrum.
Stopping rules (oracle/sp2.py, Alg. 2 and Alg. 3): the hand-worked dyadic
fixture (both clauses of Alg. 2, C_pt, FroErr^(0) and the n - 2 index of
Alg. 3) and the 2x2 closed form.
Self-consistent response (oracle/scc.py): the closed-form fixed point
q = (I - chi gamma)^-1 q0 from the charge susceptibility chi.
The unmutated modules pass all of them.  Nothing here touches the CUDA
path: the mistakes are planted in the oracle, on the CPU.
"""

import importlib.util
import os
import sys

import numpy as np
import pytest

import oracle
from oracle.sos import response2_sos
from paper_2203_09621_gb300.workloads import make_workload

SP2_PATH = os.path.join(os.path.dirname(oracle.__file__), "sp2.py")
SOS_PATH = os.path.join(os.path.dirname(oracle.__file__), "sos.py")
SCC_PATH = os.path.join(os.path.dirname(oracle.__file__), "scc.py")
GER_PATH = os.path.join(os.path.dirname(oracle.__file__), "gershgorin.py")

MUTATIONS = [
    ("dropped cross term of order o", "for a in range(1, o):", "for a in range(1, max(1, o - 1)):"),
    ("one-sided response product", "acc = S0 @ S[o][j] + S[o][j] @ S0", "acc = 2 * S0 @ S[o][j]"),
    ("wrong cross index", "acc = acc + S[a][j] @ S[o - a][j]", "acc = acc + S[a][j] @ S[a][j]"),
    ("sign of the initial response", "S = {1: [W0 * H1[j] for j in range(k)]}",
     "S = {1: [-W0 * H1[j] for j in range(k)]}"),
    ("bias with S_n instead of S_{n-1}", "S0 = s * X0 + (1 - s) * S0", "S0 = s * X0 + (1 - s) * X0"),
    ("response update without the bias", "S[o][j] = s * X[o][j] + (1 - s) * S[o][j]",
     "S[o][j] = s * X[o][j]"),
    ("branch rule inverted",
     "sigma[n_layer] = _sign_tie_minus(abs(2.0 * NS - NX - n_occ) - abs(NX - n_occ))",
     "sigma[n_layer] = -_sign_tie_minus(abs(2.0 * NS - NX - n_occ) - abs(NX - n_occ))"),
]


def load_variant(src, name, path=SP2_PATH):
    spec = importlib.util.spec_from_loader(f"oracle.{name}", loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    sys.modules[spec.name] = mod
    try:
        exec(compile(src, path, "exec"), mod.__dict__)
    finally:
        del sys.modules[spec.name]
    return mod


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def case():
    inst = make_workload(1, n=64)
    D1 = oracle.response_sos(inst.H, inst.H1[0], inst.n_occ)[1]
    D2 = response2_sos(inst.H, inst.H1[0], inst.n_occ)
    return inst, D1, D2


def pins_fail(mod, case):
    """Names of the pins the module fails (empty: passes them all)."""
    inst, D1, D2 = case
    failed = []
    try:
        r = mod.sp2_pt(inst.H, inst.H1, inst.n_occ, order=3, max_layers=100)
    except Exception as e:   # a mistake may also break the run
        return [f"raised {type(e).__name__}"]
    if not r.converged:
        failed.append("converged")
    if not rel(r.Pk[0][0], D1) <= 1e-9:
        failed.append("first order vs sum over states")
    if not rel(r.Pk[1][0], D2) <= 1e-9:
        failed.append("second order vs sum over states")
    Pk = [r.P] + [p[0] for p in r.Pk]
    H, H1 = inst.H, inst.H1[0]
    for o in range(1, 4):
        sc = max(np.linalg.norm(Pk[o]), 1e-300)
        if not np.linalg.norm(sum(Pk[a] @ Pk[o - a] for a in range(o + 1)) - Pk[o]) <= 1e-8 * sc:
            failed.append(f"idempotency, order {o}")
        comm = H @ Pk[o] - Pk[o] @ H + H1 @ Pk[o - 1] - Pk[o - 1] @ H1
        if not np.linalg.norm(comm) <= 1e-7 * sc * np.linalg.norm(H):
            failed.append(f"commutation, order {o}")
    # plain SP2 of the 4n x 4n block matrix with the run's own decisions
    n, m = inst.n, 3
    Hb = np.zeros(((m + 1) * n, (m + 1) * n))
    for b in range(m + 1):
        Hb[b * n:(b + 1) * n, b * n:(b + 1) * n] = H
        if b < m:
            Hb[b * n:(b + 1) * n, (b + 1) * n:(b + 2) * n] = H1
    e1, eN = r.bounds
    S = (eN * np.eye((m + 1) * n) - Hb) / (eN - e1)
    for s in r.sigma[: r.dk_layer[2][0] - 1]:
        S = S @ S if s == 1 else 2 * S - S @ S
    if not rel(S[:n, 3 * n:], Pk[3]) <= 1e-8:
        failed.append("block matrix, order 3")
    return failed


def test_unmutated_oracle_passes(case):
    src = open(SP2_PATH).read()
    assert pins_fail(load_variant(src, "sp2_copy"), case) == []


@pytest.mark.parametrize("what,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(case, what, old, new):
    src = open(SP2_PATH).read()
    assert src.count(old) == 1, what
    failed = pins_fail(load_variant(src.replace(old, new), "sp2_mutant"), case)
    assert failed, what


SOS_MUTATIONS = [
    ("sign of the divided difference", "F[mask] = df[mask] / de[mask]",
     "F[mask] = -df[mask] / de[mask]"),
    ("transposed eigenbasis", "P1 = V @ (F * Y) @ V.T", "P1 = V.T @ (F * Y) @ V"),
    ("sign of the first divided difference in the second order",
     "d1[mask] = (f[mask] - f[m]) / (eps[mask] - eps[m])",
     "d1[mask] = (f[m] - f[mask]) / (eps[mask] - eps[m])"),
    ("sign of the confluent second divided difference",
     "diag[mask] = -(f[mask] - f[m]) / (eps[mask] - eps[m]) ** 2",
     "diag[mask] = (f[mask] - f[m]) / (eps[mask] - eps[m]) ** 2"),
    ("halved second-order sum", "M += _second_divided_differences(eps, f, m) * np.outer(Y[:, m], Y[m, :])",
     "M += 0.5 * _second_divided_differences(eps, f, m) * np.outer(Y[:, m], Y[m, :])"),
]


def sos_pins_fail(mod, golden):
    failed = []
    g = golden("two_level.json")
    P, P1 = mod.response_sos(np.array(g["H"]), np.array(g["H1"]), g["n_occ"])
    if not np.abs(P1 - np.array(g["P1"])).max() <= 1e-12:
        failed.append("2x2 closed form")
    inst = make_workload(1, n=48)
    H, H1, n_occ = inst.H, inst.H1[0], inst.n_occ
    P, P1 = mod.response_sos(H, H1, n_occ)
    D2 = mod.response2_sos(H, H1, n_occ)
    D = lambda t: oracle.density_matrix(H + t * H1, n_occ)   # eigh projector, unmutated
    h = 1e-3
    if not rel((D(h) - D(-h)) / (2 * h), P1) <= 1e-4:
        failed.append("first-order finite differences")
    if not rel((D(h) - 2 * D(0.0) + D(-h)) / (2 * h * h), D2) <= 1e-3:
        failed.append("second-order finite differences")
    if not np.linalg.norm(P @ P1 + P1 @ P - P1) <= 1e-10 * np.linalg.norm(P1):
        failed.append("first-order idempotency")
    if not np.linalg.norm(P @ D2 + P1 @ P1 + D2 @ P - D2) <= 1e-10 * np.linalg.norm(D2):
        failed.append("second-order idempotency")
    if not np.linalg.norm(H @ D2 - D2 @ H + H1 @ P1 - P1 @ H1) <= 1e-9 * np.linalg.norm(D2):
        failed.append("second-order commutation")
    return failed


def test_unmutated_sos_passes(golden):
    src = open(SOS_PATH).read()
    assert sos_pins_fail(load_variant(src, "sos_copy", SOS_PATH), golden) == []


@pytest.mark.parametrize("what,old,new", SOS_MUTATIONS, ids=[m[0] for m in SOS_MUTATIONS])
def test_planted_sos_mistake_is_caught(golden, what, old, new):
    src = open(SOS_PATH).read()
    assert src.count(old) == 1, what
    failed = sos_pins_fail(load_variant(src.replace(old, new), "sos_mutant", SOS_PATH), golden)
    assert failed, what


ADJ_MUTATIONS = [
    ("one-sided adjoint product", "Gbar = s * (Sp @ Gbar + Gbar @ Sp) + (1 - s) * Gbar",
     "Gbar = s * (2 * Sp @ Gbar) + (1 - s) * Gbar"),
    ("sign of the input transform", "return -Gbar / (epsN - eps1)", "return Gbar / (epsN - eps1)"),
    ("state of the wrong layer", "Sp = states[idx]", "Sp = states[idx + 1]"),
]


def adj_pins_fail(mod):
    from paper_2203_09621_gb300.workloads import sym_gauss
    failed = []
    inst = make_workload(1, n=48)
    G = sym_gauss(48, 12)
    r = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ)
    dLdH = mod.sp2_adjoint(inst.H, G, inst.n_occ, r.sigma[: r.d0_layer - 1], r.bounds)
    _, P1G = oracle.response_sos(inst.H, G, inst.n_occ)
    if not rel(dLdH, P1G) <= 1e-9:
        failed.append("self-adjoint derivative")
    E = sym_gauss(48, 13)
    L = lambda t: np.sum(G * oracle.density_matrix(inst.H + t * E, inst.n_occ))
    h = 1e-4
    fd = (L(h) - L(-h)) / (2 * h)
    if not abs(fd - np.sum(dLdH * E)) <= 1e-6 * max(1.0, abs(fd)):
        failed.append("finite differences of Tr[G P]")
    return failed


def test_unmutated_adjoint_passes():
    assert adj_pins_fail(load_variant(open(SP2_PATH).read(), "adj_copy")) == []


@pytest.mark.parametrize("what,old,new", ADJ_MUTATIONS, ids=[m[0] for m in ADJ_MUTATIONS])
def test_planted_adjoint_mistake_is_caught(what, old, new):
    src = open(SP2_PATH).read()
    assert src.count(old) == 1, what
    assert adj_pins_fail(load_variant(src.replace(old, new), "adj_mutant")), what


SCC_MUTATIONS = [
    ("charges from the wrong diagonal", "q_out = np.diag(P1).copy()", "q_out = -np.diag(P1).copy()"),
    ("coupling transposed into a row sum",
     "_, P1 = response_from_eigs(eps, V, H1_ext + np.diag(gamma @ q), n_occ)\n        q_out",
     "_, P1 = response_from_eigs(eps, V, H1_ext + np.diag(gamma.sum(1) * q), n_occ)\n        q_out"),
    ("coupling dropped in the final response",
     "    _, P1 = response_from_eigs(eps, V, H1_ext + np.diag(gamma @ q), n_occ)\n    return",
     "    _, P1 = response_from_eigs(eps, V, H1_ext, n_occ)\n    return"),
]


def scc_pins_fail(mod):
    from paper_2203_09621_gb300.workloads import scc_gamma
    failed = []
    n = 32
    inst = make_workload(3, n=n, k=1)
    g = scc_gamma(n)
    eps, V = np.linalg.eigh(inst.H)
    chi = np.stack([np.diag(oracle.response_from_eigs(eps, V, np.diag(np.eye(n)[c]),
                                                      inst.n_occ)[1]) for c in range(n)], axis=1)
    q0 = np.diag(oracle.response_from_eigs(eps, V, inst.H1[0], inst.n_occ)[1])
    q_closed = np.linalg.solve(np.eye(n) - chi @ g, q0)
    with np.errstate(all="ignore"):
        P1, q, _ = mod.scc_response(inst.H, inst.H1[0], g, inst.n_occ)
    # "not <=" so that a non-finite result fails too
    if not np.linalg.norm(q - q_closed) <= 1e-10 * np.linalg.norm(q_closed):
        failed.append("closed-form fixed point")
    if not np.linalg.norm(np.diag(P1) - q_closed) <= 1e-9 * np.linalg.norm(q_closed):
        failed.append("response at the fixed point")
    return failed


def test_unmutated_scc_passes():
    assert scc_pins_fail(load_variant(open(SCC_PATH).read(), "scc_copy", SCC_PATH)) == []


@pytest.mark.parametrize("what,old,new", SCC_MUTATIONS, ids=[m[0] for m in SCC_MUTATIONS])
def test_planted_scc_mistake_is_caught(what, old, new):
    src = open(SCC_PATH).read()
    assert src.count(old) == 1, what
    assert scc_pins_fail(load_variant(src.replace(old, new), "scc_mutant", SCC_PATH)), what


GER_MUTATIONS = [
    ("diagonal kept in the radius", "radius = np.sum(np.abs(H[i, :])) - abs(H[i, i])",
     "radius = np.sum(np.abs(H[i, :]))"),
    ("signed radius", "radius = np.sum(np.abs(H[i, :])) - abs(H[i, i])",
     "radius = np.sum(H[i, :]) - H[i, i]"),
    ("column of the wrong index", "radius = np.sum(np.abs(H[i, :])) - abs(H[i, i])",
     "radius = np.sum(np.abs(H[:, 0])) - abs(H[0, 0])"),
]


def ger_pins_fail(mod, golden):
    from paper_2203_09621_gb300.workloads import sym_gauss
    failed = []
    g = golden("gershgorin_3x3.json")
    if list(mod.gershgorin_bounds(np.array(g["H"]))) != g["bounds"]:
        failed.append("3x3 fixture")
    H = sym_gauss(40, 7) + np.diag(np.linspace(-3, 3, 40))
    lo, hi = mod.gershgorin_bounds(H)
    ev = np.linalg.eigvalsh(H)
    if not (lo <= ev[0] and ev[-1] <= hi):
        failed.append("containment")
    return failed


def test_unmutated_gershgorin_passes(golden):
    assert ger_pins_fail(load_variant(open(GER_PATH).read(), "ger_copy", GER_PATH), golden) == []


@pytest.mark.parametrize("what,old,new", GER_MUTATIONS, ids=[m[0] for m in GER_MUTATIONS])
def test_planted_gershgorin_mistake_is_caught(golden, what, old, new):
    src = open(GER_PATH).read()
    assert src.count(old) == 1, what
    assert ger_pins_fail(load_variant(src.replace(old, new), "ger_mutant", GER_PATH), golden), what


# Stopping rules (Alg. 2 and Alg. 3): planted in the SP2 oracle, caught by the
# hand-worked dyadic fixture (tests/golden/stopping_rules_dyadic.json) and the
# 2x2 closed form (tests/golden/two_level.json), neither of which runs the
# mutated rule to obtain its expected values.
STOP_MUTATIONS = [
    ("second clause of Alg. 2 removed",
     "and iderr[n_layer] > c_d0 * iderr[n_layer - 2] ** 2):", "and False):"),
    ("IdErr_{n-1} in place of IdErr_{n-2}",
     "c_d0 * iderr[n_layer - 2] ** 2", "c_d0 * iderr[n_layer - 1] ** 2"),
    ("IdErr_{n-2} not squared", "c_d0 * iderr[n_layer - 2] ** 2", "c_d0 * iderr[n_layer - 2]"),
    ("first clause of Alg. 2 strict", "if iderr[n_layer] <= 0.0:", "if iderr[n_layer] < 0.0:"),
    ("C_pt dropped from Alg. 3", "fe >= c_pt * froerr0 * prev", "fe >= froerr0 * prev"),
    ("FroErr^(0) dropped from Alg. 3", "fe >= c_pt * froerr0 * prev", "fe >= c_pt * prev"),
    ("FroErr^(1)_{n-1} in place of FroErr^(1)_{n-2}",
     "prev = froerr[o][j].get(n_layer - 2)", "prev = froerr[o][j].get(n_layer - 1)"),
    ("strict comparison in Alg. 3 (never fires at exact zero)",
     "fe >= c_pt * froerr0 * prev", "fe > c_pt * froerr0 * prev"),
    ("FroErr^(0) of the updated state", 'froerr0 = np.linalg.norm(S0 - X0, "fro")',
     'froerr0 = np.linalg.norm(X0 - X0 @ X0, "fro")'),
    ("no sigma flip after D^(0) converged", "sigma[n_layer] = -sigma[n_layer - 1]",
     "sigma[n_layer] = sigma[n_layer - 1]"),
]


def stop_pins_fail(mod, golden):
    from fractions import Fraction
    failed = []
    g = golden("stopping_rules_dyadic.json")
    H = np.diag(np.array(g["H_diag"]))
    H1 = np.zeros_like(H)
    for i, j in g["H1_offdiag"]["pairs"]:
        H1[i, j] = H1[j, i] = g["H1_offdiag"]["value"]
    try:
        r = mod.sp2_pt(H, H1, g["n_occ"], c_pt=g["c_pt"], c_d0=g["c_d0"], max_layers=30)
        if r.d0_layer != g["d0_layer"]:
            failed.append("dyadic: D0 layer")
        if r.iderr != [float(Fraction(s)) for s in g["iderr"]]:
            failed.append("dyadic: IdErr history")
        if not abs(r.froerr0 - float(Fraction(g["froerr0_sq"])) ** 0.5) <= 1e-14 * r.froerr0:
            failed.append("dyadic: FroErr0")
        if r.d1_layer != [g["d1_layer"]] or not r.converged:
            failed.append("dyadic: D1 layer")
        if r.sigma != g["sigma"][: len(r.sigma)]:
            failed.append("dyadic: sigma")
        for v in g["variants"]:
            rv = mod.sp2_pt(H, H1, g["n_occ"], c_pt=v["c_pt"], c_d0=v["c_d0"], max_layers=30)
            if rv.d0_layer != v["d0_layer"] or ("d1_layer" in v and rv.d1_layer != [v["d1_layer"]]):
                failed.append(f"dyadic variant c_pt={v['c_pt']} c_d0={v['c_d0']}")
        t = golden("two_level.json")
        rt = mod.sp2_pt(np.array(t["H"]), np.array(t["H1"]), t["n_occ"], max_layers=30)
        if not rt.converged or rt.d0_layer != t["d0_layer"] or \
                not np.abs(rt.P1[0] - np.array(t["P1"])).max() <= 1e-15:
            failed.append("2x2 closed form")
    except Exception as e:
        failed.append(f"raised {type(e).__name__}")
    return failed


def test_unmutated_stopping_rules_pass(golden):
    assert stop_pins_fail(load_variant(open(SP2_PATH).read(), "stop_copy"), golden) == []


@pytest.mark.parametrize("what,old,new", STOP_MUTATIONS, ids=[m[0] for m in STOP_MUTATIONS])
def test_planted_stopping_mistake_is_caught(golden, what, old, new):
    src = open(SP2_PATH).read()
    assert src.count(old) == 1, what
    assert stop_pins_fail(load_variant(src.replace(old, new), "stop_mutant"), golden), what
