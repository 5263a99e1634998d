"""GPU parity of the stopping decisions (Alg. 1 branch rule, Alg. 2, Alg. 3).

Two kinds of check, both through the C ABI:

* The hand-worked dyadic case (tests/golden/stopping_rules_dyadic.json) in
  every precision: the device must take the decisions the fixture works out
  by hand -- the branch sequence, the second clause of Alg. 2 firing at layer
  4 with IdErr_4 > 0, Alg. 3 firing at layer 8 (C_pt = 9), at layer 6
  (C_pt = 1) or never (C_pt = 12), and D^(0) at layer 3 for c_d0 = 1.0.
* Full-size solves (n = 1024 and 2048, dual FP16 / BF16 and FP32): the
  per-layer N_S, N_X and FroErr^(1) the device reports in dmpt_info are fed
  to the rules as printed in the paper, restated below in plain Python, and
  every decision the device took (sigma_n, the D^(0) layer, each direction's
  D^(1) layer) must be the one the rules give for those numbers.
"""

from fractions import Fraction

import numpy as np
import pytest

from paper_2203_09621_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2203_09621_gb300 import dmpt  # noqa: E402

DEV = torch.device("cuda:0")
PRECISIONS = ["fp64", "fp32", "dual_fp16", "dual_bf16"]
# relative tolerance of the reported IdErr / FroErr values against the
# fixture's exact ones: FP64 rounding, FP32 masters, or the dual products
VAL_TOL = {"fp64": 1e-12, "fp32": 1e-5, "dual_fp16": 1e-4, "dual_bf16": 1e-3}


@pytest.fixture(scope="module")
def ctx():
    return dmpt.context(0)


@pytest.fixture(scope="module")
def fixture(golden_module):
    return golden_module("stopping_rules_dyadic.json")


@pytest.fixture(scope="module")
def golden_module():
    import json
    import os
    from tests.conftest import GOLDEN

    return lambda name: json.load(open(os.path.join(GOLDEN, name)))


def solve_fixture(ctx, g, precision, c_pt, c_d0, max_layers=30, hole_form=0):
    H = torch.from_numpy(np.diag(np.array(g["H_diag"]))).to(DEV)
    n = H.shape[0]
    H1 = torch.zeros(1, n, n, dtype=torch.float64, device=DEV)
    for i, j in g["H1_offdiag"]["pairs"]:
        H1[0, i, j] = H1[0, j, i] = g["H1_offdiag"]["value"]
    P, P1, info = ctx.sp2_response(H, H1, g["n_occ"], precision=precision, c_pt=c_pt,
                                   c_d0=c_d0, max_layers=max_layers, raise_on_error=False,
                                   hole_form=hole_form)
    torch.cuda.synchronize()
    return info


@pytest.mark.parametrize("precision", PRECISIONS)
def test_dyadic_fixture_decisions(ctx, fixture, precision):
    g = fixture
    info = solve_fixture(ctx, g, precision, g["c_pt"], g["c_d0"])
    tol = VAL_TOL[precision]
    assert (info.eps_min, info.eps_max) == tuple(g["bounds"])
    assert info.status == 0 and info.converged
    assert info.d0_layer == g["d0_layer"]
    assert info.sigma == g["sigma"]
    want = [float(Fraction(s)) for s in g["iderr"]]
    np.testing.assert_allclose(info.iderr, want, rtol=tol)
    assert info.iderr[-1] > 0.0          # the second clause of Alg. 2 fired
    assert info.froerr0 == pytest.approx(float(Fraction(g["froerr0_sq"])) ** 0.5, rel=tol)
    for layer, v in g["froerr1"].items():
        assert info.froerr1_hist[0][int(layer) - 1] == pytest.approx(v, rel=tol)
    assert info.d1_layer == [g["d1_layer"]]
    assert info.layers == g["d1_layer"]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_dyadic_fixture_complement_form(ctx, fixture, precision):
    """3 of 5 levels occupied: with hole_form = 1 the recursion runs on I - P
    (S_0 = I - (eps_N I - H) / (eps_N - eps_1), again exact dyadic values).
    N_S, N_X trade places in the branch rule, so every sigma is negated,
    while IdErr, FroErr^(0) and FroErr^(1) -- and so both stopping layers --
    are the same numbers."""
    g = fixture
    info = solve_fixture(ctx, g, precision, g["c_pt"], g["c_d0"], hole_form=1)
    tol = VAL_TOL[precision]
    assert info.hole and info.status == 0 and info.converged
    assert info.sigma == [-s for s in g["sigma"]]
    np.testing.assert_allclose(info.iderr, [float(Fraction(s)) for s in g["iderr"]], rtol=tol)
    assert info.froerr0 == pytest.approx(float(Fraction(g["froerr0_sq"])) ** 0.5, rel=tol)
    for layer, v in g["froerr1"].items():
        assert info.froerr1_hist[0][int(layer) - 1] == pytest.approx(v, rel=tol)
    assert info.d0_layer == g["d0_layer"] and info.d1_layer == [g["d1_layer"]]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("variant", range(3))
def test_dyadic_fixture_variants(ctx, fixture, precision, variant):
    g = fixture
    v = g["variants"][variant]
    info = solve_fixture(ctx, g, precision, v["c_pt"], v["c_d0"])
    assert info.d0_layer == v["d0_layer"]
    if "d1_layer" in v:
        assert info.converged == v["converged"]
        if v["converged"]:
            assert info.d1_layer == [v["d1_layer"]]
        else:
            assert info.status == 3 and info.layers == 30   # DMPT_ENOTCONV at max_layers


# --------------------------------------------------------------------------
# The rules as printed (Alg. 1, Alg. 2, Alg. 3 / Eq. (ConvCrit)), applied to
# the quantities the device reports

def rules_decisions(info, n_occ, k, c_pt=9.0, c_d0=4.5):
    """sigma_n, the D^(0) layer, the clause that fired and the D^(1) layers the
    printed rules give for the reported N_S, N_X, FroErr^(0) and FroErr^(1)."""
    sigma, iderr = {}, {}
    d0, clause = 0, 0
    for n in range(1, len(info.n_s) + 1):
        NS, NX = info.n_s[n - 1], info.n_x[n - 1]
        iderr[n] = NS - NX
        d = abs(2.0 * NS - NX - n_occ) - abs(NX - n_occ)
        sigma[n] = 1 if d > 0 else -1
        if iderr[n] <= 0.0:
            d0, clause = n, 1
            break
        if n > 2 and sigma[n - 1] != sigma[n - 2] and iderr[n] > c_d0 * iderr[n - 2] ** 2:
            d0, clause = n, 2
            break
    for n in range(d0 + 1, info.layers + 1):
        sigma[n] = -sigma[n - 1]
    d1 = []
    for j in range(k):
        fe = info.froerr1_hist[j]
        fired = 0
        for n in range(d0 + 2, info.layers + 1):
            if fe[n - 1] >= c_pt * info.froerr0 * fe[n - 3]:
                fired = n
                break
        d1.append(fired)
    return [sigma[n] for n in range(1, info.layers + 1)], d0, clause, d1, iderr


CASES = [
    # (config, n, k, precision)
    (2, 1024, 1, "dual_fp16"),
    (2, 1024, 1, "dual_bf16"),
    (2, 1024, 1, "fp32"),
    (3, 2048, 3, "dual_fp16"),
    (3, 2048, 3, "dual_bf16"),
]


@pytest.mark.parametrize("cfg,n,k,precision", CASES)
def test_device_decisions_follow_the_printed_rules(ctx, cfg, n, k, precision):
    inst = make_workload(cfg, n=n, k=k)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    _, _, info = ctx.sp2_response(H, H1, inst.n_occ, precision=precision)
    torch.cuda.synchronize()
    assert info.converged
    sigma, d0, clause, d1, iderr = rules_decisions(info, inst.n_occ, inst.k)
    # IdErr as reported is N_S - N_X as reported, in FP64 (bit for bit)
    assert info.iderr == [iderr[m] for m in range(1, len(iderr) + 1)]
    assert d0 == info.d0_layer and clause in (1, 2)
    assert sigma == info.sigma
    assert d1 == info.d1_layer
    # the response stops a few layers after D^(0) (Sec. IV A)
    assert all(info.d0_layer + 2 <= x <= info.d0_layer + 8 for x in info.d1_layer)
    print(f"cfg {cfg} n {n} {precision}: D0 at {d0} by clause {clause} "
          f"(IdErr {iderr[d0]:.3e}), D1 at {d1}")
