"""Edge cases of the method on the GPU path, each against the FP64 oracle.

* ragged sizes on both sides of every padding boundary of the pair kernel
  (multiples of 256) and of the SIMT forms;
* extreme occupations n_occ = 1 and n_occ = n - 1 (one occupied / one virtual
  level: the projector and its response have rank 1 / co-rank 1).  The
  rounding of the dual products is relative to the size of their operands
  (||S0||_F ~ ||P||_F = sqrt(n_occ)), not to the size of the response, so
  where ||P1||_F << ||P||_F the response's error is bounded by
  max(TOL ||P1||_F, TOL / 20 ||P||_F) (the second term is the half-filled
  case's error scale, ||dP1||_F / ||P||_F ~ 1e-5 at n = 300, with margin);
* a large-norm Hamiltonian (eigenvalues in [-400, 400]): Gershgorin bounds
  in the thousands, so the scaled S1 is tiny and the FP16 exponent scaling
  must keep its 16-bit copies normal;
* a narrow gap (0.04 around mu), which needs more layers.
"""

import numpy as np
import pytest

import oracle
from paper_2203_09621_gb300.workloads import make_instance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2203_09621_gb300 import dmpt  # noqa: E402

DEV = torch.device("cuda:0")
TOL = {"dual_fp16": 1e-3, "dual_bf16": 5e-3}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    return dmpt.context(0)


def solve_and_check(ctx, inst, precision, tol, p_floor=False, **kw):
    P, P1, info = ctx.sp2_response(torch.from_numpy(inst.H).to(DEV),
                                   torch.from_numpy(inst.H1).to(DEV), inst.n_occ,
                                   precision=precision, **kw)
    torch.cuda.synchronize()
    assert info.converged, (inst.name, precision, info.status, info.layers)
    Pr, P1r = oracle.response_from_eigs(inst.eps, inst.Q, inst.H1[0], inst.n_occ)
    assert rel(P.cpu().numpy(), Pr) < tol, (inst.name, rel(P.cpu().numpy(), Pr))
    err = np.linalg.norm(P1[0].cpu().numpy() - P1r)
    bound = tol * np.linalg.norm(P1r)
    if p_floor:
        bound = max(bound, tol / 20 * np.linalg.norm(Pr))
    assert err < bound, (inst.name, err / np.linalg.norm(P1r), err / np.linalg.norm(Pr))
    return info


@pytest.mark.parametrize("n", [31, 255, 257, 511, 513, 767, 769])
def test_ragged_sizes_dual(ctx, n):
    inst = make_instance(f"rag{n}", n, n // 2, (-2.0, -0.1), (0.1, 2.0), seed=7000 + n)
    solve_and_check(ctx, inst, "dual_fp16", TOL["dual_fp16"])


@pytest.mark.parametrize("n", [63, 129, 257])
def test_ragged_sizes_fp32(ctx, n):
    inst = make_instance(f"rag32_{n}", n, n // 2, (-2.0, -0.1), (0.1, 2.0), seed=7100 + n)
    # FP32 masters: tolerance 10 u (eps_N - eps_1) / gap (as in the FP32 parity tests)
    lo, hi = oracle.gershgorin_bounds(inst.H)
    tol = 10 * 2.0 ** -24 * (hi - lo) / 0.2
    solve_and_check(ctx, inst, "fp32", max(tol, 1e-5))


@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
@pytest.mark.parametrize("which", ["one_occupied", "one_virtual"])
def test_extreme_occupations(ctx, precision, which):
    """n_occ = 1 and n - 1 at the plain tolerance on P and P1.  With n - 1
    levels occupied the default complement form runs the recursion on I - P
    (one level), so the products' rounding scales with ||I - P||_F = 1."""
    n = 300
    n_occ = 1 if which == "one_occupied" else n - 1
    inst = make_instance(f"occ_{which}", n, n_occ, (-2.0, -0.1), (0.1, 2.0), seed=7200)
    info = solve_and_check(ctx, inst, precision, TOL[precision])
    assert info.hole == (which == "one_virtual")


@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
def test_extreme_occupation_particle_form(ctx, precision):
    """The recursion on P as printed (hole_form = 0) with n - 1 levels
    occupied: the rounding of the products is relative to ||P||_F =
    sqrt(n - 1), not to ||P1||_F, so P1 is bounded by the operands' scale
    (TOL / 20 ||P||_F) rather than by TOL ||P1||_F."""
    n = 300
    inst = make_instance("occ_one_virtual_particle", n, n - 1, (-2.0, -0.1), (0.1, 2.0),
                         seed=7200)
    info = solve_and_check(ctx, inst, precision, TOL[precision], p_floor=True, hole_form=0)
    assert not info.hole


@pytest.mark.parametrize("precision", ["fp64", "fp32", "dual_fp16", "dual_bf16"])
@pytest.mark.parametrize("n,n_occ", [(300, 240), (517, 400)])
def test_complement_form_matches_oracle(ctx, precision, n, n_occ):
    """More occupied than empty levels: the complement form against the
    oracle.  In FP64 every branch before the converging layers is the
    oracle's negated; the layer where IdErr first reaches rounding level may
    differ by one (the two forms round different numbers)."""
    inst = make_instance(f"hole{n}", n, n_occ, (-2.0, -0.1), (0.1, 2.0), seed=7500 + n)
    if precision == "fp32":
        lo, hi = oracle.gershgorin_bounds(inst.H)
        tol = max(10 * 2.0 ** -24 * (hi - lo) / 0.2, 1e-5)
    else:
        tol = {"fp64": 1e-10}.get(precision, TOL.get(precision))
    info = solve_and_check(ctx, inst, precision, tol)
    assert info.hole
    if precision == "fp64":
        r = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ)
        assert abs(info.d0_layer - r.d0_layer) <= 1
        nc = min(info.d0_layer, r.d0_layer)
        assert info.sigma[: nc - 1] == [-x for x in r.sigma[: nc - 1]]
        assert all(info.d0_layer + 2 <= d <= info.d0_layer + 8 for d in info.d1_layer)


@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
def test_large_norm_hamiltonian(ctx, precision):
    inst = make_instance("big_norm", 400, 200, (-400.0, -20.0), (20.0, 400.0), seed=7300,
                         scale=1.0)
    solve_and_check(ctx, inst, precision, TOL[precision])


def test_narrow_gap(ctx):
    inst = make_instance("narrow", 300, 150, (-2.0, -0.02), (0.02, 2.0), seed=7400)
    info = solve_and_check(ctx, inst, "dual_fp16", TOL["dual_fp16"])
    wide = make_instance("wide", 300, 150, (-2.0, -0.1), (0.1, 2.0), seed=7400)
    info_w = solve_and_check(ctx, wide, "dual_fp16", TOL["dual_fp16"])
    assert info.layers > info_w.layers   # a narrower gap needs more layers
