"""GPU parity of the batched solve (dmpt_sp2_response_batch).

Every instance of a batch runs the same kernels in the same order as a
single dmpt_sp2_response call, so its outputs must equal the single call's
bit for bit; they must also match the oracle within the dual tolerance.
"""

import numpy as np
import pytest

import oracle
from paper_2203_09621_gb300.workloads import make_instance, uneven_batch

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2203_09621_gb300 import dmpt  # noqa: E402

DEV = torch.device("cuda:0")


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    return dmpt.context(0)


@pytest.mark.parametrize("precision", ["dual_fp16", "fp32"])
def test_small_uneven_batch(ctx, precision):
    sizes = [64, 100, 130, 256, 300, 517, 700, 1000]
    insts = [make_instance(f"b{i}", n, n // 2, (-2.0, -0.05 - 0.02 * i), (0.05 + 0.02 * i, 2.0),
                           seed=9000 + i) for i, n in enumerate(sizes)]
    Hs = [torch.from_numpy(x.H).to(DEV) for x in insts]
    H1s = [torch.from_numpy(x.H1).to(DEV) for x in insts]
    nocc = [x.n_occ for x in insts]
    nocc[2] = 0                       # a trivial instance inside the batch
    Ps, P1s, infos = ctx.sp2_response_batch(Hs, H1s, nocc, precision=precision)
    torch.cuda.synchronize()
    for i, x in enumerate(insts):
        P_single, P1_single, info_s = ctx.sp2_response(Hs[i], H1s[i], nocc[i], precision=precision)
        torch.cuda.synchronize()
        assert torch.equal(Ps[i], P_single) and torch.equal(P1s[i], P1_single), i
        assert infos[i].converged and infos[i].layers == info_s.layers
        if nocc[i] == 0:
            assert not P1s[i].any()
            continue
        Pr, P1r = oracle.response_sos(x.H, x.H1[0], x.n_occ)
        tol = 1e-3 if precision == "dual_fp16" else 5e-4
        assert rel(P1s[i][0].cpu().numpy(), P1r) < tol, (i, rel(P1s[i][0].cpu().numpy(), P1r))


def test_uneven_batch_64_instances(ctx):
    """The 64-instance uneven batch (n log-uniform in [256, 2048]) in one call."""
    insts = uneven_batch(backend="torch", device="cuda")
    Hs = [x.H for x in insts]
    H1s = [x.H1 for x in insts]
    Ps, P1s, infos = ctx.sp2_response_batch(Hs, H1s, [x.n_occ for x in insts])
    torch.cuda.synchronize()
    assert all(i.converged for i in infos)
    for i in (0, 17, 63):
        x = insts[i]
        _, P1r = oracle.response_from_eigs(x.eps.cpu().numpy(), x.Q.cpu().numpy(),
                                           x.H1[0].cpu().numpy(), x.n_occ)
        assert rel(P1s[i][0].cpu().numpy(), P1r) < 1e-3
        _, P1_single, _ = ctx.sp2_response(Hs[i], H1s[i], x.n_occ)
        assert torch.equal(P1s[i], P1_single)


def test_grouped_bf16_matches_single_calls(ctx):
    """The grouped batch kernel with BF16 operands: bit-exact against single
    calls and within the BF16 tolerance of the oracle."""
    sizes = [256, 300, 777, 1024, 513]
    insts = [make_instance(f"g{i}", n, n // 2, (-2.0, -0.1), (0.1, 2.0), seed=9300 + i, k=2)
             for i, n in enumerate(sizes)]
    Hs = [torch.from_numpy(x.H).to(DEV) for x in insts]
    H1s = [torch.from_numpy(x.H1).to(DEV) for x in insts]
    Ps, P1s, infos = ctx.sp2_response_batch(Hs, H1s, [x.n_occ for x in insts], precision="dual_bf16")
    torch.cuda.synchronize()
    for i, x in enumerate(insts):
        P, P1, info = ctx.sp2_response(Hs[i], H1s[i], x.n_occ, precision="dual_bf16")
        torch.cuda.synchronize()
        assert torch.equal(Ps[i], P) and torch.equal(P1s[i], P1), i
        assert infos[i].converged and infos[i].layers == info.layers
        for j in range(2):
            _, P1r = oracle.response_sos(x.H, x.H1[j], x.n_occ)
            assert rel(P1s[i][j].cpu().numpy(), P1r) < 5e-3


# --------------------------------------------------------------------------
# The grouped kernel on 256 x 128 tiles (group_tile_n = 128): instances padded
# to a multiple of 128, four 128-column accumulators.  Its tiles differ from
# the single-instance kernels', so it is checked against the oracle (and
# against the 256 x 256 batch to rounding), not bit for bit.

@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
def test_grouped_256x128_tiles(ctx, precision):
    # sizes on both sides of every multiple of 128, k = 2, one trivial and one
    # complement-form instance
    sizes = [64, 127, 128, 129, 255, 300, 383, 385, 640, 700, 1000]
    insts = [make_instance(f"h{i}", n, n // 2 if i != 6 else (3 * n) // 4, (-2.0, -0.1),
                           (0.1, 2.0), seed=9500 + i, k=2) for i, n in enumerate(sizes)]
    Hs = [torch.from_numpy(x.H).to(DEV) for x in insts]
    H1s = [torch.from_numpy(x.H1).to(DEV) for x in insts]
    nocc = [x.n_occ for x in insts]
    nocc[4] = x_full = sizes[4]      # a trivial instance (P = I)
    P128, P1_128, inf128 = ctx.sp2_response_batch(Hs, H1s, nocc, precision=precision,
                                                   group_tile_n=128)
    P256, P1_256, _ = ctx.sp2_response_batch(Hs, H1s, nocc, precision=precision)
    torch.cuda.synchronize()
    tol = 1e-3 if precision == "dual_fp16" else 5e-3
    for i, x in enumerate(insts):
        assert inf128[i].converged, i
        if nocc[i] == x_full and i == 4:
            assert torch.equal(P128[i], torch.eye(x.n, dtype=torch.float64, device=DEV))
            continue
        Pr = oracle.density_matrix(x.H, nocc[i])
        assert rel(P128[i].cpu().numpy(), Pr) < tol, (i, rel(P128[i].cpu().numpy(), Pr))
        for j in range(2):
            _, P1r = oracle.response_from_eigs(x.eps, x.Q, x.H1[j], nocc[i])
            assert rel(P1_128[i][j].cpu().numpy(), P1r) < tol, (i, j)
            # the same method on the other tile shape: equal to rounding
            assert rel(P1_128[i][j].cpu().numpy(), P1_256[i][j].cpu().numpy()) < tol
        assert torch.equal(P1_128[i], P1_128[i].transpose(1, 2))
    # deterministic: a second call gives the same bits
    P128b, P1_128b, _ = ctx.sp2_response_batch(Hs, H1s, nocc, precision=precision,
                                                group_tile_n=128)
    torch.cuda.synchronize()
    for i in range(len(insts)):
        assert torch.equal(P1_128[i], P1_128b[i]) and torch.equal(P128[i], P128b[i])


def test_grouped_256x128_uneven_batch_64(ctx):
    insts = uneven_batch(backend="torch", device="cuda")
    Hs = [x.H for x in insts]
    H1s = [x.H1 for x in insts]
    Ps, P1s, infos = ctx.sp2_response_batch(Hs, H1s, [x.n_occ for x in insts], group_tile_n=128)
    torch.cuda.synchronize()
    assert all(i.converged for i in infos)
    for i in (0, 17, 40, 63):
        x = insts[i]
        _, P1r = oracle.response_from_eigs(x.eps.cpu().numpy(), x.Q.cpu().numpy(),
                                           x.H1[0].cpu().numpy(), x.n_occ)
        assert rel(P1s[i][0].cpu().numpy(), P1r) < 1e-3, i
