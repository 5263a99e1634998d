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
