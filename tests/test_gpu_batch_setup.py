"""The batched initial layer and outputs of dmpt_sp2_response_batch.

The batch path forms the control blocks, the Gershgorin bounds, the initial
layer (Alg. 1; Sec. III A, S_0 and S_1), its decide step, the 16-bit split and
the outputs of all instances with one launch per step.  Each instance must
keep the values of its own single-instance call, bit for bit, and match the
oracle:
* P only (k = 0), dual FP16 and FP64, with tiny and trivial instances and
  sizes on both sides of the initial layer's 64-element tiles;
* the FP64 form with a response;
* row strides larger than n (the C ABI's ld), through the C entry point,
  with the padding columns of the outputs left as they were.
"""

import ctypes

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
TOL = {"dual_fp16": 1e-3, "fp64": 1e-9}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    return dmpt.context(0)


def instances(sizes, seed, k=1):
    out = []
    for i, n in enumerate(sizes):
        out.append(make_instance(f"s{i}-n{n}", n, n // 2, (-2.0, -0.1), (0.1, 2.0), k=k,
                                 seed=seed + 17 * i))
    return out


@pytest.mark.parametrize("precision", ["dual_fp16", "fp64"])
def test_batch_density_only(ctx, precision):
    sizes = [1, 2, 3, 63, 64, 65, 200, 513]
    insts = instances(sizes, 7100)
    Hs = [torch.from_numpy(x.H).to(DEV) for x in insts]
    occ = [x.n_occ for x in insts]          # n = 1: n_occ = 0, a trivial instance
    Pb, P1b, infos = ctx.sp2_response_batch(Hs, None, occ, precision=precision)
    torch.cuda.synchronize()
    assert P1b is None
    for i, x in enumerate(insts):
        P, _, info = ctx.sp2_response(Hs[i], None, occ[i], precision=precision)
        torch.cuda.synchronize()
        assert torch.equal(Pb[i], P), (i, sizes[i])
        assert infos[i].converged and infos[i].layers == info.layers
        want = oracle.density_matrix(x.H, x.n_occ)
        if x.n_occ == 0:
            assert not Pb[i].any()
        else:
            assert rel(Pb[i].cpu().numpy(), want) < TOL[precision], (i, sizes[i])


def test_batch_fp64_with_response(ctx):
    insts = instances([100, 300, 517], 7200)
    Hs = [torch.from_numpy(x.H).to(DEV) for x in insts]
    H1s = [torch.from_numpy(x.H1).to(DEV) for x in insts]
    occ = [x.n_occ for x in insts]
    Pb, P1b, infos = ctx.sp2_response_batch(Hs, H1s, occ, precision="fp64")
    torch.cuda.synchronize()
    for i, x in enumerate(insts):
        P, P1, info = ctx.sp2_response(Hs[i], H1s[i], occ[i], precision="fp64")
        torch.cuda.synchronize()
        assert torch.equal(Pb[i], P) and torch.equal(P1b[i], P1), i
        assert infos[i].sigma == info.sigma and infos[i].d1_layer == info.d1_layer
        _, want = oracle.response_from_eigs(x.eps, x.Q, x.H1[0], x.n_occ)
        assert rel(P1b[i][0].cpu().numpy(), want) < TOL["fp64"]


@pytest.mark.parametrize("precision", ["dual_fp16", "fp64"])
def test_batch_row_stride(ctx, precision):
    """ld = n + 7 for inputs and outputs, through the C entry point."""
    sizes = [150, 300, 257]
    k = 2
    insts = instances(sizes, 7300, k=k)
    lds = [n + 7 for n in sizes]
    Hp, H1p, Pp, P1p = [], [], [], []
    for x, n, ld in zip(insts, sizes, lds):
        h = torch.zeros(n, ld, dtype=torch.float64, device=DEV)
        h[:, :n] = torch.from_numpy(x.H)
        h1 = torch.zeros(k, n, ld, dtype=torch.float64, device=DEV)
        h1[:, :, :n] = torch.from_numpy(x.H1)
        Hp.append(h)
        H1p.append(h1)
        Pp.append(torch.full((n, ld), 7.0, dtype=torch.float64, device=DEV))
        P1p.append(torch.full((k, n, ld), 7.0, dtype=torch.float64, device=DEV))
    count = len(sizes)
    I64 = ctypes.c_int64 * count
    VP = ctypes.c_void_p * count
    opts = dmpt.options(precision=precision)
    n_arr = I64(*sizes)
    nbytes = ctx.lib.dmpt_workspace_size_batch(count, n_arr, k, ctypes.byref(opts))
    ws_ptr, ws_len = ctx.workspace(nbytes)
    infos = (dmpt.DmptInfo * count)()
    st = ctx.lib.dmpt_sp2_response_batch(
        ctx.h, count, VP(*[h.data_ptr() for h in Hp]), VP(*[h.data_ptr() for h in H1p]), k,
        n_arr, I64(*lds), I64(*[x.n_occ for x in insts]), ctypes.byref(opts),
        VP(*[p.data_ptr() for p in Pp]), VP(*[p.data_ptr() for p in P1p]), infos,
        ctypes.c_void_p(ws_ptr), ws_len,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == 0
    for i, (x, n, ld) in enumerate(zip(insts, sizes, lds)):
        assert infos[i].converged
        P, P1, _ = ctx.sp2_response(torch.from_numpy(x.H).to(DEV),
                                    torch.from_numpy(x.H1).to(DEV), x.n_occ,
                                    precision=precision)
        torch.cuda.synchronize()
        assert torch.equal(Pp[i][:, :n], P) and torch.equal(P1p[i][:, :, :n], P1), i
        assert bool((Pp[i][:, n:] == 7.0).all()) and bool((P1p[i][:, :, n:] == 7.0).all())
        for j in range(k):
            _, want = oracle.response_from_eigs(x.eps, x.Q, x.H1[j], x.n_occ)
            assert rel(P1[j].cpu().numpy(), want) < TOL[precision], (i, j)
