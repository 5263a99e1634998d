"""dmpt_sp2_response_static: the solve for callers that cannot allocate.

Some callers cannot call cudaMalloc or pass a workspace -- a host framework
that owns every device allocation, code that must keep its memory fixed
after start-up, or a plug-in that only receives input and output pointers.
For them the library offers an entry point whose scratch space is one fixed
device array inside the library.  This file checks, through the C ABI, that
it gives the same results as the workspace entry point on two calls in a
row (the array keeps the previous call's contents, which must not leak into
the next result), and that it rejects sizes beyond its limit.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2203_09621_gb300 import dmpt  # noqa: E402
from paper_2203_09621_gb300.workloads import make_workload  # noqa: E402

DEV = torch.device("cuda:0")
TOL = {"dual_fp16": 1e-3, "fp64": 1e-10}


def static_call(ctx, H, H1, n_occ, precision):
    n = H.shape[0]
    k = H1.shape[0]
    P = torch.empty(n, n, dtype=torch.float64, device=DEV)
    P1 = torch.empty(k, n, n, dtype=torch.float64, device=DEV)
    opts = dmpt.options(precision=precision)
    info = dmpt.DmptInfo()
    st = ctx.lib.dmpt_sp2_response_static(
        ctx.h, H.data_ptr(), H1.data_ptr(), k, n, n, n_occ, ctypes.byref(opts), P.data_ptr(),
        P1.data_ptr(), ctypes.byref(info), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, P.cpu().numpy(), P1.cpu().numpy(), info


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("precision", ["dual_fp16", "fp64"])
def test_static_matches_workspace_entry_point_twice(precision):
    ctx = dmpt.context(0)
    # two different problems in a row: the second must not see the first's leftovers
    for cfg, n in ((2, 300), (1, 128)):
        inst = make_workload(cfg, n=n)
        H = torch.from_numpy(inst.H).to(DEV)
        H1 = torch.from_numpy(inst.H1).to(DEV)
        st, P, P1, info = static_call(ctx, H, H1, inst.n_occ, precision)
        assert st == 0 and info.converged
        Pw, P1w, iw = ctx.sp2_response(H, H1, inst.n_occ, precision=precision)
        torch.cuda.synchronize()
        assert rel(P, Pw.cpu().numpy()) <= TOL[precision]
        assert rel(P1[0], P1w[0].cpu().numpy()) <= TOL[precision]
        assert info.layers == iw.layers


def test_static_rejects_sizes_beyond_its_limit():
    ctx = dmpt.context(0)
    n = 513
    H = torch.eye(n, dtype=torch.float64, device=DEV)
    H1 = torch.zeros(1, n, n, dtype=torch.float64, device=DEV)
    st, _, _, _ = static_call(ctx, H, H1, n // 2, "dual_fp16")
    assert st == 1  # DMPT_EINVAL
    H1b = torch.zeros(2, 64, 64, dtype=torch.float64, device=DEV)
    st, _, _, _ = static_call(ctx, torch.eye(64, dtype=torch.float64, device=DEV), H1b, 32,
                              "dual_fp16")
    assert st == 1
