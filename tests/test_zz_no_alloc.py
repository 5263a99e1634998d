"""dmpt_sp2_response_static: the solve for callers that cannot allocate.

Some callers cannot call cudaMalloc or pass a workspace -- a host framework
that owns every device allocation, code that must keep its memory fixed
after start-up, or a plug-in that only receives input and output pointers.
For them the library offers an entry point whose scratch space is one fixed
device array inside the library.  This file checks, through the C ABI, that
it gives the same results as the workspace entry point, bit for bit, on two
calls in a row (the array keeps the previous call's contents, which must not
leak into the next result), that both match the FP64 oracle, and that it
refuses what it cannot do without allocating (sizes beyond its limit, the
per-launch timing and autotuning options, the S0 tape) with a status in
dmpt_info and a message.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""

import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2203_09621_gb300 import dmpt  # noqa: E402
from paper_2203_09621_gb300.workloads import make_workload  # noqa: E402

DEV = torch.device("cuda:0")
# against the FP64 oracle (relative Frobenius), as in the parity tests
TOL = {"dual_fp16": 1e-3, "fp64": 1e-10}


def static_call(ctx, H, H1, n_occ, precision, **kw):
    n = H.shape[0]
    k = H1.shape[0]
    P = torch.empty(n, n, dtype=torch.float64, device=DEV)
    P1 = torch.empty(k, n, n, dtype=torch.float64, device=DEV)
    opts = dmpt.options(precision=precision, **kw)
    info = dmpt.DmptInfo()
    info.status = -99
    info.layers = -99
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
        assert st == 0 and info.status == 0 and info.converged
        Pw, P1w, iw = ctx.sp2_response(H, H1, inst.n_occ, precision=precision)
        torch.cuda.synchronize()
        # the same kernels on the same inputs with the same options: bit for bit
        assert np.array_equal(P, Pw.cpu().numpy())
        assert np.array_equal(P1[0], P1w[0].cpu().numpy())
        assert info.layers == iw.layers and info.d0_layer == iw.d0_layer
        # and the oracle at the parity tolerance
        P_ref, P1_ref = oracle.response_sos(inst.H, inst.H1[0], inst.n_occ)
        assert rel(P, P_ref) <= TOL[precision]
        assert rel(P1[0], P1_ref) <= TOL[precision]


def test_static_refusals_set_status_and_message():
    ctx = dmpt.context(0)
    n = 64
    H = torch.eye(n, dtype=torch.float64, device=DEV)
    H1 = torch.zeros(1, n, n, dtype=torch.float64, device=DEV)
    cases = [
        (dict(), torch.eye(513, dtype=torch.float64, device=DEV),
         torch.zeros(1, 513, 513, dtype=torch.float64, device=DEV), 1, "limit"),
        (dict(), H, torch.zeros(2, n, n, dtype=torch.float64, device=DEV), 1, "limit"),
        (dict(timing=True), H, H1, 7, "timing"),
        (dict(autotune=1), H, H1, 7, "autotune"),
        (dict(ckpt_every=1), H, H1, 7, "tape"),
    ]
    for kw, Hc, H1c, want, word in cases:
        st, _, _, info = static_call(ctx, Hc, H1c, Hc.shape[0] // 2, "dual_fp16", **kw)
        assert st == want, (kw, st)
        assert info.status == want and info.layers == 0   # cleared on entry, then set
        assert word in ctx.lib.dmpt_last_error(ctx.h).decode(), kw
    # a refused call leaves the array usable: the next call still matches
    inst = make_workload(1, n=128)
    Ht = torch.from_numpy(inst.H).to(DEV)
    H1t = torch.from_numpy(inst.H1).to(DEV)
    st, P, P1, info = static_call(ctx, Ht, H1t, inst.n_occ, "dual_fp16")
    assert st == 0 and info.converged
    _, P1w, _ = ctx.sp2_response(Ht, H1t, inst.n_occ, precision="dual_fp16")
    torch.cuda.synchronize()
    assert np.array_equal(P1[0], P1w[0].cpu().numpy())
