"""Failure detection on the GPU without a GPU fault.

Every spin wait in the layer-product kernels is bounded in time.  The test
hook `inject_stall` makes the MMA issuer wait on a barrier that nothing
arrives on; the waits of every role then run out (50 ms here), the kernel
raises its timeout flag, drains its own copies and MMAs, frees tensor
memory and returns, and the call reports DMPT_ETIMEOUT.  The context must
stay usable: the next normal call on the same handle converges to the
oracle's result.
"""

import numpy as np
import pytest

import oracle
from paper_2203_09621_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2203_09621_gb300 import dmpt  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.mark.parametrize("cta_pair", [1, 0])
def test_stalled_wait_times_out_and_context_survives(cta_pair):
    ctx = dmpt.context(0)
    inst = make_workload(2, n=512)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    _, _, info = ctx.sp2_response(H, H1, inst.n_occ, cta_pair=cta_pair, inject_stall=1,
                                  timeout_s=0.05, raise_on_error=False)
    torch.cuda.synchronize()
    assert info.status == 5          # DMPT_ETIMEOUT
    assert not info.converged
    # the same handle, stream and workspace work afterwards
    P, P1, info = ctx.sp2_response(H, H1, inst.n_occ, cta_pair=cta_pair)
    torch.cuda.synchronize()
    assert info.converged
    _, P1r = oracle.response_sos(inst.H, inst.H1[0], inst.n_occ)
    assert np.linalg.norm(P1[0].cpu().numpy() - P1r) / np.linalg.norm(P1r) < 1e-3
