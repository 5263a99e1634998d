"""GPU parity of the second-order response (dmpt_sp2_response2).

D2 = (1/2) d^2 P / dlambda^2 from S2_n = sigma (S0 S2 + S1 S1 + S2 S0) +
(1 - sigma) S2 on the tensor cores, against the oracle's second-order
Daleckii-Krein formula, within the dual tolerances of the first order
(1e-3 FP16, 5e-3 BF16; measured 1e-5 .. 9e-5 and 1e-4 .. 4e-4 at n <= 1024).  P and P1 of
the same call must equal the first-order call's bit for bit (S2 never
feeds back into S0 or S1).
"""

import numpy as np
import pytest

from oracle.sos import response2_sos
from paper_2203_09621_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2203_09621_gb300 import dmpt  # noqa: E402

DEV = torch.device("cuda:0")
TOL2 = {"dual_fp16": 1e-3, "dual_bf16": 5e-3}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    return dmpt.context(0)


def test_two_level_order2(ctx, golden):
    g = golden("two_level_order2.json")
    H = torch.tensor(g["H"], dtype=torch.float64, device=DEV)
    H1 = torch.tensor(g["H1"], dtype=torch.float64, device=DEV)
    P, P1, P2, info = ctx.sp2_response2(H, H1, g["n_occ"])
    torch.cuda.synchronize()
    np.testing.assert_allclose(P2[0].cpu().numpy(), g["P2"], atol=1e-6)


@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
@pytest.mark.parametrize("cfg,n,k", [(1, None, 1), (2, 300, 1), (3, 512, 2)])
def test_order2_matches_oracle(ctx, precision, cfg, n, k):
    inst = make_workload(cfg, n=n, k=k)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    P, P1, P2, info = ctx.sp2_response2(H, H1, inst.n_occ, precision=precision)
    torch.cuda.synchronize()
    assert info.converged
    for j in range(k):
        want = response2_sos(inst.H, inst.H1[j], inst.n_occ)
        assert rel(P2[j].cpu().numpy(), want) < TOL2[precision], (j, rel(P2[j].cpu().numpy(), want))
    # first-order call on the same inputs: identical P and P1
    Pa, P1a, infoa = ctx.sp2_response(H, H1, inst.n_occ, precision=precision)
    torch.cuda.synchronize()
    assert torch.equal(P, Pa) and torch.equal(P1, P1a)
    assert info.d1_layer[:k] == infoa.d1_layer


def test_order2_rejects_tape_and_large_k(ctx):
    inst = make_workload(1, n=64)
    H = torch.from_numpy(inst.H).to(DEV)
    with pytest.raises(dmpt.DmptError) as e:
        ctx.sp2_response2(H, torch.from_numpy(inst.H1).to(DEV), inst.n_occ, ckpt_every=1)
    assert e.value.status == 7
    H1 = torch.zeros(5, 64, 64, dtype=torch.float64, device=DEV)
    with pytest.raises(dmpt.DmptError):
        ctx.sp2_response2(H, H1, inst.n_occ)
