"""GPU parity of the response replay and the self-consistent response.

* dmpt_response_replay with the forward's own perturbations reproduces the
  forward's P1 bit for bit (same operands, same order, deterministic);
  with new perturbations it matches the oracle's response.
* dmpt_scc_response matches the oracle's self-consistent fixed point
  (oracle/scc.py) within the dual-FP16 tolerance, and at a larger size its
  result satisfies the fixed-point property P1 = R(H1_ext + diag(gamma
  diag(P1))) when R is evaluated by an independent replay.
"""

import numpy as np
import pytest

import oracle
from paper_2203_09621_gb300.workloads import make_workload, scc_gamma, sym_gauss

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


def forward_with_tape(ctx, H, H1, n_occ, precision="dual_fp16"):
    opts = dmpt.options(precision=precision, ckpt_every=1)
    ws = torch.empty(ctx.workspace_size(H.shape[0], H1.shape[0], opts) + 256,
                     dtype=torch.uint8, device=DEV)
    P, P1, info = ctx.sp2_response(H, H1, n_occ, precision=precision, ckpt_every=1,
                                   workspace=ws)
    torch.cuda.synchronize()
    return P, P1, info, ws


@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
def test_replay_reproduces_forward_bitwise(ctx, precision):
    inst = make_workload(3, n=512)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    _, P1f, info, ws = forward_with_tape(ctx, H, H1, inst.n_occ, precision)
    P1f = P1f.clone()
    P1r, rinfo = ctx.response_replay(H1, ws)
    torch.cuda.synchronize()
    assert torch.equal(P1r, P1f)
    assert rinfo.layers == info.layers and rinfo.d1_layer == info.d1_layer


def test_replay_new_perturbations(ctx):
    inst = make_workload(2, n=300)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    _, _, _, ws = forward_with_tape(ctx, H, torch.cat([H1, H1]), inst.n_occ)
    new = np.stack([sym_gauss(300, 500, 0.05), sym_gauss(300, 501, 0.002)])
    P1, rinfo = ctx.response_replay(torch.from_numpy(new).to(DEV), ws)
    torch.cuda.synchronize()
    assert rinfo.converged
    for j in range(2):
        _, want = oracle.response_sos(inst.H, new[j], inst.n_occ)
        assert rel(P1[j].cpu().numpy(), want) < 1e-3


@pytest.mark.parametrize("n,k", [(256, 1), (512, 3)])
def test_scc_matches_oracle_fixed_point(ctx, n, k):
    inst = make_workload(3, n=n, k=k)
    g = scc_gamma(n)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    _, _, _, ws = forward_with_tape(ctx, H, H1, inst.n_occ)
    P1, its, res, sinfo = ctx.scc_response(H1, torch.from_numpy(g).to(DEV), ws, tol=1e-5)
    torch.cuda.synchronize()
    assert res < 1e-5 and its < 100
    for j in range(k):
        want, _, _ = oracle.scc_response(inst.H, inst.H1[j], g, inst.n_occ)
        assert rel(P1[j].cpu().numpy(), want) < 1e-3, (j, rel(P1[j].cpu().numpy(), want))


def test_scc_fixed_point_property_n2048(ctx):
    n = 2048
    inst = make_workload(3, n=n, backend="torch", device="cuda")
    g = scc_gamma(n, backend="torch", device="cuda")
    _, _, _, ws = forward_with_tape(ctx, inst.H, inst.H1, inst.n_occ)
    P1, its, res, _ = ctx.scc_response(inst.H1, g, ws, tol=1e-5)
    P1 = P1.clone()
    torch.cuda.synchronize()
    assert res < 1e-5
    # independent replay at the self-consistent perturbation
    H1_eff = inst.H1 + torch.diag_embed(torch.einsum("rc,kc->kr", g, torch.diagonal(P1, dim1=1, dim2=2)))
    P1b, _ = ctx.response_replay(H1_eff, ws)
    torch.cuda.synchronize()
    for j in range(inst.k):
        assert rel(P1b[j].cpu().numpy(), P1[j].cpu().numpy()) < 1e-4
    # the coupling changes the response well beyond the tolerance (about 1 %
    # for these dipole perturbations, whose diagonal dominates)
    P1_0, _ = ctx.response_replay(inst.H1, ws)
    assert rel(P1_0[0].cpu().numpy(), P1[0].cpu().numpy()) > 5e-3


def test_replay_requires_a_tape(ctx):
    inst = make_workload(1, n=64)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    opts = dmpt.options()
    ws = torch.empty(ctx.workspace_size(64, 1, opts) + 256, dtype=torch.uint8, device=DEV)
    ctx.sp2_response(H, H1, inst.n_occ, workspace=ws)
    with pytest.raises(dmpt.DmptError) as e:
        ctx.response_replay(H1, ws)
    assert e.value.status == 1
