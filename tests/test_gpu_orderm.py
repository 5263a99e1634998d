"""GPU parity of the responses of any order (dmpt_sp2_response_m).

Dual forms on the tensor cores; the FP64 and FP32 forms run the same passes
on the CUDA cores.

P_o = (1/o!) d^o P / dlambda^o from S_o,n = sigma (S0 S_o + S_o S0 +
sum_{a=1}^{o-1} S_a S_{o-a}) + (1 - sigma) S_o on the tensor cores (o + 1 K
passes per term), against the FP64 oracle's SP2 recursion of the same order
(itself pinned to the block upper-triangular matrix of Sec. III B, sympy
derivatives and finite differences).  Tolerances are those of the second
order: 1e-3 (dual FP16) and 5e-3 (dual BF16) relative Frobenius error per
term.  Lower orders never see higher ones, so P and every term up to m - 1
must equal those of the order-(m - 1) call bit for bit.
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
TOL = {"dual_fp16": 1e-3, "dual_bf16": 5e-3}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    return dmpt.context(0)


@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
@pytest.mark.parametrize("cfg,n,k,order", [(1, None, 1, 3), (2, 300, 1, 4), (3, 512, 2, 3),
                                           (1, 200, 1, 8)])
def test_order_m_matches_oracle(ctx, precision, cfg, n, k, order):
    inst = make_workload(cfg, n=n, k=k)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    P, terms, info = ctx.sp2_response_m(H, H1, inst.n_occ, order, precision=precision)
    torch.cuda.synchronize()
    assert info.converged, info
    assert len(terms) == order and all(t.shape == (k, inst.n, inst.n) for t in terms)
    ref = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ, order=order)
    assert ref.converged
    errs = [[rel(terms[o][j].cpu().numpy(), ref.Pk[o][j]) for j in range(k)] for o in range(order)]
    assert max(max(e) for e in errs) < TOL[precision], errs
    # symmetric terms (both halves written with the same value)
    for t in terms:
        assert torch.equal(t, t.transpose(1, 2))


@pytest.mark.parametrize("cfg,n,k,order", [(2, 300, 1, 3), (3, 256, 2, 4)])
def test_order_m_fp64_form(ctx, cfg, n, k, order):
    """The FP64 form runs the same recursion as the FP64 oracle: the same
    first-order stop layers, every term to 1e-9.  A higher order's stop test
    compares rounding-level residuals, so its layer may differ by a sigma-flip
    pair without changing the converged term."""
    inst = make_workload(cfg, n=n, k=k)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    P, terms, info = ctx.sp2_response_m(H, H1, inst.n_occ, order, precision="fp64")
    torch.cuda.synchronize()
    ref = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ, order=order)
    assert info.converged and ref.converged
    assert abs(info.layers - ref.layers) <= 2
    assert info.d1_layer[:k] == ref.dk_layer[0]
    for o in range(order):
        for j in range(k):
            assert rel(terms[o][j].cpu().numpy(), ref.Pk[o][j]) < 1e-9, (o, j)


def test_order_m_fp32_form(ctx):
    """The FP32 form carries about the precision of the dual forms, and is
    held to the dual-FP16 tolerance per term."""
    inst = make_workload(2, n=300, k=1)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    P, terms, info = ctx.sp2_response_m(H, H1, inst.n_occ, 3, precision="fp32")
    torch.cuda.synchronize()
    assert info.converged
    ref = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ, order=3)
    errs = [rel(terms[o][0].cpu().numpy(), ref.Pk[o][0]) for o in range(3)]
    assert max(errs) < TOL["dual_fp16"], errs
    # first-order terms bit-identical to the first-order call of the same form
    P1c, P1r, _ = ctx.sp2_response(H, H1, inst.n_occ, precision="fp32")
    torch.cuda.synchronize()
    assert torch.equal(P, P1c) and torch.equal(terms[0], P1r)


@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
def test_order_m_one_cta_tiles(ctx, precision):
    """The 1-CTA kernel (128 x 256 tiles) runs the same order-o jobs."""
    inst = make_workload(2, n=300, k=2)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    P, terms, info = ctx.sp2_response_m(H, H1, inst.n_occ, 3, precision=precision, cta_pair=0)
    torch.cuda.synchronize()
    assert info.converged
    ref = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ, order=3)
    errs = [[rel(terms[o][j].cpu().numpy(), ref.Pk[o][j]) for j in range(2)] for o in range(3)]
    assert max(max(e) for e in errs) < TOL[precision], errs


@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
def test_lower_orders_bitwise(ctx, precision):
    inst = make_workload(3, n=384, k=2)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    P1c, P1r, info1 = ctx.sp2_response(H, H1, inst.n_occ, precision=precision)
    P2c, P1b, P2b, info2 = ctx.sp2_response2(H, H1, inst.n_occ, precision=precision)
    P4c, terms, info4 = ctx.sp2_response_m(H, H1, inst.n_occ, 4, precision=precision)
    Pm1, terms1, _ = ctx.sp2_response_m(H, H1, inst.n_occ, 1, precision=precision)
    torch.cuda.synchronize()
    assert info4.converged
    assert torch.equal(P4c, P1c) and torch.equal(terms[0], P1r)
    assert torch.equal(P2c, P1c) and torch.equal(terms[1], P2b)
    assert torch.equal(Pm1, P1c) and torch.equal(terms1[0], P1r)
    assert info4.d1_layer[:4] == info2.d1_layer[:4]


def test_trivial_occupations(ctx):
    inst = make_workload(1, n=96)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    for n_occ, want in ((0, torch.zeros(96, 96)), (96, torch.eye(96))):
        P, terms, info = ctx.sp2_response_m(H, H1, n_occ, 3)
        torch.cuda.synchronize()
        assert info.converged and info.layers == 0
        assert torch.equal(P.cpu(), want.double())
        assert all(not t.any() for t in terms)


def test_rejections(ctx):
    inst = make_workload(1, n=64)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    with pytest.raises(dmpt.DmptError) as e:          # no tape for orders >= 2
        ctx.sp2_response_m(H, H1, inst.n_occ, 3, ckpt_every=1)
    assert e.value.status == 7
    H1x3 = torch.zeros(3, 64, 64, dtype=torch.float64, device=DEV)
    with pytest.raises(dmpt.DmptError):               # order * k = 9 > DMPT_MAX_K
        ctx.sp2_response_m(H, H1x3, inst.n_occ, 3)
    with pytest.raises(dmpt.DmptError):               # order 9 > DMPT_MAX_ORDER
        ctx.sp2_response_m(H, H1, inst.n_occ, 9)
