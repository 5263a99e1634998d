"""GPU parity of the adjoint (dmpt_sp2_backward) and the autograd wrapper.

L = Tr[G P].  The adjoint of the S0 recursion, run on the tensor cores over
the stored S0 states, must give dL/dH equal to
  * the first-order response to the perturbation G (the Daleckii-Krein
    derivative of a spectral function is self-adjoint), from the oracle;
  * the oracle's own reverse-mode recursion (same branches and bounds);
  * <dL/dH, E> = Tr[G P1(E)] for random directions E, with P1(E) from the
    GPU forward response (one call with k = 8 directions);
  * central finite differences of the oracle's L.
Tolerance: the dual-precision tolerances (1e-3 FP16, 5e-3 BF16).
"""

import numpy as np
import pytest

import oracle
from paper_2203_09621_gb300.workloads import make_workload, make_instance, sym_gauss

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


def forward_with_tape(ctx, H, H1, n_occ, precision, ckpt_every=1):
    opts = dmpt.options(precision=precision, ckpt_every=ckpt_every)
    k = 0 if H1 is None else (1 if H1.dim() == 2 else H1.shape[0])
    ws = torch.empty(ctx.workspace_size(H.shape[0], k, opts) + 256, dtype=torch.uint8,
                     device=DEV)
    P, P1, info = ctx.sp2_response(H, H1, n_occ, precision=precision, ckpt_every=ckpt_every,
                                   workspace=ws)
    torch.cuda.synchronize()
    return P, P1, info, ws


@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
@pytest.mark.parametrize("n", [256, 300])
def test_backward_equals_response_to_G(ctx, precision, n):
    inst = make_workload(2, n=n)
    G = sym_gauss(n, 77)
    H = torch.from_numpy(inst.H).to(DEV)
    P, _, info, ws = forward_with_tape(ctx, H, None, inst.n_occ, precision)
    assert info.converged
    dLdH = ctx.sp2_backward(torch.from_numpy(G).to(DEV), ws).cpu().numpy()
    _, P1G = oracle.response_sos(inst.H, G, inst.n_occ)
    assert rel(dLdH, P1G) < TOL[precision], rel(dLdH, P1G)
    # the oracle's reverse-mode recursion with the same branches and bounds
    sig = info.sigma[: info.d0_layer - 1]
    adj = oracle.sp2_adjoint(inst.H, G, inst.n_occ, sig, (info.eps_min, info.eps_max))
    assert rel(dLdH, adj) < TOL[precision]
    assert np.array_equal(dLdH, dLdH.T)


def test_backward_repeated_calls_and_nonsymmetric_G(ctx):
    inst = make_workload(1)
    H = torch.from_numpy(inst.H).to(DEV)
    _, _, info, ws = forward_with_tape(ctx, H, None, inst.n_occ, "dual_fp16")
    for seed in (1, 2, 3):
        Gn = np.random.default_rng(seed).standard_normal((128, 128))   # not symmetric
        dLdH = ctx.sp2_backward(torch.from_numpy(Gn).to(DEV), ws).cpu().numpy()
        _, P1G = oracle.response_sos(inst.H, 0.5 * (Gn + Gn.T), inst.n_occ)
        assert rel(dLdH, P1G) < 1e-3


def test_directional_derivatives_match_forward_response(ctx):
    """Config-4 style check: 8 random symmetric directions in one k = 8 call."""
    n = 512
    inst = make_workload(4, n=n)
    G = torch.from_numpy(inst.H1[0]).to(DEV)          # loss weight, symmetric Gaussian
    E = torch.stack([torch.from_numpy(sym_gauss(n, 400 + i)) for i in range(8)]).to(DEV)
    H = torch.from_numpy(inst.H).to(DEV)
    _, P1E, info, ws = forward_with_tape(ctx, H, E, inst.n_occ, "dual_fp16")
    assert info.converged
    dLdH = ctx.sp2_backward(G, ws)
    lhs = torch.einsum("ij,kij->k", dLdH, E).cpu().numpy()     # <dL/dH, E_k>
    rhs = torch.einsum("ij,kij->k", G, P1E).cpu().numpy()      # Tr[G P1(E_k)]
    scale = np.abs(rhs).max()
    assert np.abs(lhs - rhs).max() < 2e-3 * scale, (lhs, rhs)
    # central finite differences of the oracle's L = Tr[G P] along E_0
    Gn, E0 = G.cpu().numpy(), E[0].cpu().numpy()
    L = lambda t: float(np.sum(Gn * oracle.density_matrix(inst.H + t * E0, inst.n_occ)))
    h = 1e-4
    fd = (L(h) - L(-h)) / (2 * h)
    assert abs(fd - lhs[0]) < 2e-3 * max(abs(fd), scale)


def test_autograd_function(ctx):
    inst = make_workload(1)
    G = torch.from_numpy(sym_gauss(128, 9)).to(DEV)
    H = torch.from_numpy(inst.H).to(DEV).requires_grad_(True)
    P = dmpt.density(H, inst.n_occ)
    loss = (G * P).sum()
    loss.backward()
    Pr = oracle.density_matrix(inst.H, inst.n_occ)
    assert rel(P.detach().cpu().numpy(), Pr) < 1e-3
    _, P1G = oracle.response_sos(inst.H, G.cpu().numpy(), inst.n_occ)
    assert rel(H.grad.cpu().numpy(), P1G) < 1e-3


def test_p_only_forward(ctx):
    inst = make_workload(2, n=300)
    H = torch.from_numpy(inst.H).to(DEV)
    P, P1, info = ctx.sp2_response(H, None, inst.n_occ, precision="dual_fp16")
    torch.cuda.synchronize()
    assert P1 is None and info.converged
    assert rel(P.cpu().numpy(), oracle.density_matrix(inst.H, inst.n_occ)) < 1e-3


def test_backward_without_tape_is_rejected(ctx):
    inst = make_workload(1, n=64)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    opts = dmpt.options(precision="dual_fp16")
    ws = torch.empty(ctx.workspace_size(64, 1, opts) + 256, dtype=torch.uint8, device=DEV)
    ctx.sp2_response(H, H1, inst.n_occ, workspace=ws)
    with pytest.raises(dmpt.DmptError) as e:
        ctx.sp2_backward(H, ws)
    assert e.value.status == 1
    # the tape needs a dual precision
    with pytest.raises(dmpt.DmptError) as e:
        ctx.sp2_response(H, H1, inst.n_occ, precision="fp32", ckpt_every=1)
    assert e.value.status == 7


def test_adjoint_full_size_n4096(ctx):
    """Config 4 at its full size: n = 4096, dual-FP16 forward and adjoint."""
    inst = make_workload(4, backend="torch", device="cuda")
    G = inst.H1[0]
    P, _, info, ws = forward_with_tape(ctx, inst.H, None, inst.n_occ, "dual_fp16")
    assert info.converged
    dLdH = ctx.sp2_backward(G, ws).cpu().numpy()
    _, P1G = oracle.response_from_eigs(inst.eps.cpu().numpy(), inst.Q.cpu().numpy(),
                                       G.cpu().numpy(), inst.n_occ)
    assert rel(dLdH, P1G) < 1e-3, rel(dLdH, P1G)


# --------------------------------------------------------------------------
# Checkpoints every k S0 states (ckpt_every = k >= 2): the backward recomputes
# each segment from its FP32 checkpoint with the forward's own products, so
# the states, and therefore dL/dH, are bit-identical to the full tape's.

@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
@pytest.mark.parametrize("n,ck", [(256, 2), (300, 3), (300, 8), (520, 5)])
def test_checkpointed_backward_equals_full_tape(ctx, precision, n, ck):
    inst = make_workload(2, n=n)
    G = torch.from_numpy(sym_gauss(n, 78)).to(DEV)
    H = torch.from_numpy(inst.H).to(DEV)
    P1_, _, info1, ws1 = forward_with_tape(ctx, H, None, inst.n_occ, precision, 1)
    Pk, _, infok, wsk = forward_with_tape(ctx, H, None, inst.n_occ, precision, ck)
    assert info1.converged and infok.converged
    assert torch.equal(P1_, Pk) and info1.sigma == infok.sigma
    g1 = ctx.sp2_backward(G, ws1)
    gk = ctx.sp2_backward(G, wsk)
    torch.cuda.synchronize()
    assert torch.equal(g1, gk), (n, ck, precision)
    # the checkpoints survive the backward: a second call gives the same result
    gk2 = ctx.sp2_backward(G, wsk)
    torch.cuda.synchronize()
    assert torch.equal(gk, gk2)
    _, P1G = oracle.response_sos(inst.H, G.cpu().numpy(), inst.n_occ)
    assert rel(gk.cpu().numpy(), P1G) < TOL[precision]


def test_checkpoint_workspace_is_smaller_and_replay_needs_the_tape(ctx):
    n = 1024
    o1 = dmpt.options(ckpt_every=1)
    o8 = dmpt.options(ckpt_every=8)
    assert ctx.workspace_size(n, 1, o8) < 0.4 * ctx.workspace_size(n, 1, o1)
    inst = make_workload(2, n=300)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    _, _, info, ws = forward_with_tape(ctx, H, H1, inst.n_occ, "dual_fp16", 8)
    assert info.converged
    with pytest.raises(dmpt.DmptError) as e:          # replay reads every state
        ctx.response_replay(H1, ws)
    assert e.value.status == 1


@pytest.mark.parametrize("ck", [1, 8])
def test_config4_n4096_checkpoints(ctx, ck):
    """Config 4 at its full size (n = 4096, n_occ = 2048, L = Tr[G P]) with
    the full tape and with checkpoints every 8 S0 states: dL/dH against the
    oracle (the response to G), against Tr[G P1(E_k)] for 8 random symmetric
    directions from one k = 8 forward call, and a central finite difference
    of the oracle's L along E_0."""
    inst = make_workload(4, backend="torch", device="cuda")
    n = inst.n
    G = inst.H1[0]
    E = torch.stack([torch.from_numpy(sym_gauss(n, 900 + i)) for i in range(8)]).to(DEV)
    _, P1E, info, ws = forward_with_tape(ctx, inst.H, E, inst.n_occ, "dual_fp16", ck)
    assert info.converged
    dLdH = ctx.sp2_backward(G, ws)
    torch.cuda.synchronize()
    eps, Q = inst.eps.cpu().numpy(), inst.Q.cpu().numpy()
    _, P1G = oracle.response_from_eigs(eps, Q, G.cpu().numpy(), inst.n_occ)
    assert rel(dLdH.cpu().numpy(), P1G) < TOL["dual_fp16"]
    lhs = torch.einsum("ij,kij->k", dLdH, E).cpu().numpy()
    rhs = torch.einsum("ij,kij->k", G, P1E).cpu().numpy()
    scale = np.abs(rhs).max()
    assert np.abs(lhs - rhs).max() < 2e-3 * scale, (lhs, rhs)
    if ck == 8:
        Hn, Gn, E0 = inst.H.cpu().numpy(), G.cpu().numpy(), E[0].cpu().numpy()
        L = lambda t: float(np.sum(Gn * oracle.density_matrix(Hn + t * E0, inst.n_occ)))
        h = 1e-4
        fd = (L(h) - L(-h)) / (2 * h)
        assert abs(fd - lhs[0]) < 2e-3 * max(abs(fd), scale), (fd, lhs[0])


@pytest.mark.parametrize("n,ck", [(520, 4), (1300, 8)])
def test_checkpointed_backward_after_a_response_forward(ctx, n, ck):
    """The forward also ran K = 3 response directions in each layer launch;
    the recompute launches run the square alone.  The square's tiles come
    first in every launch, so they keep their schedule and the recomputed
    states, and dL/dH, stay bit-identical to the full tape's."""
    inst = make_workload(3, n=n, k=3)
    G = torch.from_numpy(sym_gauss(n, 79)).to(DEV)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    _, P1a, _, ws1 = forward_with_tape(ctx, H, H1, inst.n_occ, "dual_fp16", 1)
    _, P1b, info, wsk = forward_with_tape(ctx, H, H1, inst.n_occ, "dual_fp16", ck)
    assert info.converged and torch.equal(P1a, P1b)
    g1 = ctx.sp2_backward(G, ws1)
    gk = ctx.sp2_backward(G, wsk)
    torch.cuda.synchronize()
    assert torch.equal(g1, gk)


def _ckpt_cases(count=10, seed=3131):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(40, 900))
        out.append((i, n, int(rng.integers(2, 10)), int(rng.integers(0, 4)),
                    str(rng.choice(["dual_fp16", "dual_bf16"])), int(rng.integers(0, 2)),
                    int(rng.choice([0, 4, 8]))))
    return out


@pytest.mark.parametrize("case", _ckpt_cases(), ids=lambda c: f"c{c[0]}_n{c[1]}_k{c[2]}_d{c[3]}")
def test_checkpoint_soak_bit_identical(ctx, case):
    """Random sizes, checkpoint intervals, response counts, precisions, tile
    shapes and bands: the checkpointed backward equals the full tape's bit
    for bit."""
    i, n, ck, kdir, precision, cta_pair, band = case
    inst = make_instance(f"cks{i}", n, n // 2, (-2.0, -0.1), (0.1, 2.0), seed=9100 + i,
                         k=max(kdir, 1))
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1[:kdir]).to(DEV) if kdir else None
    G = torch.from_numpy(sym_gauss(n, 9200 + i)).to(DEV)
    kw = dict(cta_pair=cta_pair, tile_band=band)
    outs = []
    for c in (1, ck):
        opts = dmpt.options(precision=precision, ckpt_every=c, **kw)
        ws = torch.empty(ctx.workspace_size(n, kdir, opts) + 256, dtype=torch.uint8, device=DEV)
        _, _, info = ctx.sp2_response(H, H1, inst.n_occ, precision=precision, ckpt_every=c,
                                      workspace=ws, **kw)
        assert info.converged
        outs.append(ctx.sp2_backward(G, ws, **kw))
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1]), case
