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


def forward_with_tape(ctx, H, H1, n_occ, precision):
    opts = dmpt.options(precision=precision, ckpt_every=1)
    k = 0 if H1 is None else (1 if H1.dim() == 2 else H1.shape[0])
    ws = torch.empty(ctx.workspace_size(H.shape[0], k, opts) + 256, dtype=torch.uint8,
                     device=DEV)
    P, P1, info = ctx.sp2_response(H, H1, n_occ, precision=precision, ckpt_every=1,
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
