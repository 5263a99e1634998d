"""The complement form (hole_form, on by default for n_occ > n/2) through
every entry point that runs the recursion, each against the oracle.

With more occupied than empty levels the library runs the recursion on
I - P and returns P = I - Q, P_o = -Q_o.  These tests take occupations of
about 0.7 n and check:
* the adjoint: dL/dH equals the oracle's response to G (the same formula
  holds for the complement form), with the full tape and with checkpoints;
* the response replay (bit for bit against the forward) and the
  self-consistent response (the oracle's fixed point);
* the second- and third-order terms;
* an uneven batch that mixes occupations below and above half filling,
  bit for bit against single calls;
* the static-scratch entry point, bit for bit against the workspace call.
"""

import ctypes

import numpy as np
import pytest

import oracle
from paper_2203_09621_gb300.workloads import make_instance, scc_gamma, sym_gauss

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle.sos import response2_sos  # noqa: E402
from paper_2203_09621_gb300 import dmpt  # noqa: E402

DEV = torch.device("cuda:0")
TOL = {"dual_fp16": 1e-3, "dual_bf16": 5e-3}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    return dmpt.context(0)


def hole_instance(n, k=1, seed=8800, frac=0.7):
    return make_instance(f"hole{n}", n, int(round(frac * n)), (-2.0, -0.1), (0.1, 2.0),
                         k=k, seed=seed + n)


def with_states(ctx, H, H1, n_occ, ck, precision="dual_fp16"):
    k = 0 if H1 is None else H1.shape[0]
    opts = dmpt.options(precision=precision, ckpt_every=ck)
    ws = torch.empty(ctx.workspace_size(H.shape[0], k, opts) + 256, dtype=torch.uint8,
                     device=DEV)
    P, P1, info = ctx.sp2_response(H, H1, n_occ, precision=precision, ckpt_every=ck,
                                   workspace=ws)
    torch.cuda.synchronize()
    return P, P1, info, ws


@pytest.mark.parametrize("ck", [1, 8])
@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
def test_adjoint_complement(ctx, ck, precision):
    inst = hole_instance(400)
    H = torch.from_numpy(inst.H).to(DEV)
    G = sym_gauss(400, 8801)
    P, _, info, ws = with_states(ctx, H, None, inst.n_occ, ck, precision)
    assert info.converged and info.hole
    assert rel(P.cpu().numpy(), oracle.density_matrix(inst.H, inst.n_occ)) < TOL[precision]
    dLdH = ctx.sp2_backward(torch.from_numpy(G).to(DEV), ws).cpu().numpy()
    _, P1G = oracle.response_from_eigs(inst.eps, inst.Q, G, inst.n_occ)
    assert rel(dLdH, P1G) < TOL[precision], rel(dLdH, P1G)


def test_replay_and_scc_complement(ctx):
    n = 300
    inst = hole_instance(n, k=2)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    _, P1f, info, ws = with_states(ctx, H, H1, inst.n_occ, 1)
    assert info.hole
    P1f = P1f.clone()
    P1r, rinfo = ctx.response_replay(H1, ws)
    torch.cuda.synchronize()
    assert torch.equal(P1r, P1f) and rinfo.hole
    for j in range(2):
        _, want = oracle.response_from_eigs(inst.eps, inst.Q, inst.H1[j], inst.n_occ)
        assert rel(P1r[j].cpu().numpy(), want) < 1e-3
    g = scc_gamma(n)
    P1s, its, res, _ = ctx.scc_response(H1, torch.from_numpy(g).to(DEV), ws, tol=1e-5)
    torch.cuda.synchronize()
    assert res < 1e-5
    for j in range(2):
        want, _, _ = oracle.scc_response(inst.H, inst.H1[j], g, inst.n_occ)
        assert rel(P1s[j].cpu().numpy(), want) < 1e-3


@pytest.mark.parametrize("precision", ["dual_fp16", "fp64"])
def test_higher_orders_complement(ctx, precision):
    n = 300
    inst = hole_instance(n)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    P, terms, info = ctx.sp2_response_m(H, H1, inst.n_occ, 3, precision=precision)
    torch.cuda.synchronize()
    assert info.converged and info.hole
    tol = 1e-9 if precision == "fp64" else 1e-3
    r = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ, order=3)
    for o in range(1, 4):
        got = terms[o - 1][0].cpu().numpy()
        assert rel(got, r.Pk[o - 1][0]) < tol, (o, rel(got, r.Pk[o - 1][0]))
    D2 = response2_sos(inst.H, inst.H1[0], inst.n_occ)
    assert rel(terms[1][0].cpu().numpy(), D2) < tol * 10


def test_batch_mixed_occupations(ctx):
    sizes = [(260, 0.3), (300, 0.7), (517, 0.5), (640, 0.85), (333, 0.6)]
    insts = [make_instance(f"mix{i}", n, int(round(f * n)), (-2.0, -0.1), (0.1, 2.0),
                           seed=8900 + i) for i, (n, f) in enumerate(sizes)]
    Hs = [torch.from_numpy(x.H).to(DEV) for x in insts]
    H1s = [torch.from_numpy(x.H1).to(DEV) for x in insts]
    occ = [x.n_occ for x in insts]
    Pb, P1b, infos = ctx.sp2_response_batch(Hs, H1s, occ)
    torch.cuda.synchronize()
    for i, x in enumerate(insts):
        assert infos[i].converged and infos[i].hole == (2 * x.n_occ > x.n)
        P, P1, _ = ctx.sp2_response(Hs[i], H1s[i], x.n_occ)
        torch.cuda.synchronize()
        assert torch.equal(P1b[i], P1) and torch.equal(Pb[i], P)
        _, want = oracle.response_from_eigs(x.eps, x.Q, x.H1[0], x.n_occ)
        assert rel(P1[0].cpu().numpy(), want) < 1e-3


def test_static_entry_point_complement(ctx):
    inst = hole_instance(200)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    n = 200
    P = torch.empty(n, n, dtype=torch.float64, device=DEV)
    P1 = torch.empty(1, n, n, dtype=torch.float64, device=DEV)
    opts = dmpt.options()
    info = dmpt.DmptInfo()
    st = ctx.lib.dmpt_sp2_response_static(
        ctx.h, H.data_ptr(), H1.data_ptr(), 1, n, n, inst.n_occ, ctypes.byref(opts),
        P.data_ptr(), P1.data_ptr(), ctypes.byref(info),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == 0 and info.hole == 1
    Pw, P1w, _ = ctx.sp2_response(H, H1, inst.n_occ)
    torch.cuda.synchronize()
    assert torch.equal(P, Pw) and torch.equal(P1, P1w)
