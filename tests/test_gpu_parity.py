"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative Frobenius norm of P1 and P against the oracle):
  FP64 form       1e-10, and the branch sequence / layer counts of the FP64
                  oracle SP2 exactly (both sides decide in FP64)
  FP32 form       10 * u32 * (eps_N - eps_1) / gap, u32 = 2^-24: the FP32
                  rounding of the masters amplified by the condition of the
                  step at the gap after Gershgorin scaling
  dual FP16       1e-3    dual BF16   5e-3
"""

import numpy as np
import pytest

import oracle
from oracle.sos import response_columns
from paper_2203_09621_gb300.workloads import make_workload, make_instance, sym_gauss

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2203_09621_gb300 import dmpt  # noqa: E402

DEV = torch.device("cuda:0")
U32 = 2.0 ** -24
TOL = {"dual_fp16": 1e-3, "dual_bf16": 5e-3}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ctx():
    return dmpt.context(0)


def run(ctx, inst, precision, **kw):
    H = torch.from_numpy(np.ascontiguousarray(inst.H)).to(DEV)
    H1 = torch.from_numpy(np.ascontiguousarray(inst.H1)).to(DEV)
    P, P1, info = ctx.sp2_response(H, H1, inst.n_occ, precision=precision, **kw)
    torch.cuda.synchronize()
    return P.cpu().numpy(), P1.cpu().numpy(), info


def fp32_tol(inst, bounds):
    gap = inst.eps[inst.n_occ] - inst.eps[inst.n_occ - 1]
    return 10.0 * U32 * (bounds[1] - bounds[0]) / gap


# --------------------------------------------------------------------------
# Gershgorin bounds

@pytest.mark.parametrize("n,ld", [(128, 128), (300, 301), (1000, 1024)])
def test_bounds(ctx, n, ld):
    Hn = sym_gauss(n, 5 + n) + np.diag(np.linspace(-3, 3, n))
    Hp = np.zeros((n, ld))
    Hp[:, :n] = Hn
    H = torch.from_numpy(Hp).to(DEV)
    eps = torch.empty(2, dtype=torch.float64, device=DEV)
    st = ctx.lib.dmpt_bounds(ctx.h, H.data_ptr(), n, ld, eps.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == 0
    lo, hi = oracle.gershgorin_bounds(Hn)
    got = eps.cpu().numpy()
    assert abs(got[0] - lo) <= 1e-12 * abs(lo) and abs(got[1] - hi) <= 1e-12 * abs(hi)


def test_bounds_golden(ctx, golden):
    g = golden("gershgorin_3x3.json")
    H = torch.tensor(g["H"], dtype=torch.float64, device=DEV)
    got = ctx.bounds(H).cpu().numpy().tolist()
    assert got == g["bounds"]


# --------------------------------------------------------------------------
# FP64 form: same algorithm, same decisions as the FP64 oracle

@pytest.mark.parametrize("cfg,n", [(1, None), (2, 300), (3, 256)])
def test_fp64_matches_oracle(ctx, cfg, n):
    inst = make_workload(cfg, n=n)
    P, P1, info = run(ctx, inst, "fp64")
    r = oracle.sp2_pt(inst.H, inst.H1, inst.n_occ)
    Pr, P1r = oracle.response_sos(inst.H, inst.H1, inst.n_occ)
    assert info.converged and r.converged
    # branch decisions before D0 converges are unique; at the converging layer
    # N_S ~ N_X ~ n_occ and sigma is decided by rounding noise (a near tie),
    # after it the branches must alternate (the sigma flip)
    nc = r.d0_layer
    assert info.d0_layer == nc
    assert info.sigma[: nc - 1] == r.sigma[: nc - 1]
    tail = info.sigma[nc - 1:]
    assert all(tail[i] == -tail[i - 1] for i in range(1, len(tail)))
    assert info.layers == r.layers
    assert info.d1_layer == r.d1_layer
    assert abs(info.eps_min - r.bounds[0]) < 1e-12 * abs(r.bounds[0])
    assert rel(P, Pr) < 1e-10
    for j in range(inst.k):
        assert rel(P1[j], P1r[j]) < 1e-10
        assert rel(P1[j], r.P1[j]) < 1e-10


# --------------------------------------------------------------------------
# FP32 and dual forms against the oracle

@pytest.mark.parametrize("cfg,n", [(1, None), (2, 300), (2, 1024)])
def test_fp32(ctx, cfg, n):
    inst = make_workload(cfg, n=n)
    P, P1, info = run(ctx, inst, "fp32")
    Pr, P1r = oracle.response_sos(inst.H, inst.H1, inst.n_occ)
    tol = fp32_tol(inst, (info.eps_min, info.eps_max))
    assert info.converged
    assert rel(P, Pr) < tol and rel(P1[0], P1r[0]) < tol, (rel(P, Pr), rel(P1[0], P1r[0]), tol)


@pytest.mark.parametrize("cta_pair", [0, 1])
@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
@pytest.mark.parametrize("cfg,n", [(1, None), (2, 300), (2, 1024), (3, 512)])
def test_dual(ctx, precision, cfg, n, cta_pair):
    inst = make_workload(cfg, n=n)
    P, P1, info = run(ctx, inst, precision, cta_pair=cta_pair)
    Pr, P1r = oracle.response_sos(inst.H, inst.H1, inst.n_occ)
    assert info.converged, info
    assert rel(P, Pr) < TOL[precision]
    for j in range(inst.k):
        assert rel(P1[j], P1r[j]) < TOL[precision], (j, rel(P1[j], P1r[j]))
    # D1 stops a sigma-flip pair or more after D0 (Alg. 3 with the +inf reading)
    assert all(d >= info.d0_layer + 2 for d in info.d1_layer)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "dual_fp16", "dual_bf16"])
def test_two_level_closed_form(ctx, golden, precision):
    g = golden("two_level.json")
    H = torch.tensor(g["H"], dtype=torch.float64, device=DEV)
    H1 = torch.tensor(g["H1"], dtype=torch.float64, device=DEV)
    P, P1, info = ctx.sp2_response(H, H1, g["n_occ"], precision=precision)
    torch.cuda.synchronize()
    tol = 1e-12 if precision == "fp64" else 1e-6
    np.testing.assert_allclose(P.cpu().numpy(), g["P"], atol=tol)
    np.testing.assert_allclose(P1[0].cpu().numpy(), g["P1"], atol=tol)
    assert info.d0_layer == g["d0_layer"] and info.converged


@pytest.mark.parametrize("precision,cta_pair", [("fp32", 0), ("dual_fp16", 0), ("dual_fp16", 1)])
def test_deterministic(ctx, precision, cta_pair):
    inst = make_workload(2, n=512)
    a = run(ctx, inst, precision, cta_pair=cta_pair)
    b = run(ctx, inst, precision, cta_pair=cta_pair)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2].sigma == b[2].sigma


# --------------------------------------------------------------------------
# Edge cases and error paths

@pytest.mark.parametrize("n_occ", [0, 64])
def test_trivial_occupations(ctx, n_occ):
    inst = make_workload(1, n=64)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    P, P1, info = ctx.sp2_response(H, H1, n_occ, precision="dual_fp16")
    torch.cuda.synchronize()
    want = np.zeros((64, 64)) if n_occ == 0 else np.eye(64)
    assert np.array_equal(P.cpu().numpy(), want)
    assert not P1.cpu().numpy().any()
    assert info.layers == 0 and info.converged


def test_one_by_one(ctx):
    H = torch.tensor([[0.3]], dtype=torch.float64, device=DEV)
    H1 = torch.tensor([[1.0]], dtype=torch.float64, device=DEV)
    P, P1, _ = ctx.sp2_response(H, H1, 1, precision="dual_fp16")
    torch.cuda.synchronize()
    assert P.item() == 1.0 and P1.item() == 0.0


def test_errors(ctx):
    lib, h = ctx.lib, ctx.h
    inst = make_workload(1, n=64)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    P1 = torch.empty_like(H1)
    opts = dmpt.options(precision="fp32")
    ws, wlen = ctx.workspace(ctx.workspace_size(64, 1, opts))
    import ctypes
    call = lambda **kw: lib.dmpt_sp2_response(
        h, kw.get("H", H.data_ptr()), H1.data_ptr(), kw.get("k", 1), kw.get("n", 64),
        kw.get("ld", 64), kw.get("nocc", 32), ctypes.byref(opts), None, P1.data_ptr(), None,
        ctypes.c_void_p(kw.get("ws", ws)), kw.get("wlen", wlen), None)
    assert call(n=0) == 1
    assert call(ld=10) == 1
    assert call(nocc=65) == 1
    assert call(nocc=-1) == 1
    assert call(k=0) == 1 and call(k=9) == 1
    assert call(H=None) == 1
    assert call(wlen=100) == 2
    assert call(ws=ws + 8) == 2
    assert call() == 0
    torch.cuda.synchronize()


def test_not_converged(ctx):
    inst = make_workload(1)
    P, P1, info = ctx.sp2_response(torch.from_numpy(inst.H).to(DEV),
                                   torch.from_numpy(inst.H1).to(DEV), inst.n_occ,
                                   precision="fp32", max_layers=5, raise_on_error=False)
    assert info.status == 3 and not info.converged and info.layers == 5


@pytest.mark.parametrize("precision", ["fp32", "dual_fp16"])
def test_numeric_errors(ctx, precision):
    # H = c I: Gershgorin gives eps_N = eps_1, the initial layer is undefined
    H = 0.5 * torch.eye(16, dtype=torch.float64, device=DEV)
    H1 = torch.from_numpy(sym_gauss(16, 3, 0.01)).to(DEV)
    _, _, info = ctx.sp2_response(H, H1, 8, precision=precision, raise_on_error=False)
    assert info.status == 4
    Hn = torch.from_numpy(sym_gauss(16, 4)).to(DEV)
    Hn[3, 5] = float("nan")
    Hn[5, 3] = float("nan")
    _, _, info = ctx.sp2_response(Hn, H1, 8, precision=precision, raise_on_error=False)
    assert info.status == 4


# --------------------------------------------------------------------------
# Full size, launch configuration of the benchmark: sampled columns of P1
# against the oracle evaluated from the known eigendecomposition.

@pytest.fixture(scope="module")
def dipole3_full():
    """The benchmark workload (n = 8192, k = 3) and its whole oracle result:
    P = Vo Vo^T and every column of each P1_k from the known eigenpairs
    (occupied-virtual block form, about 5e12 FP64 flops on the host)."""
    inst = make_workload(3, backend="torch", device="cuda")
    eps = inst.eps.cpu().numpy()
    Q = inst.Q.cpu().numpy()
    Pr = oracle.density_from_eigs(eps, Q, inst.n_occ)
    cols = np.arange(inst.n)
    P1r = [response_columns(eps, Q, inst.H1[j].cpu().numpy(), inst.n_occ, cols)
           for j in range(inst.k)]
    return inst, Pr, P1r


@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
def test_full_size_dipole3_n8192(ctx, dipole3_full, precision):
    """The benchmark's launch configuration at its full size: the whole P and
    all three P1_k against the oracle, element by element (relative
    Frobenius), plus Tr P = n_occ, Tr P1 = 0 and exact symmetry."""
    inst, Pr, P1r = dipole3_full
    P, P1, info = ctx.sp2_response(inst.H, inst.H1, inst.n_occ, precision=precision,
                                   timing=True)
    torch.cuda.synchronize()
    assert info.converged, info
    errs = [rel(P1[j].cpu().numpy(), P1r[j]) for j in range(inst.k)]
    eP = rel(P.cpu().numpy(), Pr)
    print(f"n=8192 {precision}: rel err P {eP:.3e}, P1 {[f'{e:.3e}' for e in errs]}")
    assert max(errs) < TOL[precision], errs
    assert eP < TOL[precision], eP
    assert abs(torch.trace(P).item() - inst.n_occ) < 1e-2
    for j in range(inst.k):
        assert abs(torch.trace(P1[j]).item()) < 1e-2
        assert torch.equal(P1[j], P1[j].T)


@pytest.mark.parametrize("precision", ["dual_fp16", "dual_bf16"])
def test_full_size_cfg2_n4096(ctx, precision):
    """Config 2 at its full size (n = 4096, n_occ = 2048, gap 0.2, one H1).
    Whole P and P1 against the
    oracle evaluated from the known eigendecomposition, plus the idempotency
    identities P P = P and P P1 + P1 P = P1 on the GPU result."""
    inst = make_workload(2, backend="torch", device="cuda")
    assert inst.H.shape[0] == 4096
    P, P1, info = ctx.sp2_response(inst.H, inst.H1, inst.n_occ, precision=precision)
    torch.cuda.synchronize()
    assert info.converged, info
    Pr, P1r = oracle.response_from_eigs(inst.eps.cpu().numpy(), inst.Q.cpu().numpy(),
                                        inst.H1[0].cpu().numpy(), inst.n_occ)
    assert rel(P1[0].cpu().numpy(), P1r) < TOL[precision]
    assert rel(P.cpu().numpy(), Pr) < TOL[precision]
    PP = P @ P
    assert (torch.linalg.norm(PP - P) / torch.linalg.norm(P)).item() < TOL[precision]
    X1 = P @ P1[0] + P1[0] @ P
    assert (torch.linalg.norm(X1 - P1[0]) / torch.linalg.norm(P1[0])).item() < TOL[precision]


def test_max_directions_k8(ctx):
    """DMPT_MAX_K = 8 responses sharing one S0 recursion (one square and
    eight response jobs per D0 layer), each against the oracle."""
    inst = make_workload(2, n=300)
    n = inst.H.shape[0]
    H1 = np.stack([sym_gauss(n, 8181 + j, 0.01) for j in range(8)])
    P, P1, info = ctx.sp2_response(torch.from_numpy(inst.H).to(DEV), torch.from_numpy(H1).to(DEV),
                                   inst.n_occ)
    torch.cuda.synchronize()
    assert info.converged
    eps, V = np.linalg.eigh(inst.H)
    for j in range(8):
        _, P1r = oracle.response_from_eigs(eps, V, H1[j], inst.n_occ)
        assert rel(P1[j].cpu().numpy(), P1r) < TOL["dual_fp16"], j


@pytest.mark.parametrize("precision", ["dual_fp16", "fp32"])
def test_leading_dimension(ctx, precision):
    """Row-major inputs and outputs with ld > n (views into wider buffers)
    give the same result as the contiguous call, bit for bit."""
    inst = make_workload(2, n=520, k=2)
    n, ld = 520, 537
    Hb = torch.zeros(n, ld, dtype=torch.float64, device=DEV)
    H1b = torch.zeros(2, n, ld, dtype=torch.float64, device=DEV)
    Hb[:, :n] = torch.from_numpy(inst.H).to(DEV)
    H1b[:, :, :n] = torch.from_numpy(inst.H1).to(DEV)
    Hv, H1v = Hb[:, :n], H1b[:, :, :n]
    assert Hv.stride(0) == ld
    Pc, P1c, _ = ctx.sp2_response(torch.from_numpy(inst.H).to(DEV), torch.from_numpy(inst.H1).to(DEV),
                                  inst.n_occ, precision=precision)
    Pv, P1v, info = ctx.sp2_response(Hv, H1v, inst.n_occ, precision=precision)
    torch.cuda.synchronize()
    assert info.converged
    assert torch.equal(Pc, Pv.contiguous()) and torch.equal(P1c, P1v.contiguous())


@pytest.mark.parametrize("opts", [dict(k_snake=0), dict(tile_band=0), dict(tile_band=3),
                                  dict(tile_band=16), dict(accum_chunk=64),
                                  dict(accum_chunk=1024), dict(sync_every=1),
                                  dict(cta_pair=0, accum_chunk=512), dict(round_align=0)])
def test_options_keep_parity(ctx, opts):
    """Scheduling and accumulation options change the order of the work
    (tile order, K direction, chunk length, host polling, round alignment),
    not the method: every setting stays within the dual-FP16 tolerance of the
    oracle.  Tile order, host polling and round alignment leave the result
    bit-identical to the defaults."""
    inst = make_workload(2, n=1300, k=2)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    P, P1, info = ctx.sp2_response(H, H1, inst.n_occ, **opts)
    torch.cuda.synchronize()
    assert info.converged
    eps, V = np.linalg.eigh(inst.H)
    for j in range(2):
        _, P1r = oracle.response_from_eigs(eps, V, inst.H1[j], inst.n_occ)
        assert rel(P1[j].cpu().numpy(), P1r) < TOL["dual_fp16"], (opts, j)
    if set(opts) <= {"tile_band", "sync_every", "round_align"}:
        Pd, P1d, _ = ctx.sp2_response(H, H1, inst.n_occ)
        torch.cuda.synchronize()
        assert torch.equal(P, Pd) and torch.equal(P1, P1d), opts
