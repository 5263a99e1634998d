"""Randomised soak of the other entry points on the GPU.

* uneven batches (dmpt_sp2_response_batch): random sizes, occupations
  (trivial ones included), k and dual precision; every instance bit-exact
  against its single call and within tolerance of the oracle;
* the host-buffer pipeline (dmpt_sp2_response_host): random instance
  counts and sizes; bit-exact against the device calls;
* the second-order response (dmpt_sp2_response2): random sizes and
  occupations against the oracle's second-order formula;
* responses of orders 3-5 (dmpt_sp2_response_m): random sizes, occupations,
  k, precision and tile shape (CTA pair or 1 CTA) against the oracle's SP2
  recursion of the same order.  An order-o term is formed from the products
  S_a S_{o-a}, so its rounding scales with sum_a ||P_a|| ||P_{o-a}||, which
  can exceed ||P_o|| (cancellation); the tolerance is relative to the larger
  of the two.
"""

import numpy as np
import pytest

import oracle
from oracle.sos import response2_sos
from paper_2203_09621_gb300.workloads import make_instance

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


def random_instance(rng, tag, n_lo, n_hi, k, trivial_ok=True):
    n = int(rng.integers(n_lo, n_hi))
    r = rng.random()
    if trivial_ok and r < 0.1:
        n_occ = int(rng.choice([0, n]))
    else:
        n_occ = int(rng.integers(max(1, n // 5), n - max(1, n // 5) + 1))
    gap = float(rng.uniform(0.15, 0.4))
    return make_instance(tag, n, n_occ, (-2.0, -gap / 2), (gap / 2, 2.0), k=max(k, 1),
                         seed=int(rng.integers(1, 2**31)))


@pytest.mark.parametrize("trial", range(4))
def test_soak_batch(ctx, trial):
    rng = np.random.default_rng(31000 + trial)
    count = int(rng.integers(3, 12))
    k = int(rng.integers(1, 4))
    precision = str(rng.choice(["dual_fp16", "dual_bf16"]))
    insts = [random_instance(rng, f"b{trial}_{i}", 60, 900, k) for i in range(count)]
    Hs = [torch.from_numpy(x.H).to(DEV) for x in insts]
    H1s = [torch.from_numpy(x.H1[:k]).to(DEV) for x in insts]
    Ps, P1s, infos = ctx.sp2_response_batch(Hs, H1s, [x.n_occ for x in insts], precision=precision)
    torch.cuda.synchronize()
    for i, x in enumerate(insts):
        P, P1, info = ctx.sp2_response(Hs[i], H1s[i], x.n_occ, precision=precision)
        torch.cuda.synchronize()
        assert infos[i].converged and torch.equal(Ps[i], P) and torch.equal(P1s[i], P1), i
        if x.n_occ in (0, x.H.shape[0]):
            continue
        for j in range(k):
            _, P1r = oracle.response_from_eigs(x.eps, x.Q, x.H1[j], x.n_occ)
            assert rel(P1s[i][j].cpu().numpy(), P1r) < TOL[precision], (i, j)


@pytest.mark.parametrize("trial", range(3))
def test_soak_host_pipeline(ctx, trial):
    rng = np.random.default_rng(32000 + trial)
    n = int(rng.integers(40, 700))
    k = int(rng.integers(1, 4))
    count = int(rng.integers(1, 5))
    insts = [random_instance(rng, f"h{trial}_{i}", n, n + 1, k, trivial_ok=False)
             for i in range(count)]
    occ = insts[0].n_occ   # one occupation for the sequence
    Hs = [torch.from_numpy(x.H).pin_memory() for x in insts]
    H1s = [torch.from_numpy(x.H1[:k]).pin_memory() for x in insts]
    _, P1s, infos = ctx.solve_host(Hs, H1s, occ)
    for i, x in enumerate(insts):
        _, P1d, info = ctx.sp2_response(torch.from_numpy(x.H).to(DEV),
                                        torch.from_numpy(x.H1[:k]).to(DEV), occ)
        torch.cuda.synchronize()
        assert infos[i].converged and torch.equal(P1s[i], P1d.cpu()), i


@pytest.mark.parametrize("trial", range(4))
def test_soak_second_order(ctx, trial):
    rng = np.random.default_rng(33000 + trial)
    k = int(rng.integers(1, 4))
    precision = str(rng.choice(["dual_fp16", "dual_bf16"]))
    x = random_instance(rng, f"o2_{trial}", 50, 500, k, trivial_ok=False)
    H = torch.from_numpy(x.H).to(DEV)
    H1 = torch.from_numpy(x.H1[:k]).to(DEV)
    P, P1, P2, info = ctx.sp2_response2(H, H1, x.n_occ, precision=precision)
    torch.cuda.synchronize()
    assert info.converged
    tol2 = {"dual_fp16": 1e-3, "dual_bf16": 5e-3}[precision]
    for j in range(k):
        want = response2_sos(x.H, x.H1[j], x.n_occ)
        assert rel(P2[j].cpu().numpy(), want) < tol2, (j, rel(P2[j].cpu().numpy(), want))


@pytest.mark.parametrize("trial", range(4))
def test_soak_any_order(ctx, trial):
    rng = np.random.default_rng(34000 + trial)
    order = int(rng.integers(3, 6))
    k = int(rng.integers(1, 8 // order + 1))
    precision = str(rng.choice(["dual_fp16", "dual_bf16"]))
    cta_pair = int(rng.integers(0, 2))
    x = random_instance(rng, f"om_{trial}", 40, 400, k, trivial_ok=False)
    H = torch.from_numpy(x.H).to(DEV)
    H1 = torch.from_numpy(x.H1[:k]).to(DEV)
    P, terms, info = ctx.sp2_response_m(H, H1, x.n_occ, order, precision=precision,
                                        cta_pair=cta_pair)
    torch.cuda.synchronize()
    assert info.converged
    ref = oracle.sp2_pt(x.H, x.H1[:k], x.n_occ, order=order)
    for j in range(k):
        Pj = [ref.P] + [ref.Pk[o][j] for o in range(order)]
        for o in range(1, order + 1):
            scale = max(np.linalg.norm(Pj[o]),
                        sum(np.linalg.norm(Pj[a]) * np.linalg.norm(Pj[o - a]) for a in range(1, o)))
            err = np.linalg.norm(terms[o - 1][j].cpu().numpy() - Pj[o]) / scale
            assert err < TOL[precision], (order, k, cta_pair, j, o, err)
