"""Randomised soak of the C ABI on the GPU: many small configurations.

A fixed seed draws the size n in [1, 1100] (with a bias toward tiny and
boundary sizes), the occupation (including 0, 1, n - 1 and n), the number of
directions k in [0, 8], the precision and the scheduling options (tile
shape, K-snake, tile band, chunk length).  Every case is checked against the
oracle: P and each P1 within the form's tolerance, with the floor relative
to the operands' scale that uneven occupations need (FP32: its derived bound
10 u (eps_N - eps_1) / gap times ||P||_F; dual forms: TOL / 20 times the
norm of the projector the recursion runs on, sqrt(min(n_occ, n - n_occ))
with the default complement form), and the trivial occupations exactly.
"""

import numpy as np
import pytest

import oracle
from paper_2203_09621_gb300.workloads import make_instance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2203_09621_gb300 import dmpt  # noqa: E402

DEV = torch.device("cuda:0")
TOL = {"dual_fp16": 1e-3, "dual_bf16": 5e-3}


def draw_cases(count=60, seed=20221):
    rng = np.random.default_rng(seed)
    special = [1, 2, 3, 31, 32, 33, 255, 256, 257, 511, 512, 513]
    cases = []
    for i in range(count):
        n = int(rng.choice(special)) if rng.random() < 0.4 else int(rng.integers(4, 1100))
        r = rng.random()
        if n == 1 or r < 0.08:
            n_occ = int(rng.choice([0, n]))
        elif r < 0.16:
            n_occ = int(rng.choice([1, n - 1]))
        else:
            n_occ = int(rng.integers(1, n))
        k = int(rng.integers(0, 9)) if n_occ not in (0, n) else int(rng.integers(0, 3))
        precision = str(rng.choice(["dual_fp16", "dual_fp16", "dual_bf16", "fp32"]))
        opts = {}
        if precision.startswith("dual"):
            opts = dict(cta_pair=int(rng.integers(0, 2)), k_snake=int(rng.integers(0, 2)),
                        tile_band=int(rng.choice([0, 3, 8])),
                        accum_chunk=int(rng.choice([0, 128, 512])))
        gap = float(rng.uniform(0.1, 0.4))
        cases.append((i, n, n_occ, k, precision, opts, gap, 50000 + i))
    return cases


@pytest.fixture(scope="module")
def ctx():
    return dmpt.context(0)


@pytest.mark.parametrize("case", draw_cases(), ids=lambda c: f"c{c[0]}_n{c[1]}_o{c[2]}_k{c[3]}_{c[4]}")
def test_soak(ctx, case):
    i, n, n_occ, k, precision, opts, gap, seed = case
    inst = make_instance(f"soak{i}", n, n_occ, (-2.0, -gap / 2), (gap / 2, 2.0), seed=seed,
                         k=max(k, 1))
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1[:k]).to(DEV) if k else None
    P, P1, info = ctx.sp2_response(H, H1, n_occ, precision=precision, **opts)
    torch.cuda.synchronize()
    assert info.status == 0 and info.converged, (case, info.status, info.layers)
    if n_occ in (0, n):
        assert torch.equal(P.cpu(), torch.eye(n, dtype=torch.float64) * (n_occ == n))
        if k:
            assert not P1.any()
        return
    Pr = oracle.density_matrix(inst.H, n_occ)
    if precision == "fp32":
        lo, hi = oracle.gershgorin_bounds(inst.H)
        tol = max(10 * 2.0 ** -24 * (hi - lo) / gap, 1e-5)
    else:
        tol = TOL[precision]
    nP = np.linalg.norm(Pr)
    assert np.linalg.norm(P.cpu().numpy() - Pr) <= tol * nP, case
    # the dual forms' operands are S0 -> P, or I - P in the complement form
    # that runs by default when more than half the levels are occupied
    n_ops = np.sqrt(min(n_occ, n - n_occ)) if precision != "fp32" else nP
    assert info.hole == (2 * n_occ > n)
    for j in range(k):
        _, P1r = oracle.response_from_eigs(inst.eps, inst.Q, inst.H1[j], n_occ)
        err = np.linalg.norm(P1[j].cpu().numpy() - P1r)
        # floor relative to the operands' scale ||P||_F: the FP32 bound
        # 10 u (eps_N - eps_1) / gap is itself that scale's bound; the dual
        # forms' floor is the half-filled error scale (see the edge-case tests)
        floor = tol * nP if precision == "fp32" else tol / 20 * n_ops
        bound = max(tol * np.linalg.norm(P1r), floor)
        assert err <= bound, (case, j, err / max(np.linalg.norm(P1r), 1e-300))
