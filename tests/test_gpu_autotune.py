"""Autotuning of the layer products (dmpt_autotune, options.autotune).

The tuner times short probe solves under each candidate tile shape (CTA
pairs with 256 x 256 tiles, single CTAs with 128 x 256 tiles) and tile-band
rasterisation, and keeps the fastest per (padded n, k, precision); batches
choose between the grouped and per-instance paths.  The choice changes the
order of the work only, so results stay within the method's accuracy, and an
autotuned solve equals the solve with the chosen configuration given
explicitly, bit for bit.
"""

import numpy as np
import pytest

import oracle
from paper_2203_09621_gb300.workloads import make_instance, make_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2203_09621_gb300 import dmpt  # noqa: E402

DEV = torch.device("cuda:0")


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_autotune_choice_and_autotuned_solve():
    ctx = dmpt.Context(0)   # a fresh handle: empty tuning table
    inst = make_workload(2, n=1300, k=2)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    best, ms = ctx.autotune(H, H1, inst.n_occ)
    assert best["cta_pair"] in (0, 1) and best["tile_band"] in (0, 4, 8, 16) and ms > 0
    P, P1, info = ctx.sp2_response(H, H1, inst.n_occ, autotune=1)
    torch.cuda.synchronize()
    assert info.converged
    Pe, P1e, _ = ctx.sp2_response(H, H1, inst.n_occ, **best)
    torch.cuda.synchronize()
    assert torch.equal(P, Pe) and torch.equal(P1, P1e)
    eps, V = np.linalg.eigh(inst.H)
    for j in range(2):
        _, P1r = oracle.response_from_eigs(eps, V, inst.H1[j], inst.n_occ)
        assert rel(P1[j].cpu().numpy(), P1r) < 1e-3


def test_autotune_on_first_use_then_table():
    """autotune=1 without a prior dmpt_autotune tunes on first use; the next
    call reuses the table and gives the same result."""
    ctx = dmpt.Context(0)
    inst = make_workload(3, n=700, k=3)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    P, P1, info = ctx.sp2_response(H, H1, inst.n_occ, autotune=1)
    P2, P12, info2 = ctx.sp2_response(H, H1, inst.n_occ, autotune=1)
    torch.cuda.synchronize()
    assert info.converged and info2.converged
    assert torch.equal(P1, P12) and torch.equal(P, P2)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotune_plain_forms_have_no_candidates(precision):
    ctx = dmpt.Context(0)
    inst = make_workload(1)
    H = torch.from_numpy(inst.H).to(DEV)
    H1 = torch.from_numpy(inst.H1).to(DEV)
    best, ms = ctx.autotune(H, H1, inst.n_occ, precision=precision)
    assert ms == 0.0 and best["cta_pair"] == 1 and best["tile_band"] == 8


def test_autotuned_batch():
    ctx = dmpt.Context(0)
    sizes = [256, 300, 700, 1024, 513, 1500]
    insts = [make_instance(f"t{i}", n, n // 2, (-2.0, -0.1), (0.1, 2.0), seed=9400 + i)
             for i, n in enumerate(sizes)]
    Hs = [torch.from_numpy(x.H).to(DEV) for x in insts]
    H1s = [torch.from_numpy(x.H1).to(DEV) for x in insts]
    occ = [x.n_occ for x in insts]
    Ps, P1s, infos = ctx.sp2_response_batch(Hs, H1s, occ, autotune=1)
    Ps2, P1s2, infos2 = ctx.sp2_response_batch(Hs, H1s, occ, autotune=1)   # from the table
    torch.cuda.synchronize()
    for i, x in enumerate(insts):
        assert infos[i].converged and infos2[i].converged
        assert torch.equal(P1s[i], P1s2[i])
        _, P1r = oracle.response_sos(x.H, x.H1[0], x.n_occ)
        assert rel(P1s[i][0].cpu().numpy(), P1r) < 1e-3
