"""GPU parity of the host-buffer pipeline (dmpt_sp2_response_host).

Each instance's upper triangles are copied in (the device mirrors them),
solved by the same kernels in the same order as dmpt_sp2_response on device
buffers, and copied out, with the copies of the neighbouring instances
overlapping the solve; for symmetric inputs the results must equal the
device call's bit for bit and the oracle within the dual tolerance.
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


@pytest.fixture(scope="module")
def ctx():
    return dmpt.context(0)


@pytest.mark.parametrize("pinned", [True, False])
def test_pipeline_matches_device_calls(ctx, pinned):
    n, k = 520, 2
    insts = [make_instance(f"h{i}", n, n // 2, (-2.0, -0.1 - 0.05 * i), (0.1 + 0.05 * i, 2.0),
                           seed=7100 + i, k=k) for i in range(5)]
    Hs = [torch.from_numpy(x.H) for x in insts]
    H1s = [torch.from_numpy(x.H1) for x in insts]
    if pinned:
        Hs = [h.pin_memory() for h in Hs]
        H1s = [h.pin_memory() for h in H1s]
    P_out = [torch.empty(n, n, dtype=torch.float64) for _ in insts]
    Ps, P1s, infos = ctx.solve_host(Hs, H1s, n // 2, P_out=P_out)
    for i, x in enumerate(insts):
        Pd, P1d, info_d = ctx.sp2_response(torch.from_numpy(x.H).to(DEV),
                                           torch.from_numpy(x.H1).to(DEV), n // 2)
        torch.cuda.synchronize()
        assert torch.equal(P1s[i], P1d.cpu()) and torch.equal(Ps[i], Pd.cpu()), i
        assert infos[i].converged and infos[i].layers == info_d.layers
        for j in range(k):
            _, P1r = oracle.response_sos(x.H, x.H1[j], x.n_occ)
            assert rel(P1s[i][j].numpy(), P1r) < 1e-3


def test_only_upper_triangles_are_read(ctx):
    """The pipeline copies the upper triangles only: NaN in the strict lower
    triangles of the host inputs changes nothing (n = 1100 spans three
    512-row copy blocks and a ragged tail)."""
    n, k = 1100, 2
    x = make_instance("upper", n, n // 2, (-2.0, -0.1), (0.1, 2.0), seed=7300, k=k)
    low = np.tril(np.ones((n, n), dtype=bool), -1)
    Hn = x.H.copy()
    Hn[low] = np.nan
    H1n = x.H1.copy()
    H1n[:, low] = np.nan
    P_out = [torch.empty(n, n, dtype=torch.float64)]
    Ps, P1s, infos = ctx.solve_host([torch.from_numpy(Hn).pin_memory()],
                                    [torch.from_numpy(H1n).pin_memory()], x.n_occ, P_out=P_out)
    Pd, P1d, info_d = ctx.sp2_response(torch.from_numpy(x.H).to(DEV),
                                       torch.from_numpy(x.H1).to(DEV), x.n_occ)
    torch.cuda.synchronize()
    assert infos[0].converged and infos[0].layers == info_d.layers
    assert torch.equal(Ps[0], Pd.cpu()) and torch.equal(P1s[0], P1d.cpu())
    assert ctx.host_copy_in_bytes(n, k) < n * n * 8 * (1 + k)


def test_single_instance_and_trivial(ctx):
    inst = make_workload(2, n=300)
    P, P1, info = ctx.sp2_response_host(torch.from_numpy(inst.H).pin_memory(),
                                        torch.from_numpy(inst.H1).pin_memory(), inst.n_occ)
    assert info.converged
    Pr, P1r = oracle.response_sos(inst.H, inst.H1[0], inst.n_occ)
    assert rel(P1[0].numpy(), P1r) < 1e-3
    assert rel(P.numpy(), Pr) < 1e-3
    # n_occ = 0: P = 0, P1 = 0, no layer
    P0, P10, info0 = ctx.sp2_response_host(torch.from_numpy(inst.H), torch.from_numpy(inst.H1), 0)
    assert info0.converged and info0.layers == 0
    assert not P0.any() and not P10.any()


def test_argument_errors(ctx):
    inst = make_workload(1, n=64)
    H = torch.from_numpy(inst.H)
    with pytest.raises(ValueError):
        ctx.solve_host([H], [torch.from_numpy(inst.H1).float()], inst.n_occ)
    with pytest.raises(dmpt.DmptError) as e:
        ctx.solve_host([H], [torch.from_numpy(inst.H1)], inst.n_occ, order=2)
    assert e.value.status == 1
