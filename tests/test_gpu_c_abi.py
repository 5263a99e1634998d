"""The C ABI from a plain C program (no Python between caller and library).

tests/c_abi/dmpt_host_solve.c is compiled against include/dmpt.h and linked
to the in-tree libdmpt.so and the CUDA runtime; it solves one problem from
host buffers through dmpt_sp2_response_host.  Its P and P1 must equal the
Python binding's device call bit for bit and match the oracle.
"""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2203_09621_gb300.workloads import make_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2203_09621_gb300 import dmpt  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2203_09621_gb300")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    dmpt.load_library()   # the library is built
    exe = str(tmp_path_factory.mktemp("c_abi") / "dmpt_host_solve")
    cmd = [cc, "-O2", "-std=c99", os.path.join(ROOT, "tests", "c_abi", "dmpt_host_solve.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           "-L", PKG, "-ldmpt", "-Wl,-rpath," + PKG,
           "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(CUDA, "lib64"),
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_caller_matches_binding_and_oracle(driver, tmp_path):
    inst = make_workload(2, n=300, k=2)
    n, k = 300, 2
    src = tmp_path / "in.bin"
    dst = tmp_path / "out.bin"
    np.concatenate([inst.H.ravel(), inst.H1.ravel()]).astype(np.float64).tofile(src)
    r = subprocess.run([driver, str(n), str(inst.n_occ), str(k), str(src), str(dst)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    status, layers, d0, conv = map(int, r.stdout.split())
    assert status == 0 and conv == 1
    out = np.fromfile(dst, dtype=np.float64)
    P = out[:n * n].reshape(n, n)
    P1 = out[n * n:].reshape(k, n, n)
    Pb, P1b, info = dmpt.context(0).sp2_response(torch.from_numpy(inst.H).cuda(),
                                                 torch.from_numpy(inst.H1).cuda(), inst.n_occ)
    torch.cuda.synchronize()
    assert info.layers == layers and info.d0_layer == d0
    assert np.array_equal(P, Pb.cpu().numpy()) and np.array_equal(P1, P1b.cpu().numpy())
    for j in range(k):
        _, P1r = oracle.response_sos(inst.H, inst.H1[j], inst.n_occ)
        assert np.linalg.norm(P1[j] - P1r) / np.linalg.norm(P1r) < 1e-3
