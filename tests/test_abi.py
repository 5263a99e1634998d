"""The C ABI library builds, loads without a GPU and exports what dmpt.h declares."""

import ctypes
import os
import re

import numpy as np
import subprocess

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "dmpt.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2203_09621_gb300.build import build_library
    from paper_2203_09621_gb300 import dmpt

    build_library()
    return dmpt.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\*?\s+\**(dmpt_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dmpt_bounds", "dmpt_sp2_response", "dmpt_create", "dmpt_workspace_size"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (dmpt_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_struct_layouts_match_the_header(tmp_path):
    from paper_2203_09621_gb300 import dmpt

    src = tmp_path / "sz.c"
    src.write_text('#include "dmpt.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(dmpt_options), '
                   'sizeof(dmpt_info), offsetof(dmpt_info, sigma), offsetof(dmpt_options, timeout_s));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    so, si, osig, oto = map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split())
    assert so == ctypes.sizeof(dmpt.DmptOptions)
    assert si == ctypes.sizeof(dmpt.DmptInfo)
    assert osig == dmpt.DmptInfo.sigma.offset
    assert oto == dmpt.DmptOptions.timeout_s.offset


def test_host_only_calls(lib):
    from paper_2203_09621_gb300 import dmpt

    o = dmpt.DmptOptions()
    lib.dmpt_default_options(ctypes.byref(o))
    assert (o.precision, o.max_layers, o.c_pt, o.c_d0) == (2, 100, 9.0, 4.5)
    assert lib.dmpt_status_string(0) == b"DMPT_OK"
    # workspace grows with n and k, is 0 for invalid arguments
    w1 = lib.dmpt_workspace_size(1000, 1, ctypes.byref(o))
    w3 = lib.dmpt_workspace_size(1000, 3, ctypes.byref(o))
    assert 0 < w1 < w3
    assert lib.dmpt_workspace_size(0, 1, ctypes.byref(o)) == 0
    assert lib.dmpt_workspace_size(100, -1, ctypes.byref(o)) == 0
    assert lib.dmpt_workspace_size(100, 9, ctypes.byref(o)) == 0
    # k = 0 (P only) is valid and smaller than k = 1
    assert 0 < lib.dmpt_workspace_size(1000, 0, ctypes.byref(o)) < w1
    # the S0 tape (ckpt_every = 1) adds (max_layers + 2) hi/lo states
    t = dmpt.DmptOptions()
    lib.dmpt_default_options(ctypes.byref(t))
    t.ckpt_every = 1
    t.max_layers = 50
    wt = lib.dmpt_workspace_size(1000, 1, ctypes.byref(t))
    assert wt - w1 >= 52 * 2 * 1024 * 1024 * 2
    # checkpoints every k states: (max_layers / k + 1) FP32 masters plus a
    # k-state hi/lo tape for the segment being recomputed
    t.ckpt_every = 8
    wc = lib.dmpt_workspace_size(1000, 1, ctypes.byref(t))
    assert wc - w1 >= (50 // 8 + 1) * 4 * 1024 * 1024 + 8 * 2 * 2 * 1024 * 1024
    assert wc < wt
    t.ckpt_every = 257      # above DMPT_MAX_LAYERS
    assert lib.dmpt_workspace_size(1000, 1, ctypes.byref(t)) == 0
    t.ckpt_every = -1
    assert lib.dmpt_workspace_size(1000, 1, ctypes.byref(t)) == 0
    bad = dmpt.DmptOptions()
    lib.dmpt_default_options(ctypes.byref(bad))
    bad.precision = 9
    assert lib.dmpt_workspace_size(100, 1, ctypes.byref(bad)) == 0
    # n = 8192, k = 3, dual: 2 x 4 FP32 masters + 2 x 4 x 2 16-bit halves of 8192^2
    big = lib.dmpt_workspace_size(8192, 3, ctypes.byref(o))
    assert big >= (2 * 4 * 4 + 2 * 4 * 2 * 2) * 8192 * 8192
    # null handle / null pointer paths need no device
    assert lib.dmpt_sp2_response(None, None, None, 1, 4, 4, 2, None, None, None, None, None, 0,
                                 None) == 1
    assert lib.dmpt_destroy(None) == 1


def test_higher_order_workspace_and_options(lib):
    """Responses of order m keep m k response slots (m k <= DMPT_MAX_K = 8,
    m <= DMPT_MAX_ORDER = 8); round_align defaults to 1 and takes 0 or 1."""
    from paper_2203_09621_gb300 import dmpt

    o = dmpt.DmptOptions()
    lib.dmpt_default_options(ctypes.byref(o))
    assert o.round_align == 1 and o.order == 1
    w = {}
    for m, k in ((1, 1), (2, 1), (4, 1), (8, 1), (2, 4), (4, 2)):
        o.order = m
        w[(m, k)] = lib.dmpt_workspace_size(1000, k, ctypes.byref(o))
        assert w[(m, k)] > 0, (m, k)
    assert w[(1, 1)] < w[(2, 1)] < w[(4, 1)] < w[(8, 1)]
    assert w[(2, 4)] == w[(8, 1)] == w[(4, 2)]      # the same 8 slots
    for m, k in ((3, 3), (9, 1), (2, 5), (0, 1), (2, 0)):
        o.order = m
        assert lib.dmpt_workspace_size(1000, k, ctypes.byref(o)) == 0, (m, k)
    o.order = 1
    for v, ok in ((0, True), (1, True), (2, False), (-1, False)):
        o.round_align = v
        assert (lib.dmpt_workspace_size(100, 1, ctypes.byref(o)) > 0) == ok, v
    # null handle
    assert lib.dmpt_sp2_response_m(None, None, None, 1, 4, 4, 2, 3, None, None, None, None,
                                   None, None, 0, None) == 1


def test_host_pipeline_sizes_and_argument_errors(lib):
    """dmpt_sp2_response_host: the workspace is the solver's plus two input
    and two output buffer sets of (1 + k) n x n float64; argument errors are
    reported before any device work."""
    from paper_2203_09621_gb300 import dmpt

    o = dmpt.DmptOptions()
    lib.dmpt_default_options(ctypes.byref(o))
    for n, k in ((1000, 1), (8192, 3), (300, 0)):
        ws = lib.dmpt_workspace_size(n, k, ctypes.byref(o))
        io = -(-(n * n * 8 * (1 + k)) // 256) * 256
        assert lib.dmpt_workspace_size_host(n, k, ctypes.byref(o)) == -(-ws // 256) * 256 + 4 * io
    assert lib.dmpt_workspace_size_host(0, 1, ctypes.byref(o)) == 0
    assert lib.dmpt_workspace_size_host(100, 9, ctypes.byref(o)) == 0
    # the copy-in moves the upper triangles in row blocks of 512 rows
    lib.dmpt_host_copy_in_bytes.restype = ctypes.c_size_t
    lib.dmpt_host_copy_in_bytes.argtypes = [ctypes.c_int64, ctypes.c_int]
    for n, k in ((1000, 1), (8192, 3), (300, 0), (512, 2), (513, 2)):
        want = sum(min(512, n - r0) * (n - r0) * 8 for r0 in range(0, n, 512)) * (1 + k)
        got = lib.dmpt_host_copy_in_bytes(n, k)
        assert got == want, (n, k, got, want)
        assert n <= 512 or got < n * n * 8 * (1 + k)
    assert lib.dmpt_host_copy_in_bytes(8192, 3) == 4 * 8192 * 8704 * 4
    assert lib.dmpt_host_copy_in_bytes(0, 1) == 0 and lib.dmpt_host_copy_in_bytes(10, 9) == 0
    # null handle
    assert lib.dmpt_sp2_response_host(None, 1, None, None, 1, 4, 2, None, None, None, None,
                                      None, 0, None) == 1


def test_c_caller_builds_and_reports_missing_gpu(lib, tmp_path):
    """The plain-C caller (tests/c_abi/dmpt_host_solve.c) compiles against
    include/dmpt.h and links to the in-tree library; without a GPU,
    dmpt_create returns a status and the program exits 1 with a message."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if cc is None or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("no C compiler or CUDA headers")
    pkg = os.path.join(ROOT, "paper_2203_09621_gb300")
    exe = str(tmp_path / "dmpt_host_solve")
    r = subprocess.run([cc, "-O2", "-std=c99", os.path.join(ROOT, "tests", "c_abi", "dmpt_host_solve.c"),
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                        "-L", pkg, "-ldmpt", "-Wl,-rpath," + pkg,
                        "-L", os.path.join(cuda, "lib64"), "-lcudart",
                        "-Wl,-rpath," + os.path.join(cuda, "lib64"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present: tests/test_gpu_c_abi.py runs the program")
    except ImportError:
        pass
    src = tmp_path / "in.bin"
    np.zeros(2 * 16, dtype=np.float64).tofile(src)
    r = subprocess.run([exe, "4", "2", "1", str(src), str(tmp_path / "out.bin")],
                       capture_output=True, text=True, timeout=60)
    assert r.returncode == 1 and "dmpt_create" in r.stderr, (r.returncode, r.stderr)


def test_timeout_must_be_finite_and_capped(lib):
    """timeout_s bounds every device-side wait; it is converted to
    nanoseconds in 64 bits on the device, so inf, NaN and values above
    DMPT_MAX_TIMEOUT_S are rejected before any launch."""
    from paper_2203_09621_gb300 import dmpt

    text = open(HEADER).read()
    cap = float(re.search(r"#define DMPT_MAX_TIMEOUT_S ([0-9.]+)", text).group(1))
    o = dmpt.DmptOptions()
    lib.dmpt_default_options(ctypes.byref(o))
    for v, ok in ((2.0, True), (cap, True), (1e-3, True), (cap * 1.01, False),
                  (float("inf"), False), (float("nan"), False), (1.8e10, False), (0.0, False),
                  (-1.0, False)):
        o.timeout_s = v
        assert (lib.dmpt_workspace_size(100, 1, ctypes.byref(o)) > 0) == ok, v


def test_info_carries_stopping_histories():
    """dmpt_info exposes the per-layer quantities the stopping rules test, so
    a caller can re-check each decision (Alg. 1-3)."""
    from paper_2203_09621_gb300 import dmpt

    names = [f[0] for f in dmpt.DmptInfo._fields_]
    for f in ("n_s", "n_x", "iderr", "froerr1_hist"):
        assert f in names
    assert dmpt.DmptInfo.froerr1_hist.size == 8 * dmpt.DMPT_MAX_K * dmpt.DMPT_MAX_LAYERS
