"""Benchmark: converged-P1 TFLOP/s and time-to-solution of DNN-SP2-PT.

Workload: n = 8192, n_occ = 4096, gapped spectrum (occupied U[-2, -0.1],
virtual U[0.1, 2]), three dipole-like perturbations diag(x_k) + 0.001
sym-Gauss sharing one S_0 recursion, dual-FP16 tensor-core products
(synthetic stand-in for the paper's water systems; seeded, generated on
the device).

One step = one full dmpt_sp2_response call: Gershgorin bounds, initial
layer, every SP2 layer with its response until the Alg. 2 / Alg. 3
criteria fire, and the FP64 outputs P and P1 -- with H and H1 resident in
HBM.  value = algorithmic flops of the converged solve ((2 + 3K) 2n^3 per
D0 layer, 3K 2n^3 per D1-only layer) / device time per step.  The inputs
(2 GiB) exceed L2, so no flush is needed between steps.

`e2e` times the C ABI's host-buffer entry point (dmpt_sp2_response_host) on
`steps` instances in pinned host memory: every step's copy-in of H and H1 and
copy-out of P1 are inside the timed region, overlapped with the neighbouring
steps' solves.  `roofline` reports the layer-product
kernel against the measured dense 16-bit tensor peak.  `cpu_baseline`
times the FP64 oracle (numpy) on the host on a bounded sample.

--impl reference times the FP64 CPU oracle as the reference arm.
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged-P1 TFLOP/s and time-to-solution at N=8192, dual-FP16 vs FP32 vs FP64"
N_DEFAULT = 8192
K_DEFAULT = 3

# DRAM traffic of the layer-product kernel, averaged over the 41 layer launches
# of one timed solve of the default workload (ncu dram__bytes_read.sum +
# dram__bytes_write.sum, 1-pass capture; profiles/layer_tc2_kernel_dipole3_
# n8192_k3_dram.md).  Valid only for that kernel source and that workload.
TRAFFIC_RECORD = {
    "source": "paper_2203_09621_gb300/csrc/kernels_tc.cu",
    "sha256": "2fbf3b6c3790a556bc0eefccba34a722af386f17f0221acce63cadb195c2ce36",
    "workload": {"n": 8192, "k": 3, "precision": "dual_fp16", "cta_pair": 1, "k_snake": 1,
                 "tile_band": 8, "accum_chunk": 0},
    "bytes_per_launch": 9.7699e9 + 1.5409e9,
}


def recorded_traffic(workload):
    """Bytes per launch from the ncu record, or None once the kernel or the workload differs."""
    import hashlib
    path = os.path.join(ROOT, TRAFFIC_RECORD["source"])
    try:
        with open(path, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    if sha != TRAFFIC_RECORD["sha256"] or workload != TRAFFIC_RECORD["workload"]:
        return None
    return TRAFFIC_RECORD["bytes_per_launch"]


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            try:
                pw.append(float(parts[3]))
            except ValueError:
                pass
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm_sorted = sorted(sm)
        pw_sorted = sorted(pw)
        return {"sm_mhz": sm_sorted[len(sm_sorted) // 2], "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w": pw_sorted[len(pw_sorted) // 2] if pw_sorted else None}


def measure_matmul_peaks(n, dev, dtype_name, sustained_s=4.0, best_of=10):
    """torch.matmul n^3 (2 n^3 flops) in `dtype_name`: best of `best_of` single
    products (burst) and the mean rate of back-to-back products for about
    `sustained_s` seconds (sustained, under the power cap)."""
    import torch
    dt = {"fp16": torch.float16, "bf16": torch.bfloat16, "fp64": torch.float64}[dtype_name]
    a = torch.randn(n, n, device=dev).to(dt)
    b = torch.randn(n, n, device=dev).to(dt)
    for _ in range(3):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(best_of):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    flops = 2.0 * n ** 3
    out = {"burst_tflops": flops / (best * 1e-3) / 1e12}
    if sustained_s > 0:
        reps = max(1, int(sustained_s / (best * 1e-3)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        out["sustained_tflops"] = reps * flops / (e0.elapsed_time(e1) * 1e-3) / 1e12
        out["sustained_reps"] = reps
    out["how"] = (f"torch.matmul {dtype_name} {n}^3 (2 n^3 flops): best of {best_of} (burst)"
                  + (f", {out.get('sustained_reps')} back to back (sustained)" if sustained_s > 0 else ""))
    del a, b
    return out


def measure_copy_bandwidth(host, dev_t, stream, reps=5):
    """Pinned host <-> device copy rates (GB/s) of one tensor each way: the
    median and the slowest of `reps` copies after a warm-up copy."""
    import torch
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    dev_t.copy_(host, non_blocking=True)
    host.copy_(dev_t, non_blocking=True)
    torch.cuda.synchronize()
    nb = host.numel() * host.element_size()
    h2d, d2h = [], []
    for _ in range(reps):
        e0.record(stream)
        dev_t.copy_(host, non_blocking=True)
        e1.record(stream)
        host.copy_(dev_t, non_blocking=True)
        e2.record(stream)
        torch.cuda.synchronize()
        h2d.append(nb / (e0.elapsed_time(e1) * 1e-3) / 1e9)
        d2h.append(nb / (e1.elapsed_time(e2) * 1e-3) / 1e9)
    h2d.sort()
    d2h.sort()
    return h2d[reps // 2], d2h[reps // 2], h2d[0], d2h[0]


INPUT_BACKEND = "torch"


def make_inputs(n, k, device):
    """The workload's matrices on `device` (torch: built on the device;
    numpy: built on the host and copied, used where torch.linalg is not
    loadable, e.g. under a profiler)."""
    from paper_2203_09621_gb300.workloads import make_workload
    if INPUT_BACKEND == "numpy":
        import torch
        inst = make_workload(3, n=n, k=k)
        inst.H = torch.from_numpy(inst.H).to(device)
        inst.H1 = torch.from_numpy(inst.H1).to(device)
        inst.eps = torch.from_numpy(inst.eps)
        inst.Q = torch.from_numpy(inst.Q)
        return inst
    return make_workload(3, n=n, k=k, backend="torch", device=device)


def oracle_sample(inst_cpu_H, inst_cpu_H1, n_occ, layers):
    """FP64 oracle on the host: the first `layers` layers of Alg. 1-3."""
    import numpy as np
    import oracle
    t = time.perf_counter()
    oracle.sp2_pt(inst_cpu_H, inst_cpu_H1, n_occ, max_layers=layers)
    return time.perf_counter() - t


_ONE_CORE_SNIPPET = """
import sys, time
sys.path.insert(0, {root!r})
import oracle
from paper_2203_09621_gb300.workloads import make_workload
inst = make_workload(3, n={n}, k={k})
t = time.perf_counter()
oracle.sp2_pt(inst.H, inst.H1, inst.n_occ, max_layers=1)
print(time.perf_counter() - t)
"""


def cpu_oracle_extra(k, n_small=2048):
    """The oracle on one host core (a child process with the BLAS thread pools
    set to 1) on one layer at n = n_small, and the sum-over-states oracle
    (eigh + Daleckii-Krein transforms) on all cores at the same size."""
    import numpy as np
    import oracle
    from paper_2203_09621_gb300.workloads import make_workload
    out = {}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", _ONE_CORE_SNIPPET.format(root=ROOT, n=n_small, k=k)],
                           capture_output=True, text=True, env=env, timeout=300)
        t1 = float(r.stdout.strip().splitlines()[-1])
        out["one_core"] = {"value": alg_flops_layers(n_small, k, 1) / t1 / 1e12, "unit": "TFLOP/s",
                           "cores": 1, "sample": f"first layer of Alg. 1-3 at n={n_small}, k={k} "
                                                 f"({t1:.1f} s)"}
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        out["one_core"] = {"unavailable": f"{type(e).__name__}"}
    inst = make_workload(3, n=n_small, k=k)
    t = time.perf_counter()
    oracle.response_sos(inst.H, inst.H1, inst.n_occ)
    t = time.perf_counter() - t
    out["sum_over_states"] = {"seconds": t, "cores": cpu_cores(),
                              "sample": f"eigh + {k} Daleckii-Krein transforms at n={n_small}"}
    return out


def alg_flops_layers(n, k, layers):
    # D0-phase layers: square (2 products) + 3 products per direction
    return layers * (2 + 3 * k) * 2.0 * float(n) ** 3


def aggregate(ms_local, units_local, world):
    """Whole-job rate over replicas: max step time over ranks, units summed.

    Each rank solves its own replica of the workload (the path shards only
    as independent problems), so the job processes world * units per step in
    the time of the slowest rank.  Returns (ms_max, value in units / s).
    """
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64)
    u = torch.tensor([float(units_local)], dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        dev = torch.device("cuda", torch.cuda.current_device()) \
            if dist.get_backend() == "nccl" else torch.device("cpu")
        t, u = t.to(dev), u.to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    return ms_max, float(u.item()) / (ms_max * 1e-3)


def cpu_cores():
    try:
        import numpy as np  # noqa
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count()
    return n


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on a bounded sample."""
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            dist.destroy_process_group()
            return
    import numpy as np
    from paper_2203_09621_gb300.workloads import make_workload
    n, k = args.oracle_n, args.k
    layers = args.oracle_layers
    # bounded sample: the first `layers` layers of the same recipe at
    # n = --oracle-n, generated on the device when one is available (host QR
    # at full size alone takes minutes), else on the host
    try:
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
    except ImportError:
        dev = "cpu"
    if dev == "cuda":
        inst = make_inputs(n, k, "cuda")
        H = inst.H.cpu().numpy()
        H1 = inst.H1.cpu().numpy()
    else:
        inst = make_workload(3, n=n, k=k)
        H, H1 = inst.H, inst.H1
    for _ in range(args.warmup):
        oracle_sample(H, H1, n // 2, layers)
    times = [oracle_sample(H, H1, n // 2, layers) for _ in range(args.steps)]
    t = sum(times) / len(times)
    flops = alg_flops_layers(n, k, layers)
    val = flops / t / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"dipole3 n={args.n} k={k} n_occ={args.n // 2}; FP64 oracle "
                               f"(numpy, Algorithms 1-3) sampled: first {layers} layer(s) "
                               f"at n={n} per step"},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cpu_cores(),
                         "kind": "oracle",
                         "sample": f"first {layers} layer(s) of Alg. 1-3 on the same recipe "
                                   f"at n={n}, k={k} per step"},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--k", type=int, default=K_DEFAULT)
    ap.add_argument("--precision", default="dual_fp16")
    ap.add_argument("--forms", default="fp32,dual_bf16,fp64",
                    help="extra precision forms timed once to convergence (comma list); fp64 on "
                         "a bounded sample unless --fp64-full")
    ap.add_argument("--fp64-layers", type=int, default=2,
                    help="layers of the FP64 form timed (its full solve takes minutes at n = 8192)")
    ap.add_argument("--fp64-full", action="store_true",
                    help="run the FP64 form to convergence (about two minutes at n = 8192)")
    ap.add_argument("--paper-sizes", action="store_true",
                    help="also solve the paper's Fig. 4 sizes (n = 5904 ... 19008, n_occ = 2n/3, "
                         "K = 1) once each, as context beside its A100 figures")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip measuring the FP16 / FP64 matmul peaks used as denominators")
    ap.add_argument("--oracle-layers", type=int, default=1)
    ap.add_argument("--oracle-n", type=int, default=4096,
                    help="size of the bounded oracle sample (same recipe)")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--accum-chunk", type=int, default=0)
    ap.add_argument("--input-backend", default="torch", choices=["torch", "numpy"])
    ap.add_argument("--cta-pair", type=int, default=1, choices=[0, 1])
    ap.add_argument("--k-snake", type=int, default=1, choices=[0, 1])
    ap.add_argument("--tile-band", type=int, default=8)
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip reporting the autotuner's choice for the workload")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the uneven-batch measurement (64 instances, n in [256, 2048])")
    ap.add_argument("--no-scc", action="store_true",
                    help="skip the self-consistent response measurement (same workload + tape)")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint measurement (n=4096 forward with tape + backward)")
    args = ap.parse_args()
    global INPUT_BACKEND
    INPUT_BACKEND = args.input_backend
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    from paper_2203_09621_gb300 import dmpt

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    n, k = args.n, args.k
    inst = make_inputs(n, k, dev)
    H, H1 = inst.H.contiguous(), inst.H1.contiguous()
    ctx = dmpt.Context(local)
    P = torch.empty(n, n, dtype=torch.float64, device=dev)
    P1 = torch.empty(k, n, n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    kw = dict(precision=args.precision, out=(P, P1), stream=stream,
              accum_chunk=args.accum_chunk, cta_pair=args.cta_pair, k_snake=args.k_snake,
              tile_band=args.tile_band)

    # warm-up (also sizes the workspace)
    for _ in range(args.warmup):
        ctx.sp2_response(H, H1, inst.n_occ, **kw)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---- timed: device-resident inputs
    infos = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            _, _, info = ctx.sp2_response(H, H1, inst.n_occ, **kw)
            infos.append(info)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    clocks = clk.summary()
    alg = sum(i.alg_flops for i in infos) / len(infos)
    ms_max, rate = aggregate(ms, alg, world)
    value = rate / 1e12

    # ---- e2e: the C ABI's host-buffer entry point (dmpt_sp2_response_host),
    #      measured right after the resident steps, before the tuning and peak
    #      measurements heat the part;
    #      copies of every step's inputs and of its P1 inside the timed region
    Hh = H.cpu().pin_memory()
    H1h = H1.cpu().pin_memory()
    P1h = [torch.empty(k, n, n, dtype=torch.float64).pin_memory() for _ in range(2)]
    kwh = {key: v for key, v in kw.items() if key != "out"}
    e_steps = max(1, args.steps)
    # untimed warm-up: one pass of the same pipeline, which sizes the buffers
    # and makes the first copies to and from every pinned host buffer (on these
    # hosts a buffer's first transfers can run at a tenth of the link rate)
    ctx.solve_host([Hh] * e_steps, [H1h] * e_steps, inst.n_occ,
                   P1_out=[P1h[i % 2] for i in range(e_steps)], **kwh)
    # the host link just before the timed steps (it is measured again after them)
    Htmp = torch.empty_like(H)
    link_before = measure_copy_bandwidth(Hh, Htmp, stream)
    del Htmp
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    _, P1e, _ = ctx.solve_host([Hh] * e_steps, [H1h] * e_steps, inst.n_occ,
                               P1_out=[P1h[i % 2] for i in range(e_steps)], **kwh)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms, e2e_rate = aggregate(e0.elapsed_time(e1) / e_steps, alg, world)
    e2e_val = e2e_rate / 1e12
    e2e_same = bool(torch.equal(P1e[-1], P1.cpu()))
    h2d = ctx.host_copy_in_bytes(n, k)   # the upper triangles of H and H1
    d2h = P1.numel() * 8
    # the host link, measured alone: what the copies of one step cost if
    # nothing overlapped them, against the step's exposed extra time
    Htmp = torch.empty_like(H)
    h2d_gbs, d2h_gbs, h2d_min, d2h_min = measure_copy_bandwidth(Hh, Htmp, stream)
    del Htmp
    copy_ms_serial = (h2d / (h2d_gbs * 1e9) + d2h / (d2h_gbs * 1e9)) * 1e3
    # the same pipeline once more with per-launch timing of the layer products
    # (outside the timed region): their device time per instance while the
    # copies of the neighbouring instances run, against the resident solve's
    _, _, hinfos = ctx.solve_host([Hh] * e_steps, [H1h] * e_steps, inst.n_occ,
                                  P1_out=[P1h[i % 2] for i in range(e_steps)], timing=True, **kwh)
    torch.cuda.synchronize()
    kernel_ms_pipeline = sum(i.ms_layers for i in hinfos) / len(hinfos)

    # ---- the autotuner's choice for this workload (reported, not used by the
    #      timed steps, whose configuration is the one in `config`)
    tune = None
    if not args.no_autotune:
        tctx = dmpt.Context(local)
        choice, tms = tctx.autotune(H, H1, inst.n_occ, precision=args.precision,
                                    accum_chunk=args.accum_chunk, k_snake=args.k_snake)
        tune = {"choice": choice, "ms_per_layer": tms,
                "candidates": "cta_pair 1 x tile_band {8, 0, 4, 16}, cta_pair 0 (128 x 256 tiles)"}
        del tctx
        torch.cuda.synchronize()

    # ---- per-launch timing of the layer products (CUDA events on the stream)
    _, _, tinfo = ctx.sp2_response(H, H1, inst.n_occ, timing=True, **kw)
    torch.cuda.synchronize()
    peaks, peak_src = load_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    peak_source = f"{peak_src} bf16_tflops_sustained (FP16 dense = BF16 dense)"
    measured_peaks = None
    if not args.no_peaks:
        # the products run in FP16: measure the dense FP16 rate (cuBLAS through
        # torch.matmul, 8192^3) as the denominator, sustained like the layer
        # kernel inside a seconds-long solve; FP64 as context for the FP64 form
        measured_peaks = {"fp16": measure_matmul_peaks(8192, dev, "fp16"),
                          "fp64": measure_matmul_peaks(min(n, 8192), dev, "fp64",
                                                       sustained_s=0.0, best_of=3)}
        if args.precision == "dual_fp16":
            peak = measured_peaks["fp16"]["sustained_tflops"]
            peak_source = ("measured in this run: torch.matmul fp16 8192^3 back to back "
                           "(sustained); burst (best of 10) in measured_peaks")
        elif args.precision == "dual_bf16":
            measured_peaks["bf16"] = measure_matmul_peaks(8192, dev, "bf16")
            peak = measured_peaks["bf16"]["sustained_tflops"]
            peak_source = "measured in this run: torch.matmul bf16 8192^3 back to back (sustained)"
    achieved = tinfo.alg_flops / (tinfo.ms_layers * 1e-3) / 1e12 if tinfo.ms_layers else None
    executed = tinfo.mma_flops / (tinfo.ms_layers * 1e-3) / 1e12 if tinfo.ms_layers else None

    # ---- other precision forms, one timed solve each (time-to-solution)
    forms = {}
    form_results = {}      # precision -> (P, P1) on the host, for the accuracy check
    for f in [x for x in args.forms.split(",") if x and x != "fp64"]:
        kwf = dict(kw, precision=f)
        ctx.sp2_response(H, H1, inst.n_occ, **kwf)  # warm-up
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, _, fi = ctx.sp2_response(H, H1, inst.n_occ, **kwf)
        b.record(stream)
        torch.cuda.synchronize()
        fms = a.elapsed_time(b)
        forms[f] = {"ms": fms, "tflops": fi.alg_flops / (fms * 1e-3) / 1e12,
                    "layers": fi.layers, "d0_layer": fi.d0_layer, "converged": fi.converged}
        if not args.no_check and rank == 0:
            form_results[f] = (P.cpu().numpy(), P1.cpu().numpy())
    if "fp32" in forms:
        # context only: cuBLAS SGEMM (TF32 off) at the same n, one product
        # (2 n^3 flops), beside the SIMT form's per-layer rate
        prev_tf32 = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        a32 = torch.randn(n, n, dtype=torch.float32, device=dev)
        b32 = torch.randn(n, n, dtype=torch.float32, device=dev)
        for _ in range(2):
            torch.matmul(a32, b32)
        torch.cuda.synchronize()
        ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ga.record(stream)
        for _ in range(3):
            torch.matmul(a32, b32)
        gb.record(stream)
        torch.cuda.synchronize()
        torch.backends.cuda.matmul.allow_tf32 = prev_tf32
        forms["fp32"]["cublas_sgemm_tflops"] = 3 * 2.0 * n ** 3 / (ga.elapsed_time(gb) * 1e-3) / 1e12
        del a32, b32
    if "fp64" in args.forms.split(",") and args.fp64_full:
        # the FP64 form to convergence (time to solution and accuracy)
        kwf = dict(kw, precision="fp64")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, _, fi = ctx.sp2_response(H, H1, inst.n_occ, **kwf)
        b.record(stream)
        torch.cuda.synchronize()
        fms = a.elapsed_time(b)
        forms["fp64"] = {"ms": fms, "tflops": fi.alg_flops / (fms * 1e-3) / 1e12,
                         "layers": fi.layers, "d0_layer": fi.d0_layer,
                         "converged": fi.converged, "sample": "full solve"}
        if not args.no_check and rank == 0:
            form_results["fp64"] = (P.cpu().numpy(), P1.cpu().numpy())
    elif "fp64" in args.forms.split(",") and args.fp64_layers > 0:
        # bounded sample: the first layers of the FP64 form (each a full D0
        # layer), per-launch times by CUDA events; the time to solution is
        # extrapolated to the dual form's layer count
        kwf = dict(kw, precision="fp64", max_layers=args.fp64_layers, timing=True)
        _, _, fi = ctx.sp2_response(H, H1, inst.n_occ, raise_on_error=False, **kwf)
        torch.cuda.synchronize()
        per_layer = fi.ms_layers / max(1, fi.timed_launches)
        lay = infos[0].layers
        forms["fp64"] = {"ms_per_layer": per_layer, "layers_timed": fi.timed_launches,
                         "tflops": fi.alg_flops / (fi.ms_layers * 1e-3) / 1e12 if fi.ms_layers else None,
                         "estimated_ms": per_layer * lay, "estimated_for_layers": lay,
                         "sample": f"first {fi.timed_launches} layer(s) of the FP64 form at n={n}, "
                                   f"k={k}; estimated_ms = time per layer x the dual form's layer "
                                   f"count (an estimate, not a measured solve)"}
    # restore the dual-FP16 result in P1 for the accuracy check
    _, _, info = ctx.sp2_response(H, H1, inst.n_occ, **kw)
    torch.cuda.synchronize()

    # ---- self-consistent response on the same workload: forward with the S0
    #      tape, then H1 <- H1_ext + diag(gamma diag(P1)) by response replays
    scc = None
    if not args.no_scc and rank == 0:
        from paper_2203_09621_gb300.workloads import scc_gamma
        gam = scc_gamma(n, backend="torch", device=dev)
        sopts = dmpt.options(precision=args.precision, ckpt_every=1, max_layers=64)
        sws = torch.empty(ctx.workspace_size(n, k, sopts) + 256, dtype=torch.uint8, device=dev)
        s0, s1, s2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        s0.record(stream)
        ctx.sp2_response(H, H1, inst.n_occ, precision=args.precision, ckpt_every=1,
                         max_layers=64, workspace=sws, out=(P, P1))
        s1.record(stream)
        P1s, its, res, sinfo = ctx.scc_response(H1, gam, sws, tol=1e-5, max_iter=50,
                                                precision=args.precision)
        s2.record(stream)
        torch.cuda.synchronize()
        scc_ms = s1.elapsed_time(s2)
        scc = {"workload": f"dipole3 n={n} k={k} + gamma_ij = (40/n)/sqrt(r^2+1)",
               "iterations": its, "residual": res, "forward_with_tape_ms": s0.elapsed_time(s1),
               "scc_ms": scc_ms, "ms_per_iteration": scc_ms / max(its, 1),
               "replay_tflops": sinfo.alg_flops / (scc_ms * 1e-3) / 1e12}
        del sws, P1s

    # ---- uneven batch: 64 independent instances, n log-uniform in [256, 2048]
    batch = None
    if not args.no_batch and rank == 0:
        from paper_2203_09621_gb300.workloads import uneven_batch
        binst = uneven_batch(backend="torch", device=dev)
        bH = [x.H for x in binst]
        bH1 = [x.H1 for x in binst]
        bocc = [x.n_occ for x in binst]
        for _ in range(2):
            ctx.sp2_response_batch(bH, bH1, bocc, precision=args.precision)
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        _, _, binfos = ctx.sp2_response_batch(bH, bH1, bocc, precision=args.precision)
        b1.record(stream)
        torch.cuda.synchronize()
        bms = b0.elapsed_time(b1)
        balg = sum(i.alg_flops for i in binfos)
        # the same instances one call after another
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for x_h, x_h1, x_o in zip(bH, bH1, bocc):
            ctx.sp2_response(x_h, x_h1, x_o, precision=args.precision)
        q1.record(stream)
        torch.cuda.synchronize()
        sms_ = q0.elapsed_time(q1)
        batch = {"workload": "64 instances, n log-uniform in [256, 2048], n_occ = n/2, "
                             "gap U[0.1, 0.5], k = 1",
                 "ms": bms, "tflops": balg / (bms * 1e-3) / 1e12,
                 "sequential_ms": sms_, "speedup_vs_sequential": sms_ / bms,
                 "converged": int(sum(i.converged for i in binfos))}
        # autotuned batch: the first call times the grouped and per-instance
        # paths on a short probe and keeps the faster; the timed call reuses it
        ctx.sp2_response_batch(bH, bH1, bocc, precision=args.precision, autotune=1)
        torch.cuda.synchronize()
        b0.record(stream)
        ctx.sp2_response_batch(bH, bH1, bocc, precision=args.precision, autotune=1)
        b1.record(stream)
        torch.cuda.synchronize()
        batch["autotuned_ms"] = b0.elapsed_time(b1)
        del binst, bH, bH1

    # ---- adjoint (L = Tr[G P]): n = 4096 forward keeping the S0 states, then
    #      the backward; with the full tape (ckpt_every = 1) and with a
    #      checkpoint every 8 states (ckpt_every = 8, segments recomputed)
    adjoint = None
    if not args.no_adjoint and rank == 0:
        from paper_2203_09621_gb300.workloads import make_workload
        a_inst = make_workload(4, backend="torch", device=dev)
        Ga = a_inst.H1[0]
        na = float(a_inst.n)
        P1G = None
        if not args.no_check:
            from oracle.sos import response_from_eigs
            _, P1G = response_from_eigs(a_inst.eps.cpu().numpy(), a_inst.Q.cpu().numpy(),
                                        Ga.cpu().numpy(), a_inst.n_occ)
        adjoint = {"workload": f"adjoint n={a_inst.n} (L = Tr[G P], G sym-Gauss)"}
        for ck in (1, 8):
            aopts = dmpt.options(precision=args.precision, ckpt_every=ck)
            ws_bytes = ctx.workspace_size(a_inst.n, 0, aopts)
            aws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
            for _ in range(2):  # warm-up
                ctx.sp2_response(a_inst.H, None, a_inst.n_occ, precision=args.precision,
                                 ckpt_every=ck, workspace=aws)
                ctx.sp2_backward(Ga, aws)
            torch.cuda.synchronize()
            t0, t1, t2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            t0.record(stream)
            _, _, ainfo = ctx.sp2_response(a_inst.H, None, a_inst.n_occ,
                                           precision=args.precision, ckpt_every=ck,
                                           workspace=aws)
            t1.record(stream)
            dLdH = ctx.sp2_backward(Ga, aws)
            t2.record(stream)
            torch.cuda.synchronize()
            U = ainfo.d0_layer - 1
            f_bwd = U * 3 * 2 * na ** 3       # one dual response product per adjoint layer
            rec = {"workspace_bytes": ws_bytes,
                   "state_bytes": (U + 1) * 4 * int(na) ** 2 if ck == 1 else
                   ((U // ck + 1) * 4 + ck * 4) * int(na) ** 2,
                   "forward_ms": t0.elapsed_time(t1), "backward_ms": t1.elapsed_time(t2),
                   "backward_tflops": f_bwd / (t1.elapsed_time(t2) * 1e-3) / 1e12,
                   "forward_tflops": ainfo.alg_flops / (t0.elapsed_time(t1) * 1e-3) / 1e12,
                   "adjoint_layers": U,
                   "recomputed_squares": 0 if ck == 1 else U - (U - 1) // ck - 1}
            if P1G is not None:
                g = dLdH.cpu().numpy()
                rec["rel_err_vs_oracle"] = float(np.linalg.norm(g - P1G) / np.linalg.norm(P1G))
            adjoint["full_tape" if ck == 1 else f"checkpoint_every_{ck}"] = rec
            del aws, dLdH
        del a_inst

    # ---- the paper's Fig. 4 sizes (context): n_occ = 2n/3 as in its water
    #      boxes, one perturbation, gap 0.2; one solve each after one warm-up
    paper_sizes = None
    if args.paper_sizes and rank == 0:
        from paper_2203_09621_gb300.workloads import make_instance
        from oracle.sos import response_columns
        # the paper's dual-FP16 rates on one A100, converted to 2 flops per FMA
        a100 = {5904: 158.4, 10266: 172.2, 12720: 178.0, 16512: 197.2, 19008: 238.0}
        paper_sizes = []
        for npap, ref in a100.items():
            pi = make_instance(f"paper-n{npap}", npap, round(2 * npap / 3), (-2.0, -0.1),
                               (0.1, 2.0), "gauss", 1, 0.01, seed=7000 + npap,
                               backend="torch", device=dev)
            ctx.sp2_response(pi.H, pi.H1, pi.n_occ, precision=args.precision)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            Pp, P1p, pinf = ctx.sp2_response(pi.H, pi.H1, pi.n_occ, precision=args.precision)
            b.record(stream)
            torch.cuda.synchronize()
            pms = a.elapsed_time(b)
            rec = {"n": npap, "n_occ": pi.n_occ, "ms": pms, "layers": pinf.layers,
                   "d0_layer": pinf.d0_layer, "hole_form": pinf.hole,
                   "tflops": pinf.alg_flops / (pms * 1e-3) / 1e12,
                   "paper_1xA100_tflops_2_per_fma": ref}
            if not args.no_check:
                cols = [0, 1, pi.n_occ - 1, pi.n_occ, npap - 1]
                want = response_columns(pi.eps.cpu().numpy(), pi.Q.cpu().numpy(),
                                        pi.H1[0].cpu().numpy(), pi.n_occ, cols)
                got = P1p[0][:, cols].cpu().numpy()
                rec["rel_err_P1_sampled_columns"] = float(np.linalg.norm(got - want) /
                                                          np.linalg.norm(want))
            paper_sizes.append(rec)
            del pi, Pp, P1p
        torch.cuda.empty_cache()

    # ---- accuracy against the oracle: the whole P and every P1_k, from the
    #      known eigenpairs (outside every timed region)
    accuracy = None
    if not args.no_check and rank == 0:
        import oracle
        from oracle.sos import response_columns
        t_or = time.perf_counter()
        eps = inst.eps.cpu().numpy()
        Q = inst.Q.cpu().numpy()
        Pr = oracle.density_from_eigs(eps, Q, inst.n_occ)
        P1r = [response_columns(eps, Q, H1[j].cpu().numpy(), inst.n_occ, np.arange(n))
               for j in range(k)]
        t_or = time.perf_counter() - t_or

        def errs(Pg, P1g):
            return {"rel_err_P": float(np.linalg.norm(Pg - Pr) / np.linalg.norm(Pr)),
                    "rel_err_P1_max_k": max(float(np.linalg.norm(P1g[j] - P1r[j]) /
                                                  np.linalg.norm(P1r[j])) for j in range(k))}
        accuracy = dict(errs(P.cpu().numpy(), P1.cpu().numpy()), precision=args.precision,
                        norm="relative Frobenius, whole matrices", oracle_s=t_or)
        for f, (Pg, P1g) in form_results.items():
            forms[f].update(errs(Pg, P1g))
        del Pr, P1r, form_results

    # ---- CPU baseline: FP64 oracle, first layer(s) of the same workload
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ns = min(args.oracle_n, n)
        sub = make_inputs(ns, k, dev)
        Hc, H1c = sub.H.cpu().numpy(), sub.H1.cpu().numpy()
        del sub
        t = oracle_sample(Hc, H1c, ns // 2, args.oracle_layers)
        cpu = {"value": alg_flops_layers(ns, k, args.oracle_layers) / t / 1e12, "unit": "TFLOP/s",
               "cores": cpu_cores(), "kind": "oracle",
               "sample": f"first {args.oracle_layers} layer(s) of the FP64 numpy Alg. 1-3 on the "
                         f"same recipe at n={ns}, k={k} ({t:.1f} s)"}
        cpu.update(cpu_oracle_extra(k))

    traffic = recorded_traffic({"n": n, "k": k, "precision": args.precision, "cta_pair": args.cta_pair,
                                "k_snake": args.k_snake, "tile_band": args.tile_band,
                                "accum_chunk": args.accum_chunk})
    launches_per_step = 7 + (1 if args.precision.startswith("dual") else 0) + 2 * infos[0].product_launches
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16x2->f32" if args.precision == "dual_fp16" else args.precision, "data": "synthetic",
            "config": {"workload": f"dipole3 n={n} k={k} n_occ={n // 2} gap 0.2, {args.precision}",
                       "n": n, "k": k, "precision": args.precision, "cta_pair": args.cta_pair,
                       "l2": "inputs (2 GiB) larger than L2; no flush",
                       "parallelism": "replicas" if world > 1 else "single"},
            "time_to_solution_ms": ms_max,
            "layers": infos[0].layers, "d0_layer": infos[0].d0_layer,
            "accuracy": accuracy,
            "paper_sizes": paper_sizes,
            "forms": forms,
            "adjoint": adjoint,
            "batch": batch,
            "autotune": tune,
            "scc": scc,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "kernel": "layer_tc2_kernel" if args.cta_pair else "layer_tc_kernel",
                         "executed_mma_tflops": executed,
                         "peak_source": peak_source},
            "measured_peaks": measured_peaks,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "api": "dmpt_sp2_response_host", "equals_device_result": e2e_same,
                    "h2d_gbs": h2d_gbs, "d2h_gbs": d2h_gbs,
                    "h2d_gbs_slowest_of_5": h2d_min, "d2h_gbs_slowest_of_5": d2h_min,
                    "link_gbs_before_timed_steps": {
                        "h2d": link_before[0], "d2h": link_before[1],
                        "h2d_slowest_of_5": link_before[2], "d2h_slowest_of_5": link_before[3]},
                    "copy_ms_if_serial": copy_ms_serial,
                    "exposed_ms_per_step": e2e_ms - ms_max,
                    # the pipeline hides every copy but the first copy-in and the
                    # last copy-out of the sequence
                    "unhidden_copy_ms_per_step": copy_ms_serial / e_steps,
                    "layer_kernel_ms_per_step_in_pipeline": kernel_ms_pipeline,
                    "layer_kernel_ms_per_step_resident": tinfo.ms_layers},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
