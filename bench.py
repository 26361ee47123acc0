"""Benchmark of the fused metric-evolution chain on GB300 (one JSON line on stdout).

A step is one pass of the fused forward chain (inverse metric -> Christoffel symbols -> covariant
derivative of the shift -> d_t g_ij) over one grid of N = 2^24 (256^3) points with the seeded random
grid recipe, all 43 inputs and 39 outputs resident in HBM.  The metric is grid points per second;
achieved HBM GB/s counts the paper's effective bandwidth, 8 bytes x (43 + 39) components x N per pass
(Eq. 8).  Inputs plus outputs (11 GB) exceed the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--variant f64|f64_ff|f32]

With N > 1 every rank runs its own grid on its own GPU (the points are independent; no collective on
the data path): weak scaling, value = all ranks' points / max over ranks of the timed region.  Under
torchrun the ranks come from WORLD_SIZE / RANK / LOCAL_RANK, which must agree with --gpus; without a
launcher, --gpus N > 1 re-runs this script under torch.distributed.run with N ranks.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid points/s and HBM GB/s, fused Christoffel+dt g_ij, fwd and fwd+adjoint"
UNIT = "grid points/s"
N_FULL = 1 << 24
BYTES_PER_POINT = {"f64": 656, "f64_ff": 656, "f32": 328}
KERNEL_NAME = {"f64": "dtg_fwd_f64_kernel", "f64_ff": "dtg_fwd_ff_kernel", "f32": "dtg_fwd_f32_staged_kernel"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default=os.environ.get("TL_BENCH_VARIANT", "f64"), choices=["f64", "f64_ff", "f32"])
    ap.add_argument("--n", type=int, default=N_FULL)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the measurements of the other forms")
    ap.add_argument("--only", default=None, choices=["forward", "adjoint", "fwdbwd", "batched", "fd", "generated"],
                    help="run just one form on --n points (or --grids subgrids) and print its timing; for profiling")
    ap.add_argument("--grids", type=int, default=600)
    ap.add_argument("--order", type=int, default=4, choices=[2, 4], help="difference order of --only fd")
    ap.add_argument("--suite", default=None, help="comma-separated grid sizes: run the Eqs. 9-21 expression suite")
    ap.add_argument("--probe", action="store_true",
                    help="issue rates of the FP64 pipe (DFMA, DADD, DMUL, F2F pairs) per SM and clock, one JSON line")
    ap.add_argument("--launcher-check", action="store_true",
                    help="no GPU work: each rank builds its grid and reports it; rank 0 prints the ranks' view")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# The source files that define each profiled kernel (its own translation unit and the headers it uses).
_COMMON = ["tl_common.cuh", "tl_kernels.h"]
KERNEL_SOURCES = {
    "dtg_fwd_f64_kernel": ["dtg_fwd.cu", "dtg_fwd_body.cuh", "dtg_batched.cuh"] + _COMMON,
    "dtg_fwd_f32_kernel": ["dtg_fwd.cu", "dtg_fwd_body.cuh", "dtg_batched.cuh"] + _COMMON,
    "dtg_fwd_f32_staged_kernel": ["dtg_fwd.cu", "dtg_fwd_body.cuh", "dtg_batched.cuh", "bulk.cuh"] + _COMMON,
    "dtg_fwd_ff_kernel": ["dtg_fwd_ff.cu", "dtg_fwd_body.cuh", "dtg_ff_body.cuh", "ff.cuh", "dtg_batched.cuh"] + _COMMON,
    "dtg_bwd_f64_kernel": ["dtg_bwd.cu", "dtg_bwd_body.cuh", "dtg_fwd_body.cuh", "ff.cuh"] + _COMMON,
    "dtg_bwd_ff_kernel": ["dtg_bwd.cu", "dtg_bwd_body.cuh", "dtg_fwd_body.cuh", "ff.cuh"] + _COMMON,
    "dtg_fwdbwd_f64_kernel": ["dtg_fwd_bwd.cu", "dtg_bwd_body.cuh", "dtg_fwd_body.cuh", "dtg_ff_body.cuh", "ff.cuh"]
    + _COMMON,
    "dtg_fwdbwd_ff_kernel": ["dtg_fwd_bwd.cu", "dtg_bwd_body.cuh", "dtg_fwd_body.cuh", "dtg_ff_body.cuh", "ff.cuh"]
    + _COMMON,
    "dtg_batched_f64_kernel": ["dtg_fwd.cu", "dtg_fwd_body.cuh", "dtg_batched.cuh"] + _COMMON,
    "dtg_fd_kernel": ["dtg_fd.cu", "dtg_fwd_body.cuh", "dtg_ff_body.cuh", "ff.cuh"] + _COMMON,
    "tl_jit_kernel": ["jit.cu"],
}


def _code_only(text):
    """C/CUDA source without comments and with whitespace collapsed: what the compiler sees."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def src_digest(kernel=None):
    """Digest of a kernel's source files, comments and layout ignored (all kernel sources when kernel is
    None)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1804_10120_gb300", "csrc")
    names = sorted(KERNEL_SOURCES[kernel]) if kernel else sorted(
        n for n in os.listdir(csrc) if n.endswith((".cu", ".cuh", ".h")))
    for name in names:
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(name.encode() + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def traffic_per_launch(kernel, n):
    """DRAM bytes per launch from the committed ncu summary, scaled to n points; None when the kernel's
    sources changed since the capture (or none exists)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d[kernel]
        if e.get("src_digest") != src_digest(kernel):
            return None
        return float(e["dram_bytes"]) * n / float(e["n"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 7:
                    try:
                        rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
                    except ValueError:
                        pass
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def replica_command(gpus, argv, port):
    """The command that runs this script as `gpus` ranks on one node (one rank per GPU)."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(gpus),
            "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + list(argv)


def check_ranks(args):
    """Returns None when the rank layout matches --gpus, else an exit code after re-running under a
    launcher (no WORLD_SIZE and --gpus > 1) or refusing a layout that contradicts --gpus."""
    if "WORLD_SIZE" not in os.environ:
        if args.gpus > 1:
            return subprocess.call(replica_command(args.gpus, sys.argv[1:], _free_port()))
        return None
    world = int(os.environ["WORLD_SIZE"])
    if world != args.gpus:
        print("bench.py: WORLD_SIZE=%d but --gpus %d" % (world, args.gpus), file=sys.stderr)
        return 2
    return None


def launcher_check(args):
    """The replica layout without GPU work: every rank builds its own grid (gloo process group when
    there are several ranks), the ranks agree on the slowest rank's time, and rank 0 prints what each
    rank held.  Exercises the launcher, the per-rank seeds and the max over ranks on any machine."""
    import gridgen
    world, rank, _ = dist_setup()
    t0 = time.perf_counter()
    if args.only == "batched":
        # the sharded multi-domain batch: this rank's subgrids by the LPT rule, and their point count
        from paper_1804_10120_gb300.shard import lpt_partition
        sides = gridgen.subgrid_sides(args.grids, 2)
        mine = lpt_partition([s ** 3 for s in sides], world)[rank]
        digest = hashlib.sha256(json.dumps(mine).encode()).hexdigest()[:16]
        views = [(rank, len(mine), sum(sides[d] ** 3 for d in mine), digest)]
    else:
        x = gridgen.random_grid(4096, rank_seed(rank))
        digest = hashlib.sha256(x.tobytes()).hexdigest()[:16]
        views = [(rank, rank_seed(rank), digest)]
    local_ms = (time.perf_counter() - t0) * 1e3
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("gloo")

        def max_over(v):
            t = torch.tensor([v], dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())
        t_max, _ = replica_throughput(local_ms, 4096, 1, world, max_over)
        gathered = [None] * world
        dist.all_gather_object(gathered, views[0])
        views = gathered
        dist.destroy_process_group()
    else:
        t_max = local_ms
    if rank == 0:
        if args.only == "batched":
            ranks = [{"rank": r, "grids": g, "points": p, "indices_sha": d} for r, g, p, d in views]
        else:
            ranks = [{"rank": r, "seed": s, "grid_sha": d} for r, s, d in views]
        print(json.dumps({"launcher_check": True, "n_gpus": world, "gpus_arg": args.gpus, "t_max_ms": t_max,
                          "ranks": ranks}), flush=True)


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(x_host, budget_s=10.0, max_s=30.0):
    """The oracle as it stands, on all host cores, over the first points of the workload grid, repeated
    until ~budget_s of CPU work.  Returns (points/s, threads, sample description)."""
    import numpy as np
    import oracle
    threads = cpu_threads()
    n = x_host.shape[1]
    out = np.empty((39, n), dtype=np.float64)
    reps, points = 0, 0
    t0 = time.perf_counter()
    while True:
        oracle.forward_threaded(x_host, out, threads)
        reps += 1
        points += n
        el = time.perf_counter() - t0
        if el >= budget_s or el + el / reps > max_s:
            break
    return points / el, threads, "%d pass(es) of the oracle over %d points of the workload grid, %.1f s" % (reps, n, el)


def time_oracle_single(x_host, budget_s=3.0, n_max=1 << 18):
    """The same oracle loop on ONE host thread (no split), over the first n_max points of the workload
    grid, repeated until ~budget_s.  Returns (points/s, sample description)."""
    import numpy as np
    import oracle
    x = np.ascontiguousarray(x_host[:, :n_max])
    n = x.shape[1]
    out = np.empty((39, n), dtype=np.float64)
    reps = 0
    t0 = time.perf_counter()
    while True:
        oracle.forward_threaded(x, out, 1)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return reps * n / el, "%d pass(es) over the first %d points of the workload grid, one thread, %.1f s" % (reps, n, el)


def reference_arm(args):
    """The oracle (plain CPU loop nest) as the reference implementation, on this host's cores."""
    import numpy as np
    import gridgen
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    n_sample = min(args.n, 1 << 22)
    x = gridgen.random_grid(n_sample, 1)
    import oracle
    threads = cpu_threads()
    out = np.empty((39, n_sample), dtype=np.float64)
    for _ in range(max(1, min(args.warmup, 1))):
        oracle.forward_threaded(x, out, threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.forward_threaded(x, out, threads)
        times.append(time.perf_counter() - t0)
    t = sum(times)
    value = n_sample * args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded random grid)",
        "config": {"workload": "fused forward chain, single grid N=2^24 (256^3), SoA, seed 1",
                   "sample": "each reference step runs the CPU oracle on the first %d points of that grid" % n_sample,
                   "global_batch": n_sample, "parallelism": "host threads (%d)" % threads},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%d points per step (first points of the N=2^24 seed-1 grid)" % n_sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# Algorithmic work per grid point:
#   bytes: 8 x (43 + 39) for binary64, 4 x 82 for binary32 (each component array crosses HBM once);
#   binary64 flops of the fused chain as this library formulates it (FMA = 2): inverse 35, Eq. 6 bracket
#   18, Eq. 6 contraction 90, covariant shift derivative 39 (the 6 distinct sums Gamma^k_ij beta_k and 9
#   subtractions), Eq. 5 15.
FLOPS_F64_PER_POINT = 197
# Of the 197 flops, the 37 products that are not fused into an FMA run on the integer pipes (mul_int,
# bit-identical to the FP64 multiply), and the FP64 pipe executes 71 DFMA + 18 DADD = 89 operations per
# point.  The pipe issues DFMA and DADD at different rates on this part (measured live by
# tl_testing_pipe_rate: about 2.0 and 1.68 per clock per SM), so the kernel's second ceiling is the time
# those operations take at the measured rates: n (71 / r_DFMA + 18 / r_DADD).
FP64_OPS_PER_POINT = 89
FWD_FP64_MIX = (71, 18)                  # (DFMA, DADD) per point, counted by ncu
# The fused forward + adjoint for the loss sum W d_t g + V Gamma: 1192 bytes per point (43 inputs and
# 24 upstream gradients read, 39 outputs and 43 input gradients written) and 223 FP64-pipe operations
# (the forward's 89; Kbar/alphabar 5, betabar 15, Gammabar 18, Tbar 36, the bracket scatter 12 and the
# folded -H A H as 2 Tbar Gamma^T 48): 193 DFMA + 30 DADD.  The adjoint alone: 808 bytes and 181
# operations (163 DFMA + 18 DADD); the forward and the adjoint launched one after the other: 1464 bytes
# and 270 operations.
FWDBWD_BYTES_PER_POINT, FWDBWD_FP64_OPS, FWDBWD_FP64_MIX = 1192, 223, (193, 30)
BWD_BYTES_PER_POINT, BWD_FP64_OPS, BWD_FP64_MIX = 808, 181, (163, 18)


def fp64_floor_ms(mix, n, rates):
    """Time the FP64 pipe needs for n points of an operation mix (DFMA, DADD) at the measured rates."""
    return (mix[0] / rates[0] + mix[1] / rates[1]) * n * 1e3


def device_facts(dev):
    """SM count from the device, maximum SM clock from nvidia-smi (MHz; None if unavailable)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(dev.index), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        mhz = float(out.stdout.strip().splitlines()[0])
    except Exception:
        pass
    return sms, mhz


def nominal_hbm_gbs(dev):
    """Nominal HBM bandwidth from the device properties: memory clock x 2 (double data rate) x bus width
    (from PyTorch's device properties, else the library's device query); None when neither has them."""
    import torch
    p = torch.cuda.get_device_properties(dev)
    khz, bits = getattr(p, "memory_clock_rate", None), getattr(p, "memory_bus_width", None)
    if not khz or not bits:
        try:
            import ctypes
            import paper_1804_10120_gb300 as tl
            L = tl.lib()
            L.tl_testing_memory_info.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                                 ctypes.POINTER(ctypes.c_int32)]
            L.tl_testing_memory_info.restype = ctypes.c_int
            c, b = ctypes.c_int32(), ctypes.c_int32()
            if L.tl_testing_memory_info(dev.index or 0, ctypes.byref(c), ctypes.byref(b)) == 0:
                khz, bits = c.value, b.value
        except Exception:
            khz = bits = None
    if not khz or not bits:
        return None
    return (khz * 1e3 * 2 * bits / 8 / 1e9,
            "device properties: memory clock %d kHz x 2 x %d-bit bus" % (khz, bits))


PROBE_OPS = {0: "DFMA", 1: "DADD", 2: "DMUL", 3: "F2F pair (binary64->binary32->binary64)",
             4: "addition as DFMA by 1.0 (immediate)", 5: "DFMA, register operands", 6: "DADD, register operands",
             7: "DMUL, register operands", 8: "addition as DFMA by 1.0 from constant memory"}


def pipe_rates(dev, stream, ops=tuple(range(9)), target_ms=40.0):
    """Issue rate of each probed operation, operations (op 3: conversion pairs) per second over the whole
    GPU: 8 blocks of 256 threads per SM, 8 independent chains per thread, timed with CUDA events on
    `stream` (the kernel: tl_testing_pipe_rate)."""
    import ctypes
    import torch
    import paper_1804_10120_gb300 as tl
    L = tl.lib()
    L.tl_testing_pipe_rate.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p]
    L.tl_testing_pipe_rate.restype = ctypes.c_int
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = 8 * sms, 256
    sink = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    h = ctypes.c_void_p(stream.cuda_stream)
    rates = {}
    for op in ops:
        iters = 256
        while True:
            def run(it=iters):
                assert L.tl_testing_pipe_rate(op, it, blocks, threads, ctypes.c_void_p(sink.data_ptr()), h) == 0
            ms = cuda_time(run, 3, stream, warmup=1)
            if ms >= target_ms or iters >= (1 << 24):
                break
            iters *= 2 if ms < target_ms / 4 else 1 + int(target_ms / max(ms, 1e-3))
        rates[op] = blocks * threads * 8 * iters / (ms * 1e-3)
    return rates


def probe_main(args):
    """--probe: the FP64 pipe's issue rates on this GPU, per SM per clock at the clocks sampled meanwhile."""
    import torch
    from paper_1804_10120_gb300 import build as tlbuild
    tlbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    sms, max_mhz = device_facts(dev)
    pipe_rates(dev, stream, ops=(0,), target_ms=10.0)      # warm up clocks and module
    with ClockSampler(dev.index) as clk:
        rates = pipe_rates(dev, stream)
    c = clk.summary()
    mhz = c.get("sm_mhz") or max_mhz
    print(json.dumps({"probe": "FP64 pipe issue rates", "sms": sms, "sm_max_mhz": max_mhz, "clocks": c,
                      "ops": {PROBE_OPS[k]: {"per_s": v, "per_clk_per_sm_at_sampled_clock": v / (sms * mhz * 1e6),
                                             "per_clk_per_sm_at_max_clock": v / (sms * max_mhz * 1e6) if max_mhz else None}
                              for k, v in rates.items()}}), flush=True)


def _max_over_ranks(v, dev):
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(local_ms, points_per_rank, steps, world, max_over_ranks=None):
    """Weak-scaling aggregate of independent per-rank grids: the job's time is the slowest rank's timed
    region, its throughput all ranks' points over that time.  Returns (t_max_ms, points/s)."""
    t_max = max_over_ranks(local_ms) if (world > 1 and max_over_ranks) else local_ms
    return t_max, world * points_per_rank * steps / (t_max * 1e-3)


def rank_seed(rank):
    """Each rank times its own grid of the same recipe (seed 1 on rank 0)."""
    return 1 + 1000 * rank


def cuda_time(fn, steps, stream, warmup=3):
    """Mean ms per call of fn over `steps` calls, CUDA events on `stream`, after `warmup` calls."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def small_grid(dev, stream):
    """One small grid (N = 4096, seed 0; inputs + outputs 2.7 MB, resident in L2): launch-bound, so
    microseconds per launch, warm (inputs in L2 from the previous launch) and cold (a 256 MB write,
    twice the L2, before every launch).  Every launch is enqueued behind a fixed-length GPU spin, so
    the GPU runs them back to back and the events around each launch time the kernel, not the host's
    enqueue rate."""
    import torch
    import gridgen
    import paper_1804_10120_gb300 as tl
    n0 = 4096
    x0 = torch.from_numpy(gridgen.random_grid(n0, 0)).to(dev)
    y0 = torch.empty((39, n0), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    reps = 21

    def per_launch_us(cold):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            torch.cuda._sleep(50_000_000)       # ~25-50 ms of clock cycles: time to enqueue what follows
            for i in range(reps):
                if cold:
                    flush.fill_(i & 0xff)
                ev[2 * i].record(stream)
                tl.tl_dtg_forward(x0, y0, stream=stream)
                ev[2 * i + 1].record(stream)
        torch.cuda.synchronize()
        return sorted(1e3 * ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(1, reps))

    tl.tl_dtg_forward(x0, y0, stream=stream)
    warm, cold = per_launch_us(False), per_launch_us(True)
    return {"workload": "single grid N=4096, seed 0 (2.7 MB: fits in L2); launch-bound, microseconds per launch",
            "us_warm_median": warm[len(warm) // 2], "us_cold_median": cold[len(cold) // 2],
            "us_cold_min": cold[0], "us_cold_max": cold[-1],
            "method": "20 launches queued behind a GPU spin, events around each; cold: 256 MB written on "
                      "the launching stream before each launch"}


def padded_rows(host, dev, row_bytes=256):
    """The rows of a [c, n] host tensor copied into a device buffer whose rows are padded to a multiple
    of row_bytes; returns the c row views (length n each)."""
    import torch
    c, n = host.shape
    per = max(1, row_bytes // host.element_size())
    buf = torch.empty((c, (n + per - 1) // per * per), dtype=host.dtype, device=dev)
    buf[:, :n].copy_(host)
    return [buf[k, :n] for k in range(c)]


BATCH_STAGED = {"f64": [(128, 2), (128, 3), (256, 2)], "f32": [(128, 2), (128, 3), (256, 2), (256, 3), (512, 2)]}


def batched_depths(plan, stream, steps, dtype):
    """Best time of a batch plan at each staging depth (0: registers; 2, 3: shared memory), over the
    block sizes provided at that depth and 1, 2 or the most blocks per SM.  Restores the plan's config."""
    import paper_1804_10120_gb300 as tl
    keep = plan.config, plan.points_per_thread, plan.staging
    best = {}
    combos = [(t, 0) for t in (128, 256, 512)] + BATCH_STAGED[dtype]
    for threads, depth in combos:
        plan.set_staging(0)
        plan.set_config(threads, 1, 1)
        if depth:
            plan.set_staging(depth)
        for b in (1, 2, 3, 4):
            try:
                plan.set_config(threads, b)
            except tl.TLError:
                break
            ms = cuda_time(lambda: plan.launch(stream), max(3, steps // 2), stream)
            if depth not in best or ms < best[depth][0]:
                best[depth] = (ms, {"threads": threads, "blocks_per_sm": b})
    plan.set_staging(0)
    plan.set_config(keep[0][0], keep[0][1], keep[1])
    plan.set_staging(keep[2])
    return {str(k): {"ms": v[0], **v[1]} for k, v in sorted(best.items())}


def extras(dev, stream, steps, x64, hbm, fp64_rates=None):
    """The other forms of the path, each against the plain binary64 single-grid kernel, same GPU."""
    import torch
    import gridgen
    import paper_1804_10120_gb300 as tl
    out = {}
    n = x64.shape[1]
    y = torch.empty((39, n), dtype=torch.float64, device=dev)
    ms = cuda_time(lambda: tl.tl_dtg_forward(x64, y, dtype="f64_ff", stream=stream), steps, stream)
    out["f64_ff_forward"] = {"workload": "single grid N=2^24, seed 1", "ms": ms, "points_per_s": n / ms * 1e3,
                             "GB_s": 656 * n / ms / 1e6, "hbm_frac": 656 * n / ms / 1e6 / hbm,
                             "arith": "binary64 inverse, Eq. 6 bracket and Eq. 5; float-float contractions"}
    del y
    x32 = x64.float()
    y32 = torch.empty((39, n), dtype=torch.float32, device=dev)
    ms = cuda_time(lambda: tl.tl_dtg_forward(x32, y32, dtype="f32", stream=stream), steps, stream)
    out["f32_forward"] = {"workload": "single grid N=2^24, seed 1 rounded to binary32", "ms": ms,
                          "points_per_s": n / ms * 1e3, "GB_s": 328 * n / ms / 1e6, "hbm_frac": 328 * n / ms / 1e6 / hbm,
                          "arith": "binary32; det(g) and inverse in binary64"}
    del x32, y32
    # forward + adjoint, N = 2^22, loss sum W dtg + V Gamma (seed 3)
    n3 = 1 << 22
    x3 = torch.from_numpy(gridgen.random_grid(n3, 3)).to(dev)
    W = torch.from_numpy(gridgen.normal_fields(6, n3, 3, 1000)).to(dev)
    V = torch.from_numpy(gridgen.normal_fields(18, n3, 3, 1100)).to(dev)
    gout = [None] * 6 + [V[i] for i in range(18)] + [None] * 9 + [W[i] for i in range(6)]
    y3 = torch.empty((39, n3), dtype=torch.float64, device=dev)
    g3 = torch.empty((43, n3), dtype=torch.float64, device=dev)
    ms_f = cuda_time(lambda: tl.tl_dtg_forward(x3, y3, stream=stream), steps, stream)
    ms_b = cuda_time(lambda: tl.tl_dtg_backward(x3, gout, g3, stream=stream), steps, stream)
    ms_fb = cuda_time(lambda: (tl.tl_dtg_forward(x3, y3, stream=stream), tl.tl_dtg_backward(x3, gout, g3, stream=stream)),
                      steps, stream)
    ms_fb_ff = cuda_time(lambda: (tl.tl_dtg_forward(x3, y3, dtype="f64_ff", stream=stream),
                                  tl.tl_dtg_backward(x3, gout, g3, dtype="f64_ff", stream=stream)), steps, stream)
    ms_b_ff = cuda_time(lambda: tl.tl_dtg_backward(x3, gout, g3, dtype="f64_ff", stream=stream), steps, stream)
    ms_fused = cuda_time(lambda: tl.tl_dtg_forward_backward(x3, gout, y3, g3, stream=stream), steps, stream)
    ms_fused_ff = cuda_time(lambda: tl.tl_dtg_forward_backward(x3, gout, y3, g3, dtype="f64_ff", stream=stream),
                            steps, stream)
    out["fwd_adjoint_ff"] = {"workload": "N=2^22, seed 3, L = sum W dtg + V Gamma", "ms_adjoint": ms_b_ff,
                             "fused_ms": ms_fused_ff, "fused_points_per_s": n3 / ms_fused_ff * 1e3,
                             "fused_hbm_frac": FWDBWD_BYTES_PER_POINT * n3 / ms_fused_ff / 1e6 / hbm,
                             "ms": ms_fb_ff, "points_per_s": n3 / ms_fb_ff * 1e3, "GB_s": 1464 * n3 / ms_fb_ff / 1e6,
                             "hbm_frac": 1464 * n3 / ms_fb_ff / 1e6 / hbm,
                             "arith": "float-float forward and adjoint (binary64 inverse, bracket, folds)"}
    out["fwd_adjoint"] = {
        "workload": "N=2^22, seed 3, L = sum W dtg + V Gamma (W, V ~ N(0,1)), binary64",
        "fused": {"entry_point": "tl_dtg_forward_backward", "ms": ms_fused, "points_per_s": n3 / ms_fused * 1e3,
                  "bytes_per_point": FWDBWD_BYTES_PER_POINT,
                  "GB_s": FWDBWD_BYTES_PER_POINT * n3 / ms_fused / 1e6,
                  "hbm_frac": FWDBWD_BYTES_PER_POINT * n3 / ms_fused / 1e6 / hbm,
                  "fp64_ops_per_point": {"DFMA": FWDBWD_FP64_MIX[0], "DADD": FWDBWD_FP64_MIX[1]},
                  "fp64_floor_ms": fp64_floor_ms(FWDBWD_FP64_MIX, n3, fp64_rates) if fp64_rates else None,
                  "fp64_frac": fp64_floor_ms(FWDBWD_FP64_MIX, n3, fp64_rates) / ms_fused if fp64_rates else None,
                  "traffic": traffic_per_launch("dtg_fwdbwd_f64_kernel", n3)},
        "separate": {"ms_forward": ms_f, "ms_adjoint": ms_b, "ms": ms_fb, "points_per_s": n3 / ms_fb * 1e3,
                     "bytes_per_point": 656 + BWD_BYTES_PER_POINT, "GB_s": 1464 * n3 / ms_fb / 1e6,
                     "hbm_frac": 1464 * n3 / ms_fb / 1e6 / hbm,
                     "adjoint_hbm_frac": BWD_BYTES_PER_POINT * n3 / ms_b / 1e6 / hbm,
                     "adjoint_fp64_floor_ms": fp64_floor_ms(BWD_FP64_MIX, n3, fp64_rates) if fp64_rates else None,
                     "adjoint_fp64_frac": fp64_floor_ms(BWD_FP64_MIX, n3, fp64_rates) / ms_b if fp64_rates else None,
                     "adjoint_traffic": traffic_per_launch("dtg_bwd_f64_kernel", n3)},
        "bytes_per_point": "fused 1192 (43 inputs + 24 upstream gradients read, 39 outputs + 43 input gradients "
                           "written); adjoint alone 808 (34 inputs: d_j beta_i is not needed, 24 upstream "
                           "gradients, 43 input gradients)",
        "fp64_rate_source": "DFMA and DADD issue rates of tl_testing_pipe_rate, same run; frac = the time the "
                            "kernel's DFMA + DADD mix needs at those rates / its time"}
    del x3, W, V, gout, y3, g3
    # batched: 600 subgrids n^3, n ~ U{8..48} (seed 2)
    # each subgrid's 43 input and 39 output arrays are rows of one buffer whose row length is rounded up
    # to 256 bytes, so that every array starts on a 32-byte sector (the padding is never read)
    sides = gridgen.subgrid_sides(600, 2)
    xs, ys = [], []
    for d, side in enumerate(sides):
        xs.append(padded_rows(torch.from_numpy(gridgen.random_grid(side ** 3, 2, stream_base=gridgen.STREAMS_PER_FIELD * d)), dev))
        ys.append(padded_rows(torch.empty((39, side ** 3), dtype=torch.float64), dev))
    tot = sum(side ** 3 for side in sides)
    plan = tl.BatchPlan(xs, ys)
    cfg = plan.tune(stream)
    ms_b = cuda_time(lambda: plan.launch(stream), steps, stream)
    g = torch.cuda.CUDAGraph()
    side_stream = torch.cuda.Stream(dev)
    side_stream.wait_stream(stream)
    with torch.cuda.graph(g, stream=side_stream):
        plan.launch(side_stream)
    ms_bg = cuda_time(g.replay, steps, torch.cuda.current_stream(dev))

    def separate():
        for xd, yd in zip(xs, ys):
            tl.tl_dtg_forward(xd, yd, stream=stream)
    ms_sep = cuda_time(separate, max(2, steps // 10), stream)
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=side_stream):
        for xd, yd in zip(xs, ys):
            tl.tl_dtg_forward(xd, yd, stream=side_stream)
    ms_sepg = cuda_time(g2.replay, max(2, steps // 2), torch.cuda.current_stream(dev))
    by_depth = batched_depths(plan, stream, steps, "f64")
    out["batched"] = {"workload": "600 subgrids, N_d = n^3, n ~ U{8..48} (seed 2), %d points; each subgrid's "
                                  "arrays are rows of one buffer padded to 256-byte rows" % tot,
                      "config": {"threads": cfg[0], "blocks_per_sm": cfg[1],
                                 "points_per_thread": plan.points_per_thread, "staging": plan.staging},
                      "best_ms_by_staging_depth": by_depth,
                      "ms": ms_b, "points_per_s": tot / ms_b * 1e3, "GB_s": 656 * tot / ms_b / 1e6,
                      "hbm_frac": 656 * tot / ms_b / 1e6 / hbm,
                      "ms_in_graph": ms_bg,
                      "ms_600_launches": ms_sep, "ms_600_launches_in_graph": ms_sepg}
    plan.close()
    # the same batch stored in binary32, where the single grid gains from staging
    xs32 = [padded_rows(torch.stack(x).float(), dev) for x in xs]
    ys32 = [padded_rows(torch.empty((39, x[0].shape[0]), dtype=torch.float32), dev) for x in xs]
    del xs, ys
    plan = tl.BatchPlan(xs32, ys32, dtype="f32")
    cfg = plan.tune(stream)
    ms_b32 = cuda_time(lambda: plan.launch(stream), steps, stream)
    out["batched_f32"] = {"workload": "the same 600 subgrids rounded to binary32",
                          "config": {"threads": cfg[0], "blocks_per_sm": cfg[1],
                                     "points_per_thread": plan.points_per_thread, "staging": plan.staging},
                          "ms": ms_b32, "points_per_s": tot / ms_b32 * 1e3, "GB_s": 328 * tot / ms_b32 / 1e6,
                          "hbm_frac": 328 * tot / ms_b32 / 1e6 / hbm,
                          "best_ms_by_staging_depth": batched_depths(plan, stream, steps, "f32")}
    plan.close()
    del xs32, ys32
    # the chain with its 27 derivative inputs formed on the grid (periodic 256^3, 4th-order differences)
    fshape = (256, 256, 256)
    fd_fields = torch.from_numpy(gridgen.periodic_fields(fshape, 1)).to(dev)
    y = torch.empty((39, n), dtype=torch.float64, device=dev)
    fh = tuple(1.0 / m for m in fshape)
    for dt in ("f64", "f64_ff"):
        for order in (2, 4):
            ms_fd = cuda_time(lambda: tl.tl_dtg_forward_fd(fd_fields, fshape, fh, order, y, dtype=dt, stream=stream),
                              steps, stream)
            out["fd_forward_%s_order%d" % (dt, order)] = {
                "workload": "periodic 256^3 grid (2^24 points), smooth Fourier-mode fields, seed 1",
                "ms": ms_fd, "points_per_s": n / ms_fd * 1e3, "GB_s": 440 * n / ms_fd / 1e6,
                "hbm_frac": 440 * n / ms_fd / 1e6 / hbm,
                "bytes_per_point": "16 arrays read + 39 written = 440"}
    del fd_fields, y
    # the same chain written as a tensor-index program, emitted and compiled at run time
    from paper_1804_10120_gb300.programs import CHAIN
    k = tl.JitKernel(CHAIN)
    y = torch.empty((39, n), dtype=torch.float64, device=dev)
    ms_gen = cuda_time(lambda: k.launch(x64, y, stream=stream), steps, stream)
    out["generated_chain"] = {"workload": "single grid N=2^24, seed 1; the chain as a 16-statement index program "
                                          "compiled by the runtime generator (NVRTC, sm_103a)",
                              "ms": ms_gen, "points_per_s": n / ms_gen * 1e3, "GB_s": 656 * n / ms_gen / 1e6,
                              "hbm_frac": 656 * n / ms_gen / 1e6 / hbm}
    k.close()
    # the same chain with the footnote's sum written as a symmetric temporary (6 sums, not 9 chains)
    from paper_1804_10120_gb300.programs import CHAIN_SYM
    k = tl.JitKernel(CHAIN_SYM)
    ms_sym = cuda_time(lambda: k.launch(x64, y, stream=stream), steps, stream)
    out["generated_chain"]["symmetric_footnote_sum"] = {
        "ms": ms_sym, "points_per_s": n / ms_sym * 1e3, "hbm_frac": 656 * n / ms_sym / 1e6 / hbm,
        "program": "as the chain, with S(i,j) = Sum(k, Gamma(k,i,j)*beta(k)) a temporary symmetric in ij"}
    k.close()
    # the same program unfused: one kernel per assigned tensor, then per stored component, with the
    # intermediates through device memory (the paper's evaluation model and its "Arrays" baseline)
    from paper_1804_10120_gb300.statements import StatementPipeline
    for mode in ("statement", "component"):
        pl = StatementPipeline(CHAIN, mode)
        ms_st = cuda_time(lambda: pl.run(x64, y, stream=stream), steps, stream)
        elems = pl.elements_per_point()
        out["generated_chain"]["per_" + mode] = {
            "launches": pl.launches, "ms": ms_st, "points_per_s": n / ms_st * 1e3,
            "bytes_per_point": 8 * elems, "GB_s": 8 * elems * n / ms_st / 1e6,
            "hbm_frac": 8 * elems * n / ms_st / 1e6 / hbm, "fused_speedup": ms_st / ms_gen}
        pl.close()
    del y
    # the expression suite of Sec. 5.1 at a realistic multi-domain grid size and at a large one
    rows = suite(dev, stream, [32768, 1 << 22], reps=max(3, steps // 2))
    out["expression_suite"] = {
        "workload": "Eqs. 9-21, binary64, N(0,1) components; BW_eff = 8 B x N_e x N / t (Eq. 8)",
        "rows": [{"eq": r["eq"], "n": r["n"], "fused_GB_s": round(r["fused_GB_s"], 1),
                  "arrays_GB_s": round(r["arrays_GB_s"], 1), "fused_graph_GB_s": round(r["fused_graph_GB_s"], 1),
                  "arrays_graph_GB_s": round(r["arrays_graph_GB_s"], 1), "arrays_launches": r["arrays_launches"]}
                 for r in rows]}
    try:
        out["small_grid"] = small_grid(dev, stream)
    except Exception as e:      # context for the small case; never blocks the bench line
        out["small_grid"] = {"unavailable": repr(e)[:200]}
    return out


def only_form(args):
    """One form alone, for profilers: forward (--variant), adjoint (loss W dtg + V Gamma), batched
    (--grids subgrids of the multi-domain recipe), fd (derivatives on a periodic cube of about --n
    points, --order) or generated (the chain program through the runtime generator).  Under several
    ranks the batched form splits its subgrids across them; the other forms run one replica each."""
    import torch
    import gridgen
    import paper_1804_10120_gb300 as tl
    from paper_1804_10120_gb300 import build as tlbuild
    world, rank, local = dist_setup()
    if rank == 0 or world == 1:
        tlbuild.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=dev)
        torch.distributed.barrier()
        tlbuild.build()
    stream = torch.cuda.current_stream(dev)
    n = args.n
    if args.only == "forward":
        td = torch.float32 if args.variant == "f32" else torch.float64
        x = torch.from_numpy(gridgen.random_grid(n, 1)).to(dev, td)
        y = torch.empty((39, n), dtype=td, device=dev)
        fn = lambda: tl.tl_dtg_forward(x, y, dtype=args.variant, stream=stream)
        units = n
    elif args.only == "adjoint":
        x = torch.from_numpy(gridgen.random_grid(n, 3)).to(dev)
        W = torch.from_numpy(gridgen.normal_fields(6, n, 3, 1000)).to(dev)
        V = torch.from_numpy(gridgen.normal_fields(18, n, 3, 1100)).to(dev)
        gout = [None] * 6 + [V[i] for i in range(18)] + [None] * 9 + [W[i] for i in range(6)]
        g = torch.empty((43, n), dtype=torch.float64, device=dev)
        adj_dtype = "f64_ff" if args.variant == "f64_ff" else "f64"
        fn = lambda: tl.tl_dtg_backward(x, gout, g, dtype=adj_dtype, stream=stream)
        units = n
    elif args.only == "fwdbwd":
        x = torch.from_numpy(gridgen.random_grid(n, 3)).to(dev)
        W = torch.from_numpy(gridgen.normal_fields(6, n, 3, 1000)).to(dev)
        V = torch.from_numpy(gridgen.normal_fields(18, n, 3, 1100)).to(dev)
        gout = [None] * 6 + [V[i] for i in range(18)] + [None] * 9 + [W[i] for i in range(6)]
        y = torch.empty((39, n), dtype=torch.float64, device=dev)
        g = torch.empty((43, n), dtype=torch.float64, device=dev)
        fb_dtype = "f64_ff" if args.variant == "f64_ff" else "f64"
        fn = lambda: tl.tl_dtg_forward_backward(x, gout, y, g, dtype=fb_dtype, stream=stream)
        units = n
    elif args.only == "fd":
        side = round(n ** (1.0 / 3.0))
        shape = (side, side, side)
        f = torch.from_numpy(gridgen.periodic_fields(shape, 1)).to(dev)
        y = torch.empty((39, side ** 3), dtype=torch.float64, device=dev)
        h = tuple(1.0 / m for m in shape)
        fd_dtype = "f64_ff" if args.variant == "f64_ff" else "f64"
        fn = lambda: tl.tl_dtg_forward_fd(f, shape, h, args.order, y, dtype=fd_dtype, stream=stream)
        units = side ** 3
    elif args.only == "generated":
        from paper_1804_10120_gb300.programs import CHAIN
        x = torch.from_numpy(gridgen.random_grid(n, 1)).to(dev)
        y = torch.empty((39, n), dtype=torch.float64, device=dev)
        k = tl.JitKernel(CHAIN)
        fn = lambda: k.launch(x, y, stream=stream)
        units = n
    else:
        # the multi-domain batch; under several ranks each GPU takes its share of the subgrids by the
        # LPT rule (strong scaling: the same 600 subgrids in total, no exchange between the ranks)
        from paper_1804_10120_gb300.shard import lpt_partition
        sides = gridgen.subgrid_sides(args.grids, 2)
        mine = lpt_partition([s ** 3 for s in sides], world)[rank]
        xs, ys = [], []
        for d in mine:
            side = sides[d]
            xs.append(padded_rows(torch.from_numpy(gridgen.random_grid(side ** 3, 2, stream_base=gridgen.STREAMS_PER_FIELD * d)), dev))
            ys.append(padded_rows(torch.empty((39, side ** 3), dtype=torch.float64), dev))
        plan = tl.BatchPlan(xs, ys, dtype=args.variant if args.variant != "f32" else "f64")
        fn = lambda: plan.launch(stream)
        units = sum(side ** 3 for side in sides)
    if world > 1:
        torch.distributed.barrier()
    ms = cuda_time(fn, args.steps, stream, warmup=args.warmup)
    if world > 1:
        ms = _max_over_ranks(ms, dev)
    if rank == 0:
        line = {"form": args.only, "variant": args.variant, "points": units, "ms": ms,
                "points_per_s": units / ms * 1e3}
        if world > 1:
            line.update({"n_gpus": world, "scaling": "strong" if args.only == "batched" else "weak"})
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


EXPR_NAMES = {9: "A_i=B_i", 10: "A_ij=B_ij", 11: "A_ijk=B_ijk", 12: "A_i=B_i+C_i", 13: "A_i=B_i+C_i+D_i",
              14: "A_i=B_i+C_i+D_i+E_i", 15: "A_ij=B_iC_j", 16: "A_ijk=B_iC_jD_k", 17: "A_ijkl=B_iC_jD_kE_l",
              18: "A_ijkl=B_i^mE_mjkl", 19: "A_ijkl=C_j^nB_i^mE_mnkl", 20: "A_ijkl=D_k^oC_j^nB_i^mE_mnol",
              21: "K_ij=2alpha g_ij+beta_i beta_j"}


def suite(dev, stream, sizes, reps=10):
    """Effective bandwidth (Eq. 8, N_d = 0) of the benchmark expressions of Sec. 5.1, fused ("Tensors")
    and one launch per component / contracted index ("Arrays"), at each grid size.  Each evaluation is
    one direct call of the C entry point with prebuilt pointer tables (`*_ms`: host launches included),
    and the same evaluation captured once in a CUDA graph and replayed (`*_graph_ms`)."""
    import ctypes
    import torch
    import gridgen
    import paper_1804_10120_gb300 as tl
    L = tl.lib()
    L.tl_expr_eval.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                               ctypes.c_void_p]
    L.tl_expr_eval.restype = ctypes.c_int
    side = torch.cuda.Stream(dev)
    rows = []
    for eq in range(9, 22):
        n_in, n_out = tl.tl_expr_arity(eq)
        for n in sizes:
            x = torch.from_numpy(gridgen.normal_fields(n_in, n, eq, 5000)).to(dev)
            y = torch.empty((n_out, n), dtype=torch.float64, device=dev)
            tin = (ctypes.c_void_p * n_in)(*[x[q].data_ptr() for q in range(n_in)])
            tout = (ctypes.c_void_p * n_out)(*[y[q].data_ptr() for q in range(n_out)])
            row = {"eq": eq, "expr": EXPR_NAMES[eq], "n": n, "N_e": n_in + n_out}
            for mode, code in (("fused", 0), ("arrays", 1)):
                h = ctypes.c_void_p(stream.cuda_stream)
                launches = 1 if code == 0 else n_out * (3 ** (eq - 17) if eq in (18, 19, 20) else 1)
                r = reps if launches < 300 else max(2, reps // 4)

                def call(hs=h):
                    assert L.tl_expr_eval(eq, ctypes.byref(tin), ctypes.byref(tout), n, code, hs) == 0
                ms = cuda_time(call, r, stream, warmup=2)
                side.wait_stream(stream)
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=side):
                    call(ctypes.c_void_p(side.cuda_stream))
                gms = cuda_time(g.replay, r, torch.cuda.current_stream(dev), warmup=2)
                del g
                row.update({mode + "_launches": launches, mode + "_ms": ms, mode + "_GB_s": 8 * (n_in + n_out) * n / ms / 1e6,
                            mode + "_graph_ms": gms, mode + "_graph_GB_s": 8 * (n_in + n_out) * n / gms / 1e6})
            rows.append(row)
            del x, y
    return rows


def main():
    args = parse()
    rc = check_ranks(args)
    if rc is not None:
        sys.exit(rc)
    if args.launcher_check:
        return launcher_check(args)
    if args.probe:
        return probe_main(args)
    if args.suite:
        import torch
        from paper_1804_10120_gb300 import build as tlbuild
        tlbuild.build()
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        for row in suite(dev, torch.cuda.current_stream(dev), [int(v) for v in args.suite.split(",")], args.steps):
            print(json.dumps(row), flush=True)
        return
    if args.impl == "reference":
        return reference_arm(args)
    if args.only:
        return only_form(args)
    import numpy as np
    import torch
    import torch.distributed as dist
    import gridgen
    import paper_1804_10120_gb300 as tl
    from paper_1804_10120_gb300 import build as tlbuild

    world, rank, local = dist_setup()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    tlbuild.build()
    tl.lib()

    n = args.n
    variant = args.variant
    td = torch.float32 if variant == "f32" else torch.float64
    esz = 4 if variant == "f32" else 8
    x_host = gridgen.random_grid(n, rank_seed(rank))
    x_pinned = torch.from_numpy(x_host).to(td).pin_memory()
    x = x_pinned.to(dev)
    if world > 1 or args.no_cpu:
        x_host = None        # only the single-rank CPU baseline reads the numpy copy; free the host memory
    y = torch.empty((39, n), dtype=td, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        tl.tl_dtg_forward(x, y, dtype=variant, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(dev.index) as clk:
        ev[0].record(stream)
        for i in range(args.steps):
            step()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    t_max, value = replica_throughput(total_ms, n, args.steps, world,
                                      (lambda v: _max_over_ranks(v, dev)) if world > 1 else None)
    avg_launch_s = statistics.mean(per) * 1e-3
    hbm, peak_kind = peaks()
    bpp = BYTES_PER_POINT[variant]
    gbs = bpp * n / avg_launch_s / 1e9
    traffic = traffic_per_launch(KERNEL_NAME[variant], n)
    roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "traffic": traffic, "peak_source": peak_kind + " (MEASURED_PEAKS.json copy bandwidth)",
                "kernel": KERNEL_NAME[variant], "bytes_per_point": bpp, "avg_launch_ms": avg_launch_s * 1e3}
    sms, max_mhz = device_facts(dev)
    nominal = nominal_hbm_gbs(dev)
    if nominal:
        roofline["nominal_peak"] = {"GB_s": nominal[0], "frac": gbs / nominal[0], "source": nominal[1]}
    fp64 = None
    if variant == "f64":
        # the second ceiling of the binary64 chain: the FP64 pipe (1/64 of the FP32 rate on this part),
        # whose DFMA issue rate is measured here by the probe kernel, after the timed region
        r = pipe_rates(dev, stream, ops=(0, 1), target_ms=20.0)
        rates = (r[0], r[1])
        floor = fp64_floor_ms(FWD_FP64_MIX, n, rates)
        fp64 = {"ops_per_point": {"DFMA": FWD_FP64_MIX[0], "DADD": FWD_FP64_MIX[1]},
                "achieved_gops": FP64_OPS_PER_POINT * n / avg_launch_s / 1e9,
                "peak_gops": {"DFMA": rates[0] / 1e9, "DADD": rates[1] / 1e9},
                "floor_ms": floor, "frac": floor / (avg_launch_s * 1e3),
                "floor_ms_at_dfma_rate": fp64_floor_ms((FWD_FP64_MIX[0] + FWD_FP64_MIX[1], 0), n, rates),
                "frac_at_dfma_rate": fp64_floor_ms((FWD_FP64_MIX[0] + FWD_FP64_MIX[1], 0), n, rates) / (avg_launch_s * 1e3),
                "peak_source": "measured: issue rates of tl_testing_pipe_rate on this GPU, same run (8 x 256-thread "
                               "blocks per SM, 8 chains per thread); frac = time the 71 DFMA + 18 DADD per point need "
                               "at those rates / the kernel's time; the additions written as DFMAs (same bits) "
                               "ran no faster, so the floor with all 89 at the DFMA rate is given beside it",
                "nominal_peak_gops": 2 * sms * max_mhz / 1e3 if max_mhz else None,
                "nominal_source": "2 operations/clk/SM x %d SMs x %s MHz (device, nvidia-smi)" % (sms, max_mhz)}
        roofline["second_ceiling"] = {"unit": "FP64 pipe", **fp64}

    # end to end through the host-buffer C entry point: H2D of the inputs and D2H of the outputs inside
    # the timed region, page-locked host memory
    e2e = None
    if not args.no_e2e:
        y_pinned = torch.empty((39, n), dtype=td).pin_memory()
        ws = torch.empty(max(16, tl.tl_dtg_host_workspace_bytes(n, variant)), dtype=torch.uint8, device=dev)
        e2e_steps = max(1, min(args.steps, 5))
        tl.tl_dtg_forward_host(x_pinned, y_pinned, ws, dtype=variant, stream=stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            tl.tl_dtg_forward_host(x_pinned, y_pinned, ws, dtype=variant, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_ms = float(t.item())
        e2e = {"value": world * n * e2e_steps / (e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": 43 * n * esz, "d2h_bytes_per_step": 39 * n * esz,
               "steps": e2e_steps, "entry_point": "tl_dtg_forward_host"}
        del ws, y_pinned

    forms = None
    if rank == 0 and world == 1 and not args.no_extras and variant != "f32" and n == N_FULL:
        forms = extras(dev, stream, max(5, min(args.steps, 20)), x, hbm,
                       (fp64["peak_gops"]["DFMA"] * 1e9, fp64["peak_gops"]["DADD"] * 1e9) if fp64 else None)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, sample = time_oracle(x_host)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
        try:
            v1, sample1 = time_oracle_single(x_host)
            cpu["single_thread"] = {"value": v1, "unit": UNIT, "cores": 1, "sample": sample1}
        except Exception as e:     # the all-core figure above is the baseline; this one is context
            cpu["single_thread"] = {"unavailable": repr(e)[:200]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"f64": "f64", "f64_ff": "f64 storage, float-float contractions", "f32": "f32"}[variant],
            "data": "synthetic (seeded random grid: g = delta + 0.1 S, dg ~ U[-0.1,0.1], K, beta, dbeta ~ N(0,0.1), alpha ~ U[0.5,1.5])",
            "config": {"workload": "fused forward chain, single grid N=2^24 (256^3), SoA, seed 1",
                       "variant": variant, "global_batch": world * n, "points_per_gpu": n,
                       "parallelism": "replicas (independent grids per GPU)" if world > 1 else "single GPU",
                       "l2": "inputs+outputs %.1f GB > 129 MB L2; no flush" % (82 * n * esz / 1e9)},
            "roofline": roofline,
            # per-step spread, as the paper reports its runs (median of the timed steps, with min and max)
            "step_ms": {"median": statistics.median(per), "min": min(per), "max": max(per)},
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
