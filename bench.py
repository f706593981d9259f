"""Benchmark: exact Hankel matvecs/s at n = 8000, b = 33220 bits (10^4 digits).

One step = one whole y = A x through the C ABI (encode x, Algorithm 1 steps
3/5 for every level, tensor-core leaf products, step 8 for every level,
exact rows, b-bit rounding), inputs resident in device memory.  Prints ONE
JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The default line (N = 1) also carries the comparisons a user of the library
asks for, each measured in the same run: the plain schoolbook GPU kernel on
the same inputs (vs_plain_kernel), the exact NTT path on the same inputs
with its own roofline (exact_ntt), the batched workload of 64 matrices x 8
right-hand sides (batched) and a short Poisson serving run (serving);
--no-extras leaves them out.

--impl reference times the CPU oracle (the plain schoolbook definition,
threaded over rows) on a bounded sample of rows of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Hankel matvecs/s at n=8000, 10^4 digits"
UNIT = "matvecs/s"
WORKLOAD = "large"
WORKLOAD_DESC = "Hankel y=Ax, n=8000, b=33220 bits (10^4 decimal digits), h and x uniform signed fixed-point in (-1,1)"


# ---------------------------------------------------------------- distributed helpers

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def init_dist(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def reduce_max(dist, value: float) -> float:
    """Largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / seconds_max if seconds_max > 0 else 0.0


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="hmv_clocks_", suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- CPU oracle timing

def oracle_sample(n, h, x, seconds_target=(10.0, 30.0), rows_per_batch=None):
    """Times the oracle on whole rows of the workload until ~10-30 s of work;
    returns (matvecs/s extrapolated from rows/s, cores, rows timed)."""
    import random

    import numpy as np

    import oracle
    cores = oracle.default_threads()
    batch = rows_per_batch or cores
    rng = random.Random(7)
    done, t_used = 0, 0.0
    while t_used < seconds_target[0]:
        rows = np.array(sorted(rng.sample(range(n), batch)), dtype=np.int32)
        t0 = time.perf_counter()
        oracle.exact_rows(oracle.HANKEL, n, h.b, h, x, rows, cores)
        t_used += time.perf_counter() - t0
        done += batch
        if t_used > seconds_target[1] * 0.5:
            break
    per_matvec = t_used / done * n
    return 1.0 / per_matvec, cores, done, t_used


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n, b, h, x = load_workload(args)
    cores = oracle.default_threads()
    import numpy as np
    import random
    rng = random.Random(11)
    per_step = []
    for step in range(args.warmup + args.steps):
        rows = np.array(sorted(rng.sample(range(n), cores)), dtype=np.int32)
        t0 = time.perf_counter()
        oracle.exact_rows(oracle.HANKEL, n, b, h, x, rows, cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            per_step.append(dt)
    mean = sum(per_step) / len(per_step)
    value = 1.0 / (mean * n / cores)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32 limbs (exact)", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "n": n, "b": b, "method": "CPU oracle: schoolbook definition"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: {cores} random rows of the n={n} product, one per thread; "
                                       f"matvecs/s extrapolated as cores/(step time * n)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import numpy as np
    import torch

    from paper_1402_5287_gb300 import hmv
    from paper_1402_5287_gb300.inputs import workload
    import paper_1402_5287_gb300 as pkg

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    pkg.build()
    n, b, h, x = load_workload(args)
    L32 = (b + 31) // 32
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    method = {"auto": hmv.AUTO, "karatsuba": hmv.KARATSUBA, "fft64": hmv.FFT64, "schoolbook": hmv.SCHOOLBOOK,
              "ntt": hmv.NTT}[args.method]
    split_flag = {-1: 0, 0: 0, 1: hmv.FLAG_DIGIT_SPLIT1, 2: hmv.FLAG_DIGIT_SPLIT2, 4: hmv.FLAG_DIGIT_TOOM4,
                  6: hmv.FLAG_DIGIT_TOOM6, 8: hmv.FLAG_DIGIT_TOOM8}[args.digit_split]
    if args.digit_split == 0 and method == hmv.AUTO:
        method = hmv.KARATSUBA  # no digit split
    tile_flag = {128: hmv.FLAG_TILE128, 256: hmv.FLAG_TILE256}.get(args.tile, 0)
    plan = hmv.Plan(n, b, method=method, levels=args.levels, flags=hmv.FLAG_TIMING | split_flag | tile_flag,
                    stream=stream.cuda_stream)
    plan.load_matrix(h)
    with torch.cuda.stream(stream):
        xl = torch.from_numpy(x.limbs.view(np.int32)).to(dev)
        xn = torch.from_numpy(x.neg).to(dev)
        yl = torch.empty_like(xl)
        yn = torch.empty_like(xn)
    stream.synchronize()

    def step():
        return plan.matvec_device(xl.data_ptr(), xn.data_ptr(), x.exponent, yl.data_ptr(), yn.data_ptr())

    for _ in range(max(args.warmup, 0)):
        step()
    plan.reset_stats()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    secs = ev0.elapsed_time(ev1) / 1e3
    secs_max = reduce_max(dist, secs)
    st = plan.stats()
    value = aggregate_rate(args.steps, world, secs_max)

    # roofline of the dominant kernel (leaf products): useful digit MACs x 2 per
    # launch over its mean CUDA-event duration (the library's events bracket the
    # leaf launches of each matvec: one launch, or two back to back on the
    # plan's two streams when a Toom plan runs its products in two halves)
    launches_per_mv = st["launches_leaf"] / max(st["matvecs"], 1)
    leaf_ms = st["ms_leaf"] / max(st["launches_leaf"], 1)
    flops_per_launch = 2.0 * st["leaf_macs"] / max(launches_per_mv, 1)
    achieved_tflops = flops_per_launch / (leaf_ms / 1e3) / 1e12 if leaf_ms > 0 else 0.0
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    # the leaf is one launch of about 55 ms per matvec, timed launch by launch:
    # the burst figure is its denominator; the sustained one (a seconds-long
    # cuBLAS loop under the power cap) is reported beside it
    peak = peaks.get("bf16_tflops")
    peak_src = "of measured: burst bf16 (MEASURED_PEAKS.json)"
    if peak is None:
        peak, peak_src = 1900.0, "of fallback: burst bf16"
    peak_sust = peaks.get("bf16_tflops_sustained") or 1700.0
    issued_over_useful = st["leaf_macs_issued"] / st["leaf_macs"] if st["leaf_macs"] else None

    traffic = leaf_traffic(st["leaf_tiles"], n, b, DIGIT_SPLIT_NAMES.get(st["digit_products"]),
                           st["leaf_tile_digits"])
    roofline = {"bound": "tensor", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak if peak else None, "traffic": traffic,
                "kernel": "k_leaf_tc", "peak_source": peak_src,
                "flops_per_launch": flops_per_launch, "launch_ms": leaf_ms,
                "launches_per_matvec": launches_per_mv,
                "issued_over_useful": issued_over_useful,
                # the MMAs the tensor pipe actually ran (band edges included)
                "frac_issued": achieved_tflops * issued_over_useful / peak if issued_over_useful else None,
                "peak_sustained": peak_sust, "frac_of_sustained": achieved_tflops / peak_sust}
    path, dtype = "karatsuba+tcgen05", "bf16"
    if st["launches_leaf"] == 0:  # a comparison path was asked for: no tensor-core leaf ran
        path, dtype = {"ntt": ("exact NTT, two 31-bit primes", "u32"), "fft64": ("split-FP64 FFT", "f64"),
                       "schoolbook": ("schoolbook, 32-bit limbs", "u32")}.get(args.method, (args.method, "u32"))
        roofline = (ntt_roofline(hmv, st, n, b, secs_max / args.steps, stream) if args.method == "ntt" else None)

    # end to end through the public API: host x in, host y out, copies inside the timed region
    e2e = None
    if True:
        pin_x_l = torch.from_numpy(x.limbs.view(np.int32)).pin_memory()
        pin_x_n = torch.from_numpy(x.neg).pin_memory()
        pin_y_l = torch.empty_like(pin_x_l).pin_memory()
        pin_y_n = torch.empty_like(pin_x_n).pin_memory()
        xv = hmv.Vec(n, 1, b, x.exponent, pin_x_l.data_ptr(), pin_x_n.data_ptr(), 0, 0)
        yv = hmv.Vec(n, 1, b, 0, pin_y_l.data_ptr(), pin_y_n.data_ptr(), 0, 0)
        import ctypes
        for _ in range(max(args.warmup, 1)):
            plan.lib.hmv_matvec(plan.handle, ctypes.byref(xv), ctypes.byref(yv))
        k2 = max(1, args.steps)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(k2):
            rc = plan.lib.hmv_matvec(plan.handle, ctypes.byref(xv), ctypes.byref(yv))
            if rc != 0:
                raise RuntimeError(f"hmv_matvec failed: {rc}")
        t_e2e = time.perf_counter() - t0
        t_e2e = reduce_max(dist, t_e2e)
        e2e = {"value": aggregate_rate(k2, world, t_e2e), "unit": UNIT, "steps": k2,
               "h2d_bytes_per_step": n * L32 * 4 + n, "d2h_bytes_per_step": n * L32 * 4 + n,
               "timing": "wall clock around synchronous hmv_matvec calls with pinned host x and y"}
    plan.close()

    comparisons = {}
    if args.compare and rank == 0:
        comparisons = compare_kernels(hmv, h, x, n, b, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, rows, t_used = oracle_sample(n, h, x)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{rows} random rows of the n={n}, b={b} product ({t_used:.1f} s on {cores} threads); "
                         f"matvecs/s extrapolated from rows/s"}

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras and (n, b) == (8000, 33220):
        plain = measure_plain_kernel(hmv, h, x, n, b, stream)
        plain["factor"] = value / plain["value"]
        extras["vs_plain_kernel"] = plain
        extras["exact_ntt"] = measure_ntt(hmv, h, x, n, b, stream, args.steps, args.warmup)
        extras["exact_ntt"]["vs_plain_kernel"] = extras["exact_ntt"]["value"] / plain["value"]
        extras["batched"] = measure_batched(3, 2, args.wave_gb)
        extras["batched_exact_ntt"] = measure_batched(3, 2, args.wave_gb, "ntt")
        extras["serving"] = measure_serving(args.extra_requests, args.rate, args.matvecs_per_request,
                                            args.serve_gb, False)
        extras["serving_exact_ntt"] = measure_serving(args.extra_requests, args.rate, args.matvecs_per_request,
                                                      args.serve_gb, False, "ntt")

    if rank != 0:
        return 0
    metric = METRIC if (n, b) == (8000, 33220) else f"Hankel matvecs/s at n={n}, b={b} bits"  # profiling sizes
    line = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs_max / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "n": n, "b": b, "kind": "hankel", "method": path,
                   "digit_split": DIGIT_SPLIT_NAMES.get(st["digit_products"], str(st["digit_products"])),
                   "digit_products": st["digit_products"],
                   "levels": st["levels"], "leaves": st["leaves"], "leaf_rows_max": st["leaf_rows_max"],
                   "digits_per_operand": st["digits"], "leaf_tiles": st["leaf_tiles"],
                   "leaf_tile_digits": st["leaf_tile_digits"],
                   "digit_format": "balanced radix-2^8 digits held exactly in bf16, fp32 windows < 2^24",
                   "l2": "working set of several GB per step (inputs larger than L2)",
                   "parallelism": f"{world} independent replica(s), one per GPU"},
        "roofline": roofline,
        "stage_ms": {"prepass": st["ms_prepass"] / max(st["matvecs"], 1), "leaf": st["ms_leaf"] / max(st["matvecs"], 1),
                     "post": st["ms_post"] / max(st["matvecs"], 1), "round": st["ms_round"] / max(st["matvecs"], 1)},
        # the plain definition's work (n^2 products of D = ceil(b/8)-digit numbers, D^2 digit
        # multiply-adds each, x 2 flops) over the matvec time: exceeds the tensor peak because
        # Algorithm 1 and the digit split do less work than the definition
        "schoolbook_equivalent": {"tflops": 2.0 * n * n * ((b + 7) // 8) ** 2 / (secs_max / args.steps) / 1e12,
                                  "unit": "TFLOP/s"},
        "gpu_launches": int(st["launches_total"]),
        "clocks": clocks.summary(),
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    line.update(extras)
    if comparisons:
        line["comparisons"] = comparisons
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def compare_kernels(hmv, h, x, n, b, stream):
    """Same workload through the comparison paths (one timed matvec each)."""
    import numpy as np
    import torch
    out = {}
    for name, method, levels, w in (("exact_ntt_two_primes", hmv.NTT, -1, 0),
                                    ("split_fp64_fft_auto_width", hmv.FFT64, -1, 0),
                                    ("split_fp64_fft_16bit_pieces", hmv.FFT64, -1, 16),
                                    ("tensor_core_schoolbook_L0", hmv.KARATSUBA, 0, 0),
                                    ("plain_schoolbook_cuda_cores", hmv.SCHOOLBOOK, -1, 0)):
        plan = hmv.Plan(n, b, method=method, levels=levels, stream=stream.cuda_stream, piece_bits=w,
                        flags=hmv.FLAG_TIMING)
        plan.load_matrix(h)
        dev = torch.device("cuda", torch.cuda.current_device())
        xl = torch.from_numpy(x.limbs.view(np.int32)).to(dev)
        xn = torch.from_numpy(x.neg).to(dev)
        yl = torch.empty_like(xl)
        yn = torch.empty_like(xn)
        torch.cuda.synchronize()
        reps = 1 if method == hmv.SCHOOLBOOK else 2
        plan.matvec_device(xl.data_ptr(), xn.data_ptr(), x.exponent, yl.data_ptr(), yn.data_ptr())
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.matvec_device(xl.data_ptr(), xn.data_ptr(), x.exponent, yl.data_ptr(), yn.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) / 1e3 / reps
        out[name] = {"value": 1.0 / s, "unit": UNIT, "ms_per_matvec": s * 1e3}
        if method == hmv.FFT64:
            st = plan.stats()
            out[name].update({"piece_bits": st["fft_piece_bits"], "log2_len": st["fft_log2_len"],
                              "error_bound": st["fft_bound"], "max_rounding_distance": st["fft_max_dist"],
                              "fft_matvecs": st["fft_matvecs"], "fallbacks_to_integer_path": st["fft_fallbacks"],
                              "ms_fft_per_matvec": st["ms_fft"] / max(st["fft_matvecs"], 1)})
        plan.close()
    return out


LEAF_SOURCES = ["paper_1402_5287_gb300/csrc/hmv_leaf_tc.cu", "paper_1402_5287_gb300/csrc/tc_ptx.cuh",
                "paper_1402_5287_gb300/csrc/hmv_leaf.h"]


DIGIT_SPLIT_NAMES = {1: "none", 3: "karatsuba, one level", 9: "karatsuba, two levels", 7: "toom-4",
                     11: "toom-6", 15: "toom-8"}


def leaf_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in LEAF_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def leaf_traffic(tiles, n, b, digit_split, tile_digits):
    """DRAM bytes per launch of the leaf kernel from the committed ncu capture
    of a small case (profiles/k_leaf_tc_traffic.json), scaled to this launch
    by its tile count (the capture shows bytes per tile constant across
    sizes); None when the capture is for another b, digit split or tile width,
    or the kernel has changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_leaf_tc_traffic.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if (rec.get("sources_sha256_16") != leaf_sources_hash() or rec.get("b") != b
            or rec.get("digit_split") != digit_split or rec.get("leaf_tile_digits") != tile_digits):
        return None
    cap = rec["captures"][0]
    return (cap["dram_bytes_read"] + cap["dram_bytes_write"]) * tiles / cap["leaf_tiles"]


def load_workload(args):
    """The benchmark workload, or a smaller one of the same recipe (--n/--b,
    for profiling captures)."""
    from paper_1402_5287_gb300.inputs import BASE_SEED, uniform_vec, workload
    global WORKLOAD_DESC
    if args.n is None and args.b is None:
        return workload(WORKLOAD)
    n = args.n or 8000
    b = args.b or 33220
    WORKLOAD_DESC = f"Hankel y=Ax, n={n}, b={b} bits, h and x uniform signed fixed-point in (-1,1)"
    return n, b, uniform_vec(BASE_SEED + 2, 0, 2 * n - 1, b, 0), uniform_vec(BASE_SEED + 2, 1, n, b, 0)


def measure_batched(steps, warmup, wave_gb, method="auto"):
    """Config 4: 64 matrices x 8 right-hand sides per hmv_batch_matvec call
    (one CUDA graph launch), device-resident inputs; wall clock per call.
    method: "auto" (the tensor-core Karatsuba path) or "ntt" (every member
    on the exact NTT path)."""
    import torch

    from paper_1402_5287_gb300 import hmv
    from paper_1402_5287_gb300.inputs import batched_workload
    nrhs = 8
    probs = batched_workload(64, nrhs)
    mcode = {"auto": hmv.AUTO, "ntt": hmv.NTT}[method]
    specs = [dict(n=n, b=b, nrhs=nrhs, method=mcode) for n, b, _, _ in probs]
    stream = torch.cuda.Stream()
    bt = hmv.Batch(specs, stream=stream.cuda_stream, wave_bytes=wave_gb << 30)
    for i, (_, _, h, _) in enumerate(probs):
        bt.load_matrix(i, h)
    dev = torch.device("cuda", torch.cuda.current_device())
    xs, ys = [], []
    for n, b, _, x in probs:
        xs.append((torch.from_numpy(x.limbs.view(np.int32)).to(dev), torch.from_numpy(x.neg).to(dev)))
        ys.append((torch.empty_like(xs[-1][0]), torch.empty_like(xs[-1][1])))
    xp = [(a.data_ptr(), c.data_ptr()) for a, c in xs]
    yp = [(a.data_ptr(), c.data_ptr()) for a, c in ys]
    ex = [x.exponent for *_, x in probs]
    torch.cuda.synchronize()
    for _ in range(max(warmup, 1)):
        bt.matvec_device(xp, yp, ex)
    t0 = time.perf_counter()
    with ClockSampler(torch.cuda.current_device()) as clocks:
        for _ in range(steps):
            bt.matvec_device(xp, yp, ex)
    secs = time.perf_counter() - t0
    info = bt.info()
    bt.close()
    mv = 64 * nrhs * steps
    return {"value": mv / secs, "unit": UNIT, "steps": steps, "warmup": max(warmup, 1),
            "ms_per_step": secs / steps * 1e3,
            "workload": "64 Hankel matrices, n ~ U[32,2048], b in {4096,16384,33220}, 8 RHS each, "
                        "uniform fixed-point in (-1,1); one CUDA graph launch per step",
            "method": "exact NTT path" if method == "ntt" else "tensor-core Karatsuba path",
            "waves": info["waves"], "pairs": info["pairs"], "leaf_tiles": info["leaf_tiles"],
            "kernels_per_graph": info["kernels_per_graph"], "wave_budget_gb": wave_gb,
            "device_gb": info["device_bytes"] / 1e9,
            "useful_leaf_tflops": 2 * info["leaf_macs"] * steps / secs / 1e12, "clocks": clocks.summary()}


def run_batched(args):
    import paper_1402_5287_gb300 as pkg
    pkg.build()
    r = measure_batched(args.steps, args.warmup, args.wave_gb, "ntt" if args.method == "ntt" else "auto")
    line = {"metric": "batched Hankel matvecs/s (64 matrices x 8 right-hand sides)", "value": r["value"],
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": r["warmup"],
            "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "method", "waves", "pairs", "leaf_tiles", "kernels_per_graph",
                                         "wave_budget_gb", "device_gb")},
            "useful_leaf_tflops": r["useful_leaf_tflops"], "graph_launches_per_step": 1, "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def run_lanczos(args):
    """Lanczos steps on the n=8000, b=33220 matrix (one step: A v, two exact
    inner products, one exact three-term update rounded to b bits, alpha and
    beta on the host), on the cost model's plan."""
    import time

    import torch

    import paper_1402_5287_gb300 as pkg
    from paper_1402_5287_gb300 import hmv
    from paper_1402_5287_gb300.lanczos import Lanczos
    pkg.build()
    n, b, h, x = load_workload(args)
    method = {"auto": hmv.AUTO, "ntt": hmv.NTT}.get(args.method)
    if method is None:
        raise SystemExit("--workload lanczos runs --method auto (the tensor-core path) or ntt")
    plan = hmv.Plan(n, b, method=method, flags=hmv.FLAG_TIMING if method == hmv.AUTO else 0)
    plan.load_matrix(h)
    lz = Lanczos(plan, x)
    for _ in range(args.warmup):
        lz.step()
    plan.reset_stats()
    with ClockSampler(torch.cuda.current_device()) as clocks:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            lz.step()
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
    st = plan.stats()
    if method == hmv.AUTO:
        mv_ms = st["ms_total"] / max(st["matvecs"], 1)
    else:  # the NTT plan keeps no per-call events: time its product on its own
        vp, ev, wp = lz.operands()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            plan.matvec_device(*vp, ev, *wp)
        mv_ms = (time.perf_counter() - t1) / args.steps * 1e3
    out = {"metric": "Lanczos steps/s at n=8000, 10^4 digits", "value": args.steps / secs, "unit": "steps/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
           "config": {"workload": WORKLOAD_DESC + "; Lanczos from x, unnormalised three-term recurrence",
                      "n": n, "b": b, "digit_products": st["digit_products"],
                      "method": "exact NTT path" if method == hmv.NTT else "tensor-core Karatsuba path",
                      "per_step": "1 matvec + 2 exact inner products + 1 exact 3-term update, wall clock"},
           "matvec_ms": mv_ms, "vector_ops_ms": secs / args.steps * 1e3 - mv_ms, "clocks": clocks.summary()}
    print(json.dumps(out))
    plan.close()
    return 0


def measure_serving(requests, rate, matvecs_per_request, serve_gb, chains, method="auto"):
    """Config 5: Poisson arrivals of Lanczos (or chain) requests, continuous
    batching; matvecs/s and p50/p99 latency per matvec.  method: "auto" (the
    tensor-core Karatsuba path) or "ntt" (the exact NTT path)."""
    import random

    import torch

    from paper_1402_5287_gb300.inputs import BASE_SEED, uniform_vec
    from paper_1402_5287_gb300.serving import Request, Server
    rng = random.Random(BASE_SEED + 4)
    reqs, t = [], 0.0
    for i in range(requests):
        t += rng.expovariate(rate)
        n = rng.randint(64, 4096)
        b = rng.choice([2048, 8192, 33220])
        reqs.append(Request(i, n, b, uniform_vec(BASE_SEED + 4, 2 * i, 2 * n - 1, b, 0),
                            uniform_vec(BASE_SEED + 4, 2 * i + 1, n, b, 0), matvecs_per_request, arrival=t,
                            lanczos=not chains))
    from paper_1402_5287_gb300 import hmv
    srv = Server(memory_budget=serve_gb << 30, method={"auto": hmv.AUTO, "ntt": hmv.NTT}[method])
    with ClockSampler(torch.cuda.current_device()) as clocks:
        st = srv.run(reqs)
    desc = (f"{requests} requests, Poisson arrivals at {rate}/s, n ~ U[64,4096], b in {{2048,8192,33220}}, "
            + (f"{matvecs_per_request} chained matvecs" if chains else
               f"{matvecs_per_request} Lanczos steps (one matvec, two exact inner products and one exact "
               f"update each)")
            + " per request against a resident A (cap on the 2n of a full Lanczos run)")
    path = ("exact NTT path (requests it cannot take: tensor-core path)" if method == "ntt"
            else "tensor-core Karatsuba path")
    return {"value": st["matvecs_per_s"], "unit": UNIT, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "workload": desc, "method": path, "memory_budget_gb": serve_gb, "serving": st,
            "clocks": clocks.summary()}


def run_serving(args):
    import paper_1402_5287_gb300 as pkg
    pkg.build()
    r = measure_serving(args.requests, args.rate, args.matvecs_per_request, args.serve_gb, args.serve_chains,
                        args.serve_method)
    line = {"metric": "served Hankel matvecs/s with p50/p99 matvec latency", "value": r["value"],
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic", "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"],
            "config": {"workload": r["workload"], "method": r["method"], "memory_budget_gb": r["memory_budget_gb"]},
            "serving": r["serving"], "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def measure_ntt(hmv, h, x, n, b, stream, steps, warmup):
    """The exact NTT path on the same inputs (device-resident x and y, CUDA
    events), with its roofline: Montgomery products per matvec (each radix-2
    butterfly of both transforms, the pointwise product and the Chinese
    remainder of every kept coefficient, for both primes) over the rate this
    GPU sustains for independent products, measured in the same run."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    plan = hmv.Plan(n, b, method=hmv.NTT, stream=stream.cuda_stream)
    plan.load_matrix(h)
    with torch.cuda.stream(stream):
        xl = torch.from_numpy(x.limbs.view(np.int32)).to(dev)
        xn = torch.from_numpy(x.neg).to(dev)
        yl = torch.empty_like(xl)
        yn = torch.empty_like(xn)
    stream.synchronize()
    for _ in range(max(warmup, 3)):
        plan.matvec_device(xl.data_ptr(), xn.data_ptr(), x.exponent, yl.data_ptr(), yn.data_ptr())
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.matvec_device(xl.data_ptr(), xn.data_ptr(), x.exponent, yl.data_ptr(), yn.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    st = plan.stats()
    plan.close()
    s = e0.elapsed_time(e1) / 1e3 / steps
    K = st["fft_log2_len"]
    return {"value": 1.0 / s, "unit": UNIT, "ms_per_matvec": s * 1e3, "steps": steps, "warmup": max(warmup, 3),
            "method": "exact NTT: 16-bit pieces, one cyclic convolution of 2^%d points modulo two 31-bit primes, "
                      "Chinese remainder, carries; bit-exact" % K,
            "roofline": ntt_roofline(hmv, st, n, b, s, stream)}


def ntt_roofline(hmv, st, n, b, s, stream):
    """The NTT path's roofline for a matvec of s seconds: Montgomery products
    per matvec (each radix-2 butterfly of both transforms, the pointwise
    product and the Chinese remainder of every kept coefficient, for both
    primes) over the rate this GPU sustains for independent products,
    measured now."""
    K = st["fft_log2_len"]
    N = 1 << K
    P = (b + 15) // 16
    products = 2.0 * K * N + 2.0 * N + n * (2 * P - 1)
    peak = hmv.measure_montgomery_rate(stream.cuda_stream)
    return {"bound": "alu", "achieved": products / s, "peak": peak, "unit": "Montgomery products/s",
            "frac": products / s / peak, "traffic": None, "products_per_matvec": products,
            "kernel": "k_ntt_rpass, k_ntt_rmid (the transform passes)",
            "peak_source": "of measured: independent Montgomery products on this GPU, same run"}


def measure_plain_kernel(hmv, h, x, n, b, stream):
    """One timed matvec of the plain schoolbook kernel (32-bit limbs, CUDA
    cores) on the benchmark workload, after a warm-up on a small problem."""
    import torch
    from paper_1402_5287_gb300.inputs import uniform_vec
    hs, xs = uniform_vec(5, 0, 127, 2048, 0), uniform_vec(5, 1, 64, 2048, 0)
    with hmv.Plan(64, 2048, method=hmv.SCHOOLBOOK, stream=stream.cuda_stream) as p:
        p.load_matrix(hs)
        p.matvec(xs)
    dev = torch.device("cuda", torch.cuda.current_device())
    plan = hmv.Plan(n, b, method=hmv.SCHOOLBOOK, stream=stream.cuda_stream)
    plan.load_matrix(h)
    with torch.cuda.stream(stream):
        xl = torch.from_numpy(x.limbs.view(np.int32)).to(dev)
        xn = torch.from_numpy(x.neg).to(dev)
        yl = torch.empty_like(xl)
        yn = torch.empty_like(xn)
    stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.matvec_device(xl.data_ptr(), xn.data_ptr(), x.exponent, yl.data_ptr(), yn.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    plan.close()
    s = e0.elapsed_time(e1) / 1e3
    return {"value": 1.0 / s, "unit": UNIT, "ms_per_matvec": s * 1e3, "steps": 1,
            "kernel": "k_schoolbook (32-bit limbs, CUDA cores), same inputs"}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--levels", type=int, default=-1, help="Karatsuba depth (-1: cost model)")
    ap.add_argument("--digit-split", type=int, choices=[-1, 0, 1, 2, 4, 6, 8], default=-1,
                    help="split of the mantissas on top of the index recursion: Karatsuba levels 1 or 2, "
                         "Toom-4, Toom-6 or Toom-8 (4, 6, 8), none (0) or the cost model's choice (-1)")
    ap.add_argument("--method", choices=["auto", "karatsuba", "fft64", "schoolbook", "ntt"], default="auto",
                    help="product method (profiling runs; the metric uses auto = Karatsuba + tcgen05)")
    ap.add_argument("--tile", type=int, choices=[0, 128, 256], default=0,
                    help="leaf tile width in product digits (profiling runs; 0: the plan's default)")
    ap.add_argument("--compare", action="store_true", help="also time the schoolbook comparison kernels")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the plain-kernel, batched and serving keys of the default line")
    ap.add_argument("--extra-requests", type=int, default=40,
                    help="requests of the short serving run in the default line")
    ap.add_argument("--n", type=int, default=None, help="matrix order (profiling runs; default 8000)")
    ap.add_argument("--b", type=int, default=None, help="mantissa bits (profiling runs; default 33220)")
    ap.add_argument("--workload", choices=["matvec", "batched", "serving", "lanczos"], default="matvec",
                    help="matvec: the n=8000 metric; batched: 64 matrices x 8 RHS per graph launch; "
                         "serving: Poisson requests with continuous batching; lanczos: Lanczos steps on the "
                         "n=8000 matrix")
    ap.add_argument("--wave-gb", type=int, default=48, help="batched: device memory per wave")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=4.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--matvecs-per-request", type=int, default=16)
    ap.add_argument("--serve-gb", type=int, default=200, help="serving: device memory budget")
    ap.add_argument("--serve-method", choices=["auto", "ntt"], default="auto",
                    help="serving: the tensor-core Karatsuba path (auto) or the exact NTT path")
    ap.add_argument("--serve-chains", action="store_true",
                    help="serving: plain chains v <- A v instead of Lanczos steps")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "lanczos":
        return run_lanczos(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
