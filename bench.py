"""Throughput of the skew-symmetric LABS walk on GB300: exact flip evaluations per second.

One bench step = one full run of the L=201 workload: every walker restarts from its
Philox start (labs_reset) and takes 10^4 walk steps (labs_walk), each step evaluating
all n = 101 free-variable flips exactly (int32 ISL).  Default: 16384 walkers, HT of 2^16
slots per walker (8.6 GB of tables, far larger than the 129 MB L2), seed 7.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/, plain C, all host cores) on a bounded
sample of the same workload.  Under torchrun every rank runs its own walkers (seed
offset by rank, no collective on the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact flip evaluations/sec"
UNIT = "flip evaluations/s"
# The neighbourhood's work is one multiply-add per lag term (s_j x C_{2|j-i|}, Toeplitz
# form), n(n-1) lag terms per walker step, run as exact fp32 FMAs.  Derived peak of the
# FMA pipe: 152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz (maximum SM clock).
FP32_LANES_PER_SM = 128
ALGO_FLOP_PER_LAG_TERM = 2
# For comparison with an int32 formulation: one int32 multiply-add per lag term is the
# least such a path executes, and IMAD issues at half the FP32 FMA rate (64 lanes/clk/SM).
INT32_MAD_LANES_PER_SM = 64


def int32_equivalent(lag_terms_per_s, sms, sm_mhz):
    peak = INT32_MAD_LANES_PER_SM * sms * sm_mhz * 1e6
    return {"lag_terms_per_s": lag_terms_per_s, "int32_mad_peak": peak, "frac": lag_terms_per_s / peak,
            "note": "lag terms per second over the int32 multiply-add rate (%d SMs x %d lanes x %.0f MHz)"
                    % (sms, INT32_MAD_LANES_PER_SM, sm_mhz)}
# The PSL objective adds, per lag term of every flip, C' = C + cs (a + b) and max |C'|:
# an add, an FMA and a max beside the Toeplitz FMA, i.e. four FP32 lane operations,
# against the pipe's 128 lane operations per clock per SM.
PSL_LANE_OPS_PER_LAG_TERM = 4
WALK_KERNELS = {4: "walk_quad_kernel", 2: "walk_pair_kernel", 1: "walk_chunk_kernel"}  # by walkers per warp
# DRAM bytes per walker step of the L=201 walk kernel (ncu: dram__bytes_read.sum +
# dram__bytes_write.sum of a 4864-walker x 256-step launch of the current kernel,
# 373.1 + 33.6 MB over 1,245,184 walker steps, profiles/walk_pair_kernel_L201_16384w.md);
# None when not captured for the current kernel
DRAM_BYTES_PER_WALKER_STEP = 326.7


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--L", type=int, default=201)
    ap.add_argument("--walkers", type=int, default=16384)
    ap.add_argument("--walk-steps", type=int, default=10000)
    ap.add_argument("--tabu-log2", type=int, default=16)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--cpu-walkers", type=int, default=128)
    ap.add_argument("--cpu-steps", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-delta", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-length line (52 odd lengths 201..303 x 2048 walkers in one launch)")
    ap.add_argument("--no-scaleup", action="store_true",
                    help="skip the scale-up key (L=303 and 501, 131072 walkers x 2e4 steps each)")
    ap.add_argument("--mixed-walkers", type=int, default=2048)
    ap.add_argument("--mixed-steps", type=int, default=5000)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--config", choices=["walk", "learned", "scaleup", "long", "secondhash"], default="walk")
    ap.add_argument("--long-walkers", type=int, default=608)
    ap.add_argument("--long-steps", type=int, default=512)
    ap.add_argument("--scaleup-walkers", type=int, default=131072)
    ap.add_argument("--scaleup-steps", type=int, default=20000)
    ap.add_argument("--search", choices=["walk", "bestfirst", "psl"], default="walk",
                    help="walk: the self-avoiding walk; bestfirst: Algorithm 1 as printed (queue of 32); "
                         "psl: the walk under the PSL objective")
    ap.add_argument("--cpu-steps-psl", type=int, default=600,
                    help="oracle steps per walker of the CPU sample for --search psl (its oracle rebuilds "
                         "every neighbour: O(L^3) per step)")
    ap.add_argument("--learned-L", type=int, default=255)
    ap.add_argument("--learned-walkers", type=int, default=32768)
    ap.add_argument("--learned-steps", type=int, default=20000)
    ap.add_argument("--learned-train-steps", type=int, default=20000)
    ap.add_argument("--learned-seconds", type=float, default=None,
                    help="wall-clock cap per arm of --config learned (default: the step count alone)")
    ap.add_argument("--learned-segment", type=int, default=1024)
    ap.add_argument("--learned-arms", default="plain,learned,restarts",
                    help="comma list: learned (the full learned mode), restarts (restart proposals only)")
    ap.add_argument("--delta-rows", type=int, default=1 << 20)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def tensor_peak():
    """Dense FP16 tensor rate (FLOP/s): the measured sustained BF16 GEMM rate (FP16 and
    BF16 share the nominal dense rate), else the fallback 1.7 PFLOP/s."""
    return float(measured_peaks().get("bf16_tflops_sustained", 1700.0)) * 1e12


def lag_roofline(n, flips, st, fma_peak):
    """Lag-term FLOP/s (one multiply-add per lag term, n - 1 per flip evaluation) against
    the FP32 FMA peak and the FP16 tensor peak; `roofline_frac` takes the pipe that runs
    the Toeplitz product (labs_counters.tensor_cores)."""
    flops = ALGO_FLOP_PER_LAG_TERM * (n - 1) * flips
    tc = bool(st.get("tensor_cores"))
    d = {"toeplitz": "tensor cores" if tc else "fp32", "fma_frac": flops / fma_peak,
         "tensor_frac": flops / tensor_peak()}
    d["roofline_frac"] = d["tensor_frac"] if tc else d["fma_frac"]
    return d


def cpu_baseline(args):
    """The oracle as it stands, all host cores, on a bounded sample of the workload."""
    import oracle

    cores = os.cpu_count() or 1
    steps = cpu_steps(args)
    t0 = time.perf_counter()
    oracle_run(args, steps, cores)
    dt = time.perf_counter() - t0
    n = (args.L + 1) // 2
    flips = args.cpu_walkers * steps * n
    return {"value": flips / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "L=%d, %d walkers x %d steps (walkers 0..%d of the workload), %.2f s" %
                      (args.L, args.cpu_walkers, steps, args.cpu_walkers - 1, dt)}


def cpu_steps(args):
    return args.cpu_steps_psl if args.search == "psl" else args.cpu_steps


def oracle_run(args, steps, cores):
    import oracle

    if args.search == "bestfirst":
        oracle.bestfirst(args.L, args.seed, args.cpu_walkers, steps, tabu_log2=args.tabu_log2, nthreads=cores)
    else:
        oracle.walk(args.L, args.seed, args.cpu_walkers, steps, tabu_log2=args.tabu_log2, nthreads=cores,
                    objective="psl" if args.search == "psl" else "isl")


def config_of(args, world):
    what = {"bestfirst": "best-first search (Algorithm 1, queue of 32)",
            "psl": "self-avoiding walk under the PSL objective"}.get(args.search, "self-avoiding walk")
    return {"workload": "L=%d skew-symmetric %s, %d walkers/GPU x %d steps, HT 2^%d slots/walker, "
                        "uniform random +-1 Philox starts, seed %d" % (args.L, what, args.walkers, args.walk_steps,
                                                                      args.tabu_log2, args.seed),
            "L": args.L, "walkers_per_gpu": args.walkers, "walk_steps": args.walk_steps,
            "tabu_slots_per_walker": 1 << args.tabu_log2,
            "l2": "inputs larger than L2: %.1f GB of HT tables per GPU" %
                  ((args.walkers << args.tabu_log2) * 8 / 1e9),
            "parallelism": "independent walkers, %d rank(s)" % world}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    n = (args.L + 1) // 2
    steps = cpu_steps(args)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle_run(args, steps, cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tmax = sum(times) / len(times)
    flips = args.cpu_walkers * steps * n
    value = flips / tmax
    sample = "L=%d, %d walkers x %d steps per step (a bounded sample of the workload)" % (args.L, args.cpu_walkers, steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_of(args, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def delta_kernel_line(args, dev, stream, labs):
    """labs_neighbor_delta (the stateless neighbourhood evaluation, Algorithm 1's flip
    loop over given sequences) on a batch larger than L2, timed with CUDA events on
    the library's stream: throughput and its fp32 FMA roofline."""
    import torch

    import labs_inputs

    L, B = args.L, args.delta_rows
    n, c = (L + 1) // 2, (L + 1) // 2 - 1
    with torch.cuda.stream(stream):
        x = torch.from_numpy(labs_inputs.random_free_vars(B, L, seed=args.seed)).to(dev)
        j = torch.arange(1, n, device=dev)
        sign = torch.where(j % 2 == 1, -1, 1).to(torch.int8)
        rows = torch.cat([x, x[:, c - j] * sign], dim=1).contiguous()  # Eq. 4
        out = labs.neighbor_delta(rows, stream=stream)
        ms = []
        for _ in range(args.warmup + args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            labs.neighbor_delta(rows, stream=stream)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
    ms = statistics.mean(ms[args.warmup:])
    flips = B * n / (ms / 1e3)
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = FP32_LANES_PER_SM * 2 * sms * sm_mhz * 1e6
    achieved = ALGO_FLOP_PER_LAG_TERM * (n - 1) * flips
    del out
    return {"kernel": "delta_kernel", "rows": B, "L": L, "ms_per_launch": ms, "value": flips, "unit": UNIT,
            "input_bytes": B * L, "output_bytes": B * n * 4,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None},
            "int32_equivalent": int32_equivalent((n - 1) * flips, sms, sm_mhz)}


def mixed_line(args, dev, labs):
    """All 52 odd lengths L = 201..303 as walkers of one context (one persistent,
    graph-captured chunk chain; launch shape from the tuner), mixed_walkers walkers per
    length x mixed_steps steps, seed 7: flips/s timed with CUDA events on the
    library's stream around labs_walk, after an untimed run of the same length."""
    import torch

    from paper_2011_00068_gb300 import tune

    Ls = list(range(201, 304, 2))
    counts = [args.mixed_walkers] * len(Ls)
    best = tune.tune(Ls, counts, tabu_log2=args.tabu_log2, device=dev, steps=256)
    s = labs.Search(Ls, counts, 7, device=dev, tabu_log2=args.tabu_log2, warps_per_cta=best["warps_per_cta"],
                    chunk_steps=best["chunk_steps"])
    s.walk(args.mixed_steps)  # untimed: graph capture and first touch of the tables
    s.sync()
    s.reset()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s.stream)
    s.walk(args.mixed_steps)
    b.record(s.stream)
    s.sync()
    ms = a.elapsed_time(b)
    st = s.stats()
    assert st["steps"] == sum(counts) * args.mixed_steps, st
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    lag_terms = sum(c * args.mixed_steps * ((L + 1) // 2) * ((L + 1) // 2 - 1) for L, c in zip(Ls, counts))
    peak = FP32_LANES_PER_SM * 2 * sms * sm_mhz * 1e6
    b = s.best()
    out = {"workload": "52 odd L = 201..303, %d walkers each (%d walkers), %d steps, one context, seed 7, "
                       "HT 2^%d slots/walker (%.1f GB)" % (args.mixed_walkers, sum(counts), args.mixed_steps,
                                                         args.tabu_log2,
                                                         (sum(counts) << args.tabu_log2) * 8 / 1e9),
           "value": st["flip_evaluations"] / (ms / 1e3), "unit": UNIT, "ms": ms,
           "launch": {"warps_per_cta": best["warps_per_cta"], "chunk_steps": best["chunk_steps"]},
           "roofline_frac": ALGO_FLOP_PER_LAG_TERM * lag_terms / (ms / 1e3) / peak,
           "best": {"isl": b["isl"], "F": b["F"], "L": b["L"]}}
    s.close()
    del s
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch

    import paper_2011_00068_gb300 as labs

    rank, world, local = dist_env()
    pg = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        pg = dist
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(dev)
    n = (args.L + 1) // 2
    from paper_2011_00068_gb300 import replicas

    seed = replicas.rank_seed(args.seed, rank)
    shape = {}
    from paper_2011_00068_gb300 import _native

    flags = {"bestfirst": _native.LABS_FLAG_BEST_FIRST, "psl": _native.LABS_FLAG_PSL}.get(args.search, 0)
    if not args.no_tune:
        from paper_2011_00068_gb300 import tune

        best = tune.tune(args.L, args.walkers, tabu_log2=args.tabu_log2, device=dev, flags=flags)
        shape = {"warps_per_cta": best["warps_per_cta"], "chunk_steps": best["chunk_steps"]}
    s = labs.Search(args.L, args.walkers, seed, device=dev, stream=stream, tabu_log2=args.tabu_log2, flags=flags,
                    **shape)
    chunk = int(s.cfg.chunk_steps) or 1024
    nchunks = -(-args.walk_steps // chunk)

    def barrier():
        torch.cuda.synchronize(dev)
        if pg:
            pg.barrier()

    def one_step():
        s.reset()
        s.walk(args.walk_steps)

    for _ in range(args.warmup):
        one_step()
    s.sync()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    wall = []
    with ClockSampler(local) as clk:
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            # walk-kernel time: events on the library's stream around labs_walk
            s.reset()
            ev[i][0].record(stream)
            s.walk(args.walk_steps)
            ev[i][1].record(stream)
        s.sync()
        barrier()
        t1 = time.perf_counter()
    walk_ms = [a.elapsed_time(b) for a, b in ev]
    elapsed = replicas.max_over_ranks(t1 - t0, device=dev)
    flips_per_step = args.walkers * args.walk_steps * n
    value = world * flips_per_step * args.steps / elapsed
    st = s.stats()
    assert st["steps"] == args.walkers * args.walk_steps, st

    # roofline of the walk kernel: lag terms n(n-1) per walker step, one FMA (2 FLOP) each
    avg_launch_s = statistics.mean(walk_ms) / 1e3 / nchunks
    ops_per_launch = ALGO_FLOP_PER_LAG_TERM * n * (n - 1) * args.walkers * args.walk_steps / nchunks
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = FP32_LANES_PER_SM * 2 * sms * sm_mhz * 1e6
    achieved = ops_per_launch / avg_launch_s
    unit = "TFLOP/s"
    if args.search == "psl":
        # FP32 lane operations: PSL_LANE_OPS_PER_LAG_TERM per lag term, one per lane per clock
        achieved *= PSL_LANE_OPS_PER_LAG_TERM / ALGO_FLOP_PER_LAG_TERM
        peak /= 2
        unit = "Tops/s (FP32 lane operations)"
    kernel = ("walk_psl_pair_kernel" if args.search == "psl" and st["walkers_per_warp"] == 2
              else WALK_KERNELS[st["walkers_per_warp"]])
    steps_per_launch = args.walkers * args.walk_steps / nchunks
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": unit,
                "frac": achieved / peak,
                "traffic": (DRAM_BYTES_PER_WALKER_STEP * steps_per_launch
                            if args.L == 201 and args.search == "walk" and DRAM_BYTES_PER_WALKER_STEP else None),
                "traffic_note": ("bytes per launch: %.1f B per walker step from one ncu capture of a small "
                                 "launch, scaled by walker steps" % DRAM_BYTES_PER_WALKER_STEP
                                 if DRAM_BYTES_PER_WALKER_STEP and args.search == "walk" and args.L == 201
                                 else "not captured for this kernel and workload"),
                "kernel": kernel, "lane_block": st["lane_block"],
                "peak_source": "derived: %d SMs x %d FP32 lanes x %s x %.0f MHz (FMA pipe)" % (
                    sms, FP32_LANES_PER_SM, "1 op" if args.search == "psl" else "2 FLOP", sm_mhz),
                "toeplitz": ("tensor cores: mma.sync.m16n8k16, FP16 operands (exact small integers), FP32 "
                             "accumulation; the step around it is issue- and latency-bound on the FP32, integer "
                             "and load/store pipes, so lag terms are counted against the FP32 FMA peak"
                             if st.get("tensor_cores") else "FP32 FMA pipe"),
                "tensor_frac": (ops_per_launch / avg_launch_s / tensor_peak() if args.search != "psl" else None)}

    e2e = None
    if not args.no_e2e:
        # the user's whole call: fresh start, walk, and the per-walker results read back
        e2e_times = []
        d2h = 0
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            s.reset()
            s.walk(args.walk_steps)
            r = s.results()
            b = s.best()
            e2e_times.append(time.perf_counter() - t0)
            d2h = sum(v.nbytes for v in r.values()) + b["seq"].nbytes + 16
        e2e = {"value": world * flips_per_step / statistics.mean(e2e_times), "unit": UNIT,
               "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(d2h)}

    delta = None if args.no_delta else delta_kernel_line(args, dev, stream, labs)
    mixed = scaleup = None
    if world == 1 and args.search == "walk" and not (args.no_mixed and args.no_scaleup):
        s.close()
        torch.cuda.empty_cache()
        if not args.no_mixed:
            mixed = mixed_line(args, dev, labs)
        if not args.no_scaleup:
            # config 5 (the walks; its learned arm is --config learned's measurement)
            total, per_L, workload, _ = scaleup_measure(args, dev, labs)
            scaleup = {"workload": workload, "value": total, "unit": UNIT, "per_L": per_L}
    if args.search == "psl":
        # lowest (PSL, ISL) pair over ranks: PSL < 2^9 above ISL < 2^26 in one key
        obj, best_rank = replicas.best_over_ranks((st["best_psl"] << 26) | st["best_isl"], device=dev)
        best_isl, best_psl = obj & ((1 << 26) - 1), obj >> 26
    else:
        best_isl, best_rank = replicas.best_over_ranks(st["best_isl"], device=dev)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(config_of(args, world), launch={
                    "warps_per_cta": int(s.cfg.warps_per_cta) or 8, "chunk_steps": chunk,
                    "tuned": not args.no_tune}),
                "roofline": roofline,
                "int32_equivalent": int32_equivalent(value / world * (n - 1), sms, sm_mhz),
                "clocks": clk.summary(), "e2e": e2e,
                "gpu_launches": args.steps * (2 + nchunks),
                "walk_ms_per_step": statistics.mean(walk_ms),
                "best": dict({"isl": best_isl, "F": args.L ** 2 / (2 * best_isl), "L": st["best_L"],
                              "rank": best_rank}, **({"psl": best_psl} if args.search == "psl" else {})),
                "delta_kernel": delta,
                "mixed_201_303": mixed,
                "scaleup_303_501": scaleup,
                "restarts": st["restarts"]}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line))
    s.close()
    if pg:
        pg.destroy_process_group()
    return 0


def run_learned(args):
    """Config 4: the learned proposal vs the plain walk at L=255 on the same GPU
    (time-to-F thresholds and flips/s of both); one JSON line."""
    import torch

    from paper_2011_00068_gb300 import compare

    torch.cuda.set_device(0)
    arms = args.learned_arms.split(",")
    r = compare.run(L=args.learned_L, walkers=args.learned_walkers, steps=args.learned_steps,
                    train_steps=args.learned_train_steps, batch=4096, seconds=args.learned_seconds,
                    segment=args.learned_segment, full_arm="learned" in arms, restart_arm="restarts" in arms)
    for k in ("plain", "learned", "learned_restarts"):
        if r[k] is None:
            continue
        curve = r[k].pop("curve", None) or []
        # the best-F curve, thinned to about 40 points: (steps, seconds, best ISL)
        r[k]["curve"] = curve[::max(1, len(curve) // 40)] + curve[-1:]
    tt = {k: (r[k]["time_to_F"]["8.5"] if r[k] else None) for k in ("plain", "learned", "learned_restarts")}
    best_arm = "learned_restarts" if r["learned_restarts"] else "learned"
    cap = ("%d steps or %.0f s per arm" % (args.learned_steps, args.learned_seconds) if args.learned_seconds
           else "%d steps" % args.learned_steps)
    line = {"metric": "time-to-F>=8.5 at L=%d, learned vs plain (censored at %s)" % (args.learned_L, cap),
            "value": tt[best_arm]["seconds"] if tt[best_arm] else None, "unit": "s", "higher_is_better": False,
            "value_arm": best_arm,
            "n_gpus": 1, "dtype": "f32 walk / bf16 net", "data": "synthetic",
            "config": {"workload": "L=%d, %d walkers, %d steps, trained %d steps x batch 4096 on the walk log" %
                                   (args.learned_L, args.learned_walkers, args.learned_steps,
                                    args.learned_train_steps)},
            "vs_baseline": None, "comparison": r}
    sustained = measured_peaks().get("bf16_tflops_sustained")
    line["train_tflops"] = r["train"]["tflops"]
    line["train_frac_of_bf16_sustained"] = r["train"]["tflops"] / sustained if sustained else None
    print(json.dumps(line))
    return 0


def scaleup_measure(args, dev, labs):
    """Config 5's walks: L=303 and L=501, scaleup_walkers walkers each, scaleup_steps
    steps (segments of 1000, best ISL read after each): per-length flips/s, roofline
    fractions, best F and the time to F >= 8; and the time-weighted aggregate."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = float(measured_peaks().get("sm_max_mhz", 2070.0))
    peak = FP32_LANES_PER_SM * 2 * sms * sm_mhz * 1e6
    out = {}
    seg = 1000
    for L in (303, 501):
        n = (L + 1) // 2
        s = labs.Search(L, args.scaleup_walkers, 42, device=dev)
        s.walk(64)
        s.sync()
        s.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done, t8 = 0, None
        while done < args.scaleup_steps:
            k = min(seg, args.scaleup_steps - done)
            s.walk(k)
            done += k
            b = s.best()
            if t8 is None and 2 * 8 * b["isl"] <= L * L:
                t8 = {"steps": done, "seconds": time.perf_counter() - t0}
        dt = time.perf_counter() - t0
        st = s.stats()
        flips = st["flip_evaluations"] / dt
        b = s.best()
        out[str(L)] = {"flips_per_s": flips, "seconds": dt, "steps": done, "walkers": args.scaleup_walkers,
                       "best_isl": b["isl"], "best_F": b["F"], "best_hex": b["hex"], "time_to_F8": t8,
                       "kernel": WALK_KERNELS[st["walkers_per_warp"]],
                       **lag_roofline(n, flips, st, peak),
                       "tabu_bytes": (args.scaleup_walkers << 16) * 8}
        s.close()
        del s
        torch.cuda.empty_cache()
    total = sum(v["flips_per_s"] * v["seconds"] for v in out.values()) / sum(v["seconds"] for v in out.values())
    workload = ("L=303 and L=501, %d walkers each, %d steps, seed 42, uniform random +-1 Philox starts, HT 2^16 "
                "slots/walker" % (args.scaleup_walkers, args.scaleup_steps))
    peak_source = ("fma_frac: derived, %d SMs x %d FP32 lanes x 2 FLOP x %.0f MHz (FMA pipe); tensor_frac: of "
                   "measured sustained BF16 GEMM rate %.1f TFLOP/s (FP16 shares the dense rate)"
                   % (sms, FP32_LANES_PER_SM, sm_mhz, tensor_peak() / 1e12))
    return total, out, workload, peak_source


def run_scaleup(args):
    """Config 5: L=303 and L=501, 131072 walkers each, 2e4 steps of the plain walk (the
    learned proposal is measured by --config learned): flips/s, the walk kernel's
    roofline fraction, best F and the time to F >= 8 (sampled every 1000 steps); one
    JSON line."""
    import torch

    import paper_2011_00068_gb300 as labs

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    total, out, workload, peak_source = scaleup_measure(args, dev, labs)
    line = {"metric": "exact flip evaluations/sec, L=303 and L=501 scale-up", "value": total,
            "unit": "flip evaluations/s", "higher_is_better": True, "n_gpus": 1, "dtype": "f32",
            "data": "synthetic", "vs_baseline": None,
            "config": {"workload": workload, "peak_source": peak_source},
            "per_L": out}
    print(json.dumps(line))
    return 0


def run_long(args):
    """Long sequences (one walker per CTA): L = 2047, 4095, 8191 and 11263, long_walkers
    walkers x long_steps steps each of the walk (ISL or PSL objective) or the best-first
    search: flips/s, the kernel's roofline fraction (one FMA per lag term, as the warp
    kernels), best F; one JSON line."""
    import torch

    import paper_2011_00068_gb300 as labs
    from paper_2011_00068_gb300 import _native

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = float(measured_peaks().get("sm_max_mhz", 2070.0))
    peak = FP32_LANES_PER_SM * 2 * sms * sm_mhz * 1e6
    out = {}
    objective = "psl" if args.search == "psl" else "isl"
    flags = _native.LABS_FLAG_BEST_FIRST if args.search == "bestfirst" else 0
    for L in (2047, 4095, 8191, 11263):
        n = (L + 1) // 2
        s = labs.Search(L, args.long_walkers, 42, device=dev, objective=objective, flags=flags)
        s.walk(8)  # warm-up: graph capture, first touch of the tables
        s.sync()
        s.reset()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s.stream)
        s.walk(args.long_steps)
        b.record(s.stream)
        s.sync()
        ms = a.elapsed_time(b)
        st = s.stats()
        flips = st["flip_evaluations"] / (ms / 1e3)
        best = s.best()
        out[str(L)] = {"flips_per_s": flips, "ms": ms, "steps": args.long_steps, "walkers": args.long_walkers,
                       "walker_steps_per_s": st["steps"] / (ms / 1e3), "best_isl": best["isl"],
                       "best_F": best["F"], "lane_block": st["lane_block"], **lag_roofline(n, flips, st, peak)}
        if objective == "psl":
            # FP32 lane operations of the PSL terms: PSL_LANE_OPS_PER_LAG_TERM per lag term
            out[str(L)]["psl_lane_op_frac"] = PSL_LANE_OPS_PER_LAG_TERM * (n - 1) * flips / (peak / 2)
        if objective == "psl":
            out[str(L)]["best_psl"] = best["psl"]
        s.close()
        del s
        torch.cuda.empty_cache()
    total = sum(v["flips_per_s"] * v["ms"] for v in out.values()) / sum(v["ms"] for v in out.values())
    what = {"psl": ", PSL objective", "bestfirst": ", best-first search"}.get(args.search, "")
    line = {"metric": "exact flip evaluations/sec, long sequences" + what,
            "value": total, "unit": "flip evaluations/s",
            "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic", "vs_baseline": None,
            "config": {"workload": "L=2047, 4095, 8191 and 11263, %d walkers each (one per CTA of 128, 256 or 512 threads), %d steps, "
                                   "seed 42, uniform random +-1 Philox starts, HT 2^16 slots/walker"
                                   % (args.long_walkers, args.long_steps),
                       "kernel": "long_walk_kernel",
                       "peak_source": "fma_frac: derived, %d SMs x %d FP32 lanes x 2 FLOP x %.0f MHz (FMA pipe); "
                                      "tensor_frac: of measured sustained BF16 GEMM rate %.1f TFLOP/s (FP16 shares "
                                      "the dense rate)" % (sms, FP32_LANES_PER_SM, sm_mhz, tensor_peak() / 1e12)},
            "per_L": out}
    print(json.dumps(line))
    return 0


def run_secondhash(args):
    """The ablation of Section 3: the best-first search at L = args.L with and without
    xLastovka's second table of evaluated neighbours, args.walkers walkers x
    args.walk_steps steps each: time, flips/s, the share of neighbours the table
    skipped, best F; one JSON line."""
    import torch

    import paper_2011_00068_gb300 as labs
    from paper_2011_00068_gb300 import _native

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = (args.L + 1) // 2
    out = {}
    plain, cached = _native.LABS_FLAG_BEST_FIRST, _native.LABS_FLAG_BEST_FIRST | _native.LABS_FLAG_SECOND_HASH
    runs = [("without", plain, args.walk_steps), ("with", cached, args.walk_steps), ("without_equal_time", plain, 0)]
    for name, flags, steps in runs:
        if name == "without_equal_time":  # as many steps as fit in the time the table's run took
            steps = int(round(args.walk_steps * out["with"]["ms"] / out["without"]["ms"]))
        s = labs.Search(args.L, args.walkers, args.seed, device=dev, flags=flags)
        s.walk(64)
        s.sync()
        s.reset()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s.stream)
        s.walk(steps)
        b.record(s.stream)
        s.sync()
        ms = a.elapsed_time(b)
        st = s.stats()
        best = s.best()
        out[name] = {"ms": ms, "steps": steps, "flips_per_s": st["flip_evaluations"] / (ms / 1e3),
                     "skipped_share": st["cache_hits"] / st["flip_evaluations"],
                     "new_evaluations_per_s": (st["flip_evaluations"] - st["cache_hits"]) / (ms / 1e3),
                     "best_isl": best["isl"], "best_F": best["F"], "restarts": st["restarts"]}
        s.close()
        del s
        torch.cuda.empty_cache()
    line = {"metric": "best-first search with and without the second table", "value": out["with"]["flips_per_s"],
            "unit": "flip evaluations/s", "higher_is_better": True, "n_gpus": 1, "dtype": "f32",
            "data": "synthetic", "vs_baseline": None,
            "config": {"workload": "L=%d best-first search (queue of 32), %d walkers x %d steps, seed %d, HT and "
                                   "second table 2^16 slots/walker each" % (args.L, args.walkers, args.walk_steps,
                                                                           args.seed), "n": n},
            "runs": out}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "secondhash":
        return run_secondhash(args)
    if args.config == "long":
        return run_long(args)
    if args.config == "learned":
        return run_learned(args)
    if args.config == "scaleup":
        return run_scaleup(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
