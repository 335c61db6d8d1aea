"""Benchmark: paths/s of the GPU path tracker on the cyclic 7 batch.

Workload: cyclic 7-roots plus 8 copies with its supports and random complex
Gaussian coefficients (seed 2), total-degree homotopies, 9 x 5040 = 45,360
paths per step.  One step = track every path of the 9 systems (one batch
handle: the tracker launch, the tail launch that finishes the paths still
running when most threads are idle, and classification), then refine the
ill-conditioned endpoints in double double.  The homotopy tables are
resident in HBM before the timed region; the L2 is flushed (a 256 MiB
write) between steps.

Line printed (rank 0, one JSON object): the device-timed value and Newton
steps/s, an end-to-end value through the C ABI with host buffers (table
upload and endpoint download inside the timed region), the roofline of the
tracking call (track + tail kernels, FP64 ALU bound), the served latency of
Poisson-arriving small requests (continuous batching), the oracle timed on
the host cores, SM clocks sampled during the timed region and the kernel
launch count.

``--impl reference`` times the CPU oracle (the reference of this project)
on the same workload instead.  ``--gpus N`` under torchrun runs N
independent replicas (paths are independent; nothing is exchanged).
``--workload serving`` runs the serving workload alone; ``--workload
configs`` measures all five workloads, one line each (``--configs 9,10,11``:
cyclic 9 D=2 stages, double double tracking, polyhedral homotopies).
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

METRIC = "paths/s at 1e-10 endpoint acc; % FP64 peak; served p50/p99 latency"
WORKLOAD = "cyclic7 + 8 random-coefficient copies (seed 2): 9 x 5040 = 45,360 total-degree paths"
# FP64 peak: 152 SMs x 2 FP64 FMA lanes/clk x 2 flops x 2.07 GHz = 1.259 TFLOP/s (the nominal 1.25);
# an FMA-chain probe on this GPU measured 1.257 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 peak: 152 SMs x 128 FP32 FMA lanes/clk x 2 flops x 2.07 GHz = 80.5 TFLOP/s (probe: 73.4).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# ------------------------------------------------------------------ flop model

def unit_flops(tab_terms, n: int) -> float:
    """FP64 flops of one evaluate+factor+solve unit as the tracker executes it
    (a fused multiply-add counts 2, a multiplication, addition or division 1;
    comparisons and absolute values 0), for a homotopy whose terms are
    (support size k, sum of (a_j - 1)) pairs.  Per term: c(t) = c0 + t c1
    (2 FMA); a constant adds c(t) to its row of the right-hand side (2);
    an exponent-one term (sum 0) runs k - 1 prefix and k - 1 suffix complex
    multiplications (6 each), k - 1 complex fused multiply-adds into H_x (8
    each), one complex addition (2) and one into the right-hand side (8):
    20k - 6; a term with powers adds the common factor (sum (a_j - 1)
    complex multiplications), c(t) times it (6), the exponent scalings
    (2 per variable) and x^a = cf * suffix (6): 22k + 6 sum + 6.  Complex LU
    with partial pivoting: per column the |.|_1 sums of the pivot search (1
    each), the reciprocal of the pivot (6), m multipliers (6 each) and m^2
    trailing updates (8 each), m = n - 1 - column; one solve: n(n-1)/2
    complex fused multiply-adds forward and backward (8 each) and n
    multiplications by the reciprocal pivots (6).  The step logic between
    units (Runge-Kutta combinations, norms) is not counted."""
    f = 0.0
    for k, extra in tab_terms:
        f += 4  # c(t)
        if k == 0:
            f += 2
        elif extra == 0:
            f += 20 * k - 10
        else:
            f += 22 * k + 6 * extra + 2
    for col in range(n):
        m = n - 1 - col
        f += (m + 1) + 6 + 6 * m + 8 * m * m
    f += 8 * n * (n - 1) + 6 * n
    return f


def poly_unit_flops(sys_) -> float:
    """FP64 flops of one unit of the polyhedral tracker: the terms of the
    system itself (no start system), each with the coefficient c t^p and
    c p t^(p-1) (6 flops; the exponential is not counted), and the LU and
    solve of unit_flops."""
    exps = np.asarray(sys_.exps, dtype=np.int64).reshape(-1, sys_.n_var)
    terms = []
    for e in exps:
        nz = e[e > 0]
        terms.append((len(nz), int((nz - 1).sum())))
    return unit_flops(terms, sys_.n_var) + 2 * len(terms)


def homotopy_terms(sys_):
    """(k, sum(a_j-1)) of the terms of the total-degree homotopy of sys_ (an
    object with terms_per_eq and exps [T, n])."""
    out = []
    exps = np.asarray(sys_.exps, dtype=np.int64).reshape(-1, sys_.n_var)
    tpe = np.asarray(sys_.terms_per_eq, dtype=np.int64)
    bounds = np.concatenate([[0], np.cumsum(tpe)])
    degs = [int(exps[bounds[i]:bounds[i + 1]].sum(axis=1).max()) for i in range(len(tpe))]
    for e in exps:
        nz = e[e > 0]
        out.append((len(nz), int((nz - 1).sum())))
    for d in degs:
        out.append((1, int(d) - 1))  # x_i^{d_i}
        out.append((0, 0))  # constant
    return out


# ------------------------------------------------------------------ clocks

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
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ distributed helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, paths_per_rank: int, steps: int, max_total_ms: float) -> float:
    """Whole-job paths/s of N independent replicas: every rank tracks the same
    workload, timed by the slowest rank (weak scaling)."""
    return world * paths_per_rank * steps / (max_total_ms / 1e3)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ CPU oracle arm

def oracle_sample(systems, gammas, per_system: int, seed: int = 7, threads: int | None = None):
    """Time the oracle (work crew on every host core, or `threads`) on
    per_system seeded random paths of every system (all of them when
    per_system >= the system's path count); returns (paths/s, cores, paths,
    secs).  The start solutions of the sample are computed before the timed
    region."""
    import oracle
    rng = np.random.Generator(np.random.PCG64(seed))
    cores = threads or oracle.host_threads()
    jobs = []
    for s, g in zip(systems, gammas):
        h = oracle.total_degree(s, g)
        P = oracle.num_paths(h)
        if per_system >= P:
            jobs.append((h, None, P))
        else:
            idx = np.sort(rng.choice(P, size=per_system, replace=False))
            starts = np.array([oracle.start_solution(h, int(p)) for p in idx])
            jobs.append((h, starts, per_system))
    t0 = time.perf_counter()
    n = 0
    for h, starts, k in jobs:
        if starts is None:
            oracle.track(h, threads=cores)
        else:
            oracle.track(h, starts=starts, threads=cores)
        n += k
    dt = time.perf_counter() - t0
    return n / dt, cores, n, dt


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from workloads import configs
    w = configs.cyclic7_batch()
    per = args.ref_sample
    for _ in range(args.warmup):
        oracle_sample(w.systems, w.gammas, max(50, per // 10))
    vals, secs = [], []
    for _ in range(args.steps):
        v, cores, n, dt = oracle_sample(w.systems, w.gammas, per)
        vals.append(v)
        secs.append(dt)
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{per} seeded random paths per system, 9 systems"},
        "cpu_baseline": {"value": value, "unit": "paths/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per} x 9 seeded random paths per step"},
        "e2e": {"value": value, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def run_gpu(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1804_03807_gb300 import build as pbuild
    pbuild.build()
    import paper_1804_03807_gb300 as P
    from workloads import configs

    w = configs.cyclic7_batch()
    systems, gammas = w.systems, w.gammas
    # one handle for the 9 systems (shared supports): one launch, one path queue
    h = P.phc_make_homotopy_batch(systems, gammas)
    total_paths = P.phc_num_paths(h)
    main = torch.cuda.current_stream(dev)
    x = torch.empty((h.n, total_paths), dtype=torch.complex128, device=dev)
    cls = torch.empty(total_paths, dtype=torch.int8, device=dev)
    st = torch.empty((total_paths, P.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    xlo = torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    opts = P.phc_default_opts(precision=args.precision)
    if args.tail_drain is not None:
        opts.tail_drain = args.tail_drain
    if args.block_threads:
        opts.block_threads = args.block_threads
    if args.tail_threads:
        opts.tail_threads = args.tail_threads
    tail_on = opts.tail_drain > 0  # FP32 interior too: its double-only paths hand off
    launches_per_step = 4 if tail_on else 3  # track, (tail,) classify, refine

    def step(pair=None):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(main)
        P.phc_track_paths(h, 0, total_paths, opts, x, cls, st, stream=main)
        e1.record(main)
        P.phc_refine_endpoints(h, x, xlo, total_paths, 1e6, 1e12, 8, cls, st, stream=main)
        if pair is not None:
            pair.append((e0, e1))

    for _ in range(args.warmup):
        step()
        flush.fill_(1)
    torch.cuda.synchronize()

    # flop model per unit (all systems share the structure)
    uf = unit_flops(homotopy_terms(systems[0]), systems[0].n_var)

    barrier(world)
    torch.cuda.synchronize()
    times, pairs = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(main)
            step(pairs)
            b.record(main)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.summary()
    total_ms = max_over_ranks(float(np.sum(times)), world, dev)
    value = replica_value(world, total_paths, args.steps, total_ms)

    # roofline of track_kernel: algorithmic flops / duration of the tracking
    # call; units done in single precision count against the FP32 peak
    stn = P.stats_numpy(st)
    tail_paths, tail_units = P.phc_tail_paths(h, main, units=True)
    units = int(stn["n_solve"].sum())
    units32 = int(stn["n_fp32"].sum())
    f64 = (units - units32) * uf
    f32 = units32 * uf
    kern_ms = float(np.mean([p0.elapsed_time(p1) for p0, p1 in pairs]))
    # DRAM bytes (read + write) per tracking call: ncu counters of track_kernel<7,0>
    # (985,344 + 82,688 B) and tail_kernel<7,32> (785,664 + 0 B) tracking one system
    # of this batch (5040 paths, 3,969,533 units), scaled by the units of this step.
    # Only meaningful for the default FP64 configuration those kernels ran in.
    traffic = args.traffic
    if traffic is None and args.precision == 0 and tail_on and (opts.tail_threads or 32) == 32:
        traffic = (985_344 + 82_688 + 785_664) * units / 3_969_533
    secs = kern_ms / 1e3
    # the same peak measured on this device (independent FMA chains, every SM)
    probe = P.phc_fp64_probe(16, 200_000, stream=main)
    frac = (f64 / secs / 1e12) / FP64_PEAK_TFLOPS
    frac32 = (f32 / secs / 1e12) / FP32_PEAK_TFLOPS
    roofline = {"bound": "alu", "achieved": f64 / secs / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": frac, "fp32_frac": frac32, "traffic": traffic,
                "kernel": (f"track_kernel<7> + tail_kernel<7,{opts.tail_threads or 32}>" if tail_on else "track_kernel<7>") +
                          " (+classify_kernel<7>, <0.1 %)",
                "tail_paths_per_step": tail_paths, "tail_units_per_step": tail_units,
                "tail_drain": opts.tail_drain if tail_on else 0.0,
                "fp64_flops_per_step": f64,
                "fp32_flops_per_step": f32, "fp32_peak": FP32_PEAK_TFLOPS, "units_per_step": units,
                "fp32_units_per_step": units32, "kernel_ms": kern_ms,
                "flops_per_unit": uf,
                "peak_source": "derived: 152 SMs x 2 FP64 (128 FP32) FMA/clk x 2 flops x 2.07 GHz",
                "peak_probe": probe, "frac_of_probe": f64 / secs / 1e12 / probe if probe > 0 else None,
                "frac_formula": "frac = fp64_flops/peak/T; fp32_frac = fp32_flops/fp32_peak/T; "
                                "flops = units x flops_per_unit (FP64 flops the kernel executes per unit)"}

    # end to end through the C ABI with host buffers
    e2e = end_to_end(P, systems, gammas, dev, args)

    # correctness summary of the last step
    counts = np.bincount(cls.cpu().numpy(), minlength=4)

    line = {
        "metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(total_ms / args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": ["fp64", "fp32-interior"][args.precision],
                   "l2": "flushed (256 MiB write) between steps",
                   "parallelism": f"replicas x{world}", "classes_last_step": counts.tolist()},
        "roofline": roofline, "e2e": e2e, "clocks": clocks, "gpu_launches": launches_per_step * args.steps,
        # Newton corrections (corrector and end game) per second of the same steps, all ranks
        "newton_steps_per_s": world * int(stn["n_newton"].sum()) * args.steps / (total_ms / 1e3),
    }
    if rank == 0 and world == 1 and args.serving_requests > 0:
        # served latency (the third figure of the metric): Poisson arrivals of
        # small requests plus the cyclic 9 D=2 request (362,880 paths, two
        # cascade stages) arriving first, continuous batching
        sv, _ = serving_session(args.serving_requests, not args.no_big, args.slots, args.batch_paths)
        line["serving"] = {k: sv[k] for k in ("requests", "rate_per_s", "wall_s", "tracked_paths_per_s",
                                              "offered_small_paths_per_s", "achieved_small_paths_per_s",
                                              "latency_small", "latency_cyclic9_d2") if k in sv}
        line["serving"]["workload"] = (f"{args.serving_requests} Poisson (200/s) sparse requests, "
                                       "Bezout 1e2..1e3" + ("" if args.no_big else
                                       " + cyclic 9 D=2 (362,880 paths, 2 cascade stages) at t=0") +
                                       "; small requests batched on high-priority streams (phc_track_many), "
                                       "the large one in chunks on low-priority streams")
    if rank == 0 and world == 1 and args.batching:
        line["batching"] = batching_numbers()
    if rank == 0 and not args.no_cpu_baseline:
        # the whole workload on every host core, and a seeded sample on one core
        v, cores, n, dt = oracle_sample(systems, gammas, 10 ** 9)
        v1, _, n1, dt1 = oracle_sample(systems, gammas, 100, threads=1)
        line["cpu_baseline"] = {"value": v, "unit": "paths/s", "cores": cores, "kind": "oracle",
                                "sample": f"the whole workload ({n} paths), {dt:.1f} s wall",
                                "one_core": {"value": v1, "unit": "paths/s", "cores": 1,
                                             "sample": f"{n1} seeded random paths (100 per system), {dt1:.1f} s"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batching_numbers():
    """The batching workload (256 random sparse systems of uneven size,
    4,322,140 paths): one phc_track_many call against one phc_track_paths
    launch per system, device time (CUDA events), one run each after a
    warm-up run of each."""
    import paper_1804_03807_gb300 as P
    from workloads import configs
    w = configs.sparse_batch()
    hs = [P.phc_make_homotopy(s, g) for s, g in zip(w.systems, w.gammas)]
    npaths = sum(P.phc_num_paths(x) for x in hs)
    ms = _timed(lambda: P.track_many(hs), 1, 1)
    ms1 = _timed(lambda: [P.track(x) for x in hs], 1, 1)
    return {"workload": f"256 random sparse systems, n 3..10, {npaths:,} total-degree paths",
            "paths_per_s": npaths / (ms / 1e3), "ms": ms,
            "one_launch_per_system": {"paths_per_s": npaths / (ms1 / 1e3), "ms": ms1}}


def end_to_end(P, systems, gammas, dev, args):
    """Same metric through the C ABI from host lists to host endpoints: per
    step the batch homotopy is built from host lists (tables uploaded),
    tracked, refined, and endpoints and classes are copied to pinned host
    memory."""
    import torch
    total = sum(s.bezout() for s in systems)
    xh = torch.empty((systems[0].n_var, total), dtype=torch.complex128, pin_memory=True)
    ch = torch.empty(total, dtype=torch.int8, pin_memory=True)
    opts = P.phc_default_opts(precision=args.precision)
    if args.tail_drain is not None:
        opts.tail_drain = args.tail_drain
    if args.block_threads:
        opts.block_threads = args.block_threads
    if args.tail_threads:
        opts.tail_threads = args.tail_threads

    def one():
        h = P.phc_make_homotopy_batch(systems, gammas)
        bytes_in = sum(s.exps.nbytes + s.coefs.nbytes + s.terms_per_eq.nbytes for s in systems)
        r = P.track(h, opts=opts, device=dev)
        xlo = torch.empty_like(r.x)
        P.phc_refine_endpoints(h, r.x, xlo, total, 1e6, 1e12, 8, r.cls, r.stats)
        xh.copy_(r.x, non_blocking=True)
        ch.copy_(r.cls, non_blocking=True)
        torch.cuda.synchronize()
        return bytes_in, r.x.numel() * 16 + r.cls.numel()

    one()
    reps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(reps):
        bi, bo = one()
    dt = time.perf_counter() - t0
    return {"value": total * reps / dt, "unit": "paths/s", "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo),
            "steps": reps}


def serving_session(n_requests: int, big: bool, slots: int, batch_paths: int = 60_000):
    """Continuous batching of Poisson arrivals (200/s) of sparse requests,
    optionally with cyclic 9 embedded for top dimension 2 (362,880 paths, two
    cascade stages) arriving first; returns the measurement and the requests."""
    from paper_1804_03807_gb300 import serving
    from workloads import configs
    w = configs.serving(n_requests=n_requests, rate=200.0, seed=5, bezout_range=(100, 1000),
                        big=(9, 2) if big else None)
    reqs = [serving.Request(i, s, g, float(a)) for i, (s, g, a) in
            enumerate(zip(w.systems, w.gammas, w.extra["arrivals"]))]
    small = set(r.rid for r in reqs)
    if big:
        b = w.extra["big"]
        reqs.append(serving.Request(len(reqs), b["system"], b["gamma"], b["arrival"], b["top_dim"], b["gammas"],
                                    b["hyper"]))
    srv = serving.Server(slots=2, max_inflight=slots, batch_paths=batch_paths)
    srv.run(reqs[:8], realtime=False)  # warm-up: kernels loaded, allocator primed
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        res = srv.run(reqs)
        wall = time.perf_counter() - t0
    paths = sum(r.n_paths * len(r.stages) for r in res)
    top_paths = sum(r.n_paths for r in res)
    small_paths = sum(r.n_paths for r in res if r.rid in small)
    last_small = max(r.finished for r in res if r.rid in small)
    out = {"requests": len(reqs), "rate_per_s": 200.0, "wall_s": wall, "paths_per_s": top_paths / wall,
           "tracked_paths_per_s": paths / wall,
           "offered_small_paths_per_s": small_paths / max(w.extra["arrivals"][-1], 1e-9),
           "achieved_small_paths_per_s": small_paths / max(last_small, 1e-9),
           "latency_small": serving.latency_summary(res, small), "clocks": clk.summary(), "slots": slots}
    if big:
        out["latency_cyclic9_d2"] = serving.latency_summary(res, set(r.rid for r in reqs) - small)
    return out, reqs


def run_serving(args):
    """Config 5: Poisson arrivals (200/s) of sparse requests plus cyclic 9
    embedded for top dimension 2 (362,880 paths, two cascade stages)
    arriving first; continuous batching on one GPU."""
    import torch
    from paper_1804_03807_gb300 import build as pbuild
    pbuild.build()
    torch.cuda.set_device(0)
    sv, reqs = serving_session(args.requests, not args.no_big, args.slots, args.batch_paths)
    line = {"metric": METRIC, "workload": "serving", "value": sv["paths_per_s"], "unit": "paths/s",
            "tracked_paths_per_s": sv["tracked_paths_per_s"], "n_requests": sv["requests"], "wall_s": sv["wall_s"],
            "latency_small": sv["latency_small"], "latency_cyclic9_d2": sv.get("latency_cyclic9_d2", {"count": 0}),
            "offered_small_paths_per_s": sv["offered_small_paths_per_s"], "slots": args.slots,
            "clocks": sv["clocks"],
            "config": {"workload": f"{args.requests} Poisson (200/s) sparse requests, Bezout 1e2..1e3"
                       + ("" if args.no_big else " + cyclic 9 D=2 (362,880 paths, 2 cascade stages) at t=0")}}
    if not args.no_cpu_baseline:
        v, cores, n, dt = oracle_sample([r.system for r in reqs[:40]], [r.gamma for r in reqs[:40]], 100)
        line["cpu_baseline"] = {"value": v, "unit": "paths/s", "cores": cores, "kind": "oracle",
                                "sample": f"{n} paths of the first 40 requests, {dt:.1f} s wall"}
    print(json.dumps(line), flush=True)
    return 0


def _timed(fn, reps: int, warmup: int = 2):
    """Mean device time (ms) of fn() on the current stream over reps calls
    (CUDA events, synchronised on both sides)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_configs(args):
    """Every workload of the benchmark list on one GPU (or those in
    --configs), one JSON line each: paths/s and Newton steps/s (device
    time), the FP64 fraction of the flop model, the one-launch-per-system
    (or per-stage) variant where one exists, and the oracle on a bounded
    sample of the same workload."""
    import torch
    from paper_1804_03807_gb300 import build as pbuild
    pbuild.build()
    import oracle
    import paper_1804_03807_gb300 as P
    from workloads import configs
    torch.cuda.set_device(0)
    peak = FP64_PEAK_TFLOPS * 1e12
    out = {}

    def summary(rs, flops_per_unit, ms):
        units = newton = 0
        flops = 0.0
        for r, fpu in zip(rs, flops_per_unit):
            st = P.stats_numpy(r.stats)
            live = r.cls.cpu().numpy() >= 0  # a stage's entries that tracked a path
            units += int(st["n_solve"][live].sum())
            newton += int(st["n_newton"][live].sum())
            flops += float(st["n_solve"][live].sum()) * fpu
        return {"newton_steps_per_s": newton / (ms / 1e3), "fp64_frac": flops / (ms / 1e3) / peak,
                "units": units}

    def oracle_part(systems, gammas, per_system, what):
        v, cores, n, dt = oracle_sample(systems, gammas, per_system)
        return {"paths_per_s": v, "cores": cores, "sample": f"{n} {what} ({dt:.1f} s)"}

    def config1():
        w = configs.dense4()
        h = P.phc_make_homotopy(w.systems[0], w.gammas[0])
        ms = _timed(lambda: out.__setitem__("r", P.track(h)), 50)
        d = {"config": 1, "workload": "dense n=4, degree 2, 16 paths", "paths_per_s": 16 / (ms / 1e3), "ms": ms}
        d.update(summary([out["r"]], [unit_flops(homotopy_terms(w.systems[0]), 4)], ms))
        for drain in (0.0, 0.8):
            o = P.phc_default_opts(tail_drain=drain)
            msd = _timed(lambda: P.track(h, opts=o), 50)
            d[f"tail_drain_{drain}"] = {"ms": msd, "paths_per_s": 16 / (msd / 1e3)}
        for g in (8, 16):
            o = P.phc_default_opts(tail_threads=g)
            msg = _timed(lambda: P.track(h, opts=o), 50)
            d[f"tail_threads_{g}"] = {"ms": msg, "paths_per_s": 16 / (msg / 1e3)}
        d["oracle"] = oracle_part(w.systems * 200, w.gammas * 200, 16, "paths")
        return d

    def config2():
        w = configs.cyclic7_batch()
        hb = P.phc_make_homotopy_batch(w.systems, w.gammas)
        hs = [P.phc_make_homotopy(s, g) for s, g in zip(w.systems, w.gammas)]
        ms = _timed(lambda: out.__setitem__("r", P.track(hb)), 3)
        d = {"config": 2, "workload": "cyclic 7 + 8 random copies, 45,360 paths, one batch launch",
             "paths_per_s": 45360 / (ms / 1e3), "ms": ms}
        d.update(summary([out["r"]], [unit_flops(homotopy_terms(w.systems[0]), 7)], ms))
        ms1 = _timed(lambda: [P.track(x) for x in hs], 3)
        d["one_launch_per_system"] = {"paths_per_s": 45360 / (ms1 / 1e3), "ms": ms1}
        d["oracle"] = oracle_part(w.systems, w.gammas, 400, "paths")
        return d

    def config3():
        w = configs.cyclic8_d1()
        base, gamma = w.systems[0], w.gammas[0]
        E = P.phc_embed(base, 1, w.embed["gammas"], w.embed["hyper"])
        h = P.phc_make_homotopy(E, gamma)
        fpu = unit_flops(homotopy_terms(E), 9)

        def piped():
            top, nxt = P.pipeline(h, 1)
            P.refine(h, top, cond_threshold=1e8)
            out["r"] = (top, nxt)

        def staged():
            top = P.track(h)
            P.refine(h, top, cond_threshold=1e8)
            out["s"] = (top, P.cascade_from(h, 1, top))

        ms = _timed(piped, 2, 1)
        d = {"config": 3, "workload": "cyclic 8 embedded D=1: 40,320 paths + cascade stage, pipelined in one launch",
             "paths_per_s": 40320 / (ms / 1e3), "ms": ms}
        d.update(summary(list(out["r"]), [fpu, fpu], ms))
        ms1 = _timed(staged, 2, 1)
        d["one_launch_per_stage"] = {"paths_per_s": 40320 / (ms1 / 1e3), "ms": ms1}
        Eo = oracle.embed(base, 1, w.embed["gammas"], w.embed["hyper"])
        d["oracle"] = oracle_part([Eo], [gamma], 2000, "top-stage paths")
        return d

    def config4():
        w = configs.sparse_batch()
        hs = [P.phc_make_homotopy(s, g) for s, g in zip(w.systems, w.gammas)]
        npaths = sum(P.phc_num_paths(x) for x in hs)
        fpus = [unit_flops(homotopy_terms(s), s.n_var) for s in w.systems]
        ms = _timed(lambda: out.__setitem__("r", P.track_many(hs)), 1, 1)
        d = {"config": 4, "workload": f"256 sparse systems, n 3..10, {npaths:,} paths, phc_track_many",
             "paths_per_s": npaths / (ms / 1e3), "ms": ms}
        d.update(summary(out["r"], fpus, ms))
        ms1 = _timed(lambda: [P.track(x) for x in hs], 1, 1)
        d["one_launch_per_system"] = {"paths_per_s": npaths / (ms1 / 1e3), "ms": ms1}
        # launch parameters chosen by the project's tuner on a sample of the systems
        from paper_1804_03807_gb300 import autotune
        t0 = time.perf_counter()
        o = autotune.tune_many(hs, sample_systems=16,
                               grid={"tail_threads": (16, 32), "tail_drain": (0.8, 0.9), "block_threads": (0, 128)})
        tune_s = time.perf_counter() - t0
        ms2 = _timed(lambda: P.track_many(hs, opts=o), 1, 1)
        d["autotuned"] = {"paths_per_s": npaths / (ms2 / 1e3), "ms": ms2, "tuning_s": tune_s,
                          "opts": {"tail_threads": o.tail_threads, "tail_drain": o.tail_drain,
                                   "block_threads": o.block_threads}}
        d["oracle"] = oracle_part(w.systems[:40], w.gammas[:40], 100, "paths of 40 systems")
        return d

    def config9():
        """The large request of the serving workload alone: cyclic 9 embedded
        for top dimension 2 (11 unknowns, 362,880 paths), top stage, then its
        two cascade stages chained on the device."""
        w = configs.serving(n_requests=1, big=(9, 2))
        b = w.extra["big"]
        E = P.phc_embed(b["system"], b["top_dim"], b["gammas"], b["hyper"])
        h = P.phc_make_homotopy(E, b["gamma"])
        E1 = P.phc_embed(b["system"], 1, b["gammas"][:, :1], b["hyper"][:1])
        h1 = P.phc_make_homotopy(E1, b["gamma"])
        ms = _timed(lambda: out.__setitem__("r", P.track(h)), 1, 1)
        top = out["r"]
        d = {"config": "5-big", "workload": "cyclic 9 embedded D=2: 362,880 paths, top stage alone",
             "paths_per_s": 362880 / (ms / 1e3), "ms": ms}
        d.update(summary([top], [unit_flops(homotopy_terms(E), 11)], ms))
        d["classes_top"] = np.bincount(top.cls.cpu().numpy(), minlength=4).tolist()

        def stages():
            s2 = P.cascade_from(h, 2, top)
            s1 = P.cascade_from(h1, 1, s2)
            out["s"] = (s2, s1)
        ms2 = _timed(stages, 1, 1)
        s2, s1 = out["s"]
        n2 = int((s2.cls.cpu().numpy() >= 0).sum())
        n1 = int((s1.cls.cpu().numpy() >= 0).sum())
        d["cascade"] = {"ms": ms2, "paths": [n2, n1], "paths_per_s": (n2 + n1) / (ms2 / 1e3)}
        d["cascade"].update(summary([s2, s1], [unit_flops(homotopy_terms(E), 11),
                                              unit_flops(homotopy_terms(E1), 10)], ms2))
        return d

    def config10():
        """Double double tracking (Section 5, Table 2: the solver in double
        double): one random-coefficient cyclic 7 copy (5040 paths), against
        the same paths in double precision."""
        w = configs.cyclic7_batch()
        h = P.phc_make_homotopy(w.systems[1], w.gammas[1])
        ms = _timed(lambda: out.__setitem__("r", P.track_dd(h)), 1, 1)
        r, _ = out["r"]
        ms64 = _timed(lambda: P.track(h), 3, 1)
        st = P.stats_numpy(r.stats)
        return {"config": "dd", "workload": "cyclic 7 random copy 1, 5040 paths, complex double double",
                "paths_per_s": 5040 / (ms / 1e3), "ms": ms, "units": int(st["n_solve"].sum()),
                "classes": np.bincount(r.cls.cpu().numpy(), minlength=4).tolist(),
                "fp64": {"paths_per_s": 5040 / (ms64 / 1e3), "ms": ms64}}

    def config12():
        """The precision ladder of Section 5 and Table 2 (the solver in double,
        double double and quad double): the total-degree paths of one
        random-coefficient cyclic 7 copy (5040 paths) tracked in each."""
        w = configs.cyclic7_batch()
        h = P.phc_make_homotopy(w.systems[1], w.gammas[1])
        P.track_qd(h, n_paths=64)  # first launch: module and local memory set-up
        ms_qd = _timed(lambda: out.__setitem__("q", P.track_qd(h)), 1, 0)
        r, _ = out["q"]
        ms_dd = _timed(lambda: out.__setitem__("d", P.track_dd(h)), 1, 1)
        ms64 = _timed(lambda: out.__setitem__("f", P.track(h)), 3, 1)
        st = P.stats_numpy(r.stats)
        cls = {k: np.bincount(out[k][0].cls.cpu().numpy() if k != "f" else out[k].cls.cpu().numpy(),
                              minlength=4).tolist() for k in ("q", "d", "f")}
        # the oracle beside it: the same copy's first 32 paths in each precision
        oh = oracle.total_degree(w.systems[1], w.gammas[1])
        ncores = oracle.host_threads()
        t0 = time.perf_counter()
        oracle.track(oh, first=0, n_paths=32, threads=ncores)
        t_d = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.track_dd(oh, first=0, n_paths=32, threads=ncores)
        t_dd = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.track_qd(oh, first=0, n_paths=32, threads=ncores)
        t_qd = time.perf_counter() - t0
        orc = {"sample": "paths 0..31 of the same copy", "cores": ncores, "double_paths_per_s": 32 / t_d,
               "double_double_paths_per_s": 32 / t_dd, "quad_double_paths_per_s": 32 / t_qd,
               "ratios": {"dd_over_d": t_dd / t_d, "qd_over_d": t_qd / t_d}}
        return {"config": "precision ladder", "oracle": orc,
                "workload": "cyclic 7 random copy 1, 5040 total-degree paths",
                "double": {"ms": ms64, "paths_per_s": 5040 / (ms64 / 1e3), "classes": cls["f"]},
                "double_double": {"ms": ms_dd, "paths_per_s": 5040 / (ms_dd / 1e3), "classes": cls["d"]},
                "quad_double": {"ms": ms_qd, "paths_per_s": 5040 / (ms_qd / 1e3), "classes": cls["q"],
                                "units": int(st["n_solve"].sum())},
                "ratios": {"dd_over_d": ms_dd / ms64, "qd_over_d": ms_qd / ms64, "qd_over_dd": ms_qd / ms_dd}}

    def config13():
        """The pipelined polyhedral solve against the number of host threads
        that make the cells (Section 2.2, Figure 2; the paper's tables of the
        pipelined polyhedral homotopies time 2 to 64 tasks): random cyclic 10
        (35,940 paths), the cells made by p threads while the GPU tracks."""
        from workloads import cyclic, random_lifting, rng_for, with_random_coefficients
        g = with_random_coefficients(cyclic(10), rng_for(610))
        lift = random_lifting(rng_for(620), g.n_terms)
        rows, base = [], None
        old = os.environ.get("PHC_HOST_THREADS")
        try:
            for p in (1, 2, 4, 8, 16):
                os.environ["PHC_HOST_THREADS"] = str(p)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s = P.solve_polyhedral(g, lift, 40000)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                t0 = time.perf_counter()
                P.phc_mixed_cells(g, lift)
                dc = time.perf_counter() - t0
                base = base or dt
                rows.append({"threads": p, "pipeline_s": dt, "speedup": base / dt, "cells_alone_s": dc,
                             "paths": int(s.x.shape[1])})
        finally:
            if old is None:
                os.environ.pop("PHC_HOST_THREADS", None)
            else:
                os.environ["PHC_HOST_THREADS"] = old
        return {"config": "pipelined polyhedral vs host threads", "system": "cyclic 10, random coefficients",
                "rows": rows}

    def polyhedral_large(n: int, max_paths: int):
        """Random-coefficient cyclic n by the pipelined polyhedral solve
        (Section 2.2, Figure 2: the host threads make the mixed cells while
        the GPU tracks the paths of the cells made so far)."""
        from workloads import cyclic, random_lifting, rng_for, with_random_coefficients
        g = with_random_coefficients(cyclic(n), rng_for(900 + n))
        lift = random_lifting(rng_for(950 + n), g.n_terms)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = P.solve_polyhedral(g, lift, max_paths)
        torch.cuda.synchronize()
        t_pipe = time.perf_counter() - t0
        st = P.stats_numpy(r.stats)
        c = r.cls.cpu().numpy()
        far = c != 0
        return {"config": f"polyhedral-{n}", "workload": f"random cyclic {n}, pipelined polyhedral solve",
                "not_regular": {"norm_x": sorted(float(v) for v in st["norm_x"][far]),
                                "stop": np.bincount(st["stop"][far], minlength=6).tolist(),
                                "t": sorted(float(v) for v in st["t"][far])},
                "paths": int(c.shape[0]), "pipeline_s": t_pipe, "paths_per_s": c.shape[0] / t_pipe,
                "units": int(st["n_solve"].sum()), "classes": np.bincount(c, minlength=4).tolist(),
                "host_threads": os.cpu_count()}

    def config14():
        """Random cyclic 11: 184,756 paths (the number of roots of cyclic 11,
        C(20, 10)) against 11! = 39,916,800 total-degree paths."""
        return polyhedral_large(11, 184756)

    def config15():
        """Random cyclic 12: 500,352 paths (the mixed volume of cyclic 12)
        against 12! = 479,001,600 total-degree paths."""
        return polyhedral_large(12, 500352)

    def config11():
        """Polyhedral homotopies (Section 2.2) on random-coefficient cyclic
        n systems (n = 7 .. 10): the mixed cells on the host, the polyhedral
        paths on the GPU (one launch for all cells), the two-stage pipeline
        (cells made while the paths of the cells made so far are tracked),
        and the total-degree homotopy of the same system for comparison."""
        from workloads import cyclic, random_lifting, rng_for, unit_gamma, with_random_coefficients
        res = []
        for n in (7, 8, 9, 10):
            g = with_random_coefficients(cyclic(n), rng_for(600 + n))
            lift = random_lifting(rng_for(610 + n), g.n_terms)
            t0 = time.perf_counter()
            cells, vols, mv = P.phc_mixed_cells(g, lift)
            t_cells = time.perf_counter() - t0
            t0 = time.perf_counter()
            h = P.phc_make_polyhedral_homotopy(g, lift, cells)
            t_handle = time.perf_counter() - t0
            variants = {}
            for name, o in (("one_thread_per_path", P.phc_default_opts(group_paths=-1)),
                            ("group_32", P.phc_default_opts(group_paths=1, tail_threads=32)),
                            ("group_16", P.phc_default_opts(group_paths=1, tail_threads=16))):
                variants[name] = _timed(lambda: P.track_polyhedral(h, opts=o), 3, 1)
            ms = _timed(lambda: out.__setitem__("r", P.track_polyhedral(h)), 3, 1)
            r = out["r"]
            st = P.stats_numpy(r.stats)
            units = int(st["n_solve"].sum())
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s = P.solve_polyhedral(g, lift, mv)
            torch.cuda.synchronize()
            t_pipe = time.perf_counter() - t0
            same = bool(torch.equal(s.x, r.x))
            td = None
            if n <= 9:  # cyclic 10: 3,628,800 total-degree paths, left out
                ht = P.phc_make_homotopy(g, unit_gamma(rng_for(620 + n)))
                mst = _timed(lambda: out.__setitem__("t", P.track(ht)), 1, 1)
                ct = out["t"].cls.cpu().numpy()
                stt = P.stats_numpy(out["t"].stats)
                td = {"paths": int(ct.shape[0]), "ms": mst, "regular": int((ct == 0).sum()),
                      "units": int(stt["n_solve"].sum())}
            res.append({
                "system": f"cyclic {n}, random coefficients", "mixed_volume": mv, "cells": int(cells.shape[0]),
                "cells_s": t_cells, "handle_s": t_handle,
                "track_ms": ms, "track_ms_variants": variants, "paths_per_s": mv / (ms / 1e3), "units": units,
                "newton_steps_per_s": int(st["n_newton"].sum()) / (ms / 1e3),
                "fp64_frac": units * poly_unit_flops(g) / (ms / 1e3) / peak,
                "classes": np.bincount(r.cls.cpu().numpy(), minlength=4).tolist(),
                "pipeline_s": t_pipe, "pipeline_equals_one_launch": same,
                "total_degree": td,
            })
        # the paper's solve of a top dimensional system (Sections 2.2, 2.3):
        # polyhedral paths to a random-coefficient system with the embedded
        # system's supports, then the coefficient-parameter homotopy to the
        # embedded system; against the total-degree homotopy of the same
        w = configs.cyclic8_d1()
        e = w.embed
        E_lists = P.phc_embed(w.systems[0], e["top_dim"], e["gammas"], e["hyper"])
        from workloads import PolySystem
        E = PolySystem(E_lists.n_eq, E_lists.n_var, E_lists.terms_per_eq, E_lists.exps, E_lists.coefs, name="c8E1")
        g = with_random_coefficients(E, rng_for(630))
        lift = random_lifting(rng_for(631), g.n_terms)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sp = P.solve_polyhedral(g, lift, 1 << 16)
        hp = P.phc_make_parameter_homotopy(E, g.coefs, unit_gamma(rng_for(632)))
        rp = P.track_from(hp, sp.x)
        torch.cuda.synchronize()
        t_poly = time.perf_counter() - t0
        ht = P.phc_make_homotopy(E, w.gammas[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rt = P.track(ht)
        torch.cuda.synchronize()
        t_td = time.perf_counter() - t0

        def split(r):
            x, c = r.x.cpu().numpy().T, r.cls.cpu().numpy()
            fin = (c == 0) | (c == 1)
            z = np.abs(x[:, -1])
            return {"classes": np.bincount(c, minlength=4).tolist(), "regular_z0": int(((c == 0) & (z < 1e-8)).sum()),
                    "regular_z_nonzero": int(((c == 0) & (z >= 1e-8)).sum()), "finite": int(fin.sum())}
        emb = {"system": "cyclic 8 embedded for D = 1 (9 unknowns)", "mixed_volume": int(sp.x.shape[1]),
               "polyhedral_then_parameter_s": t_poly, "polyhedral_then_parameter": split(rp),
               "total_degree_paths": int(rt.cls.shape[0]), "total_degree_s": t_td, "total_degree": split(rt)}
        # the oracle beside it, on a bounded case it finishes in seconds: its own
        # cells (exact search in Python) and polyhedral paths of random cyclic 6
        from oracle import mixed as OM
        g6 = with_random_coefficients(cyclic(6), rng_for(606))
        lift6 = random_lifting(rng_for(616), g6.n_terms)
        t0 = time.perf_counter()
        oc = OM.mixed_cells(g6, lift6)
        t_oc = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, _, ocls, _, _ = OM.track_polyhedral(g6, lift6, oc, threads=oracle.host_threads())
        t_ot = time.perf_counter() - t0
        cells6, _, mv6 = P.phc_mixed_cells(g6, lift6)
        h6 = P.phc_make_polyhedral_homotopy(g6, lift6, cells6)
        ms6 = _timed(lambda: P.track_polyhedral(h6), 5, 2)
        orc = {"system": "cyclic 6, random coefficients (mixed volume 156)", "cores": oracle.host_threads(),
               "oracle_cells_s": t_oc, "oracle_track_s": t_ot, "oracle_paths_per_s": mv6 / t_ot,
               "oracle_regular": int((ocls == 0).sum()), "gpu_track_ms": ms6, "gpu_paths_per_s": mv6 / (ms6 / 1e3)}
        return {"config": "polyhedral", "systems": res, "embedded": emb, "oracle": orc}

    def config5():
        sv, reqs = serving_session(args.requests, not args.no_big, args.slots, args.batch_paths)
        d = {"config": 5, "workload": f"{args.requests} Poisson (200/s) sparse requests"
             + ("" if args.no_big else " + cyclic 9 D=2 (362,880 paths, two cascade stages)"),
             "paths_per_s": sv["paths_per_s"], "tracked_paths_per_s": sv["tracked_paths_per_s"],
             "wall_s": sv["wall_s"], "latency_small": sv["latency_small"],
             "latency_cyclic9_d2": sv.get("latency_cyclic9_d2"), "clocks": sv["clocks"]}
        d["oracle"] = oracle_part([r.system for r in reqs[:40]], [r.gamma for r in reqs[:40]], 100,
                                  "paths of 40 requests")
        return d

    want = [int(c) for c in args.configs.split(",")] if args.configs else [1, 2, 3, 4, 5]
    table = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5, 9: config9, 10: config10, 11: config11,
             12: config12, 13: config13, 14: config14, 15: config15}
    for c in want:
        print(json.dumps(table[c]()), flush=True)
    return 0


def profile_case(which: str = "cyclic7"):
    """A small case of a bench kernel, run twice: one random-coefficient
    cyclic 7 system (5040 paths, track_kernel single mode), 40 systems of
    the sparse batch (track_kernel multi-system mode), or the polyhedral
    paths of a random cyclic 7 system (924 paths, poly_group_kernel)."""
    import torch
    import paper_1804_03807_gb300 as P
    from workloads import configs
    if which == "polyhedral":
        from workloads import cyclic, random_lifting, rng_for, with_random_coefficients
        g = with_random_coefficients(cyclic(7), rng_for(607))
        lift = random_lifting(rng_for(617), g.n_terms)
        cells, _, mv = P.phc_mixed_cells(g, lift)
        h = P.phc_make_polyhedral_homotopy(g, lift, cells)
        for _ in range(2):
            r = P.track_polyhedral(h)
            torch.cuda.synchronize()
        print(json.dumps({"profile_case": "polyhedral cyclic7", "paths": mv,
                          "units": int(P.stats_numpy(r.stats)["n_solve"].sum())}))
        return 0
    if which == "sparse":
        w = configs.sparse_batch(count=40, seed=4)
        hs = [P.phc_make_homotopy(s, g) for s, g in zip(w.systems, w.gammas)]
        for _ in range(2):
            rs = P.track_many(hs)
            torch.cuda.synchronize()
        print(json.dumps({"profile_case": "sparse40", "paths": sum(P.phc_num_paths(h) for h in hs)}))
        return 0
    w = configs.cyclic7_batch()
    h = P.phc_make_homotopy(w.systems[1], w.gammas[1])
    for _ in range(2):
        r = P.track(h)
        torch.cuda.synchronize()
    print(json.dumps({"profile_case": w.systems[1].name, "classes": np.bincount(r.cls.cpu().numpy(), minlength=4).tolist(),
                      "units": int(P.stats_numpy(r.stats)["n_solve"].sum())}))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--ref-sample", type=int, default=400, help="oracle paths per system per step")
    ap.add_argument("--traffic", type=float, default=None, help="ncu DRAM bytes per track launch, if captured")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", type=int, default=0, help="0 = FP64, 1 = FP32 interior")
    ap.add_argument("--block-threads", type=int, default=0,
                    help="tracker threads per block (multiple of 32; default: as many as shared memory holds)")
    ap.add_argument("--tail-threads", type=int, default=0, help="threads per path in the tail kernel (8, 16, 32)")
    ap.add_argument("--tail-drain", type=float, default=None,
                    help="fraction of idle tracker threads that moves running paths to the tail kernel "
                         "(default: the library's; 0 = off)")
    ap.add_argument("--workload", choices=["cyclic7_batch", "serving", "configs"], default="cyclic7_batch",
                    help="configs: every workload of the benchmark list, one line each")
    ap.add_argument("--requests", type=int, default=2000, help="serving: number of Poisson requests")
    ap.add_argument("--slots", type=int, default=4, help="serving: batches of requests on the GPU at once")
    ap.add_argument("--no-big", action="store_true", help="serving: leave out the cyclic 9 request")
    ap.add_argument("--batch-paths", type=int, default=60_000, help="serving: most paths per batch of small requests")
    ap.add_argument("--configs", default="", help="--workload configs: which (e.g. 3,5; default 1-5; 9 = the "
                    "cyclic 9 D=2 request of the serving workload alone; 10 = double double tracking; "
                    "11 = polyhedral homotopies; 12 = double, double double and quad double tracking; "
                    "13 = the pipelined polyhedral solve against the host threads; 14 / 15 = random cyclic 11 / 12 "
                    "by the pipelined polyhedral solve)")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="default workload: requests of the served-latency measurement added to the line (0 = none)")
    ap.add_argument("--no-batching", dest="batching", action="store_false",
                    help="default workload: leave out the batching numbers (256 sparse systems)")
    ap.add_argument("--profile-case", nargs="?", const="cyclic7", default=None,
                    choices=["cyclic7", "sparse", "polyhedral"],
                    help="run a small case of a bench kernel twice (for ncu) and exit")
    args = ap.parse_args(argv)
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "configs":
        return run_configs(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
