"""Benchmark of libtsqr: R factor of a tall-and-skinny FP64 matrix on GB300.

Workload (one step = one full TSQR of the matrix: leaf folds + reduction tree + normalize):
  FP64 A of 4,194,304 x 32 (1 GiB, column-major), iid N(0,1) from seed 0, the AUTO plan
  (hybrid tree: flat folds inside each CTA, binary tree across CTAs).
Metric: GFLOP/s counted as (2 m n^2 - 2 n^3 / 3) per step; A-read GB/s reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (one unblocked Householder QR, FP64) on the host cores,
each step one factorization of the whole workload (about 0.7 s on 16 cores).  Under torchrun
every rank factorizes its own replica (the method needs no exchange between GPUs); rank 0
prints one JSON line.  Unless --no-extras, the line also carries the mixed-precision and
varlen-batched paths measured against the FP64 path ("extras").
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import signal
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

M, N = 4194304, 32
SEED = 0
FP64_FMA_PER_CLK_PER_SM = 2      # DFMA lane-ops per clock per SM of a GB300 (measured)
SMS = 152
SM_MAX_MHZ = 2070.0


def flops(m, n):
    return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0


def peaks():
    p = {"hbm_gbs": 6800.0, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        p = {"hbm_gbs": float(d.get("hbm_gbs", 6800.0)), "source": "measured",
             "sm_max_mhz": float(d.get("sm_max_mhz", SM_MAX_MHZ))}
    mhz = p.get("sm_max_mhz", SM_MAX_MHZ)
    p["fp64_tflops"] = SMS * FP64_FMA_PER_CLK_PER_SM * 2 * mhz * 1e6 / 1e12
    return p


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        exe = shutil.which("nvidia-smi")
        if exe:
            self.path = f"/tmp/tsqr_clocks_{os.getpid()}.csv"
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen([exe, f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": rows[0][1],
                "reasons": reasons, "samples": len(rows), "power_w_max": max(r[2] for r in rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group(backend, init_method="env://")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Largest x over the ranks (the job's time is its slowest replica's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(local_ms, steps, world, flops_per_step):
    """Whole-job GFLOP/s: every replica's flops over the slowest replica's time, and that time."""
    ms = max_over_ranks(local_ms, world)
    return world * flops_per_step * steps / (ms / 1e3) / 1e9, ms


def run_cpu_baseline(At_cpu, threads, R_gpu, target_s=10.0, max_reps=40):
    """The oracle on the whole workload, repeated until about target_s seconds of CPU work;
    its R is also compared with the GPU's R of the same matrix."""
    import oracle
    A = oracle.from_torch_colmajor(At_cpu)
    reps, spent = 0, 0.0
    Ro = None
    while reps < max_reps and (reps == 0 or spent < target_s):
        t0 = time.perf_counter()
        Ro = oracle.householder_r(A, nthreads=threads)
        spent += time.perf_counter() - t0
        reps += 1
    out = {"value": reps * flops(M, N) / spent / 1e9, "unit": "GFLOP/s", "cores": threads,
           "kind": "oracle", "seconds": spent, "reps": reps,
           "sample": f"the whole {M:,} x {N} FP64 workload, {reps} repetitions, one unblocked "
                     f"Householder QR each, {threads} threads"}
    kap = oracle.kappa_from_r(Ro)
    out["parity"] = {
        "rel_err_vs_oracle": oracle.rel_err(R_gpu, Ro),
        "bound_50_kappa_u": 50 * kap * 2.0 ** -53,
        "bound_c_m_kappa_u": max(50.0, 2.0 * M ** 0.5) * kap * 2.0 ** -53,
        "gram_residual": oracle.gram_residual(A, R_gpu, nthreads=threads),
        "gram_tol": 1e-13}
    return out


def run_cpu_one_thread(At_cpu, rows=1 << 20):
    """The oracle on one host thread, on the first `rows` rows of the workload (about as long as
    the all-core run on the whole matrix)."""
    import oracle
    A = oracle.from_torch_colmajor(At_cpu[:, :rows].contiguous())
    t0 = time.perf_counter()
    oracle.householder_r(A, nthreads=1)
    dt = time.perf_counter() - t0
    return {"value": flops(rows, N) / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "seconds": dt, "sample": f"the first {rows:,} rows of the {M:,} x {N} workload, one "
                                     f"unblocked Householder QR on one thread"}


def bench_reference(args, world, rank):
    if rank != 0:
        return 0
    import workloads
    threads = os.cpu_count() or 1
    rows = M
    At = workloads.gaussian(rows, N, seed=SEED)
    import oracle
    A = oracle.from_torch_colmajor(At)
    for _ in range(args.warmup):
        oracle.householder_r(A, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.householder_r(A, nthreads=threads)
    dt = (time.perf_counter() - t0) / args.steps
    v = flops(rows, N) / dt / 1e9
    line = {"metric": "TSQR GFLOP/s (2mn^2-2n^3/3), FP64", "value": v, "unit": "GFLOP/s",
            "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"FP64 {M:,} x {N} N(0,1) seed {SEED}; CPU oracle, one "
                                   f"unblocked Householder QR of the whole matrix per step",
                       "m": M, "n": N},
            "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                             "sample": f"the whole {M:,} x {N} workload per step"},
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def bench_ours(args, world, rank, local):
    import torch
    import paper_1002_4250_gb300 as T
    import workloads

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    At_cpu = workloads.gaussian(M, N, seed=SEED + rank)
    A = At_cpu.to(dev).T                                   # (m, n) column-major, lda = m
    R = T.empty_r(N, dev)
    plan = T.tsqr_resolve_plan(M, N)
    fl = flops(M, N)
    bytes_a = 8.0 * M * N

    # pipe peaks measured on this GPU by libtsqr's microbenchmarks (before the timed region)
    try:
        measured = T.measure_peaks()
    except Exception as exc:  # reported, not fatal: the derived peak stays the denominator
        measured = {"error": str(exc)}

    for _ in range(max(args.warmup, 3)):
        T.tsqr_r(A, R=R)
    torch.cuda.synchronize()

    # device-timed region: inputs resident in HBM (1 GiB > the 129 MB L2: no flush needed)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches = 0
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            T.tsqr_r(A, R=R)
            ev[i][1].record(stream)
            launches += T.tsqr_last_launch_count()
        end.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    ms_local = start.elapsed_time(end)
    per_launch = [a.elapsed_time(b) for a, b in ev]
    value, ms = job_value(ms_local, args.steps, world, fl)
    status = T.tsqr_get_device_status()
    ms_step = ms / args.steps

    # end to end through the public host-buffer call (tsqr_r_host): page-locked host A read in
    # place by the leaves, R back to page-locked host memory; every step ends with the host
    # holding R.  Its R must equal the device-timed call's bytes (same plan and kernel).
    e2e = None
    if not args.no_e2e:
        A_host = At_cpu.pin_memory()
        R_host = torch.empty((N, N), dtype=torch.float64).pin_memory().T
        e2e_steps = max(3, min(args.steps, 10))
        for _ in range(2):
            T.tsqr_r_host(A_host.T, R=R_host, sync=False)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            T.tsqr_r_host(A_host.T, R=R_host, sync=False)
            torch.cuda.synchronize()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
        e2e_status = T.tsqr_get_device_status()
        e2e = {"value": world * fl / e2e_s / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": int(A_host.numel() * 8), "d2h_bytes_per_step": int(N * N * 8),
               "ms_per_step": e2e_s * 1e3, "steps": e2e_steps,
               "device_status": int(e2e_status),
               "r_equals_device_r": bool(torch.equal(R_host, R.cpu())),
               "call": "tsqr_r_host: page-locked host A read in place by the leaves through its "
                       "device mapping, R to page-locked host memory"}

    pk = peaks()
    kern_ms = statistics.mean(per_launch)
    achieved = fl / (kern_ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": pk["fp64_tflops"], "unit": "TFLOP/s",
            "frac": achieved / pk["fp64_tflops"], "traffic": None,
            "peak_note": "FP64 DFMA pipe: 152 SMs x 2 FMA/clk x 2 flop x max SM clock (derived "
                         "from the unit count and clock); beside it the DFMA microbenchmark "
                         "measured in this run (peak_measured)",
            "peak_measured": measured.get("fp64_dfma"),
            "frac_of_measured": (achieved / measured["fp64_dfma"]) if measured.get("fp64_dfma") else None,
            "measured_peaks_tflops": measured,
            "kernel": "tsqr_f64_kernel", "kernel_ms": kern_ms,
            "a_read_gbs": bytes_a / (kern_ms / 1e3) / 1e9,
            "a_read_frac_of_hbm": bytes_a / (kern_ms / 1e3) / 1e9 / pk["hbm_gbs"],
            "hbm_peak_gbs": pk["hbm_gbs"], "hbm_peak_source": pk["source"]}
    traffic_path = os.path.join(ROOT, "profiles", "tsqr_f64_kernel_traffic.json")
    if os.path.exists(traffic_path):
        with open(traffic_path) as f:
            tr = json.load(f)
        launch = {"tile_rows": plan.tile_rows, "ctas": plan.ctas, "warps": plan.warps,
                  "arity": plan.arity}
        if tr.get("kernel_sha") == kernel_sha() and tr.get("launch") == launch:
            roof["traffic"] = tr.get("bytes_per_launch")

    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        extras = bench_extras(dev, os.cpu_count() or 1, measured)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(At_cpu, os.cpu_count() or 1, R.cpu().numpy())
        cpu["one_thread"] = run_cpu_one_thread(At_cpu)

    if rank == 0:
        line = {"metric": "TSQR GFLOP/s (2mn^2-2n^3/3), FP64", "value": value, "unit": "GFLOP/s",
                "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
                "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"FP64 {M:,} x {N} N(0,1) seed {SEED}+rank, 1 GiB per GPU",
                           "m": M, "n": N, "tree": ["auto", "binary", "flat", "hybrid"][plan.tree],
                           "tile_rows": plan.tile_rows, "ctas": plan.ctas, "warps": plan.warps,
                           "parallelism": f"replicas x{world}",
                           "l2": "input 1 GiB per GPU > 129 MB L2; no flush"},
                "a_read_gbs": world * bytes_a * args.steps / (ms / 1e3) / 1e9,
                "e2e": e2e, "gpu_launches": launches, "roofline": roof,
                "cpu_baseline": cpu, "clocks": clk.summary(), "extras": extras,
                "device_status": int(status)}
        print(json.dumps(line))
    return 0


def time_call(fn, reps, warmup=2):
    """Mean device time (ms) of fn() over reps calls, CUDA events on the current stream."""
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


def bench_extras(dev, threads, measured):
    """One entry per workload of the method's configurations, each speed with its error:
    the 10,000 x 16 binary-tree call, 4,194,304 x 32 by tree and at kappa = 1e8, the FP64 width
    sweep at 2^24 rows, the mixed-precision path per kappa (FP32 and BF16) against the FP64 path,
    the varlen batch (FP64 and mixed FP32) with graph replay, and the other entry points."""
    import torch
    out = {}
    out["c1_10000x16_binary256"] = bench_c1(dev, threads)
    out["c2_4194304x32"] = bench_c2(dev, threads)
    widths = bench_widths(dev)
    out["c3_widths_2e24"] = widths
    out["c4_mixed_2e24x64"] = bench_mixed(dev, threads, widths["64"]["ms"], measured)
    out["c5_varlen_batch"] = bench_batched(dev, threads)
    out["thin_qr"] = bench_qr(dev)
    out["lstsq"] = bench_lstsq(dev)
    out["caqr"] = bench_caqr(dev)
    torch.cuda.empty_cache()
    return out


def _errors(A, R, Ro, threads, u):
    """Forward error against the oracle's R, the Gram residual, and 50 kappa u."""
    import oracle
    kap = oracle.kappa_from_r(Ro)
    return {"rel_err_vs_oracle": oracle.rel_err(R, Ro), "bound_50_kappa_u": 50.0 * kap * u,
            "gram_residual": oracle.gram_residual(A, R, nthreads=threads), "kappa": kap}


def bench_c1(dev, threads):
    """10,000 x 16 FP64 N(0,1) seed 0, 256-row tiles, binary tree (the paper's tree): time per
    call (launch-bound at this size) and the error against the oracle."""
    import paper_1002_4250_gb300 as T
    import oracle
    import workloads
    m, n = 10000, 16
    At = workloads.gaussian(m, n, seed=0)
    A = At.to(dev).T
    R = T.empty_r(n, dev)
    plan = T.make_plan("binary", tile_rows=256)
    ms = time_call(lambda: T.tsqr_r_ex(A, plan=plan, R=R), reps=200, warmup=5)
    An = oracle.from_torch_colmajor(At)
    res = {"us_per_call": ms * 1e3, "gflops": flops(m, n) / ms / 1e6}
    res.update(_errors(An, R.cpu().numpy(), oracle.householder_r(An, nthreads=threads), threads,
                       2.0 ** -53))
    return res


def bench_c2(dev, threads):
    """4,194,304 x 32 FP64: the binary (256-row tiles), flat (one CTA) and hybrid (AUTO) trees
    on N(0,1) input, and the AUTO plan on A = G diag(sigma) V^T with kappa = 1e8, with errors."""
    import torch
    import paper_1002_4250_gb300 as T
    import oracle
    import workloads
    m, n = 4194304, 32
    fl = flops(m, n)
    res = {}
    At = workloads.gaussian(m, n, seed=0)
    A = At.to(dev).T
    R = T.empty_r(n, dev)
    An = oracle.from_torch_colmajor(At)
    Ro = oracle.householder_r(An, nthreads=threads)
    for name, plan, reps in (("binary", T.make_plan("binary", tile_rows=256), 5),
                             ("flat", T.make_plan("flat"), 1), ("hybrid_auto", None, 10)):
        ms = time_call(lambda: T.tsqr_r_ex(A, plan=plan, R=R), reps=reps, warmup=1)
        r = {"ms": ms, "gflops": fl / ms / 1e6}
        r.update(_errors(An, R.cpu().numpy(), Ro, threads, 2.0 ** -53))
        res[name] = r
    del A
    Ct = workloads.conditioned(m, n, 1e8, seed=0)
    C = Ct.to(dev).T
    ms = time_call(lambda: T.tsqr_r(C, R=R), reps=10, warmup=1)
    Cn = oracle.from_torch_colmajor(Ct)
    r = {"ms": ms, "gflops": fl / ms / 1e6}
    r.update(_errors(Cn, R.cpu().numpy(), oracle.householder_r(Cn, nthreads=threads), threads,
                     2.0 ** -53))
    res["kappa_1e8_auto"] = r
    del C
    torch.cuda.empty_cache()
    return res


def mixed_roofline_ms(m, n, elem_bytes, measured, panel=16):
    """Roofline time (ms) of the blocked mixed leaf: max(bytes(A) / HBM, trailing-update flops
    as 3xTF32 on the tcgen05 TF32 pipe + the panels' flops on the FFMA pipe), with the pipe
    peaks measured in this run and the HBM copy bandwidth measured on the pool.  The trailing
    update of a panel of `panel` columns with t columns right of it costs 4 m panel t flops
    (Z = X^T C and C -= X Y); the panels take the rest of 2mn^2 - 2n^3/3."""
    hbm = peaks()["hbm_gbs"] * 1e9
    tc = measured.get("tf32_tcgen05")
    ff = measured.get("fp32_ffma")
    if not tc or not ff:
        return None
    trailing = sum(4.0 * m * panel * max(0, n - j - panel) for j in range(0, n, panel))
    panel_fl = flops(m, n) - trailing
    t_mem = elem_bytes * m * n / hbm
    t_pipe = trailing / (tc * 1e12 / 3.0) + panel_fl / (ff * 1e12)
    return {"roofline_ms": max(t_mem, t_pipe) * 1e3, "hbm_ms": t_mem * 1e3,
            "pipes_ms": t_pipe * 1e3, "trailing_flops": trailing, "panel_flops": panel_fl,
            "peaks": "tf32_tcgen05 and fp32_ffma measured in this run (TFLOP/s); HBM: "
                     + peaks()["source"]}


def bench_mixed(dev, threads, ms64, measured):
    """The mixed-precision path at 16,777,216 x 64 on A = G diag(sigma) V^T, kappa in {1e2, 1e4,
    1e6}, FP32 and BF16 storage: time of the AUTO plan (the blocked leaf) and of the fold leaf,
    the speedup over the FP64 path at 2^24 x 64 (N(0,1), ms64), the fraction of the blocked
    leaf's roofline, and the errors against the FP64 oracle on the same recipe at 1,048,576
    rows (the oracle's time at 2^24 rows is minutes)."""
    import torch
    import paper_1002_4250_gb300 as T
    import oracle
    import workloads
    m, n = 1 << 24, 64
    me = 1 << 20
    fl = flops(m, n)
    res = {"workload": f"{m:,} x {n}, A = G diag(sigma) V^T (G drawn on the GPU); errors on the "
                       f"same recipe at {me:,} rows (G from the CPU generator, seed 0)",
           "fp64_ms_2e24x64": ms64, "error_rows": me}
    R = T.empty_r(n, dev)
    u32 = 2.0 ** -24
    for kappa in (1e2, 1e4, 1e6):
        A64 = workloads.conditioned(m, n, kappa, seed=0, device=dev, device_draw=True).T
        Ae = workloads.conditioned(me, n, kappa, seed=0)
        for name, dt in (("fp32", torch.float32), ("bf16", torch.bfloat16)):
            A = A64.T.to(dt).T
            ms = time_call(lambda: T.tsqr_r_ex(A, R=R), reps=5, warmup=1)
            used = T.last_plan()
            fold = T.make_plan(leaf="fold")
            ms_fold = time_call(lambda: T.tsqr_r_ex(A, plan=fold, R=R), reps=2, warmup=1)
            del A
            Ael = Ae.to(dt)
            An = oracle.from_torch_colmajor(Ael.to(torch.float64))
            Ro = oracle.householder_r(An, nthreads=threads)
            Rp = T.tsqr_r_ex(Ael.to(dev).T).cpu().numpy()
            Rf = T.tsqr_r_ex(Ael.to(dev).T, plan=fold).cpu().numpy()
            r = {"ms": ms, "gflops": fl / ms / 1e6, "speedup_vs_fp64": ms64 / ms,
                 "a_read_gbs": torch.tensor([], dtype=dt).element_size() * m * n / ms / 1e6,
                 "leaf": ["auto", "fold", "panels"][used.leaf], "fold_ms": ms_fold,
                 "errors": _errors(An, Rp, Ro, threads, u32),
                 "fold_errors": _errors(An, Rf, Ro, threads, u32),
                 "gram_tol": 2e-6}
            roof = mixed_roofline_ms(m, n, 4 if dt == torch.float32 else 2, measured)
            if roof is not None:
                roof["frac"] = roof["roofline_ms"] / ms
                r["roofline"] = roof
            res[f"{name}_kappa_{kappa:.0e}"] = r
        del A64
        torch.cuda.empty_cache()
    return res


def bench_caqr(dev):
    """tsqr_caqr_r (R of a general m x n matrix by TSQR panels and trailing updates) on
    262,144 x 1,024 FP64 N(0,1) with the default panel: time and GFLOP/s (2mn^2 - 2n^3/3)."""
    import torch
    import paper_1002_4250_gb300 as T
    import workloads
    m, n = 262144, 1024
    A = workloads.gaussian(m, n, seed=0, device=dev).T
    R = T.empty_r(n, dev)
    ms = time_call(lambda: T.tsqr_caqr_r(A, R=R), reps=2, warmup=1)
    del A
    torch.cuda.empty_cache()
    return {"workload": f"{m:,} x {n:,} N(0,1) seed 0, default panel", "ms": ms,
            "gflops": flops(m, n) / ms / 1e6}


def bench_lstsq(dev):
    """tsqr_lstsq on 4,194,304 x 32 FP64 with k = 1 right-hand side (the augmented
    factorization of [A | B]) and k = 32 and 100 (Q^T B through the stored reflectors), beside
    tsqr_r alone."""
    import torch
    import paper_1002_4250_gb300 as T
    import workloads
    m, n = 4194304, 32
    A = workloads.gaussian(m, n, seed=0, device=dev).T
    R = T.empty_r(n, dev)
    res = {"r_only_ms": time_call(lambda: T.tsqr_r(A, R=R), reps=5, warmup=1)}
    for k in (1, 32, 100):
        g = torch.Generator(device=dev).manual_seed(k)
        B = torch.randn(k, m, generator=g, dtype=torch.float64, device=dev).T
        X = torch.empty(k, n, dtype=torch.float64, device=dev).T
        res[f"k{k}_ms"] = time_call(lambda: T.tsqr_lstsq(A, B, X=X, R=R), reps=3, warmup=1)
        del B, X
    res["path"] = {"k1": "augmented [A | B]", "k32": "stored reflectors", "k100": "stored reflectors"}
    del A
    torch.cuda.empty_cache()
    return res


def bench_qr(dev):
    """tsqr_qr (thin Q and R, FP64) on 4,194,304 x 32 and 16,777,216 x 64: time, GFLOP/s with
    LAPACK's counts (geqrf 2mn^2 - 2n^3/3 plus orgqr 2mn^2 - 2n^3/3), the Q passes' share
    (tsqr_qr minus tsqr_r_ex with the plan tsqr_qr's factorization used), and the Q passes'
    FP64 rate on the flops the
    blocked form executes (3mn^2: mn^2 for the chunks' S factors, 2mn^2 for the leaf pass)."""
    import torch
    import paper_1002_4250_gb300 as T
    import workloads
    res = {}
    for m, n in ((4194304, 32), (1 << 24, 64)):
        A = workloads.gaussian(m, n, seed=0, device=dev).T
        Q = torch.empty(n, m, dtype=torch.float64, device=dev).T
        R = T.empty_r(n, dev)
        reps = 5 if n <= 32 else 2
        ms_qr = time_call(lambda: T.tsqr_qr(A, Q=Q, R=R), reps=reps, warmup=1)
        used = T.last_plan()  # the factorization's plan: R alone timed with the same one
        ms_r = time_call(lambda: T.tsqr_r_ex(A, R=R, plan=used), reps=reps, warmup=1)
        fl = 4.0 * m * n * n - 4.0 * n ** 3 / 3
        res[f"{m}x{n}"] = {"ms": ms_qr, "gflops_lapack_count": fl / ms_qr / 1e6,
                           "r_only_ms": ms_r, "q_passes_ms": ms_qr - ms_r,
                           "q_passes_gflops_executed": 3.0 * m * n * n / (ms_qr - ms_r) / 1e6}
        del A, Q
        torch.cuda.empty_cache()
    return res


def bench_widths(dev):
    """FP64 at 16,777,216 x n for n in {4, 8, 16, 32, 64, 128}, N(0,1), with the plan chosen by
    the autotuner (tsqr_autotune; n = 128 keeps the AUTO panels, whose tuning would take a
    minute): GFLOP/s, A-read GB/s and the fraction of the roofline time max(bytes(A) / HBM,
    flops / FP64 peak); beside it the time of the built-in AUTO plan."""
    import torch
    import paper_1002_4250_gb300 as T
    import workloads
    m = 1 << 24
    pk = peaks()
    res = {}
    for n in (4, 8, 16, 32, 64, 128):
        fl = flops(m, n)
        bytes_a = 8.0 * m * n
        t_roof = max(bytes_a / (pk["hbm_gbs"] * 1e9), fl / (pk["fp64_tflops"] * 1e12)) * 1e3
        A = workloads.gaussian(m, n, seed=0, device=dev).T
        R = T.empty_r(n, dev)
        T.tsqr_autotune_reset()
        reps = 2 if n >= 64 else 5
        ms_builtin = time_call(lambda: T.tsqr_r(A, R=R), reps=reps, warmup=1)
        builtin = T.last_plan()
        tune_s = None
        if n <= 64:
            t0 = time.perf_counter()
            T.tsqr_autotune(A, R=R)
            tune_s = time.perf_counter() - t0
        ms = time_call(lambda: T.tsqr_r(A, R=R), reps=reps, warmup=1)
        used = T.last_plan()
        T.tsqr_autotune_reset()
        del A
        torch.cuda.empty_cache()
        plan_str = lambda p: (f"{['auto', 'binary', 'flat', 'hybrid', 'panels'][p.tree]} "
                              f"tile {p.tile_rows} ctas {p.ctas} warps {p.warps} arity {p.arity}")
        res[str(n)] = {"ms": ms, "gflops": fl / ms / 1e6, "a_read_gbs": bytes_a / ms / 1e6,
                       "roofline_ms": t_roof, "frac_of_roofline": t_roof / ms,
                       "bound": "hbm" if bytes_a / (pk["hbm_gbs"] * 1e9) > fl / (pk["fp64_tflops"] * 1e12)
                       else "alu",
                       "plan": plan_str(used), "autotune_s": tune_s,
                       "builtin_ms": ms_builtin, "builtin_plan": plan_str(builtin),
                       "builtin_frac_of_roofline": t_roof / ms_builtin}
    return res


def bench_batched(dev, threads):
    """The varlen batch: 4096 problems, m log-uniform in [512, 262144], n uniform in
    {8, 16, 32, 64}, packed in one buffer, one persistent launch per call; FP64 and mixed FP32.
    Each is timed with the built-in knobs and with the knobs tsqr_autotune_batched picks; beside
    the tuned time: the replay of the call captured in a CUDA graph, and the errors of a sample
    of 24 problems (every 171st) against the oracle (the largest Gram residual and forward
    error of the sample)."""
    import numpy as np
    import torch
    import paper_1002_4250_gb300 as T
    import oracle
    import workloads
    buf, ms, ns, offs = workloads.varlen_batch(4096, 512, 262144, seed=0, device=dev)
    fl = sum(flops(m, n) for m, n in zip(ms, ns))
    roff = [0]
    for n in ns:
        roff.append(roff[-1] + n * n)
    Rp = torch.empty(roff[-1], dtype=torch.float64, device=dev)
    res = {"problems": len(ms), "elements": int(offs[-1]), "gflop_per_call": fl / 1e9}
    sample = list(range(0, 4096, 171))
    for name, dt, code, prec, u in (("fp64", torch.float64, T.F64, T.PREC_F64, 2.0 ** -53),
                                    ("mixed_fp32", torch.float32, T.F32, T.PREC_MIXED, 2.0 ** -24)):
        b = buf if dt == torch.float64 else buf.to(dt)
        ptrs = [b.data_ptr() + b.element_size() * o for o in offs[:-1]]
        # the built-in knobs, then the knobs tsqr_autotune_batched picks for this batch's
        # bucket (cached: the AUTO calls below run with them)
        T.tsqr_autotune_reset()
        call = lambda: T.tsqr_r_batched(ptrs, ms, ns, roff, Rp, dtype=code, prec=prec)
        ms_builtin = time_call(call, reps=2 if name == "fp64" else 5, warmup=1)
        builtin = T.last_batch_plan().as_tuple()
        t0 = time.perf_counter()
        tuned = T.tsqr_autotune_batched(ptrs, ms, ns, roff, Rp, dtype=code, prec=prec)
        tune_s = time.perf_counter() - t0
        ms_ = time_call(call, reps=2 if name == "fp64" else 5, warmup=1)
        used = T.last_batch_plan().as_tuple()
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            call()  # workspace and problem table in place before the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            T.tsqr_r_batched(ptrs, ms, ns, roff, Rp, dtype=code, prec=prec, stream=stream)
        ms_graph = time_call(g.replay, reps=2 if name == "fp64" else 5, warmup=1)
        torch.cuda.synchronize()
        Rh = Rp.cpu().numpy()
        gram, ferr = [], []
        for i in sample:
            m, n = ms[i], ns[i]
            Ai = b[offs[i]:offs[i + 1]].view(n, m).to(torch.float64).cpu()
            An = oracle.from_torch_colmajor(Ai)
            Ri = Rh[roff[i]:roff[i] + n * n].reshape(n, n).T
            gram.append(oracle.gram_residual(An, Ri, nthreads=threads))
            ferr.append(oracle.rel_err(Ri, oracle.householder_r(An, nthreads=threads)))
        res[name] = {"ms": ms_, "gflops": fl / ms_ / 1e6, "graph_replay_ms": ms_graph,
                     "builtin_ms": ms_builtin, "builtin_knobs": builtin,
                     "tuned_knobs": used, "autotune_s": tune_s,
                     "a_read_gbs": b.element_size() * offs[-1] / ms_ / 1e6,
                     "sample_problems": len(sample), "max_gram_residual": float(np.max(gram)),
                     "max_rel_err_vs_oracle": float(np.max(ferr)),
                     "gram_tol": 1e-13 if name == "fp64" else 2e-6}
        del b
    T.tsqr_autotune_reset()
    res["knobs_fields"] = "(warps, ctas_per_sm, leaves_per_cta, arity per width bucket, leaf)"
    res["mixed_speedup_vs_fp64"] = res["fp64"]["ms"] / res["mixed_fp32"]["ms"]
    del buf
    torch.cuda.empty_cache()
    return res


# The sources the FP64 leaf + tree kernel's code comes from: its translation unit and the
# device headers (the C-ABI header it also includes holds declarations only).
KERNEL_SOURCES = ("paper_1002_4250_gb300/csrc/tsqr_f64.cu",
                  "paper_1002_4250_gb300/csrc/tsqr_f64.cuh",
                  "paper_1002_4250_gb300/csrc/tsqr_fold.cuh",
                  "paper_1002_4250_gb300/csrc/tsqr_internal.h")


def kernel_sha():
    """First 16 hex digits of SHA-256 over the FP64 kernel's sources, in KERNEL_SOURCES order."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the mixed-precision vs FP64 comparison at 16,777,216 x 64")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end host-buffer leg (e.g. under a profiler)")
    args = ap.parse_args()
    world, rank, local = dist_init() if args.impl == "ours" else (
        int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0)
    if args.impl == "reference":
        return bench_reference(args, world, rank)
    from paper_1002_4250_gb300 import _build
    _build.build()
    rc = bench_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
