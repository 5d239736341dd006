#!/usr/bin/env python
"""Benchmark of the usFFT sampling-and-detection increment on GB300.

Workload (the 2-D configuration): P1 FE on the unit square with 63x63 interior nodes
(G = 3969), affine periodic coefficient with d = 10, search domain [-32,32]^10, s = 500,
delta = 1e-10 relative, r = 2.  One step = one pass of the hot path for the coupled
increment t (default t = 3): for each of the r~ = 2 detection iterations, FE solves at all
M lattice nodes, one length-M FFT per mesh node with the gather at k.z mod M, per-node
selection and the union.  Increments 1..t-1 run untimed beforehand.

Metric: lattice samples/s (one sample = one FE solve at a lattice node, all G nodes), for
the mixed-precision path (fp32 CG + fp64 residual refinement) and for the fp64 path, both
at the 1e-10 accuracy bar; `value` is the mixed path, `fp64` holds the fp64 path.

Timing: CUDA events on the plan's stream around each step, a 256 MB L2 flush between
steps (outside the events), barrier + synchronize around the timed region, max over
ranks.  `e2e` times the public call usfft_increment (after usfft_rewind) end to end,
host planning and host<->device copies included.  `--impl reference` times the CPU
oracle on bounded samples of the same workload.
"""
import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "usFFT lattice samples/s (FE solve+FFT) mixed vs FP64 @1e-10; p50/p99 latency"
UNIT = "lattice samples/s"
FLUSH_BYTES = 256 << 20
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# ALU peaks from unit counts and the maximum SM clock: FP32 128 FMA/clk/SM; FP64 2 DFMA/clk/SM
# (the recipe's nominal 1.25 TFLOP/s fp64 over 152 SMs at 2.07 GHz).
PEAK_FP32_TFLOPS = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
PEAK_FP64_TFLOPS = SM_COUNT * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12
FLOPS_PER_CG_ITER_PER_NODE = 21      # Jacobi-PCG: SpMV 9 + two dots 4 + three AXPY 6 + scaling 2


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of the
# kernel, with a hash of the kernel source it was taken on; a changed source makes it null.
PROFILE_TRAFFIC = {
    "mixed": {"bytes": 201629696, "files": ["k_sample2d_dst.cu", "k_pcg_common.cuh", "k_theta.cuh", "k_cvt.cuh"],
              "sha": "60f1c60f50c270ae", "profile": "profiles/pcg2d_mixed_dst_c2_t3.md"},
    "fp64_dst": {"bytes": 3496581064, "files": ["k_sample2d_dst64.cu", "k_pcg_common.cuh", "k_theta.cuh"],
                 "sha": "34d37d1241cb3db6", "profile": "profiles/pcg2d_fp64_dst_c2_t3.md"},
    "fp64": {"bytes": 178385408, "files": ["k_sample2d.cu", "k_pcg_common.cuh", "k_theta.cuh"],
             "sha": "a926921e40d8c868", "profile": "profiles/pcg2d_fp64_c2_t3.md"},
    "fft": {"bytes": 518528256, "files": ["k_fft.cu", "k_cvt.cuh"],
            "sha": "44c2d4bb1a480777", "profile": "profiles/fft_c2_t3.md"},
    "big": {"bytes": 6395321000, "files": ["k_sample2d_dst.cu", "k_pcg_common.cuh", "k_theta.cuh", "k_cvt.cuh"],
            "sha": "60f1c60f50c270ae", "profile": "profiles/pcg2d_mixed_big_mesh127_t3.md"},
}


def profiled_traffic(kind):
    import hashlib
    rec = PROFILE_TRAFFIC[kind]
    h = hashlib.sha256()
    for f in rec["files"]:
        with open(os.path.join(ROOT, "paper_2109_04131_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return rec["bytes"] if h.hexdigest()[:16] == rec["sha"] else None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        for r in self.rows:
            for name, flag in zip(self.NAMES, r[4:8]):
                if "Active" in flag and "Not" not in flag:
                    reasons.add(name)
        pw = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows),
                "power_w_max": max(pw) if pw else None}


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q / 100.0
    f, c = math.floor(k), math.ceil(k)
    return xs[f] if f == c else xs[f] + (xs[c] - xs[f]) * (k - f)


def max_over_ranks(x, world, device=None):
    """The maximum of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, tot_ms):
    """Units all ranks processed per second when every rank did units_per_rank in the slowest
    rank's time tot_ms (independent instances: weak scaling)."""
    return world * units_per_rank / (tot_ms / 1e3)


def workload_config(w, t, info=None):
    p = w.params
    cfg = {"workload": f"2-D P1 FE {w.problem.n}x{w.problem.n} interior (G={w.problem.G}), affine periodic "
                       f"coefficient, d={w.problem.d}, Gamma=[-{p.N},{p.N}]^{w.problem.d}, s={p.s}, "
                       f"delta={p.delta:g} relative, r={p.r}; coupled increment t={t}",
           "G": w.problem.G, "d": w.problem.d, "N": p.N, "s": p.s, "r": p.r, "t": t,
           "l2": "inputs larger than L2 (samples M*G*8 B) and a 256 MB L2 flush between steps",
           "parallelism": "independent instances, one per GPU"}
    if info is not None:
        cfg.update({"M": int(info["M"]), "n_candidates": int(info["n_candidates"]),
                    "samples_per_step": int(info["M"]) * (p.r if t < w.problem.d else 1)})
    return cfg


# ---------------------------------------------------------------------------------------------
# CPU oracle on bounded samples (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------------------------
def oracle_shape(w, t):
    """Oracle-only setup: increments 1..t-1, then J_t, (z, M) of increment t."""
    from oracle import lattice
    from oracle.usfft import OracleRun
    run = OracleRun(w.problem, w.params)
    for _ in range(t - 1):
        run.increment()
    run.detect_1d(t)
    J = lattice.candidate_set(run.I_prefix, np.array(run.I1d[t], dtype=np.int64), w.params.N)
    z, M = lattice.search(J, t, w.params.seed)
    return run, J, z, M


def _oracle_rows(job):
    """Worker of the oracle pool: the oracle's FE samples of some lattice nodes (unchanged oracle
    code); job None only starts the worker."""
    if job is None:
        return None
    prob, nodes, rows = job
    from oracle import fe
    from oracle.usfft import sample_rows
    return sample_rows(prob, nodes, rows, fe.make_mesh(prob.kind, prob.n))


_ORACLE_POOL = None


def oracle_pool():
    """Processes for the oracle's independent FE solves, one per host core (spawn: the parent holds
    a CUDA context), BLAS single-threaded in each; started and warmed before any timing.  None if
    the workers cannot start (the solves then run in this process)."""
    global _ORACLE_POOL
    if _ORACLE_POOL is None:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            pool = ProcessPoolExecutor(max_workers=os.cpu_count() or 1, mp_context=mp.get_context("spawn"))
            list(pool.map(_oracle_rows, [None] * (os.cpu_count() or 1), timeout=300))   # workers up
            _ORACLE_POOL = pool
        except Exception:                              # a broken pool raises instead of hanging
            _ORACLE_POOL = False
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    return _ORACLE_POOL or None


def oracle_sample_time(w, t, J, z, M, rows):
    """Seconds for the oracle's sampler (the rows' FE solves shared out over one process per host
    core) and its DFT (numpy, BLAS threads on all cores) on `rows` lattice nodes of iteration 1;
    and the processes the solves used."""
    from oracle import dft, lattice, rng
    from oracle.usfft import NodeSet
    d = w.problem.d
    tails = {j - 1: rng.uniform(w.params.seed, rng.PHASE_TAIL, t, 1, j) for j in range(t + 1, d + 1)}
    nodes = NodeSet(d, list(range(t)), z, M, tails)
    m = lattice.lattice_indices(J, z, M)
    global _ORACLE_POOL
    pool = oracle_pool()
    U = None
    if pool:
        procs = os.cpu_count() or 1
        parts = [c for c in np.array_split(np.asarray(rows), procs) if len(c)]
        try:
            list(pool.map(_oracle_rows, [(w.problem, nodes, c[:1]) for c in parts], timeout=600))   # warm
            t0 = time.perf_counter()
            U = np.concatenate(list(pool.map(_oracle_rows, [(w.problem, nodes, c) for c in parts], timeout=600)))
            t1 = time.perf_counter()
        except Exception:                              # a worker died: the solves run in this process
            _ORACLE_POOL = False
            U = None
    if U is None:
        procs = 1
        t0 = time.perf_counter()
        U = _oracle_rows((w.problem, nodes, np.asarray(rows)))
        t1 = time.perf_counter()
    dft.partial_coefficients(U, np.asarray(rows), m, M)
    t2 = time.perf_counter()
    return t2 - t0, t1 - t0, t2 - t1, procs


def cpu_baseline(w, t, rows_n=None):
    t0 = time.perf_counter()
    run, J, z, M = oracle_shape(w, t)
    setup = time.perf_counter() - t0
    if rows_n is None:
        rows_n = 24 * (os.cpu_count() or 1)
    rows = np.linspace(0, M - 1, rows_n).astype(np.int64)
    tot, ts, td, procs = oracle_sample_time(w, t, J, z, M, rows)
    return {"value": rows_n / tot, "unit": UNIT, "cores": os.cpu_count() if procs > 1 else 1, "kind": "oracle",
            "sample": f"{rows_n} of the M={M} lattice nodes of increment t={t}, iteration 1 (|J|={len(J)}): "
                      f"banded-Cholesky FE solves ({ts:.2f} s, {procs} processes) + naive DFT of those rows "
                      f"at all |J| indices ({td:.2f} s, numpy BLAS on all cores); oracle setup (increments "
                      f"1..{t - 1}) and process start untimed ({setup:.1f} s)",
            "seconds": tot}


def run_reference(args, rank, world):
    import torch.distributed as dist  # noqa: F401
    if rank != 0:
        return
    w = W.c2(1)
    t = args.t
    _, J, z, M = oracle_shape(w, t)
    rows_n = args.ref_rows or 24 * (os.cpu_count() or 1)
    rng_ = np.random.default_rng(0)
    times = []
    for k in range(args.warmup + args.steps):
        rows = np.sort(rng_.choice(M, size=rows_n, replace=False))
        tot, _, _, procs = oracle_sample_time(w, t, J, z, M, rows)
        if k >= args.warmup:
            times.append(tot)
    per = [rows_n / x for x in times]
    value = rows_n * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, t, {"M": M, "n_candidates": len(J)}),
            "latency_ms": {"p50": 1e3 * percentile(times, 50), "p99": 1e3 * percentile(times, 99)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count() if procs > 1 else 1,
                             "kind": "oracle",
                             "sample": f"each step: {rows_n} random lattice nodes of increment t={t} "
                                       f"(M={M}, |J|={len(J)}): FE solves ({procs} processes) + naive DFT rows"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist
    from paper_2109_04131_gb300 import binding

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream(dev)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None

    def barrier():
        if world > 1:
            dist.barrier()

    w = W.c2(1 + rank)
    t = args.t
    # setup: increments 1..t-1 in fp64; every precision then runs increment t from that state
    p64 = binding.Plan(w.problem, W.with_precision(w, W.PRECISION_FP64).params)
    for _ in range(t - 1):
        p64.increment()
    I_prev = p64.get_set()
    info64 = p64.increment()
    plans = {"fp64_jacobi": p64}
    infos = {"fp64_jacobi": info64}
    for name, prec in (("mixed", W.PRECISION_MIXED), ("fp64", W.PRECISION_FP64_DST)):
        pl = binding.Plan(w.problem, W.with_precision(w, prec).params)
        pl.resume(t - 1, I_prev, info64["theta"])
        infos[name] = pl.increment()
        plans[name] = pl

    # accuracy of every precision against the oracle on sampled lattice nodes
    accuracy = sampled_accuracy(w, t, plans, rows=4) if rank == 0 and not args.skip_accuracy else None

    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    results = {}
    for name in (("mixed",) if args.skip_fp64 else ("mixed", "fp64", "fp64_jacobi")):
        results[name] = time_replays(plans[name], infos[name], w, t, args.steps, args.warmup, flush, stream, barrier,
                                     world, dev, uuid if rank == 0 else None)

    # end to end through the public call (rewind + usfft_increment), mixed precision
    e2e = e2e_measure(plans["mixed"], t, args.e2e_steps, barrier, world, dev)
    # the rows past the increment (reconstruction, evaluation, statistics, random lattices)
    next_rows = None
    if rank == 0 and not args.skip_next_rows:
        pk, pkind = measured_peaks()
        next_rows = next_rows_measure(w, plans["mixed"], t, args.n_test, pk, pkind, steps=args.steps)

    if rank != 0:
        for p in plans.values():
            p.close()
        return
    peaks, peak_kind = measured_peaks()
    G = w.problem.G
    if args.skip_fp64:                       # profiling runs: the mixed leg stands in for the others
        results["fp64"] = results["fp64_jacobi"] = results["mixed"]
    mx, f64, fjac = results["mixed"], results["fp64"], results["fp64_jacobi"]
    value = whole_job_rate(world, mx["samples_per_step"] * args.steps, mx["tot_ms"])
    value64 = whole_job_rate(world, f64["samples_per_step"] * args.steps, f64["tot_ms"])
    value_jac = whole_job_rate(world, fjac["samples_per_step"] * args.steps, fjac["tot_ms"])

    d_, E_ = w.problem.d, 2 * (w.problem.n + 1) ** 2
    P_ = (w.problem.n + 15) // 16 * 16
    peak_bf16 = peaks.get("bf16_tflops", 1921.8)

    def dst64_roofline(res, n_mesh, label):
        # fp64 sampler with the sine-transform preconditioner: the transforms' fused multiply-adds
        # dominate (dst64_flops_per_solve); FP64-pipe bound
        st = res["stages"]
        n = max(1, st["launches"]["sample"])
        solves = res["samples_per_step"] * args.steps
        iters = st["cg_iters_total"] / max(1, solves)
        flops = dst64_flops_per_solve(n_mesh, iters) * solves / n
        dur = st["ms"]["sample"] / n / 1e3
        ach = flops / dur / 1e12
        return {"bound": "alu", "achieved": ach, "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / PEAK_FP64_TFLOPS, "traffic": profiled_traffic("fp64_dst") if n_mesh == 63 else None,
                "kernel": f"pcg2d_fp64_dst_kernel ({label}, {n} launches timed)",
                "flops_per_launch": flops, "ms_per_launch": dur * 1e3, "cg_iters_per_solve": iters,
                "peak_note": f"fp64 peak from unit counts at {SM_MAX_MHZ:.0f} MHz (2 DFMA/clk/SM)"}

    def fp64_roofline(res):
        # FP64 Jacobi path: 21 G flops per Jacobi-PCG iteration + 2 d E flops of coefficient assembly per solve
        st = res["stages"]
        n = max(1, st["launches"]["sample"])
        solves = res["samples_per_step"] * args.steps
        flops = (FLOPS_PER_CG_ITER_PER_NODE * G * st["cg_iters_total"] + 2.0 * d_ * E_ * solves) / n
        dur = st["ms"]["sample"] / n / 1e3
        ach = flops / dur / 1e12
        return {"bound": "alu", "achieved": ach, "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / PEAK_FP64_TFLOPS, "traffic": profiled_traffic("fp64"),
                "kernel": f"pcg2d_fp64_kernel (assembly + Jacobi-PCG, {n} launches timed)",
                "flops_per_launch": flops, "ms_per_launch": dur * 1e3,
                "cg_iters_per_solve": st["cg_iters_total"] / max(1, solves),
                "peak_note": f"fp64 peak from unit counts at {SM_MAX_MHZ:.0f} MHz (2 DFMA/clk/SM)"}

    def mixed_roofline(res):
        # MIXED sampler.  Work it issues per solve (counted from the kernel's code):
        #   FP64 pipe: first refinement step x += ||r|| d (1 DFMA), r = b - K x with the fp64
        #     weights (1 DMUL, 3 DFMA, 1 DFMA, 1 DADD) and its double-float split (1 DADD): 13 flops
        #     per node; every later step only the x update (2 flops; r is updated in double-float);
        #     once per solve the fp64 edge weights (2 DADD from the double-float pairs) and
        #     diagonal (3 DADD): 5 flops per node.  The coefficient assembly runs in double-float on
        #     the FP32 pipe, not here.
        #   FP32 pipe: per inner iteration the preconditioner scaling (2), the SpMV in difference
        #     form (4 sub + 1 mul + 3 fma = 11), eight inner products (16), four updates (8): 37
        #     flops per node; per refinement step after the first the double-float update
        #     r -= ||r|| K d (K d 57, the product 7, the renormalised sum 11, the norm term 3): 78;
        #     once per solve the double-float diagonal (3 sums): 33.
        #   Tensor pipe (BF16): per inner iteration four P x P x P products, 4 * 2 P^3 flops.
        # The roof reported is the FP64 pipe's (the busiest pipe in the ncu capture); the others and
        # the HBM view (the samples written) are listed beside it.
        st = res["stages"]
        n = max(1, st["launches"]["sample"])
        solves = res["samples_per_step"] * args.steps
        inner, outer = st["cg_iters_total"], st["refine_steps_total"]
        f64 = (18.0 * G * solves + 2.0 * G * (outer - solves)) / n
        f32 = (37.0 * G * inner + 78.0 * G * (outer - solves) + 33.0 * G * solves) / n
        ftc = 4 * 2.0 * P_ ** 3 * inner / n
        dur = st["ms"]["sample"] / n / 1e3
        ach = f64 / dur / 1e12
        out_bytes = 8.0 * G * solves / n
        return {"bound": "alu", "achieved": ach, "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / PEAK_FP64_TFLOPS, "traffic": profiled_traffic("mixed"),
                "kernel": f"pcg2d_mixed_dst_kernel (fp64 and double-float refinement + fp32 flexible PCG + BF16 DST, {n} launches timed)",
                "flops_per_launch": f64, "ms_per_launch": dur * 1e3,
                "work_per_solve": {"fp64_flops": "18 G + 2 G per refinement step after the first",
                                   "fp32_flops": "37 G per inner iteration + 78 G per refinement step after the first + 33 G",
                                   "bf16_tensor_flops": f"4 * 2 * {P_}^3 per inner iteration"},
                "units": {"fp64": {"tflops": ach, "frac": ach / PEAK_FP64_TFLOPS},
                          "fp32": {"tflops": f32 / dur / 1e12, "frac": f32 / dur / 1e12 / PEAK_FP32_TFLOPS},
                          "tensor_bf16": {"tflops": ftc / dur / 1e12, "frac": ftc / dur / 1e12 / peak_bf16},
                          "hbm": {"gbs": out_bytes / dur / 1e9, "frac": out_bytes / dur / 1e9 / peaks["hbm_gbs"],
                                  "bytes_per_launch": out_bytes}},
                "inner_iters_per_solve": inner / max(1, solves), "refine_steps_per_solve": outer / max(1, solves),
                "peak_note": f"fp64 and fp32 peaks from unit counts at {SM_MAX_MHZ:.0f} MHz; bf16 and hbm {peak_kind} "
                             f"(MEASURED_PEAKS.json burst figures)"}

    def fft_roofline(res):
        st = res["stages"]
        n = max(1, st["launches"]["fft"])
        M = int(res["info"]["M"])
        nJ = int(res["info"]["n_candidates"])
        algo = 8.0 * M * G + 16.0 * nJ * G          # read the samples once, write the gathered coefficients
        dur = st["ms"]["fft"] / n / 1e3
        ach = algo / dur / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": profiled_traffic("fft"),
                "kernel": "fft_inplace_kernel<DF> (+ fft_final_kernel<DF> where the lattice does not fit on chip; double-float arithmetic, one iteration)",
                "bytes_per_launch": algo, "ms_per_launch": dur * 1e3,
                "peak_note": f"{peak_kind} hbm_gbs (burst)"}

    roof = mixed_roofline(mx)
    clocks = mx["clocks"] or {}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mx["tot_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": workload_config(w, t, mx["info"]),
        "fe_node_samples_per_s": value * G,
        "latency_ms": {"p50": percentile(mx["step_ms"], 50), "p99": percentile(mx["step_ms"], 99)},
        "fp64": {"value": value64, "unit": UNIT, "dtype": "f64", "ms_per_step": f64["tot_ms"] / args.steps,
                 "solver": "fp64 CG with the same sine-transform preconditioner as the mixed mode, applied in fp64 "
                           "(USFFT_FP64_DST): the two differ in arithmetic precision only",
                 "latency_ms": {"p50": percentile(f64["step_ms"], 50), "p99": percentile(f64["step_ms"], 99)},
                 "roofline": dst64_roofline(f64, w.problem.n, "63x63"), "clocks": f64["clocks"],
                 "stage_ms_per_step": {k: v / args.steps for k, v in f64["stages"]["ms"].items()}},
        "fp64_jacobi": {"value": value_jac, "unit": UNIT, "dtype": "f64", "ms_per_step": fjac["tot_ms"] / args.steps,
                        "solver": "fp64 Jacobi-preconditioned CG (USFFT_FP64)",
                        "latency_ms": {"p50": percentile(fjac["step_ms"], 50), "p99": percentile(fjac["step_ms"], 99)},
                        "roofline": fp64_roofline(fjac), "clocks": fjac["clocks"]},
        "speedup_mixed_vs_fp64": value / value64,
        "speedup_mixed_vs_fp64_jacobi": value / value_jac,
        "accuracy": accuracy,
        "roofline": roof,
        "roofline_fft": fft_roofline(mx),
        "stage_ms_per_step": {k: v / args.steps for k, v in mx["stages"]["ms"].items()},
        "gpu_launches": mx["launches"],
        "clocks": {"sm_mhz": clocks.get("sm_mhz"), "sm_max_mhz": clocks.get("sm_max_mhz"),
                   "reasons": clocks.get("reasons"), "samples": clocks.get("samples"),
                   "power_w_max": clocks.get("power_w_max")},
        "e2e": e2e,
        "next_rows": next_rows,
    }
    if args.skip_fp64:
        for k in ("fp64", "fp64_jacobi", "speedup_mixed_vs_fp64", "speedup_mixed_vs_fp64_jacobi"):
            line[k] = None
    if not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline(w, t)
    print(json.dumps(line), flush=True)
    for p in plans.values():
        p.close()


def time_replays(plan, info, w, t, steps, warmup, flush, stream, barrier, world, dev, clock_uuid):
    """CUDA-event time of `steps` replays of the plan's last increment (all its detection
    iterations), an L2 flush between steps, clocks sampled during the timed region."""
    import torch
    samples_per_step = int(info["M"]) * (w.params.r if t < w.problem.d else 1)
    for _ in range(warmup):
        plan.replay(sync=True)
    plan.set_timing(True)
    launches = 0
    evs = []
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(clock_uuid) if clock_uuid is not None else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    t_wall0 = time.perf_counter()
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        launches += plan.replay(sync=False)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    barrier()
    if clocks:
        clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    stages = plan.stage_times()
    plan.set_timing(False)
    tot_ms = max_over_ranks(sum(step_ms), world, dev)
    return {"samples_per_step": samples_per_step, "step_ms": step_ms, "tot_ms": tot_ms, "wall_s": wall,
            "launches": launches, "stages": stages, "clocks": clocks.summary() if clocks else None, "info": info}


def dst64_flops_per_solve(n, iters):
    """fp64 flops of one solve of the fp64 sampler with the sine-transform preconditioner: per
    preconditioner application (iters + 1 of them) four 1-D transforms of n^2 ceil(n/2) fused
    multiply-adds; per CG iteration the SpMV (9 G), two inner products and the residual norm (6 G),
    three updates (6 G) and the scalings (3 G)."""
    G = n * n
    return (iters + 1) * 4 * 2.0 * G * ((n + 1) // 2) + iters * 24.0 * G


def e2e_measure(plan, t, steps, barrier, world, dev):
    times, samples, h2d, d2h, dev_ms, host_ms = [], [], [], [], [], []
    plan.rewind(t - 1)
    plan.increment()                              # warm
    barrier()
    for _ in range(steps):
        plan.rewind(t - 1)
        t0 = time.perf_counter()
        info = plan.increment()
        times.append(time.perf_counter() - t0)
        samples.append(info["samples"])
        h2d.append(info["h2d_bytes"])
        d2h.append(info["d2h_bytes"])
        dev_ms.append(info["ms_device"])
        host_ms.append(info["ms_host_plan"])
    tot = max_over_ranks(sum(times), world, dev)
    return {"value": whole_job_rate(world, sum(samples), 1e3 * tot), "unit": UNIT, "h2d_bytes_per_step": int(np.mean(h2d)),
            "d2h_bytes_per_step": int(np.mean(d2h)), "steps": steps,
            "ms_per_step": 1e3 * tot / steps,
            "latency_ms": {"p50": 1e3 * percentile(times, 50), "p99": 1e3 * percentile(times, 99)},
            "ms_device_per_step": float(np.mean(dev_ms)), "ms_host_plan_per_step": float(np.mean(host_ms)),
            "call": "usfft_rewind(t-1) + usfft_increment (1-D detections of dimension t, J_t, lattice "
                    "search, both detection iterations, host copies)"}


def autotune_shapes(reqs, precisions):
    """usfft_autotune on the first request of every (precision, mesh-size bucket) shape, after its
    increments (untimed); the process-wide table then serves every later plan of that shape.  Returns
    the table, the reports and the seconds spent."""
    from paper_2109_04131_gb300 import binding
    t0 = time.perf_counter()
    seen, reports = set(), []
    for r in reqs:
        if r.workload.problem.kind != W.PDE_2D:
            continue
        for prec in precisions:
            key = (prec, (r.workload.problem.n + 15) // 16)
            if key in seen:
                continue
            seen.add(key)
            wl = W.with_precision(r.workload, prec)
            plan = binding.Plan(wl.problem, wl.params)
            for _ in range(r.increments):
                plan.increment()
            rep = plan.autotune(reps=2 if prec == W.PRECISION_MIXED else 1)
            reports.append({"precision": prec, "n": wl.problem.n, **rep})
            plan.close()
    return {"table": binding.usfft_tune_export(), "shapes": reports, "seconds": time.perf_counter() - t0}


def serving_measure(kind, count):
    """Batched ("batch": `count` independent instances shaped like the batching configuration, all
    present at the start, three increments each) or served ("serve": a seeded Poisson stream of
    `count` requests at 200/s, half 128x128-mesh lognormal instances, half 1-D 255-node
    instances, admitted within a 150 GB budget) against the same requests run one at a time."""
    import torch
    from paper_2109_04131_gb300 import binding, serving
    if kind == "batch":
        reqs = [serving.Request(k, 0.0, w, inc, 1 << 30) for k, (w, inc) in enumerate(W.batch_instances(count))]
    else:
        reqs = [serving.Request(k, t, w, inc, res) for k, (t, w, inc, res) in enumerate(W.serving_requests(count))]

    def make_plan(r):
        return binding.Plan(r.workload.problem, r.workload.params, stream=torch.cuda.Stream().cuda_stream)

    # launch parameters tuned per shape for both modes compared below (bit-identical results)
    tuned = autotune_shapes(reqs, (W.PRECISION_MIXED, W.PRECISION_FP64_DST))

    # continuous batching without a round barrier (one worker thread per admitted instance)
    rep = serving.AsyncServer(budget_bytes=150 << 30, make_plan=make_plan, max_active=64).run(reqs)
    torch.cuda.synchronize()
    # the same with increment rounds (usfft_increment_many over the admitted instances)
    rounds = serving.Server(budget_bytes=150 << 30, make_plan=make_plan,
                            increment_many=binding.usfft_increment_many).run(reqs)
    torch.cuda.synchronize()
    alone = serving.run_one_at_a_time(reqs, lambda r: binding.Plan(r.workload.problem, r.workload.params))
    torch.cuda.synchronize()
    alone64 = serving.run_one_at_a_time(
        reqs, lambda r: binding.Plan(r.workload.problem, W.with_precision(r.workload, W.PRECISION_FP64_DST).params))
    rep.pop("instances")
    rounds.pop("instances")
    alone.pop("results")
    alone64.pop("results")
    return {"requests": count, "autotune": tuned, "served": rep, "served_in_rounds": rounds, "one_at_a_time": alone,
            "one_at_a_time_fp64": alone64,
            "speedup_samples_per_s": rep["samples_per_s"] / alone["samples_per_s"] if alone["samples_per_s"] else None,
            "speedup_vs_fp64_one_at_a_time": rep["samples_per_s"] / alone64["samples_per_s"]
            if alone64["samples_per_s"] else None,
            "precision": "mixed",
            "note": "one-at-a-time runs the same requests in arrival order without overlap, in the mixed mode "
                    "and in fp64 with the same preconditioner (USFFT_FP64_DST; plain fp64 for the 1-D requests); "
                    "every mode meets the 1e-10 bar"}


def config_1d(seeds=10):
    """The 1-D configuration (31 interior nodes, d = 4, N = 16, s = 50, delta = 1e-12 relative, r = 1):
    every increment of full runs (seeds 1..seeds) through usfft_increment, per-increment device time and
    wall latency, fp64 (the 1-D solves are fp64 cyclic reduction in every mode; the modes differ in the
    lattice FFT) and mixed."""
    import torch
    from paper_2109_04131_gb300 import binding
    out = {"workload": "1-D P1 FE on (0,1), 31 interior nodes, affine periodic coefficient, d=4, Gamma=[-16,16]^4, "
                       "s=50, delta=1e-12 relative, r=1; full runs t=1..4"}
    for name, prec in (("fp64", W.PRECISION_FP64), ("mixed", W.PRECISION_MIXED)):
        lat, dev_ms, samples, where = [], [], 0, []
        for sd in range(1, seeds + 1):
            w = W.with_precision(W.c1(sd), prec)
            plan = binding.Plan(w.problem, w.params)
            # warm every seed's kernels, lattice sizes and buffers once (an untimed full run)
            for _ in range(w.problem.d):
                plan.increment()
            plan.close()
            plan = binding.Plan(w.problem, w.params)
            torch.cuda.synchronize()
            gc.disable()                             # no collector pause inside a timed increment
            for _ in range(w.problem.d):
                t0 = time.perf_counter()
                info = plan.increment()
                lat.append(1e3 * (time.perf_counter() - t0))
                dev_ms.append(info["ms_device"])
                where.append((sd, int(info["t"]), int(info["M"])))
                samples += info["samples"]
            gc.enable()
            plan.close()
        out[name] = {"lattice_samples": samples, "value": samples / (sum(lat) / 1e3), "unit": UNIT,
                     "device_samples_per_s": samples / (sum(dev_ms) / 1e3),
                     "increment_latency_ms": {"p50": percentile(lat, 50), "p99": percentile(lat, 99)},
                     "increment_device_ms": {"p50": percentile(dev_ms, 50), "p99": percentile(dev_ms, 99)},
                     "slowest_increment": {"seed_t_M": where[int(np.argmax(dev_ms))], "ms_device": float(np.max(dev_ms)),
                                           "ms_wall": float(lat[int(np.argmax(dev_ms))])}}
    return out


def precision_mesh127(steps, warmup, t=3):
    """Mixed vs fp64 (same preconditioner) on the 128x128-mesh lognormal workload at step t."""
    import torch
    from paper_2109_04131_gb300 import binding
    w3 = W.c3(1)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream(dev)
    base = binding.Plan(w3.problem, W.with_precision(w3, W.PRECISION_MIXED).params)
    for _ in range(t - 1):
        info = base.increment()
    I_prev, theta = base.get_set(), info["theta"]
    base.close()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    plans, res = {}, {}
    for name, prec in (("mixed", W.PRECISION_MIXED), ("fp64", W.PRECISION_FP64_DST)):
        pl = binding.Plan(w3.problem, W.with_precision(w3, prec).params)
        pl.resume(t - 1, I_prev, theta)
        inf = pl.increment()
        plans[name] = pl
        res[name] = time_replays(pl, inf, w3, t, steps, warmup, flush, stream, lambda: None, 1, dev, None)
    acc = sampled_accuracy(w3, t, plans, rows=2)
    out = {"workload": "2-D P1 FE 127x127 interior (G=16129), lognormal-type coefficient, d=20, Gamma=[-32,32]^20, "
                       f"s=1000, delta=1e-10 relative, r=2; coupled increment t={t}",
           "M": int(res["mixed"]["info"]["M"]), "n_candidates": int(res["mixed"]["info"]["n_candidates"]),
           "accuracy": acc}
    for name, r in res.items():
        st = r["stages"]
        solves = r["samples_per_step"] * steps
        leg = {"value": r["samples_per_step"] * steps / (r["tot_ms"] / 1e3), "unit": UNIT,
               "ms_per_step": r["tot_ms"] / steps,
               "stage_ms_per_step": {k: v / steps for k, v in st["ms"].items()},
               "cg_iters_per_solve": st["cg_iters_total"] / max(1, solves)}
        if name == "fp64":
            flops = dst64_flops_per_solve(w3.problem.n, leg["cg_iters_per_solve"]) * solves
            ach = flops / (st["ms"]["sample"] / 1e3) / 1e12
            leg["sampler_fp64"] = {"achieved_tflops": ach, "frac_of_fp64_peak": ach / PEAK_FP64_TFLOPS}
        out[name] = leg
        plans[name].close()
    out["speedup_mixed_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def next_rows_measure(w, pmx, t0, n_test, peaks, peak_kind, n_batch=32, n_serve=200, steps=10):
    """The rows past the detection increment, on the same workload: the remaining increments
    t0+1..d of the mixed plan (single reconstructing lattice per step), step 3 (usfft_reconstruct),
    the quantities of interest (usfft_statistics), FE solves at n_test random parameters and the
    evaluation of u^usFFT there with the errors (usfft_errors), and the same run with random
    rank-1 lattices (5 lattices, size factor 2) for the sample counts."""
    import dataclasses
    import torch
    from paper_2109_04131_gb300 import binding
    d, G = w.problem.d, w.problem.G
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_0 = time.perf_counter()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t_0)

    single = []
    for _ in range(t0 + 1, d + 1):
        info = pmx.increment()
        single.append({"t": info["t"], "M": info["M"], "samples": info["samples"], "n_detected": info["n_detected"],
                       "ms_device": info["ms_device"]})
    (I, C), ms_rec, wall_rec = timed(pmx.reconstruct)
    z_rec, M_rec = pmx.get_lattice()
    (mean, var, gsi), ms_stat, _ = timed(pmx.statistics)
    nI = len(I)
    Y = torch.from_numpy(W.parameter_points(w.problem, n_test, seed=5)).to("cuda")
    V = torch.empty((n_test, G, 2), dtype=torch.float64, device="cuda")
    Ud = torch.empty((n_test, G), dtype=torch.float64, device="cuda")
    lib, h = pmx._lib, pmx.handle
    _, ms_pts, _ = timed(lambda: lib.usfft_sample_points(h, Y.data_ptr(), n_test, Ud.data_ptr(), 1))
    timed(lambda: lib.usfft_evaluate(h, Y.data_ptr(), n_test, V.data_ptr(), 1))                # warm
    st, ms_eval, _ = timed(lambda: lib.usfft_evaluate(h, Y.data_ptr(), n_test, V.data_ptr(), 1))
    assert st == 0
    e2 = np.zeros(G)
    ei = np.zeros(G)
    st, ms_err, _ = timed(lambda: lib.usfft_errors(h, Y.data_ptr(), n_test, 1, e2.ctypes.data, ei.ctypes.data))
    assert st == 0
    # step 3 on multiple rank-1 lattices (usfft_reconstruct_multiple), then the errors with it
    (Im, Cm), ms_mrec, wall_mrec = timed(pmx.reconstruct_multiple)
    _, M_mult = pmx.get_random_lattices()
    e2m = np.zeros(G)
    eim = np.zeros(G)
    st, _, _ = timed(lambda: lib.usfft_errors(h, Y.data_ptr(), n_test, 1, e2m.ctypes.data, eim.ctypes.data))
    assert st == 0 and np.array_equal(Im, I)
    n_mult = int(np.sum(M_mult))
    mult = {"n_I": len(Im), "lattices": int(len(M_mult)), "M": [int(v) for v in M_mult], "samples": n_mult,
            "samples_bound": int(math.ceil(2 * math.log(2 * max(len(Im), 1))) * 4 * max(len(Im) - 1, 0)),
            "ms": ms_mrec, "wall_ms": wall_mrec, "lattice_samples_per_s": n_mult / (ms_mrec / 1e3),
            "err2_max": float(np.max(e2m)), "errinf_max": float(np.max(eim)), "err2_median": float(np.median(e2m)),
            "max_rel_diff_vs_single_lattice": float(np.max(np.abs(Cm - C)) / max(float(np.max(np.abs(C))), 1e-300))}
    flops_eval = 8.0 * n_test * nI * G                  # complex multiply-add per (point, frequency, node)
    ach = flops_eval / (ms_eval / 1e3) / 1e12
    stat_bytes = 16.0 * G * nI
    stat_gbs = stat_bytes / (ms_stat / 1e3) / 1e9

    # the precision configuration: 128 x 128 mesh (16129 nodes, lognormal-type coefficient, d = 20),
    # coupled step t = 3 in the mixed mode and in fp64 with the same preconditioner, both from the
    # state after increments 1-2, timed like the headline and checked against the oracle
    c3 = precision_mesh127(steps=min(steps, 10), warmup=3)
    c1 = config_1d()

    # batched and served forms (continuous batching through usfft_increment_many)
    batching = serving_measure("batch", n_batch)
    served = serving_measure("serve", n_serve)

    # random rank-1 lattices on the same workload (increments 1..d)
    prr = binding.Plan(w.problem, dataclasses.replace(W.with_precision(w, W.PRECISION_MIXED).params, rr_lattices=5,
                                                      rr_size_factor=2.0))
    rr = []
    for _ in range(d):
        info = prr.increment()
        rr.append({"t": info["t"], "samples": info["samples"], "n_detected": info["n_detected"],
                   "ms_device": info["ms_device"]})
    prr.close()
    return {
        "workload": "the 2-D workload above, increments t0+1..d after the timed increment, mixed precision",
        "increments_single_lattice": single,
        "samples_single_lattice_t0_plus_1_to_d": int(sum(r["samples"] for r in single)),
        "reconstruct": {"n_I": nI, "M": int(M_rec), "ms": ms_rec, "wall_ms": wall_rec,
                        "lattice_samples_per_s": M_rec / (ms_rec / 1e3)},
        "reconstruct_multiple": mult,
        "statistics": {"ms": ms_stat, "bytes": stat_bytes, "achieved_gbs": stat_gbs,
                       "frac_of_hbm": stat_gbs / peaks["hbm_gbs"], "peak_note": f"{peak_kind} hbm_gbs",
                       "gsi_l1_min": float(np.min(gsi[:, 0])), "variance_max": float(np.max(var))},
        "sample_points": {"n": n_test, "ms": ms_pts, "samples_per_s": n_test / (ms_pts / 1e3)},
        "evaluate": {"n": n_test, "n_I": nI, "ms": ms_eval, "flops": flops_eval, "achieved_tflops": ach,
                     "frac_of_fp64_peak": ach / PEAK_FP64_TFLOPS, "bound": "alu",
                     "kernel": "evaluate_kernel (fp64 complex contraction, E formed on chip)"},
        "errors": {"n": n_test, "ms": ms_err, "err2_max": float(np.max(e2)), "errinf_max": float(np.max(ei)),
                   "err2_median": float(np.median(e2))},
        "precision_mesh127": c3,
        "config_1d": c1,
        "batching": batching,
        "serving": served,
        "random_r1l": {"lattices": 5, "size_factor": 2.0, "precision": "mixed", "increments": rr,
                       "samples_total": int(sum(r["samples"] for r in rr)),
                       "ms_device_total": float(sum(r["ms_device"] for r in rr))},
    }


def sampled_accuracy(w, t, plans, rows=4):
    """Max relative error of the last iteration's samples on `rows` lattice nodes, against
    the oracle's banded-Cholesky solves at the same nodes (fp64 and mixed)."""
    from oracle import fe, rng
    from oracle.usfft import NodeSet, sample_rows
    out = {}
    mesh = fe.make_mesh(w.problem.kind, w.problem.n)
    d = w.problem.d
    for name, plan in plans.items():
        z, M = plan.get_lattice()
        it = w.params.r if t < d else 1
        tails = {j - 1: rng.uniform(w.params.seed, rng.PHASE_TAIL, t, it, j) for j in range(t + 1, d + 1)}
        nodes = NodeSet(d, list(range(t)), np.asarray(z), M, tails)
        idx = np.linspace(0, M - 1, rows).astype(np.int64)
        U = plan.get_samples()
        Uo = sample_rows(w.problem, nodes, idx, mesh)
        out[name + "_samples_rel_err"] = float(np.max(np.abs(U[idx] - Uo)) / np.max(np.abs(Uo)))
    out["rows"] = rows
    out["bar"] = 1e-10
    return out


def profile_case(args):
    """A short, fixed run for ncu: increments 1..K of the 2-D workload (63x63 mesh, either precision)
    or of the 127x127 lognormal-type workload (mixed precision, large-mesh sampler)."""
    import torch
    from paper_2109_04131_gb300 import binding
    prec = {"mixed": W.PRECISION_MIXED, "fp64": W.PRECISION_FP64, "fp64_dst": W.PRECISION_FP64_DST}[args.precision]
    w = W.with_precision(W.c3(1) if args.profile_workload == "mesh127" else W.c2(1), prec)
    plan = binding.Plan(w.problem, w.params)
    for _ in range(args.profile_increments):
        info = plan.increment()
        print(json.dumps({k: info[k] for k in ("t", "M", "n_candidates", "samples", "cg_iters_total", "ms_device")}))
    plan.close()
    torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--t", type=int, default=3, help="coupled increment timed as one step")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--ref-rows", type=int, default=0,
                    help="lattice nodes per reference step (0: 24 per host core, the cpu_baseline sample)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-accuracy", action="store_true")
    ap.add_argument("--skip-next-rows", action="store_true",
                    help="skip the reconstruction / evaluation / statistics / random-lattice leg")
    ap.add_argument("--n-test", type=int, default=4096, help="test points of the error evaluation")
    ap.add_argument("--profile-increments", type=int, default=0,
                    help="profiling mode: only run this many increments of the 2-D workload (no timing)")
    ap.add_argument("--precision", choices=["mixed", "fp64", "fp64_dst"], default="mixed")
    ap.add_argument("--skip-fp64", action="store_true",
                    help="time the mixed path only (profiling runs of the headline step)")
    ap.add_argument("--profile-workload", choices=["mesh63", "mesh127"], default="mesh63",
                    help="profiling mode: the 63x63 2-D workload or the 127x127 lognormal-type one")
    args = ap.parse_args()
    if args.profile_increments:
        profile_case(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" and torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
