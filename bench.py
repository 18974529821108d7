#!/usr/bin/env python3
"""Benchmark: Monte Carlo TRG trajectories per second on GB300.

One step = one call of the whole hot path (mctrg_run: sampling, split,
plaquette contraction, batched Jacobi SVD at every level, final trace,
estimator) over a batch of trajectories of the workload.  Prints one JSON
line (rank 0).  `--impl reference` times the CPU oracle on the same
workload instead.  Under torchrun every rank runs its own trajectory range
(replicas: no collective on the data path) and rank 0 reports the
whole-job rate over the slowest rank's time.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# workload name -> (description, parameters)
WORKLOADS = {
    # the metric's configuration: 2D Ising 1024 x 1024, chi = 16, plain FP64
    "ising-L1024-chi16-fp64": dict(L=1024, chi=16, beta=0.44, h=0.0, traj_per_step=1, precision=0),
    "ising-L256-chi16-fp64": dict(L=256, chi=16, beta=0.44, h=0.0, traj_per_step=8, precision=0),
    "ising-L32-chi16-fp64": dict(L=32, chi=16, beta=0.44, h=0.0, traj_per_step=512, precision=0),
    "ising-L16-chi8-fp64": dict(L=16, chi=8, beta=0.44, h=0.0, traj_per_step=4096, precision=0),
    "ising-L4-chi2-fp64": dict(L=4, chi=2, beta=0.44, h=0.0, traj_per_step=1 << 20, precision=0),
}
DEFAULT_WORKLOAD = "ising-L1024-chi16-fp64"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP64 rate of GB300 from its unit counts: 152 SMs x 2 FP64 FMA per clock x 2
# flops x 2.07 GHz = 1.26 TFLOP/s (nominal 1.25).  The roofline uses the
# library's DFMA probe measured in the same run; this is the fallback.
FP64_NOMINAL_TFLOPS = 1.25
# DRAM bytes (read + write) of one 256 x 256 matrix, from ncu captures of the
# kernels on a case of 128 such matrices (Ising 32 x 32, chi = 16):
# k_jacobi_warp 2.66 GB and k_bidiag 917.1 MB per launch of 128.
JACOBI_DRAM_BYTES_PER_MATRIX_N256 = 2.658e9 / 128
BIDIAG_DRAM_BYTES_PER_MATRIX_N256 = 917.06e6 / 128


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return dict(FALLBACK_PEAKS), "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(wl, seconds_budget=20.0, workers=None):
    """Oracle (CPU, FP64) trajectories/s for the workload, from a bounded sample.

    Runs whole oracle trajectories on a lattice small enough to finish in the
    budget with the same chi and level shapes, then scales by the number of
    per-trajectory tensors at the sampled levels (both grow as L^2), which
    holds the oracle's work.  Returns (rate, cores, sample description).
    """
    import multiprocessing as mp
    from oracle import ising
    from oracle.trg import Problem, run_trajectory
    workers = workers or os.cpu_count() or 1
    L, chi = wl["L"], wl["chi"]
    Ls = min(L, 32 if chi >= 16 else (64 if chi >= 8 else 256))
    prob = Problem(ising.site_tensor(wl["beta"], wl["h"]), Ls, chi)
    ctx = mp.get_context("spawn")
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"          # one BLAS thread per worker process
    t0 = time.perf_counter()
    done = 0
    with ctx.Pool(workers) as pool:
        batch = workers
        while True:
            pool.starmap(run_trajectory, [(prob, 12345, done + i) for i in range(batch)])
            done += batch
            if time.perf_counter() - t0 > seconds_budget / 2 or done >= 100000:
                break
            batch *= 2
    dt = time.perf_counter() - t0
    scale = (L * L) / float(Ls * Ls)
    rate = done / dt / scale
    desc = ("oracle, %d whole trajectories of the %dx%d lattice (chi=%d, beta=%g) on %d spawn workers "
            "in %.1f s, scaled by the per-trajectory tensor count ratio %.0f" % (done, Ls, Ls, chi, wl["beta"],
                                                                               workers, dt, scale))
    return rate, workers, desc


# the serving stand-in's sample cap: 2^16 (the literal workload's 2^18 would hold one job for
# minutes at these lattice sizes and keep the bench's serving phase from ending in a few minutes)
SERVE_MAX_SAMPLES = 1 << 16


def _serve_mix(rng, max_samples=SERVE_MAX_SAMPLES):
    """One job of the serving stand-in (small lattices; the literal sizes run as refusals)."""
    return (float(rng.uniform(0.3, 0.6)), float(rng.choice([0.0, 0.05])), int(rng.choice([4, 8, 16, 32])),
            int(rng.choice([2, 4, 8])), float(10 ** rng.uniform(-4, -2)), int(max_samples), int(rng.integers(1 << 62)))


def _serve_literal(rng):
    """One job at the serving workload's literal sizes: L in 2^8..2^16, chi in {8, 16, 32},
    target 1e-6..1e-4 (refused at submission or projected out of reach)."""
    return (float(rng.uniform(0.3, 0.6)), float(rng.choice([0.0, 0.05])), int(2 ** rng.integers(8, 17)),
            int(rng.choice([8, 16, 32])), float(10 ** rng.uniform(-6, -4)), 1 << 18, int(rng.integers(1 << 62)))


SERVE_ARRIVALS_PER_S = 200.0


def measure_serving(mctrg, seconds, load=0.7, seed=0xB0A7 + 5, literal_jobs=3, drain_s=120.0, burst_jobs=16):
    """Continuous batching under Poisson arrivals at 200 requests/s, job sizes scaled to a
    stated fraction of capacity.

    Job mix (small-lattice stand-in of the serving workload): beta uniform in
    [0.3, 0.6], h in {0, 0.05}, L in {4, 8, 16, 32}, chi in {2, 4, 8}, target
    standard error of ln Z log-uniform in [1e-4, 1e-2].  After the arrivals,
    `literal_jobs` jobs at the literal sizes are submitted; each must be refused at
    submission (footprint beyond the device) or stopped after its first round
    (target projected out of reach), and their latency is reported apart (a first
    round at these sizes holds a worker for seconds, which would swamp the mix's
    percentiles if they arrived with it).  The server's trajectory capacity is measured on a
    burst of `burst_jobs` jobs of the mix (at most 2^16 trajectories each); the
    job size is then scaled, through each job's sample cap, so that 200 jobs/s
    offer `load` times that capacity, and the server's job rate at that size is
    measured on a second burst (arrivals slow to `load` times it if it cannot take
    200/s).  Jobs still running `drain_s` after the last arrival are reported as
    unfinished.
    """
    import numpy as np
    rng = np.random.default_rng(seed)
    srv = mctrg.mctrg_server_create()
    try:
        t0 = time.perf_counter()
        burst = [mctrg.mctrg_server_submit(srv, *_serve_mix(rng))[1] for _ in range(burst_jobs)]
        traj = sum(mctrg.mctrg_server_wait(srv, j, 900.0)[1].n for j in burst)
        cap = traj / (time.perf_counter() - t0)
        cap_samples = int(min(SERVE_MAX_SAMPLES, max(4, round(load * cap / SERVE_ARRIVALS_PER_S))))
        t0 = time.perf_counter()
        burst = [mctrg.mctrg_server_submit(srv, *_serve_mix(rng, cap_samples))[1] for _ in range(8 * burst_jobs)]
        for j in burst:
            mctrg.mctrg_server_wait(srv, j, 900.0)
        job_cap = 8 * burst_jobs / (time.perf_counter() - t0)
        rate = min(SERVE_ARRIVALS_PER_S, load * job_cap)
        ids, lit, refused, n_arr = [], [], 0, 0
        t0 = time.perf_counter()
        t_next = 0.0
        while t_next < seconds:
            now = time.perf_counter() - t0
            if now < t_next:
                time.sleep(t_next - now)
            n_arr += 1
            st, j = mctrg.mctrg_server_submit(srv, *_serve_mix(rng, cap_samples))
            if st == 0:
                ids.append(j)
            t_next += float(rng.exponential(1.0 / rate))
        t_end = time.perf_counter()
        lat, n_traj, reached, projected, unfinished = [], 0, 0, 0, 0
        for j in ids:
            st, est, l = mctrg.mctrg_server_wait(srv, j, max(1.0, drain_s - (time.perf_counter() - t_end)))
            if st == mctrg.MCTRG_ETIMEDOUT:
                unfinished += 1
                continue
            lat.append(l)
            n_traj += est.n
            reached += st == 0
            projected += st == mctrg.MCTRG_EUNREACHABLE
        wall = time.perf_counter() - t0
        lit_lat, lit_sizes, admissible = [], [], []
        for _ in range(literal_jobs):
            job = _serve_literal(rng)
            size = "L=%d chi=%d" % (job[2], job[3])
            # a literal job the footprint admits runs a first round of matrices up to
            # 1024 on a side (a minute or more); it is reported, not run here
            fst, _fp = mctrg.mctrg_server_footprint(srv, job[2], job[3], job[5])
            if fst == 0:
                admissible.append(size)
                continue
            lit_sizes.append(size)
            ts = time.perf_counter()
            st, j = mctrg.mctrg_server_submit(srv, *job)
            if st != 0:
                refused += 1
                lit_lat.append(time.perf_counter() - ts)
                continue
            st, est, l = mctrg.mctrg_server_wait(srv, j, 600.0)
            lit.append(st)
            lit_lat.append(l)
    finally:
        mctrg.mctrg_server_destroy(srv)
    lat = np.sort(np.array(lat))
    return {"capacity_trajectories_per_s": cap, "offered_load": load, "arrivals_per_s": rate,
            "sample_cap_per_job": cap_samples, "job_capacity_per_s": job_cap,
            "jobs": len(ids), "seconds_of_arrivals": seconds,
            "latency_p50_s": float(lat[len(lat) // 2]) if len(lat) else None,
            "latency_p99_s": float(lat[min(len(lat) - 1, int(0.99 * len(lat)))]) if len(lat) else None,
            "trajectories_per_s": n_traj / wall, "jobs_reaching_target": reached,
            "jobs_projected_unreachable": projected, "jobs_unfinished_after_drain": unfinished,
            "literal_jobs": {"sizes": lit_sizes, "admissible_not_run": admissible, "refused_at_submit": refused,
                             "projected_out_of_reach": int(sum(1 for x in lit if x == mctrg.MCTRG_EUNREACHABLE)),
                             "other_status": [int(x) for x in lit if x != mctrg.MCTRG_EUNREACHABLE],
                             "latency_s": lit_lat},
            "mix": "beta U[0.3,0.6], h {0,0.05}, L {4,8,16,32}, chi {2,4,8}, target SE(ln Z) 1e-4..1e-2 "
                   "log-uniform; job size scaled by the per-job sample cap so that the arrival rate offers "
                   "%.0f%% of the measured trajectory capacity; then %d jobs at the literal sizes "
                   "(L 2^8..2^16, chi {8,16,32}, target 1e-6..1e-4)" % (100 * load, literal_jobs)}


def svd_bench(mctrg, torch, S, n=256, nv=16):
    """The band route (tensor-core dense -> band reduction) and the one-stage
    bidiagonalization route on the same S random n x n matrices, values and nv
    kept vectors: one untimed call, then one call each timed with CUDA events."""
    g = torch.Generator(device="cuda").manual_seed(0x5FD)
    A = torch.randn((S, n, n), dtype=torch.float64, device="cuda", generator=g)
    sig = torch.zeros((S, n), dtype=torch.float64, device="cuda")
    vt = torch.zeros((S, nv, n), dtype=torch.float64, device="cuda")
    out = {"matrices": S, "n": n, "kept_vectors": nv}
    for name, fn in (("band", mctrg.mctrg_svd_band_batched), ("bidiag", mctrg.mctrg_svd_bidiag_batched)):
        st = fn(A, sig, vt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = fn(A, sig, vt)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"status": st, "ms": e0.elapsed_time(e1)}
    return out


def _uneven_jobs(n_jobs, seed):
    """The uneven-batch stand-in: chi in {4, 8, 16, 24}, L in {8, 16, 32, 64} (L <= 32 for
    chi > 8), beta uniform in [0.3, 0.6], h uniform in [0, 0.1], 64-512 trajectories each."""
    import numpy as np
    rng = np.random.default_rng(seed)
    jobs = []
    for _ in range(n_jobs):
        chi = int(rng.choice([4, 8, 16, 24]))
        L = int(rng.choice([8, 16, 32, 64] if chi <= 8 else [8, 16, 32]))
        n = int(rng.integers(64, 513))
        jobs.append((float(rng.uniform(0.3, 0.6)), float(rng.uniform(0, 0.1)), L, chi, n,
                     int(rng.integers(1 << 62)), 0))
    return jobs


def _hotrg_flops(L, chi, D0=2):
    """Algorithmic FP64 flops of one Monte Carlo HOTRG trajectory: per bond the
    two pair Gram matrices, the bond Gram matrix, its bidiagonal reduction
    ((8/3) n^3) and the three contraction stages."""
    Lx = Ly = L
    Dh = Dv = D0
    total = 0.0
    while Lx * Ly > 1:
        n, q = Dh * Dh, Dh * Dv
        kc, N = min(chi, n), Lx * (Ly // 2)
        fma = (2 * q ** 3 + n * n * Dv * Dv + kc * Dv * Dh * Dh * Dv * Dh + kc * Dv * Dh * Dh * Dv * q +
               kc * kc * Dv * Dv * n)
        total += N * (2.0 * fma + 8.0 / 3.0 * n ** 3)
        Lx, Ly = Ly // 2, Lx
        Dh, Dv = Dv, kc
    return total


def measure_hotrg(mctrg, fp64_peak, L=64, chi=16, n=16, beta=0.44, seed=0xB0A7 + 6):
    """Monte Carlo HOTRG (mctrg_hotrg_run, one blocking call that allocates and
    frees its memory): trajectories/s, wall clock, on the Ising torus."""
    import time
    o = mctrg.make_options()
    mctrg.mctrg_hotrg_run(o, 8, chi, 2, seed, beta=beta)            # module load, first allocations
    t0 = time.perf_counter()
    st, est = mctrg.mctrg_hotrg_run(o, L, chi, n, seed, beta=beta)
    dt = time.perf_counter() - t0
    f = _hotrg_flops(L, chi) * n
    return {"config": {"L": L, "chi": chi, "beta": beta, "trajectories": n}, "seconds": dt,
            "trajectories_per_s": n / dt, "alg_tflops": f / dt / 1e12,
            "frac_of_fp64_peak": (f / dt / 1e12) / fp64_peak if fp64_peak else None,
            "ln_mean_Z": est.ln_mean_Z, "se_ln_Z": est.se_ln_Z, "status": mctrg.mctrg_strerror(st),
            "note": "whole call on the wall clock (allocation, every kernel, the copies); the dominant kernel, "
                    "the contraction's middle stage, runs at the FP64 rate"}


def measure_uneven(mctrg, n_jobs=24, seed=0xB0A7 + 4):
    """Jobs of uneven chi and lattice size: (a) through the server (each job on a
    worker's stream, FP64), (b) as one batch (levels advanced together, the SVD
    stages in ragged launches over every job's matrices, autotuned launch
    geometry), FP64, and (c) the batch with the FP64-accurate tensor-core
    contraction.  The same jobs and counters in every run: each job's ln Z^ must
    agree (to the rounding of the server's merge of its rounds)."""
    import numpy as np
    jobs = _uneven_jobs(n_jobs, seed)
    traj = sum(j[4] for j in jobs)
    out = {"jobs": n_jobs, "trajectories": traj,
           "mix": "chi {4,8,16,24}, L {8..64}, beta U[0.3,0.6], h U[0,0.1], 64-512 trajectories each"}
    srv = mctrg.mctrg_server_create()
    t0 = time.perf_counter()
    ids = []
    try:
        for b, h, L, chi, n, sd, _ in jobs:
            st, j = mctrg.mctrg_server_submit(srv, b, h, L, chi, 0.0, n, sd)   # fixed-sample job
            ids.append(j)
        srv_est = [mctrg.mctrg_server_wait(srv, j, 1800.0)[1] for j in ids]
        wall = time.perf_counter() - t0
    finally:
        mctrg.mctrg_server_destroy(srv)
    srv_traj = sum(e.n for e in srv_est)
    out["server_fp64"] = {"seconds": wall, "trajectories": srv_traj, "trajectories_per_s": srv_traj / wall}
    import tempfile
    cache = os.path.join(tempfile.gettempdir(), "mctrg_autotune_cache.txt")
    for name, prec in (("batch_fp64", mctrg.MCTRG_FP64), ("batch_fp64tc", mctrg.MCTRG_FP64TC)):
        opts = mctrg.make_options(precision=prec, autotune_cache=cache)
        # one trajectory per job first: every shape of the batch is tuned (and cached) before timing
        mctrg.mctrg_batch_run([(b, h, L, chi, 1, sd, 0) for b, h, L, chi, _, sd, _ in jobs], opts)
        t0 = time.perf_counter()
        st, ests = mctrg.mctrg_batch_run(jobs, opts)
        wall = time.perf_counter() - t0
        same = [(a, b) for a, b in zip(ests, srv_est) if a.n == b.n]   # jobs that ran the same trajectories
        dev = max([abs(a.ln_mean_Z - b.ln_mean_Z) / abs(b.ln_mean_Z) for a, b in same
                   if np.isfinite(a.ln_mean_Z) and np.isfinite(b.ln_mean_Z)] or [0.0])
        out[name] = {"status": mctrg.mctrg_strerror(st), "seconds": wall, "trajectories_per_s": traj / wall,
                     "max_rel_lnZ_vs_server": dev, "jobs_compared_with_server": len(same)}
    out["trajectories_per_s"] = out["batch_fp64tc"]["trajectories_per_s"]
    return out


def _time_to_se(est, rate, targets=(1e-1, 1e-2)):
    """Trajectories and seconds to reach a standard error of ln Z, projected from this run's
    estimate by the 1/sqrt(N) law (Sec. V, Eq. shrunkDev) at this run's rate."""
    if not (est.n > 1 and est.se_ln_Z > 0 and math.isfinite(est.se_ln_Z) and rate > 0):
        return None
    out = {}
    for t in targets:
        n = est.n * (est.se_ln_Z / t) ** 2
        out["se_%g" % t] = {"trajectories": n, "seconds": n / rate}
    return out


def measure_time_to_se(mctrg, precision=0, L=32, chi=16, beta=0.44, n=2048, target=1e-3, svd=0):
    """Time to a stated standard error of ln Z on the 32 x 32 lattice (chi = 16): n
    trajectories, their SE, the trajectories the target needs by the 1/sqrt(N) law and the
    time at the measured rate (this lattice's estimator is well behaved: ESS near n)."""
    ctx = mctrg.mctrg_create(mctrg.make_options(precision=precision, svd=svd))
    try:
        assert mctrg.mctrg_init_lattice(ctx, beta, 0.0, L, chi) == 0
        mctrg.mctrg_run(ctx, 64, 0x5E, 10 ** 6)             # warm
        t0 = time.perf_counter()
        st, est = mctrg.mctrg_run(ctx, n, 0x5E, 0)
        dt = time.perf_counter() - t0
    finally:
        mctrg.mctrg_destroy(ctx)
    need = n * (est.se_ln_Z / target) ** 2
    return {"lattice": "Ising %dx%d, chi=%d, beta=%g" % (L, L, chi, beta), "trajectories": n,
            "seconds": dt, "trajectories_per_s": n / dt, "se_ln_Z": est.se_ln_Z, "ess": est.ess,
            "target_se_ln_Z": target, "trajectories_needed": need, "seconds_needed": need * dt / n}


def run_reference(args, wl, rank, world):
    if rank != 0:
        return
    for _ in range(args.warmup):
        pass   # the oracle has no device state to warm; each step below is a fresh sample
    rates = []
    t_all = time.perf_counter()
    budget = max(5.0, min(20.0, 150.0 / max(1, args.steps)))
    for _ in range(args.steps):
        r, cores, desc = oracle_rate(wl, seconds_budget=budget)
        rates.append(r)
    value = sum(rates) / len(rates)
    line = {"impl": "reference", "metric": "trajectories/s", "value": value, "unit": "trajectories/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * (time.perf_counter() - t_all) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, **{k: wl[k] for k in ("L", "chi", "beta", "h")}},
            "cpu_baseline": {"value": value, "unit": "trajectories/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "trajectories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# The per-sample standard deviations of Z~/Z the paper reports (Table 1) for its
# 128-spin network (spins on the bonds of an 8 x 8 tensor network, Fig. 1).
TABLE1 = [(6, 1.5, 4.171e-2, 1 << 20), (28, 2.34826, 5.017e-4, 4096), (40, 2.34826, 1.353e-5, 512)]


def run_table1(mctrg, np):
    """Per-sample std of Z~ over its mean at the Table 1 points, on the paper's
    lattice, with the trajectory counts of TABLE1 (chi~ = 40 splits 1600 x 1600
    matrices at its deepest levels)."""
    import time
    out = []
    for chi, T, paper, n in TABLE1:
        row = {"chi": chi, "T": T, "paper_std": paper}
        ctx = mctrg.mctrg_create(mctrg.make_options())
        assert mctrg.mctrg_init_bond_lattice(ctx, 1.0 / T, 0.0, 8, chi) == 0
        ln = np.zeros(n)
        sg = np.zeros(n, np.int8)
        fl = np.zeros(n, np.uint8)
        t0 = time.perf_counter()
        st, est = mctrg.mctrg_run(ctx, n, 0x7AB1E + chi, 0, ln, sg, fl)
        dt = time.perf_counter() - t0
        mctrg.mctrg_destroy(ctx)
        x = sg * np.exp(ln - ln.max())
        mean = x.mean()
        row.update({"trajectories": n, "seconds": dt, "trajectories_per_s": n / dt,
                    "std_over_mean": float(x.std(ddof=1) / mean), "ln_mean_Z": est.ln_mean_Z,
                    "se_ln_Z": est.se_ln_Z, "n_flagged": int(est.n_flagged), "status": mctrg.mctrg_strerror(st)})
        out.append(row)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--traj-per-step", type=int, default=0)
    ap.add_argument("--precision", default="", choices=["", "fp64", "tf32", "bf16", "tf32x3", "bf16x3", "fp64tc"],
                    help="arithmetic of the contraction (default: the workload's, FP64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--serve-load", type=float, default=0.7)
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--no-time-to-se", action="store_true")
    ap.add_argument("--no-hotrg", action="store_true")
    ap.add_argument("--svd-bench", type=int, default=0, metavar="S",
                    help="time the batched SVD routes alone on S random 256 x 256 matrices (16 kept vectors), "
                         "one warm-up call each, then exit")
    ap.add_argument("--table1", action="store_true",
                    help="per-sample std of Z~ on the paper's 128-spin network (Table 1) instead of the bench line")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.traj_per_step:
        wl["traj_per_step"] = args.traj_per_step
    if args.precision:
        wl["precision"] = ["fp64", "tf32", "bf16", "tf32x3", "bf16x3", "fp64tc"].index(args.precision)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return

    import numpy as np
    import torch
    from paper_1710_03757_gb300 import build, mctrg, replicas
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        build.build()
    if args.svd_bench:
        if rank == 0:
            print(json.dumps(svd_bench(mctrg, torch, args.svd_bench)))
        return
    if args.table1:
        if rank == 0:
            print(json.dumps({"table1": run_table1(mctrg, np),
                              "lattice": "Ising spins on the bonds of an 8 x 8 periodic tensor network (128 spins)",
                              "note": "std of Z~ over the sample mean of Z~ (the paper divides by the exact Z)"}))
        return
    if dist:
        dist.barrier()
    # the FP64 roofline's denominator, measured on this device now (DFMA probe)
    with ClockSampler(local) as pclk:
        pst, fp64_peak, fp64_ms = mctrg.mctrg_measure_fp64_peak(local)
    fp64_probe = ({"tflops": fp64_peak, "launch_ms": fp64_ms, "clocks": pclk.summary()} if pst == 0
                  else {"error": mctrg.mctrg_strerror(pst)})
    stream = torch.cuda.Stream()
    B = wl["traj_per_step"]
    seed = 0x4D435452 + 2

    def make_ctx(prec, svd=None):
        if svd is None:   # FP64TC takes the tensor-core SVD route too
            svd = mctrg.SVD_BAND if prec == mctrg.MCTRG_FP64TC else mctrg.SVD_AUTO
        opts = mctrg.make_options(device=local, stream=stream.cuda_stream, precision=prec, profile=1, svd=svd)
        c = mctrg.mctrg_create(opts)
        s = mctrg.mctrg_init_lattice(c, wl["beta"], wl["h"], wl["L"], wl["chi"])
        if s != 0:
            raise RuntimeError("init failed: " + mctrg.mctrg_strerror(s))
        return c

    def first_of(step):
        # trajectory counters: rank r, step s covers [(s * world + r) * B, ...)
        return replicas.first_trajectory(step, rank, world, B)

    def one_step(c, step, ln, sg, fl):
        st, est = mctrg.mctrg_run(c, B, seed, first_of(step), ln, sg, fl)
        if st not in (0, mctrg.MCTRG_EDOMAIN, mctrg.MCTRG_ENOCONV):
            raise RuntimeError("run failed: " + mctrg.mctrg_strerror(st))
        return est

    def timed_steps(c, nsteps, warm, step0):
        """warm untimed steps, then nsteps timed steps; returns ms, estimates, per-step outputs."""
        outs = [(torch.zeros(B, dtype=torch.float64, device="cuda"), torch.zeros(B, dtype=torch.int8, device="cuda"),
                 torch.zeros(B, dtype=torch.uint8, device="cuda")) for _ in range(nsteps)]
        for w in range(warm):
            one_step(c, step0 + nsteps + 1 + w, *outs[0])   # counters outside the timed range
        torch.cuda.synchronize()
        mctrg.mctrg_reset_kernel_stats(c)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ests = []
        e0.record(stream)
        for i in range(nsteps):
            ests.append(one_step(c, step0 + i, *outs[i]))
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return e0.elapsed_time(e1), ests, outs

    ctx = make_ctx(wl["precision"])
    with ClockSampler(local) as clk:
        ms, ests, outs = timed_steps(ctx, args.steps, args.warmup, 0)
    stats = [mctrg.mctrg_kernel_stats(ctx, k) for k in range(mctrg.K_COUNT)]
    launches = int(sum(st_.launches for st_ in stats))
    # e2e: the public API calls a user makes (create, init, run), host result buffers, wall clock
    t0 = time.perf_counter()
    c2 = make_ctx(wl["precision"])
    ln_h, sg_h, fl_h = np.zeros(B), np.zeros(B, np.int8), np.zeros(B, np.uint8)
    one_step(c2, args.steps, ln_h, sg_h, fl_h)
    mctrg.mctrg_destroy(c2)
    e2e_s = time.perf_counter() - t0
    # the same trajectories with the contraction on the tensor cores: error-compensated
    # TF32 (TF32X3), and BF16 slices at FP64 accuracy (FP64TC, Ozaki scheme)
    mixed = None
    if wl["precision"] == 0 and not args.no_mixed:
        mixed = {}
        steps_m = min(args.steps, 5)
        ref = np.concatenate([o[0].cpu().numpy() for o in outs[:steps_m]])
        e64 = mctrg.mctrg_merge_estimates(ests[:steps_m])
        peaks_m, _ = measured_peaks()
        for name, prec, note, ratio in (
                ("tf32x3", mctrg.MCTRG_TF32X3, "TF32 hi/lo split, three tcgen05 passes, FP32 accumulation", 0.5),
                ("fp64tc", mctrg.MCTRG_FP64TC, "BF16 slices multiplied exactly on tcgen05, summed in FP64 "
                                               "(Ozaki scheme), in the contraction and in the SVD's dense -> "
                                               "band reduction (8-bit digits of a fixed-point trailing matrix)",
                 1.0)):
            cm = make_ctx(prec)
            # at most 5 timed steps: these legs compare paths on the same trajectories
            ms_m, ests_m, outs_m = timed_steps(cm, steps_m, 1, 0)
            gst = mctrg.mctrg_kernel_stats(cm, mctrg.K_GEMM)
            kst = [mctrg.mctrg_kernel_stats(cm, k) for k in range(mctrg.K_COUNT)]
            mctrg.mctrg_destroy(cm)
            got = np.concatenate([o[0].cpu().numpy() for o in outs_m])
            # near-tie trajectories (flagged in either run) may keep different indices: left out,
            # as in the parity tests, and counted
            fl = np.concatenate([o[2].cpu().numpy() for o in outs[:steps_m]]) | np.concatenate(
                [o[2].cpu().numpy() for o in outs_m])
            ok = np.isfinite(ref) & np.isfinite(got) & (fl == 0)
            rel = np.abs(got[ok] - ref[ok]) / np.abs(ref[ok])
            em = mctrg.mctrg_merge_estimates(ests_m)
            # executed tensor-pipe flops of the contraction: passes (TF32X3) or slice
            # products (FP64TC, 28 at inner dimension 256) times the algorithmic 2 n^2 K
            passes = 3 if prec == mctrg.MCTRG_TF32X3 else 28
            tc_rate = passes * gst.flops_alg / (gst.ms / 1e3) / 1e12 if gst.ms > 0 else None
            tc_peak = peaks_m.get("bf16_tflops_sustained", peaks_m.get("bf16_tflops")) * ratio
            mixed[name] = {
                "precision": note + ("; SVD and sampling FP64" if prec == mctrg.MCTRG_TF32X3 else
                                     "; bisection, vectors, chase and sampling FP64"),
                "steps": steps_m,
                "value": B * steps_m * world / (ms_m / 1000.0), "ms_per_step": ms_m / steps_m,
                "lnZ_rel_err_per_traj_median": float(np.median(rel)) if rel.size else None,
                "lnZ_rel_err_per_traj_max": float(np.max(rel)) if rel.size else None,
                "lnZ_abs_err_per_site_max": float(np.max(np.abs(got[ok] - ref[ok]))) / wl["L"] ** 2
                if rel.size else None,
                "lnZhat_rel_err": abs(em.ln_mean_Z - e64.ln_mean_Z) / abs(e64.ln_mean_Z)
                if np.isfinite(em.ln_mean_Z) and np.isfinite(e64.ln_mean_Z) else None,
                "errors_against": "the FP64 path on the same trajectories (parity-tested against the FP64 oracle), "
                                  "unflagged ones: %d of %d" % (int(ok.sum()), len(ok)),
                "contraction": {"launches": gst.launches, "ms": gst.ms, "share_of_step": gst.ms / ms_m,
                                "tensor_tflops": tc_rate, "tensor_peak_tflops": tc_peak,
                                "tensor_frac": tc_rate / tc_peak if tc_rate else None,
                                "peak_note": "MEASURED_PEAKS bf16 sustained" + (" x 1/2 (TF32 nominal ratio)"
                                                                                if ratio != 1.0 else "")},
                "kernels": {mctrg.KERNEL_NAMES[k]: {"launches": kst[k].launches, "ms": round(kst[k].ms, 3),
                                                     "share": round(kst[k].ms / max(1e-9, sum(x.ms for x in kst)),
                                                                    4)}
                            for k in range(mctrg.K_COUNT) if kst[k].launches}}
            bs = kst[mctrg.K_BAND]
            if bs.launches and bs.ms > 0:
                # the reduction's algorithmic (8/3) n^3 FP64 flops per matrix over its time:
                # the rate the FP64 pipe would need to match it
                eq = bs.flops_alg / (bs.ms / 1e3) / 1e12
                fpk = fp64_peak if pst == 0 and fp64_peak > 0 else FP64_NOMINAL_TFLOPS
                mixed[name]["svd_band_stage"] = {
                    "launches": bs.launches, "avg_launch_ms": bs.ms / bs.launches,
                    "fp64_equivalent_tflops": eq, "fp64_peak_tflops": fpk, "frac_of_fp64_peak": eq / fpk,
                    "note": "dense -> band reduction (tensor-core digit products, FP64 panels): algorithmic "
                            "(8/3) n^3 flops per matrix / time, against the FP64 pipe's measured peak"}
    ms_t = torch.tensor([ms, e2e_s], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max, e2e_max = float(ms_t[0]), float(ms_t[1])
    total_traj = B * args.steps * world
    value = total_traj / (ms_max / 1000.0)
    # the whole job's estimate: every rank's sufficient statistics, merged exactly
    all_ests = replicas.gather_estimates(dist, ests, device="cuda") if dist else ests
    merged = mctrg.mctrg_merge_estimates(all_ests)
    if rank != 0:
        mctrg.mctrg_destroy(ctx)
        if dist:
            dist.destroy_process_group()
        return
    # roofline of the dominant kernel (largest summed time)
    dom = max(range(mctrg.K_COUNT), key=lambda k: stats[k].ms)
    ds = stats[dom]
    peaks, peak_src = measured_peaks()
    # (K_BAND: the band route's reduction, reported as its algorithmic (8/3) n^3 FP64 flops
    # against the FP64 pipe's peak: the rate the FP64 pipe would need to match it)
    flop_classes = (mctrg.K_BIDIAG, mctrg.K_JACOBI, mctrg.K_VECTORS, mctrg.K_SAMPLE, mctrg.K_FORM_XY,
                    mctrg.K_GEMM, mctrg.K_TRACE, mctrg.K_BAND, mctrg.K_CHASE)
    fp64_dom = dom in flop_classes and (dom != mctrg.K_GEMM or wl["precision"] == 0)
    if fp64_dom and ds.flops_alg > 0:
        achieved = ds.flops_alg / (ds.ms / 1000.0) / 1e12 if ds.ms > 0 else 0.0
        peak = fp64_peak if pst == 0 and fp64_peak > 0 else FP64_NOMINAL_TFLOPS
        per_matrix = {mctrg.K_JACOBI: JACOBI_DRAM_BYTES_PER_MATRIX_N256,
                      mctrg.K_BIDIAG: BIDIAG_DRAM_BYTES_PER_MATRIX_N256}.get(dom)
        roof = {"bound": "alu", "kernel": mctrg.KERNEL_NAMES[dom], "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": ("measured: the library's DFMA throughput probe (mctrg_measure_fp64_peak) "
                                "in this run" if pst == 0 else
                                "nominal FP64 rate of GB300 from unit counts (probe failed)"),
                "peak_nominal": FP64_NOMINAL_TFLOPS, "fp64_probe": fp64_probe,
                "traffic": (per_matrix * ds.items / max(1, ds.launches)
                            if per_matrix and wl["chi"] == 16 else None),
                "traffic_note": "bytes per launch, scaled from the per-matrix DRAM bytes of the ncu capture",
                "launches": ds.launches, "avg_launch_ms": ds.ms / max(1, ds.launches),
                "alg_flops_per_launch": ds.flops_alg / max(1, ds.launches)}
        if dom == mctrg.K_BAND:
            roof["note"] = ("FP64-equivalent rate: the reduction's (8/3) n^3 flops run as tensor-core digit "
                            "products and FP64 panel factorizations, so it can exceed the FP64 pipe's peak")
    else:
        achieved = ds.bytes_alg / (ds.ms / 1000.0) / 1e9 if ds.ms > 0 else 0.0
        roof = {"bound": "hbm", "kernel": mctrg.KERNEL_NAMES[dom], "achieved": achieved,
                "peak": peaks.get("hbm_gbs"), "unit": "GB/s", "frac": achieved / peaks.get("hbm_gbs"),
                "peak_source": peak_src, "traffic": None}
    kernels = {mctrg.KERNEL_NAMES[k]: {"launches": stats[k].launches, "ms": round(stats[k].ms, 3),
                                        "share": round(stats[k].ms / max(1e-9, sum(x.ms for x in stats)), 4)}
               for k in range(mctrg.K_COUNT)}
    line = {"metric": "trajectories/s", "value": value, "unit": "trajectories/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ["f64", "f64+tf32", "f64+bf16", "f64+tf32x3", "f64+bf16x3", "f64 (bf16 slices)"][wl["precision"]],
            "data": "synthetic",
            "config": {"workload": args.workload, "L": wl["L"], "chi": wl["chi"], "beta": wl["beta"],
                       "h": wl["h"], "trajectories_per_step_per_gpu": B, "parallelism": "replicas%d" % world,
                       "l2": "working set (halves, matrices) far larger than L2; no flush needed"},
            "e2e": {"value": B * world / e2e_max if e2e_max > 0 else None,
                    "unit": "trajectories/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": B * (8 + 1 + 1) + 8 * 6,
                    "note": "mctrg_create + mctrg_init_lattice + mctrg_run with host result buffers, wall "
                            "clock; the inputs are five scalars passed by value (beta, h, L, chi, seed)"},
            "mixed": mixed,
            "gpu_launches": launches, "roofline": roof, "kernels": kernels,
            "estimate": {"ln_mean_Z": merged.ln_mean_Z, "se_ln_Z": merged.se_ln_Z, "n": merged.n,
                         "ess": merged.ess, "n_flagged": merged.n_flagged,
                         "note": ("effective sample size %.2f of %d: the estimate is dominated by its largest "
                                  "trajectories and its SE is not reliable" % (merged.ess, merged.n))
                         if merged.ess < 0.2 * merged.n else "effective sample size %.1f of %d" % (merged.ess,
                                                                                                   merged.n)},
            "time_to_se": _time_to_se(merged, value),
            "clocks": clk.summary()}
    mctrg.mctrg_destroy(ctx)
    if args.serve_seconds > 0:
        try:
            line["serve"] = measure_serving(mctrg, args.serve_seconds, args.serve_load)
        except Exception as e:
            line["serve"] = {"error": repr(e)[:200]}
    if not args.no_time_to_se:
        try:
            line["time_to_se_32x32"] = {"fp64": measure_time_to_se(mctrg, 0),
                                        "fp64tc": measure_time_to_se(mctrg, mctrg.MCTRG_FP64TC,
                                                                     svd=mctrg.SVD_BAND)}
        except Exception as e:
            line["time_to_se_32x32"] = {"error": repr(e)[:200]}
    if not args.no_hotrg:
        try:
            line["hotrg"] = measure_hotrg(mctrg, line["roofline"].get("peak") if line["roofline"]["unit"] == "TFLOP/s"
                                          else None)
        except Exception as e:
            line["hotrg"] = {"error": repr(e)[:200]}
    if not args.no_uneven:
        try:
            line["uneven_batch"] = measure_uneven(mctrg)
        except Exception as e:
            line["uneven_batch"] = {"error": repr(e)[:200]}
    if not args.no_cpu_baseline:
        try:
            r, cores, desc = oracle_rate(wl)
            line["cpu_baseline"] = {"value": r, "unit": "trajectories/s", "cores": cores, "kind": "oracle",
                                    "sample": desc}
        except Exception as e:   # never lose the GPU line over the baseline
            line["cpu_baseline"] = {"value": None, "error": repr(e)[:200]}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
