#!/usr/bin/env python
"""Throughput of the sparsified thin-wire MoM hot path on GB300: unknowns x incidences solved per
second, RCS checked against the plain FP64 path.

One step = the whole hot path on one cloud through one C-ABI call (swm_run): load the wire cloud,
S-NFC neighbour search, block fill, block-Jacobi preconditioner, right-hand sides, GMRES(50) to
1e-6 for every incidence, RCS.  Headline workload (the largest single-GPU configuration):
1,000,000 wires in 8 Gaussian clusters (sigma 40 wavelengths) in a 600-wavelength cube, lengths
U[0.3, 0.6] wavelengths, <= 0.08-wavelength segments, radius 1e-3, random directions, r_c = 3
wavelengths, 37 monostatic incidences (theta 0..180 degrees in 5-degree steps), monostatic RCS.
The 10,000-wire single-incidence workload (720-angle bistatic RCS) is measured beside it.  Inputs
are seeded and synthetic.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own cloud (seed 1 + rank): weak scaling, no data-path
collective; the timing is the max over ranks.  ``--impl reference`` times the FP64 CPU oracle on
the host cores (a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import (cloud_batching_snapshot, cloud_learned, cloud_mid, cloud_precision,  # noqa: E402
                   incidences_monostatic, incidences_single_minus_z, observations_phi_cut)

METRIC = "unknowns×incidences solved/sec at ≤0.1 dB RCS error vs plain FP64 path"
UNIT = "unknowns*incidences/s"
K0 = 2.0 * math.pi
R_C = 3.0
TOL = 1e-6
RESTART = 50
N_OBS = 720
FP32_FLOPS_PER_EVAL = 29  # algorithmic FP32 operations of one kernel evaluation of the fill
N_SM = 152


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi samples every 50 ms while the timed region runs.

    start() returns once nvidia-smi has written its first sample, so the sampler is running when
    the timed region begins; mark() notes where the timed region starts in its output, and stop()
    keeps the samples after the mark (the last one before it if the region was shorter than the
    sampling period, flagged by "samples": 0)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None and self._lines() == 0:
            time.sleep(0.02)
        self.mark0 = 0

    def _lines(self):
        try:
            with open(self.path) as f:
                return sum(1 for line in f if line.strip())
        except OSError:
            return 0

    def mark(self):
        self.mark0 = self._lines()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        lines = [line for line in open(self.path) if line.strip()]
        os.unlink(self.path)
        return self.summarise(lines, getattr(self, "mark0", 0))

    @staticmethod
    def summarise(lines, mark0):
        """Median SM clock, max clock and active slowdown reasons of the samples after the mark
        (the last one before it when the region was shorter than the sampling period)."""
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        during = lines[mark0:]
        if not during:
            during = lines[max(0, mark0 - 1):mark0]
        sm, smax, reasons = [], [], set()
        for line in during:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(lines) - mark0, "reasons": sorted(reasons)}


def rcs_db_error(s, ref, floor_db=30.0):
    s, ref = np.asarray(s).ravel(), np.asarray(ref).ravel()
    keep = ref >= ref.max() * 10 ** (-floor_db / 10)
    return float(np.max(np.abs(10 * np.log10(s[keep] / ref[keep]))))


# ---------------------------------------------------------------------------------- workloads
# The headline workload is the largest single-GPU configuration: 1,000,000 wires in 8 Gaussian
# clusters, 37 monostatic incidences, GMRES(50) to 1e-6, monostatic RCS.  The 10,000-wire
# single-incidence workload with its 720-angle bistatic RCS is measured beside it.
WORKLOADS = {
    "learned": dict(cloud=lambda seed: cloud_learned(seed=3 + seed), r_c=3.0, n_inc=37, n_obs=0,
                    text="learned: 1,000,000 wires in 8 Gaussian clusters (sigma 40) in a 600-wavelength cube, "
                         "lengths U[0.3, 0.6], r_c 3, 37 monostatic incidences (theta 0..180 deg, 5 deg), "
                         "GMRES(50) 1e-6, monostatic RCS"),
    "mid": dict(cloud=lambda seed: cloud_mid(seed=seed), r_c=3.0, n_inc=1, n_obs=N_OBS,
                text="mid: 10,000 wires, Gaussian sigma 30, r_c 3, GMRES(50) 1e-6, 1 incidence, "
                     "720-angle bistatic RCS"),
}


def workload_inputs(name, rank=0):
    w = WORKLOADS[name]
    cl = w["cloud"](rank_seed(rank))
    inc = incidences_single_minus_z() if w["n_inc"] == 1 else incidences_monostatic(w["n_inc"])
    obs = observations_phi_cut(w["n_obs"]) if w["n_obs"] else None
    return cl, inc, obs


def ball_sample(cloud, n_target, seed=0):
    """The n_target wires nearest to a randomly drawn wire of the cloud (local density kept; the
    centre is drawn with the wires' own distribution, so the sample's density is typical)."""
    rng = np.random.default_rng(seed)
    c0 = cloud.centres[rng.integers(0, cloud.nw)]
    d = np.linalg.norm(cloud.centres - c0, axis=1)
    return cloud.subset(np.sort(np.argsort(d)[:min(cloud.nw, n_target)]))


def _oracle_blocks(args):
    """Worker: the oracle's blocks of the given (p, q) pairs and the inverses of the given wires'
    self blocks."""
    import oracle as O

    cloud, k, pairs, rows = args
    blocks = [O.block(cloud, k, int(p), int(q)) for p, q in pairs]
    return blocks, O.block_jacobi(cloud.subset(rows), k)


def oracle_step(cloud, inc, obs, r_c, pool=None, n_chunks=1, solver="gmres"):
    """The whole path on the FP64 CPU oracle (test infrastructure, timed as the CPU baseline):
    pairs, blocks, block-Jacobi, RHS, GMRES per incidence, RCS.  The blocks and the self-block
    inverses are computed in ``pool`` (the oracle's own functions, rows split over the workers).
    Returns (rcs, build seconds, seconds of the per-incidence part)."""
    import scipy.sparse as sp

    import oracle as O

    t0 = time.perf_counter()
    pairs = O.neighbour_pairs(cloud.centres, r_c)
    m, off = O.numbering(cloud.nseg)
    nw = cloud.nw
    bounds = np.linspace(0, nw, n_chunks + 1).astype(np.int64)
    rowpos = np.searchsorted(pairs[:, 0], bounds)
    jobs = [(cloud, K0, pairs[rowpos[i]:rowpos[i + 1]], np.arange(bounds[i], bounds[i + 1]))
            for i in range(n_chunks)]
    res = list(pool.map(_oracle_blocks, jobs)) if pool is not None else [_oracle_blocks(j) for j in jobs]
    rows, cols, vals, Mi = [], [], [], []
    for (blocks, minv), job in zip(res, jobs):
        Mi += minv
        for (p, q), Zb in zip(job[2], blocks):
            rr, cc = np.meshgrid(off[p] + np.arange(m[p]), off[q] + np.arange(m[q]), indexing="ij")
            rows.append(rr.ravel())
            cols.append(cc.ravel())
            vals.append(Zb.ravel())
    N = int(off[-1])
    Z = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    t1 = time.perf_counter()
    b = O.rhs(cloud, K0, inc)
    X = np.zeros_like(b)
    for i in range(b.shape[1]):
        if solver == "bicgstab":
            X[:, i], _, _ = O.bicgstab(Z, b[:, i], Mi, off, TOL, 1000)
        else:
            X[:, i], _, _ = O.gmres(Z, b[:, i], Mi, off, TOL, RESTART, 1000)
    sig = O.rcs_bistatic(cloud, K0, X, obs) if obs is not None else O.rcs_monostatic(cloud, K0, X, inc)
    t2 = time.perf_counter()
    return sig, t1 - t0, t2 - t1


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_pool(cores):
    """Process pool for the oracle (spawned workers, one BLAS thread each)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    return cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"))


def cpu_oracle_sample(name, n_target, cores, steps=1, warmup=0, solver="gmres"):
    """The oracle on a bounded sample of workload ``name``: the wires nearest a random wire of the
    cloud, one incidence; with several incidences in the workload the per-incidence part is
    extrapolated (build once + n_inc x one incidence's RHS, GMRES and RCS)."""
    w = WORKLOADS[name]
    cl_full, inc_full, obs = workload_inputs(name)
    cl = ball_sample(cl_full, n_target)
    inc = inc_full[:1]
    n_inc = inc_full.shape[0]
    with oracle_pool(cores) as pool:
        for _ in range(warmup):
            oracle_step(cl, inc, obs, w["r_c"], pool, cores, solver)
        tb, ts = [], []
        for _ in range(max(1, steps)):
            _, b, s = oracle_step(cl, inc, obs, w["r_c"], pool, cores, solver)
            tb.append(b)
            ts.append(s)
    t_build, t_inc = float(np.mean(tb)), float(np.mean(ts))
    t_step = t_build + n_inc * t_inc
    value = cl.n_unknowns * n_inc / t_step
    kry = "BiCGSTAB" if solver == "bicgstab" else "GMRES(50)"
    sample = (f"{cl.nw} wires nearest a random wire of the {cl_full.nw:,}-wire cloud (N={cl.n_unknowns}), the "
              f"whole path on the FP64 NumPy oracle (blocks and self-block inverses on {cores} processes, the "
              f"solve in one): build {t_build:.2f} s, one incidence's RHS + {kry} 1e-6 + RCS {t_inc:.3f} s")
    if n_inc > 1:
        sample += f"; EXTRAPOLATED to {n_inc} incidences as build + {n_inc} x one incidence"
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "extrapolated": n_inc > 1, "seconds_per_step": t_step}


# ---------------------------------------------------------------------------------- ranks
def rank_seed(rank: int) -> int:
    """Each rank solves its own cloud of the same statistics (weak scaling): seed 1 + rank."""
    return 1 + rank


def aggregate_over_ranks(times_ms, units, device, world):
    """Max of each time over the ranks and the sum of the units they processed (whole-job
    throughput = summed units / slowest rank).  A timing reduction only: no solver data moves."""
    import torch
    import torch.distributed as dist

    tm = torch.tensor([float(t) for t in times_ms], dtype=torch.float64, device=device)
    un = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        dist.all_reduce(un, op=dist.ReduceOp.SUM)
    return tm.tolist(), un.item()


# ---------------------------------------------------------------------------------- our arm
def solve_steps(iterations, restart):
    """Arnoldi step indices j of one solve and the lengths of its restart cycles."""
    steps_j, cycles = [], []
    it = iterations
    while it > 0:
        c = min(restart, it)
        steps_j += list(range(c))
        cycles.append(c)
        it -= c
    return steps_j, cycles


def class_bytes_bicgstab(cls, st, prec, n_rhs):
    """Algorithmic bytes of one BiCGSTAB solve per kernel class.  A step: two products (E, column
    map and row descriptors once for all incidences, the source read and the image written), the
    two direction updates with their incidence-minor copies (p = r + beta (p - omega v): r, p, v
    read, p and its copy written; s = r - alpha v: r, v read, s and its copy written), the inner
    products (rh^H v; t^H s and t^H t) and y += alpha p + omega s, r = s - omega t with rh^H r and
    |r| (y, p, s, t, rh read, y and r written).  Each true-residual check: the residual product
    (b read as well) and |r|.  With the incidence-minor vectors (complex64, 2-256 incidences) the
    direction updates write no copy, and b and y are transposed once each; otherwise each update
    writes the incidence-minor copy and each check copies y."""
    esz = 16 if prec == "c128" else 8
    N, R = st["n"], n_rhs
    vec = R * N * esz
    steps = st["iterations"]
    checks = st["restarts"] + 2
    mat = st["nnz_offd"] * esz + st["ncm_offd"] * 4 + 16 * N
    xt = prec != "c128" and R >= 2
    if cls == "apply":
        return steps * 2 * (mat + 2 * vec) + checks * (mat + 3 * vec)
    minor = xt and 2 <= R <= 256
    if cls == "transpose":
        if minor:
            return steps * (4 + 3) * vec
        return steps * ((5 + 4) * vec if xt else (4 + 3) * vec) + (checks * 2 * vec if xt else 0)
    if cls == "dots":
        return steps * 4 * vec + checks * vec
    if cls == "update":
        return steps * 7 * vec
    return None


def class_bytes(cls, st, prec, n_rhs, restart, solver="gmres"):
    """Algorithmic bytes of one solve for a kernel class of the per-kernel GMRES step.
    Product: E values, column map and row descriptors once per block of incidences sharing a
    read, u read and w written per incidence, and per restart cycle the residual product
    (B and y read, W written); the transpose to incidence-minor order is not counted.  Delayed
    Gram-Schmidt at step j: dots read Q_<j, u and w ((j + 2) vectors; the closing pass of a cycle
    Q_<j and u), update reads Q_<j, u, w and writes q_j and the next u ((j + 4) vectors)."""
    if solver == "bicgstab":
        return class_bytes_bicgstab(cls, st, prec, n_rhs)
    esz = 16 if prec == "c128" else 8
    N, R = st["n"], n_rhs
    vec = R * N * esz
    steps_j, cycles = solve_steps(st["iterations"], restart)
    if cls == "apply":
        rbs = st["step_rhs_block"]
        rb = (32 if R >= 24 else 16) if rbs == 32 else max(1, rbs)
        nblk = -(-R // rb)
        mat = (st["nnz_offd"] * esz + st["ncm_offd"] * 4 + 16 * N) * nblk
        return len(steps_j) * (mat + 2 * vec) + (len(cycles) + 1) * (mat + 3 * vec)
    if cls == "transpose":
        # the copy of u (and of y at each restart) to incidence-minor order: read and written once
        return (len(steps_j) + len(cycles) + 1) * 2 * vec
    if cls == "dots":
        return sum((j + 2) * vec for j in steps_j) + sum((c + 1) * vec for c in cycles)
    if cls == "update":
        return sum((j + 4) * vec for j in steps_j)
    if cls == "gmres":
        # the persistent solve: product and delayed Gram-Schmidt as above, b formed from the wire
        # geometry, restart products, y update by the basis, x = M^-1 y
        mat = st["nnz_offd"] * esz + st["ncm_offd"] * 4 + 16 * N
        b = sum(mat + vec + (2 * j + 6) * vec for j in steps_j) + sum((c + 1) * vec for c in cycles)
        b += (st["restarts"] + 1) * (mat + 3 * vec) + sum(cycles) * vec
        b += st["nw"] * (7 * 8 + 4) + vec + st["nminv"] * esz + 2 * vec
        return b
    return None


def fp32_peak_tflops(pk):
    mhz = pk.get("sm_max_mhz", 2070.0)
    return N_SM * 128 * 2 * mhz * 1e6 / 1e12


def roofline_of(cls, st, prof_ms, launches, prec, n_rhs, restart, steps, pk, per_step_units=None, solver="gmres"):
    """Achieved algorithmic rate of one kernel class over ``steps`` profiled steps."""
    if prof_ms <= 0 or launches <= 0:
        return None
    per_launch_ms = prof_ms / launches
    if cls == "fill_mutual":
        flops = st["fill_evals"] * FP32_FLOPS_PER_EVAL * steps
        peak = fp32_peak_tflops(pk) if prec != "c128" else 1.25
        ach = flops / (prof_ms * 1e-3) / 1e12
        return {"kernel": "k_mutual_blocks_f32" if prec != "c128" else "k_mutual_blocks<double>", "bound": "alu",
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "per_launch_flops": flops / launches, "per_launch_ms": per_launch_ms,
                "peak_source": ("FP32 peak = 152 SMs x 128 lanes x 2 flops x max SM clock" if prec != "c128"
                                else "nominal FP64 peak"),
                "flops_per_eval": FP32_FLOPS_PER_EVAL, "evals_per_launch": st["fill_evals"]}
    b = class_bytes(cls, st, prec, n_rhs, restart, solver)
    if b is None:
        return {"kernel": cls, "bound": "other", "per_launch_ms": per_launch_ms}
    work = b * steps
    ach = work / (prof_ms * 1e-3) / 1e9
    peak = pk.get("hbm_gbs", 6800.0)
    names = {"apply": "block-sparse product, form %s (k_spmv_wa / k_spmv_wg / k_spmv_wm / k_spmv_wp / k_spmv_w / "
                      "k_spmv_t / k_spmv, timed per shape)" % st.get("step_rhs_block"),
             "transpose": "k_rhs_minor_all: pending vectors to incidence-minor order",
             "dots": "k_dots: delayed Gram-Schmidt inner products",
             "update": "k_update: delayed Gram-Schmidt update",
             "gmres": "k_gmres_persist: persistent GMRES solve"}
    if solver == "bicgstab":
        names.update({"transpose": "k_bp_dir (k_bi_dir): direction updates p and s",
                      "dots": "k_bp_rv, k_bp_ts (k_bi_rv, k_bi_ts): inner products r^H v, t^H s, t^H t",
                      "update": "k_bp_xr (k_bi_xr): y and r updates with r^H r and |r|"})
    return {"kernel": names.get(cls, cls), "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "peak_source": "of measured (MEASURED_PEAKS.json copy bandwidth)",
            "per_launch_bytes": work / launches, "per_launch_ms": per_launch_ms}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch over the launch's
# algorithmic bytes, from one ncu capture of the kernel's current code on the 250,000-wire cloud
# of the same density, keyed by (workload, kernel class, precision, solver, product form); the
# bench line's traffic is this ratio times its own algorithmic bytes per launch.  The capture is
# recorded with the profile summaries.  A class or form without a capture of its current code
# reports null.
MEASURED_TRAFFIC = {
    # (form 75's capture, 1.0597 GB against 1.0766 GB, predates its record-based prologue, so the
    # form reports null until it is captured again)
}

PROFILE_CLASSES = ["pairs", "fill_self", "fill_mutual", "invert", "form_e", "apply", "transpose", "dots", "update",
                   "far", "gmres"]


def workload_text(name, solver, restart):
    t = WORKLOADS[name]["text"]
    if solver == "bicgstab":
        return t.replace("GMRES(50) 1e-6", "BiCGSTAB 1e-6 (true residual)")
    return t.replace("GMRES(50)", f"GMRES({restart})")


def measure(name, args, local, world, rank, with_e2e=True, with_fp64=True, steps=None, solver=None):
    """Time workload ``name`` through swm_run (device inputs), then: the class shares (one
    profiled step per class), the dominant and the named classes' rooflines (a separate profiled
    pass), the end-to-end step from pinned host buffers, and the plain FP64 path (its RCS gates the
    fast path).  Returns the record and the summed units."""
    import torch
    import torch.distributed as dist

    from paper_2410_03060_gb300 import swm

    w = WORKLOADS[name]
    solver = solver or args.solver
    cl, inc, obs = workload_inputs(name, rank)
    R, N = inc.shape[0], cl.n_unknowns
    prec_id = swm.SWM_C64 if args.precision == "c64" else swm.SWM_C128
    restart = args.restart
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
           (cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)]
    shape = (R, 2) if obs is None else (R, obs.shape[0], 2)
    sigma = torch.zeros(shape, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    ctx = swm.swm_create(local)
    swm.swm_set_solver(ctx, solver)
    K = steps or args.steps

    def step(c=None, prec=prec_id, inputs=dev, out=sigma):
        rc = swm.swm_run(c or ctx, *inputs, K0, w["r_c"], prec, inc, obs, out, TOL, restart, 2000)
        if rc != 0:
            raise RuntimeError(f"swm_run returned {rc} (not converged)")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region: K steps, nothing profiled
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = swm.swm_get_stats(ctx)["kernel_launches"]
    clocks = ClockSampler(local)
    clocks.start()
    clocks.mark()
    evs = []
    for _ in range(K):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms_step = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    st = swm.swm_get_stats(ctx)
    launches = (st["kernel_launches"] - l0) // max(1, K)
    s_fast = sigma.cpu().numpy().copy()

    # class shares: one profiled step per class (untimed)
    share, prof = {}, {}
    for c in PROFILE_CLASSES:
        swm.swm_profile(ctx, c)
        step()
        torch.cuda.synchronize()
        s = swm.swm_get_stats(ctx)
        share[c] = s["prof_ms"]
        prof[c] = (s["prof_ms"], s["prof_launches"])
    swm.swm_profile(ctx, "none")
    dominant = max(share, key=share.get)
    # roofline pass of the dominant class: a few profiled steps of their own
    rsteps = max(1, min(3, K))
    swm.swm_profile(ctx, dominant)
    for _ in range(rsteps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    s = swm.swm_get_stats(ctx)
    swm.swm_profile(ctx, "none")
    pk = peaks()
    roof = roofline_of(dominant, st, s["prof_ms"], s["prof_launches"], args.precision, R, restart, rsteps, pk,
                       solver=solver)
    if roof is not None:
        roof["class"] = dominant
        roof["profiled_steps"] = rsteps
        ratio = MEASURED_TRAFFIC.get((name, dominant, args.precision, solver, st.get("step_rhs_block")))
        roof["traffic"] = ratio * roof["per_launch_bytes"] if ratio and "per_launch_bytes" in roof else None
    extra_roofs = {}
    for c in ("fill_mutual", "apply", "transpose", "dots", "update"):
        if c != dominant and prof[c][1] > 0:
            extra_roofs[c] = roofline_of(c, st, prof[c][0], prof[c][1], args.precision, R, restart, 1, pk,
                                         solver=solver)

    rec = {"workload": workload_text(name, solver, restart), "solver": solver, "nw": cl.nw, "unknowns": N, "incidences": R, "blocks": st["nb"],
           "ms_per_step": ms_step, "value_local": N * R / (ms_step * 1e-3), "gpu_launches": int(launches),
           "iterations": st["iterations"], "restarts": st["restarts"], "rel_residual": st["rel_residual"],
           "step_rhs_block": st["step_rhs_block"],
           "phase_ms": {k: st[k] for k in ("ms_neighbour", "ms_fill", "ms_precond", "ms_rhs", "ms_solve", "ms_rcs")},
           "kernel_ms_per_step": share, "roofline": roof, "rooflines_other": extra_roofs, "clocks": clk}

    if with_e2e:
        # end to end through the public API: pinned host inputs read in place, RCS written to a
        # pinned host buffer, inside the timed region
        host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in
                   (cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)]
        sig_host = torch.zeros(shape, dtype=torch.float64).pin_memory().numpy()
        e2e = []
        for _ in range(max(1, min(K, 10))):
            flush.zero_()
            torch.cuda.synchronize()
            t = time.perf_counter()
            step(inputs=host_in, out=sig_host)
            torch.cuda.synchronize()
            e2e.append(time.perf_counter() - t)
        rec["e2e_ms"] = 1e3 * float(np.mean(e2e))
        rec["h2d"] = int(sum(a.nbytes for a in host_in))
        rec["d2h"] = int(sig_host.nbytes)
    swm.swm_destroy(ctx)
    del flush
    torch.cuda.empty_cache()

    if with_fp64:
        # the plain FP64 path on the same cloud: its RCS gates the fast path; a few steps timed
        ctx64 = swm.swm_create(local)
        swm.swm_set_solver(ctx64, solver)
        sig64 = torch.zeros_like(sigma)
        step(c=ctx64, prec=swm.SWM_C128, out=sig64)
        torch.cuda.synchronize()
        f64 = []
        for _ in range(max(1, min(K, 3))):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            step(c=ctx64, prec=swm.SWM_C128, out=sig64)
            b.record()
            f64.append((a, b))
        torch.cuda.synchronize()
        ms64 = float(np.mean([a.elapsed_time(b) for a, b in f64]))
        s64 = sig64.cpu().numpy()
        swm.swm_destroy(ctx64)
        torch.cuda.empty_cache()
        rec["ms64"] = ms64
        rec["rcs_err_db_vs_fp64"] = rcs_db_error(s_fast[..., 0], s64[..., 0])
        rec["rcs_rel_l2_vs_fp64"] = float(np.linalg.norm(s_fast[..., 0] - s64[..., 0]) / np.linalg.norm(s64[..., 0]))
    return rec, N * R


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    name = args.workload if args.workload in WORKLOADS else "learned"
    rec, units = measure(name, args, local, world, rank)
    side = None
    if name == "learned" and not args.no_mid:
        side, _ = measure("mid", args, local, world, rank, with_e2e=False, with_fp64=True,
                          steps=max(args.steps, 200), solver="gmres")

    # max over ranks, units over all ranks
    (ms_step, e2e_ms, ms64), total_units = aggregate_over_ranks([rec["ms_per_step"], rec["e2e_ms"], rec["ms64"]],
                                                                units, "cuda", world)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    out = {
        "metric": METRIC, "value": total_units / (ms_step * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64" if args.precision == "c64" else "c128",
        "data": "synthetic (seeded wire clouds)",
        "config": {"workload": rec["workload"], "nw": rec["nw"], "unknowns": rec["unknowns"],
                   "incidences": rec["incidences"], "blocks": rec["blocks"], "precision": args.precision,
                   "solver": rec["solver"], "restart": args.restart if rec["solver"] == "gmres" else None,
                   "tol": TOL,
                   "l2": "inputs larger than L2 (E and the Krylov basis are GBs); a 256 MB write also flushes "
                         "L2 between steps",
                   "parallelism": f"{world} independent clouds (one per GPU)"},
        "gpu_launches": rec["gpu_launches"],
        "e2e": {"value": total_units / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": rec["h2d"],
                "d2h_bytes_per_step": rec["d2h"], "ms_per_step": e2e_ms,
                "path": "swm_run from page-locked host buffers (inputs copied in by DMA, RCS written in place)"},
        "rcs_err_db_vs_fp64": rec["rcs_err_db_vs_fp64"],
        "rcs_rel_l2_vs_fp64": rec["rcs_rel_l2_vs_fp64"],
        "fp64_path": {"value": total_units / (ms64 * 1e-3), "ms_per_step": ms64,
                      "speedup_of_value": ms64 / ms_step},
        "iterations": rec["iterations"], "restarts": rec["restarts"], "rel_residual": rec["rel_residual"],
        "step_rhs_block": rec["step_rhs_block"],
        "phase_ms": rec["phase_ms"],
        "kernel_share_ms_per_step": rec["kernel_ms_per_step"],
        "roofline": rec["roofline"],
        "rooflines_other": rec["rooflines_other"],
        "clocks": rec["clocks"],
    }
    if side is not None:
        out["mid"] = {k: side[k] for k in ("workload", "unknowns", "ms_per_step", "value_local", "iterations",
                                           "gpu_launches", "rcs_err_db_vs_fp64", "ms64", "roofline", "clocks")}
        out["mid"]["fp64_speedup"] = side["ms64"] / side["ms_per_step"]
    if world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        out["cpu_baseline"] = cpu_oracle_sample(name, min(30000, 600 * cores), cores, solver=args.solver)
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------------- larger workloads
SCALE = {
    "learned": dict(cloud=cloud_learned, r_c=3.0, n_inc=37,
                    text="1,000,000 wires in 8 Gaussian clusters (sigma 40) in a 600-wavelength cube, r_c 3"),
    "precision": dict(cloud=cloud_precision, r_c=4.0, n_inc=91,
                      text="200,000 wires in a 350-wavelength cube, lengths 0.35/0.45/0.5, r_c 4"),
    "batching0": dict(cloud=lambda nw=None: cloud_batching_snapshot(0, nw), r_c=3.0, n_inc=181,
                      text="batching snapshot 0 (0.005 wires per cubic wavelength), r_c 3"),
}


def run_scale(args):
    """One larger workload: the step (cloud, build, solve, monostatic RCS) in complex64, with the fill
    measured against the FP32 peak and the block-sparse product against HBM bandwidth.  Prints a
    JSON line of kind "scale"; it is a measurement record, not the benchmark line."""
    import torch

    from paper_2410_03060_gb300 import swm

    w = SCALE[args.workload]
    torch.cuda.set_device(0)
    if args.nw and args.workload == "learned" and args.same_density:
        # a smaller cloud with the full cloud's wire density (cluster sigma scaled with nw^(1/3))
        cl = cloud_learned(nw=args.nw, sigma=40.0 * (args.nw / 1e6) ** (1.0 / 3.0))
    else:
        cl = w["cloud"](nw=args.nw) if args.nw else w["cloud"]()
    n_inc = args.inc or w["n_inc"]
    inc = incidences_monostatic(n_inc)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)]
    mono = torch.zeros((n_inc, 2), dtype=torch.float64, device="cuda")
    ctx = swm.swm_create(0)
    swm.swm_set_solver(ctx, args.solver)
    restart = args.restart

    def step():
        swm.swm_set_cloud(ctx, *dev)
        swm.swm_build(ctx, K0, w["r_c"], swm.SWM_C64)
        rc = swm.swm_solve(ctx, inc, TOL, restart, 2000)
        swm.swm_rcs_monostatic(ctx, mono)
        return rc

    step()
    torch.cuda.synchronize()
    res = {}
    for cls in ("fill_mutual", "apply", "transpose", "dots", "update", "far", "pairs", "fill_self"):
        swm.swm_profile(ctx, cls)
        step()
        torch.cuda.synchronize()
        st = swm.swm_get_stats(ctx)
        res[cls] = (st["prof_ms"], st["prof_launches"])
    swm.swm_profile(ctx, "none")
    ts = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        rc = step()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t)
    st = swm.swm_get_stats(ctx)
    pk = peaks()
    roofs = {c: roofline_of(c, st, res[c][0], res[c][1], "c64", n_inc, restart, 1, pk, solver=args.solver)
             for c in ("fill_mutual", "apply", "transpose", "dots", "update") if res[c][1] > 0}
    N = st["n"]
    out = {
        "kind": "scale", "workload": args.workload, "description": w["text"], "nw": cl.nw, "unknowns": N,
        "blocks": st["nb"], "nnz": st["nnz"], "incidences": n_inc, "solver": args.solver, "restart": restart,
        "iterations": st["iterations"], "restarts": st["restarts"], "converged": st["converged"],
        "rel_residual": st["rel_residual"], "rc": rc,
        "ms_per_step": 1e3 * float(np.median(ts)),
        "value": N * n_inc / float(np.median(ts)), "unit": UNIT,
        "phase_ms": {k: st[k] for k in ("ms_neighbour", "ms_fill", "ms_precond", "ms_rhs", "ms_solve", "ms_rcs")},
        "rooflines": roofs,
        "step_rhs_block": st["step_rhs_block"],
        "kernel_ms_per_step": {k: v[0] for k, v in res.items()},
    }
    print(json.dumps(out))
    swm.swm_destroy(ctx)


def run_compare(args):
    """One larger workload solved in the three precisions (float64, complex64, bfloat16 storage with
    float64 refinement): time per step and the monostatic RCS error of each against the float64
    path.  Prints a JSON line of kind "precision_compare" (a measurement record)."""
    import torch

    from paper_2410_03060_gb300 import swm

    w = SCALE[args.workload]
    torch.cuda.set_device(0)
    cl = w["cloud"](nw=args.nw) if args.nw else w["cloud"]()
    n_inc = args.inc or w["n_inc"]
    inc = incidences_monostatic(n_inc)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)]
    res = {}
    ref = None
    for name, prec in (("c128", swm.SWM_C128), ("c64", swm.SWM_C64), ("bf16", swm.SWM_BF16)):
        ctx = swm.swm_create(0)
        mono = torch.zeros((n_inc, 2), dtype=torch.float64, device="cuda")

        def step():
            swm.swm_set_cloud(ctx, *dev)
            swm.swm_build(ctx, K0, w["r_c"], prec)
            rc = swm.swm_solve(ctx, inc, TOL, args.restart, 2000)
            swm.swm_rcs_monostatic(ctx, mono)
            return rc

        step()
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(1, args.steps)):
            torch.cuda.synchronize()
            t = time.perf_counter()
            rc = step()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t)
        st = swm.swm_get_stats(ctx)
        sig = mono.cpu().numpy()[:, 0].copy()
        if ref is None:
            ref = sig
        ms = 1e3 * float(np.median(ts))
        res[name] = {"ms_per_step": ms, "value": st["n"] * n_inc / (ms * 1e-3), "iterations": st["iterations"],
                     "outer_or_restarts": st["restarts"], "rel_residual": st["rel_residual"], "rc": rc,
                     "phase_ms": {k: st[k] for k in ("ms_neighbour", "ms_fill", "ms_precond", "ms_rhs", "ms_solve",
                                                     "ms_rcs")},
                     "rcs_err_db_vs_c128": rcs_db_error(sig, ref)}
        swm.swm_destroy(ctx)
    for name in res:
        res[name]["speedup_vs_c128"] = res["c128"]["ms_per_step"] / res[name]["ms_per_step"]
    print(json.dumps({"kind": "precision_compare", "workload": args.workload, "description": w["text"],
                      "nw": cl.nw, "incidences": n_inc, "restart": args.restart, "tol": TOL, "unit": UNIT,
                      "paths": res}))


def run_warm(args):
    """Learned warm start on the mid workload: train the network on clouds of the same statistics
    (other seeds, 8 random incidences each, currents solved to 1e-8), then time the step with and
    without it on the benchmark cloud.  Prints a JSON line of kind "warm_start" (a measurement
    record; the network's training is outside the timed steps)."""
    import torch

    from paper_2410_03060_gb300 import swm
    from synth.netinit import init_params

    torch.cuda.set_device(0)
    g = np.random.default_rng(5)

    def incs(n):
        return np.stack([np.arccos(g.uniform(-1, 1, n)), g.uniform(0, 2 * math.pi, n), g.uniform(0, math.pi, n)], 1)

    train = []
    for seed in range(11, 11 + args.train_clouds):
        c = cloud_mid(seed=seed)
        ctx = swm.swm_create(0)
        swm.swm_set_cloud(ctx, c.centres, c.dirs, c.lengths, c.radii, c.nseg)
        swm.swm_build(ctx, K0, R_C, swm.SWM_C64)
        inc = incs(8)
        X = np.zeros((8, c.n_unknowns), dtype=np.complex128)
        swm.swm_solve(ctx, inc, 1e-8, RESTART, 2000, X)
        train.append((ctx, inc, X))
    net = swm.swm_net_create(0)
    swm.swm_net_set_params(net, init_params(0))
    t0 = time.perf_counter()
    losses = []
    for it in range(args.train_steps):
        ctx, inc, X = train[it % len(train)]
        losses.append(swm.swm_net_train_step(net, ctx, inc, X, 3e-4)[0])
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    for ctx, _, _ in train:
        swm.swm_destroy(ctx)
    cl = cloud_mid(seed=1)
    inc, obs = incidences_single_minus_z(), observations_phi_cut(N_OBS)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)]
    sig = torch.zeros((1, N_OBS, 2), dtype=torch.float64, device="cuda")
    x0 = torch.zeros((1, cl.n_unknowns), dtype=torch.complex128, device="cuda")
    ctx = swm.swm_create(0)

    def step(warm):
        swm.swm_set_cloud(ctx, *dev)
        swm.swm_build(ctx, K0, R_C, swm.SWM_C64)
        if warm:
            swm.swm_net_predict(net, ctx, inc, x0)
            swm.swm_solve_guess(ctx, inc, x0, TOL, RESTART, 1000)
        else:
            swm.swm_solve(ctx, inc, TOL, RESTART, 1000)
        swm.swm_rcs_bistatic(ctx, obs, sig)

    res = {}
    for warm in (False, True):
        for _ in range(3):
            step(warm)
        torch.cuda.synchronize()
        evs = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            step(warm)
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
        st = swm.swm_get_stats(ctx)
        res["warm" if warm else "cold"] = {"ms_per_step": ms, "value": cl.n_unknowns / (ms * 1e-3),
                                           "iterations": st["iterations"], "ms_solve": st["ms_solve"],
                                           "rcs": sig.cpu().numpy()[0, :, 0].copy()}
    # quality of the initial guess on this (unseen) cloud, against its converged currents
    X = torch.zeros((1, cl.n_unknowns), dtype=torch.complex128, device="cuda")
    swm.swm_set_cloud(ctx, *dev)
    swm.swm_build(ctx, K0, R_C, swm.SWM_C64)
    swm.swm_solve(ctx, inc, 1e-8, RESTART, 2000, X)
    loss_net = swm.swm_net_train_step(net, ctx, inc, X, 0.0)[0]
    swm.swm_net_set_params(net, init_params(0) * 0)
    loss_iso = swm.swm_net_train_step(net, ctx, inc, X, 0.0)[0]
    out = {"kind": "warm_start", "workload": "mid (10,000 wires), 1 incidence, 720-angle RCS",
           "train": {"clouds": args.train_clouds, "incidences_each": 8, "steps": args.train_steps, "seconds": train_s,
                     "loss_first_100": float(np.mean(losses[:100])), "loss_last_100": float(np.mean(losses[-100:]))},
           "initial_guess_rel_sq_error": {"isolated_wires": loss_iso, "network": loss_net},
           "rcs_err_db_warm_vs_cold": rcs_db_error(res["warm"]["rcs"], res["cold"]["rcs"]),
           "cold": {k: v for k, v in res["cold"].items() if k != "rcs"},
           "warm": {k: v for k, v in res["warm"].items() if k != "rcs"}}
    print(json.dumps(out))
    swm.swm_net_destroy(net)
    swm.swm_destroy(ctx)


def run_batch(args):
    """The batching workload: 64 cloud snapshots of 2,000-50,000 wires (log-uniform sizes, 0.005
    wires per cubic wavelength), each solved for 181 monostatic incidences (complex64, GMRES to 1e-6)
    with its monostatic RCS.  Snapshots run concurrently on --streams contexts, each on its own CUDA
    stream and host thread.  Prints a JSON line of kind "batch" (a measurement record)."""
    import threading

    import torch

    from paper_2410_03060_gb300 import swm
    from synth import batching_sizes

    torch.cuda.set_device(0)
    n_snap = args.snapshots
    sizes = batching_sizes(n_snap)
    clouds = [cloud_batching_snapshot(i) for i in range(n_snap)]
    n_inc = args.inc or 181
    inc = incidences_monostatic(n_inc)
    dev = [[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (c.centres, c.dirs, c.lengths, c.radii, c.nseg)]
           for c in clouds]
    n_str = max(1, args.streams)
    streams = [torch.cuda.Stream() for _ in range(n_str)]
    ctxs = [swm.swm_create(0, stream=s.cuda_stream) for s in streams]
    monos = [torch.zeros((n_inc, 2), dtype=torch.float64, device="cuda") for _ in range(n_str)]
    its = [0] * n_snap

    def worker(w, order):
        with torch.cuda.stream(streams[w]):
            for i in order:
                ctx = ctxs[w]
                swm.swm_set_cloud(ctx, *dev[i])
                swm.swm_build(ctx, K0, R_C, swm.SWM_C64)
                swm.swm_solve(ctx, inc, TOL, args.restart, 2000)
                swm.swm_rcs_monostatic(ctx, monos[w])
                its[i] = swm.swm_get_stats(ctx)["iterations"]

    # largest snapshots first, dealt round-robin to the streams
    order = list(np.argsort(-sizes))
    plan = [order[w::n_str] for w in range(n_str)]

    def run_all():
        th = [threading.Thread(target=worker, args=(w, plan[w])) for w in range(n_str)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        torch.cuda.synchronize()

    run_all()  # warm-up (allocations, the step kernel's block size per shape)
    ts = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        run_all()
        ts.append(time.perf_counter() - t0)
    units = float(sum(c.n_unknowns for c in clouds)) * n_inc
    sec = float(np.median(ts))
    print(json.dumps({"kind": "batch", "snapshots": n_snap, "wires": int(sum(c.nw for c in clouds)),
                      "unknowns": int(sum(c.n_unknowns for c in clouds)), "incidences_each": n_inc,
                      "streams": n_str, "restart": args.restart, "seconds_per_batch": sec,
                      "value": units / sec, "unit": UNIT, "iterations_min_max": [int(min(its)), int(max(its))],
                      "step_rhs_block_last": [swm.swm_get_stats(c)["step_rhs_block"] for c in ctxs]}))
    for c in ctxs:
        swm.swm_destroy(c)


def run_block(args):
    """Block GMRES against independent GMRES on batching snapshots: per snapshot, the library's
    swm_solve (independent GMRES per incidence, the incidences sharing every read of E) and the
    block GMRES of paper_2410_03060_gb300.dist (one Krylov space per group of up to --block-size
    incidences, its vector algebra in the library's kernels, its small dense algebra on the host),
    both complex128 to 1e-6.  Prints a JSON line of kind "block_gmres" (a measurement record)."""
    import torch

    from paper_2410_03060_gb300 import dist, swm

    torch.cuda.set_device(0)
    n_inc = args.inc or 181
    inc = incidences_monostatic(n_inc)
    rows = []
    for i in range(args.snapshots):
        cl = cloud_batching_snapshot(i)
        ctx = swm.swm_create(0)
        swm.swm_set_cloud(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)
        swm.swm_build(ctx, K0, R_C, swm.SWM_C128)
        swm.swm_solve(ctx, inc, TOL, args.restart, 2000)
        torch.cuda.synchronize()
        t = time.perf_counter()
        swm.swm_solve(ctx, inc, TOL, args.restart, 2000)
        torch.cuda.synchronize()
        t_ind = time.perf_counter() - t
        it_ind = swm.swm_get_stats(ctx)["iterations"]
        owner = np.zeros(cl.nw, dtype=np.int64)
        plan = dist.Plan(cl.centres, cl.nseg, owner, 0, R_C)
        its, t_blk = [], 0.0
        for g0 in range(0, n_inc, args.block_size):
            sub = inc[g0:g0 + args.block_size]
            ops = dist.SwmOps(ctx, plan, sub.shape[0])
            b = dist.gather_rhs_own(ops, sub)
            torch.cuda.synchronize()
            t = time.perf_counter()
            y, it, rel = dist.dist_block_gmres(ops, dist.LocalComm(), plan, b, TOL, args.block_restart, 2000)
            torch.cuda.synchronize()
            t_blk += time.perf_counter() - t
            its.append(int(it))
        swm.swm_destroy(ctx)
        rows.append({"snapshot": i, "nw": cl.nw, "unknowns": cl.n_unknowns, "independent_iterations": it_ind,
                     "independent_ms": 1e3 * t_ind, "block_iterations": its, "block_ms": 1e3 * t_blk})
    print(json.dumps({"kind": "block_gmres", "incidences": n_inc, "block_size": args.block_size,
                      "block_restart": args.block_restart, "restart": args.restart, "tol": TOL, "precision": "c128",
                      "snapshots": rows}))


# ---------------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The reference arm: the FP64 CPU oracle (the paper has no code) on the host cores, on a bounded
    sample of the same workload, same metric and unit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.workload if args.workload in WORKLOADS else "learned"
    cores = host_cores()
    # sample size keeps the whole run within a few minutes: about 20 ms of oracle time per wire and
    # core-second, (steps + warmup) oracle steps
    per_step_s = 150.0 / (args.steps + args.warmup)
    n_wires = int(min(30000, max(200, per_step_s * cores / 0.02)))
    cb = cpu_oracle_sample(name, n_wires, cores, steps=args.steps, warmup=args.warmup, solver=args.solver)
    v = cb["value"]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": cb["seconds_per_step"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded wire clouds)",
        "config": {"workload": workload_text(name, args.solver, args.restart) + " (bounded sample, see cpu_baseline.sample)"},
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["c64", "c128"], default="c64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(set(WORKLOADS) | set(SCALE)), default="learned",
                    help="learned (the headline) or mid; precision and batching0 print scale records")
    ap.add_argument("--no-mid", action="store_true", help="skip the 10,000-wire side measurement")
    ap.add_argument("--inc", type=int, default=0, help="incidences of a larger workload (default: its own)")
    ap.add_argument("--restart", type=int, default=RESTART)
    ap.add_argument("--solver", choices=["gmres", "bicgstab"], default="bicgstab",
                    help="Krylov method of the solve (GMRES(restart) or BiCGSTAB)")
    ap.add_argument("--nw", type=int, default=0, help="wire count of a larger workload (default: its own)")
    ap.add_argument("--same-density", action="store_true",
                    help="with --nw on the learned workload: scale the cluster width to keep the wire density")
    ap.add_argument("--batch", action="store_true",
                    help="the 64-snapshot batching workload, snapshots spread over --streams contexts")
    ap.add_argument("--snapshots", type=int, default=64)
    ap.add_argument("--block", action="store_true",
                    help="with --batch: block GMRES against independent GMRES on the first --snapshots snapshots")
    ap.add_argument("--block-size", type=int, default=32)
    ap.add_argument("--block-restart", type=int, default=10)
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--warm-start", action="store_true",
                    help="mid workload with and without the learned warm start (trains the network first)")
    ap.add_argument("--train-clouds", type=int, default=4)
    ap.add_argument("--train-steps", type=int, default=1500)
    ap.add_argument("--compare-precisions", action="store_true",
                    help="larger workload: time the float64, complex64 and bfloat16-refinement paths")
    ap.add_argument("--scale", action="store_true",
                    help="print a scale record (kernel classes, rooflines) of a larger workload")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if (args.scale or args.compare_precisions or args.workload not in WORKLOADS) and args.impl == "ours":
        if args.compare_precisions:
            run_compare(args)
        else:
            run_scale(args)
        return
    if args.batch and args.block and args.impl == "ours":
        run_block(args)
        return
    if args.batch and args.impl == "ours":
        run_batch(args)
        return
    if args.warm_start and args.impl == "ours":
        run_warm(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
