#!/usr/bin/env python
"""Throughput of the sparsified thin-wire MoM hot path on GB300: unknowns x incidences solved per
second, RCS checked against the plain FP64 path.

One step = the whole hot path on one cloud: load the wire cloud, S-NFC neighbour search, block
fill, block-Jacobi preconditioner, right-hand side, GMRES(50) to 1e-6, and the 720-angle bistatic
RCS.  Workload: 10,000 wires (lengths U[0.3, 0.6] wavelengths, <= 0.08-wavelength segments,
radius 1e-3, Gaussian centres sigma = 30 wavelengths, random directions), r_c = 3 wavelengths, one
plane wave arriving from +z, theta-polarised.  Inputs are seeded and synthetic.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own cloud (seed 1 + rank): weak scaling, no data-path
collective; the timing is the max over ranks.  ``--impl reference`` times the FP64 CPU oracle.
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


def slab_sample(cloud, n_target):
    """The wires of the centre slab |x| < w holding about n_target wires (local density kept)."""
    x = np.abs(cloud.centres[:, 0])
    w = np.sort(x)[min(len(x) - 1, n_target)]
    return cloud.subset(np.nonzero(x < w)[0])


def oracle_step(cloud, inc, obs):
    """The whole path on the FP64 CPU oracle (test infrastructure, timed as the CPU baseline)."""
    import oracle as O

    Z = O.assemble(cloud, K0, R_C, sparse=True)
    Mi = O.block_jacobi(cloud, K0)
    m, off = O.numbering(cloud.nseg)
    b = O.rhs(cloud, K0, inc)
    X = np.zeros_like(b)
    for i in range(b.shape[1]):
        X[:, i], _, _ = O.gmres(Z, b[:, i], Mi, off, TOL, RESTART, 1000)
    return O.rcs_bistatic(cloud, K0, X, obs)


def cpu_baseline(n_wires=1000):
    cl = slab_sample(cloud_mid(), n_wires)
    inc, obs = incidences_single_minus_z(), observations_phi_cut(N_OBS)
    t = time.perf_counter()
    oracle_step(cl, inc, obs)
    dt = time.perf_counter() - t
    return {"value": cl.n_unknowns * inc.shape[0] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"centre slab of the 10,000-wire cloud: {cl.nw} wires, N={cl.n_unknowns}, full path "
                      f"(pairs, fill, block-Jacobi, RHS, GMRES(50) 1e-6, 720-angle RCS) in {dt:.1f} s; "
                      f"single-threaded NumPy"}


# dram__bytes_read.sum + dram__bytes_write.sum per launch, mid workload, from one ncu capture of
# the kernel's current code (profiles/gmres_persist_mid.md)
MEASURED_TRAFFIC = {("gmres", "c64"): 6.392e6}


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
def kernel_roofline(cls, st, prof_ms, launches, prec, n_rhs, pk, clocks):
    """Achieved algorithmic rate of one kernel class over the timed region."""
    esz = 16 if prec == "c128" else 8
    N, nw = st["n"], st["nw"]
    if prof_ms <= 0 or launches <= 0:
        return None
    per_launch_ms = prof_ms / launches
    if cls == "apply":
        # per Arnoldi step: E values + column map + x, y and V rows + row metadata, plus the V rows
        # read by the fused first Gram-Schmidt pass; per restart: the residual product (+ b)
        mat = st["nnz_offd"] * esz + st["ncm_offd"] * 4 + 4 * N + 28 * nw
        vec = N * esz * n_rhs
        per_solve = sum(mat + 3 * vec + (j + 1) * vec for j in st["_steps"]) + (st["restarts"] + 1) * (mat + 3 * vec)
        work = per_solve * st["_cycles_mult"]
        return {"bound": "hbm", "achieved": work / (prof_ms * 1e-3) / 1e9, "peak": pk.get("hbm_gbs", 6800.0),
                "unit": "GB/s", "per_launch_bytes": work / launches, "per_launch_ms": per_launch_ms}
    if cls == "gmres":
        # the persistent solve, one launch per solve.  Per Arnoldi step j: E values + column map +
        # row descriptors and the gathered vector u, then the delayed Gram-Schmidt: dots over
        # V_0..V_{j-1}, u, w and the update reading them and writing V_j and the next u; the closing
        # pass of a cycle reads V_0..V_{j-1} and u; per restart cycle: the residual product and the
        # update of y by the basis; once: b formed from the wire geometry (centre, direction, length,
        # segment count) and written, and x = M^-1 y (the inverse blocks, y read, x written).
        mat = st["nnz_offd"] * esz + st["ncm_offd"] * 4 + 16 * N
        vec = N * esz * n_rhs
        per_solve = sum(mat + vec + (2 * j + 6) * vec for j in st["_steps"])
        per_solve += sum((c + 1) * vec for c in st["_cycle_len"])
        per_solve += (st["restarts"] + 1) * (mat + 3 * vec) + sum(st["_cycle_len"]) * vec
        per_solve += nw * (7 * 8 + 4) + vec + st["nminv"] * esz + 2 * vec
        work = per_solve * st["_cycles_mult"]
        return {"bound": "hbm", "achieved": work / (prof_ms * 1e-3) / 1e9, "peak": pk.get("hbm_gbs", 6800.0),
                "unit": "GB/s", "per_launch_bytes": work / launches, "per_launch_ms": per_launch_ms,
                "note": "latency-bound at this size (E and the basis stay on chip or in L2)"}
    if cls in ("dots", "update", "finish"):
        vec = N * esz * n_rhs
        work = sum((j + 1) * vec + 2 * vec for j in st["_steps"]) * st["_cycles_mult"]
        return {"bound": "hbm", "achieved": work / (prof_ms * 1e-3) / 1e9, "peak": pk.get("hbm_gbs", 6800.0),
                "unit": "GB/s", "per_launch_bytes": work / max(1, len(st["_steps"])), "per_launch_ms": per_launch_ms}
    if cls == "fill_mutual":
        flops = st["fill_evals"] * FP32_FLOPS_PER_EVAL
        mhz = pk.get("sm_max_mhz", 2070.0)
        peak = N_SM * 128 * 2 * mhz * 1e6 / 1e12 if prec == "c64" else 1.25
        return {"bound": "alu", "achieved": flops / (per_launch_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "per_launch_flops": flops, "per_launch_ms": per_launch_ms,
                "note": ("FP32 peak = 152 SMs x 128 lanes x 2 flops x max SM clock" if prec == "c64"
                         else "nominal FP64 peak")}
    return {"bound": "other", "per_launch_ms": per_launch_ms}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2410_03060_gb300 import swm

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec_id = swm.SWM_C64 if args.precision == "c64" else swm.SWM_C128
    cl = cloud_mid(seed=rank_seed(rank))
    inc, obs = incidences_single_minus_z(), observations_phi_cut(N_OBS)
    N = cl.n_unknowns
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
           (cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)]
    sigma = torch.zeros((1, N_OBS, 2), dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    ctx = swm.swm_create(local)

    def step(prec=prec_id, inputs=dev, out=sigma):
        # set_cloud, build, solve and the bistatic RCS in one C-ABI call (swm_run)
        swm.swm_run(ctx, *inputs, K0, R_C, prec, inc, obs, out, TOL, RESTART, 1000)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st0 = swm.swm_get_stats(ctx)
    # accuracy gate against the plain FP64 path (untimed)
    s_fast = sigma.cpu().numpy()[0, :, 0].copy()
    sig64 = torch.zeros_like(sigma)
    step(prec=swm.SWM_C128, out=sig64)
    torch.cuda.synchronize()
    err_db = rcs_db_error(s_fast, sig64.cpu().numpy()[0, :, 0])

    # dominant kernel class: one profiled step per class (untimed)
    classes = ["pairs", "fill_self", "fill_mutual", "invert", "form_e", "rhs", "apply", "update", "finish", "far",
               "gmres"]
    share = {}
    for c in classes:
        swm.swm_profile(ctx, c)
        step()
        torch.cuda.synchronize()
        share[c] = swm.swm_get_stats(ctx)["prof_ms"]
    dominant = max(share, key=share.get)
    swm.swm_profile(ctx, dominant)

    # timed region
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = swm.swm_get_stats(ctx)["kernel_launches"]
    clocks = ClockSampler(local)
    clocks.start()
    clocks.mark()
    evs = []
    for _ in range(args.steps):
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
    ms = [a.elapsed_time(b) for a, b in evs]
    st = swm.swm_get_stats(ctx)
    launches = (st["kernel_launches"] - l0) // max(1, args.steps)
    ms_step = float(np.mean(ms))
    prof_ms, prof_n = st["prof_ms"], st["prof_launches"]
    swm.swm_profile(ctx, "none")

    # e2e through the public API with pinned host buffers (copies inside the timed region)
    host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in
               (cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)]
    sig_host = torch.zeros((1, N_OBS, 2), dtype=torch.float64).pin_memory().numpy()
    e2e_steps = max(1, min(args.steps, 50))
    e2e = []
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        step(inputs=host_in, out=sig_host)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t)
    e2e_ms = 1e3 * float(np.mean(e2e))
    h2d = int(sum(a.nbytes for a in host_in))
    d2h = int(sig_host.nbytes)

    # plain FP64 path on the same GPU
    f64 = []
    for _ in range(max(1, min(args.steps, 20))):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step(prec=swm.SWM_C128, out=sig64)
        b.record()
        f64.append((a, b))
    torch.cuda.synchronize()
    ms64 = float(np.mean([a.elapsed_time(b) for a, b in f64]))
    swm.swm_destroy(ctx)

    # max over ranks, units over all ranks
    (ms_step, e2e_ms, ms64), total_units = aggregate_over_ranks([ms_step, e2e_ms, ms64], N * inc.shape[0],
                                                                "cuda", world)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    pk = peaks()
    # reconstruct the Arnoldi step indices of one solve for the Gram-Schmidt byte counts
    it = st["iterations"]
    steps_j, cycle_len = [], []
    while it > 0:
        c = min(RESTART, it)
        steps_j += list(range(c))
        cycle_len.append(c)
        it -= c
    st["_steps"] = steps_j
    st["_cycle_len"] = cycle_len
    st["_cycles_mult"] = args.steps
    roof = kernel_roofline(dominant, st, prof_ms, prof_n, args.precision, 1, pk, clk)
    if roof and roof.get("peak"):
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["peak_source"] = "of measured (MEASURED_PEAKS.json)" if roof["unit"] == "GB/s" else roof.get("note")
    if roof is not None:
        # DRAM bytes per launch from one ncu capture of this kernel at this workload
        # (profiles/gmres_persist_mid.md); null for a kernel without a capture of its current code
        roof["traffic"] = MEASURED_TRAFFIC.get((dominant, args.precision))
        roof["kernel"] = dominant
    out = {
        "metric": METRIC, "value": total_units / (ms_step * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64" if args.precision == "c64" else "c128",
        "data": "synthetic (seeded wire clouds)",
        "config": {"workload": "mid: 10,000 wires, Gaussian sigma 30, r_c 3, GMRES(50) 1e-6, 1 incidence, "
                               "720-angle bistatic RCS", "nw": cl.nw, "unknowns": N, "blocks": st["nb"],
                   "precision": args.precision, "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"{world} independent clouds (one per GPU)"},
        "gpu_launches": int(launches),
        "e2e": {"value": total_units / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "rcs_err_db_vs_fp64": err_db,
        "fp64_path": {"value": total_units / (ms64 * 1e-3), "ms_per_step": ms64,
                      "speedup_of_value": ms64 / ms_step},
        "iterations": st["iterations"],
        "phase_ms": {k: st[k] for k in ("ms_neighbour", "ms_fill", "ms_precond", "ms_rhs", "ms_solve", "ms_rcs")},
        "kernel_share_ms_per_step": share,
        "roofline": roof,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
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
    cl = w["cloud"](nw=args.nw) if args.nw else w["cloud"]()
    n_inc = args.inc or w["n_inc"]
    inc = incidences_monostatic(n_inc)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)]
    mono = torch.zeros((n_inc, 2), dtype=torch.float64, device="cuda")
    ctx = swm.swm_create(0)
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
    for cls in ("fill_mutual", "apply", "dots", "update", "finish", "far", "pairs", "fill_self"):
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
    mhz = pk.get("sm_max_mhz", 2070.0)
    fp32_peak = N_SM * 128 * 2 * mhz * 1e6 / 1e12
    fill_ms, _ = res["fill_mutual"]
    fill_tf = st["fill_evals"] * FP32_FLOPS_PER_EVAL / (fill_ms * 1e-3) / 1e12
    # block-sparse product: E (+ column map, row descriptors) once per block of right-hand sides
    # sharing a read, u read and w written per right-hand side; a transpose to incidence-minor
    # order is implementation traffic, not counted
    esz, N, R = 8, st["n"], n_inc
    it = st["iterations"]
    steps_j, closing_j = [], []
    while it > 0:
        c = min(restart, it)
        steps_j += list(range(c))
        closing_j.append(c)
        it -= c
    rbs = st["step_rhs_block"]
    rb = (32 if R >= 24 else 16) if rbs == 32 else max(1, rbs)
    nblk = -(-R // rb) if R > 1 else 1
    mat = (st["nnz_offd"] * esz + st["ncm_offd"] * 4 + 16 * N) * nblk
    apply_bytes = sum(mat + 2 * R * N * esz for _ in steps_j)
    apply_ms, apply_n = res["apply"]
    # the residual products of the restarts are timed with the class too: count their bytes
    apply_bytes += (st["restarts"] + 1) * (st["nnz_offd"] * esz + st["ncm_offd"] * 4) * R
    gbs = apply_bytes / (apply_ms * 1e-3) / 1e9
    # delayed Gram-Schmidt: dots read Q_<j, u, w; update reads them and writes q_j, u; the closing
    # dots of a cycle read Q_<j and u
    gs_bytes = sum((2 * j + 6) * R * N * esz for j in steps_j) + sum((j + 1) * R * N * esz for j in closing_j)
    gs_ms = res["dots"][0] + res["update"][0]
    gs_gbs = gs_bytes / (gs_ms * 1e-3) / 1e9
    out = {
        "kind": "scale", "workload": args.workload, "description": w["text"], "nw": cl.nw, "unknowns": N,
        "blocks": st["nb"], "nnz": st["nnz"], "incidences": n_inc, "restart": restart, "iterations": st["iterations"],
        "converged": st["converged"], "rel_residual": st["rel_residual"], "rc": rc,
        "ms_per_step": 1e3 * float(np.median(ts)),
        "value": N * n_inc / float(np.median(ts)), "unit": UNIT,
        "phase_ms": {k: st[k] for k in ("ms_neighbour", "ms_fill", "ms_precond", "ms_rhs", "ms_solve", "ms_rcs")},
        "fill_roofline": {"bound": "alu", "kernel": "k_mutual_blocks<float>", "evals": st["fill_evals"],
                          "flops_per_eval": FP32_FLOPS_PER_EVAL, "ms": fill_ms, "achieved": fill_tf,
                          "peak": fp32_peak, "unit": "TFLOP/s", "frac": fill_tf / fp32_peak,
                          "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock"},
        "apply_roofline": {"bound": "hbm",
                           "kernel": "k_rhs_minor + k_spmv_t (block-sparse product, one lane per incidence)"
                           if rbs == 32 else "k_spmv (block-sparse product, %d incidences per read of E)" % rb,
                           "launches": apply_n, "ms": apply_ms, "bytes": apply_bytes, "achieved": gbs,
                           "peak": pk.get("hbm_gbs", 6800.0), "unit": "GB/s",
                           "frac": gbs / pk.get("hbm_gbs", 6800.0), "peak_source": "of measured (MEASURED_PEAKS.json)"},
        "gs_roofline": {"bound": "hbm", "kernel": "k_dots + k_update (delayed Gram-Schmidt)", "ms": gs_ms,
                        "bytes": gs_bytes, "achieved": gs_gbs, "peak": pk.get("hbm_gbs", 6800.0), "unit": "GB/s",
                        "frac": gs_gbs / pk.get("hbm_gbs", 6800.0),
                        "peak_source": "of measured (MEASURED_PEAKS.json)"},
        "step_rhs_block": rbs,
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


# ---------------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # sample size keeps the whole run within a few minutes (about 8 ms of oracle time per wire)
    n_wires = int(min(1000, max(100, 150.0 / ((args.steps + args.warmup) * 0.008))))
    cl = slab_sample(cloud_mid(), n_wires)
    inc, obs = incidences_single_minus_z(), observations_phi_cut(N_OBS)
    for _ in range(args.warmup):
        oracle_step(cl, inc, obs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(cl, inc, obs)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    v = cl.n_unknowns * inc.shape[0] / dt
    sample = (f"centre slab of the 10,000-wire cloud: {cl.nw} wires, N={cl.n_unknowns}; full path on the FP64 "
              f"NumPy oracle, single-threaded")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded wire clouds)",
        "config": {"workload": "mid (sampled): 10,000-wire cloud statistics, r_c 3, GMRES(50) 1e-6, 1 incidence, "
                               "720-angle bistatic RCS", "nw": cl.nw, "unknowns": cl.n_unknowns},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["c64", "c128"], default="c64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["mid"] + sorted(SCALE), default="mid")
    ap.add_argument("--inc", type=int, default=0, help="incidences of a larger workload (default: its own)")
    ap.add_argument("--restart", type=int, default=RESTART)
    ap.add_argument("--nw", type=int, default=0, help="wire count of a larger workload (default: its own)")
    ap.add_argument("--batch", action="store_true",
                    help="the 64-snapshot batching workload, snapshots spread over --streams contexts")
    ap.add_argument("--snapshots", type=int, default=64)
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--warm-start", action="store_true",
                    help="mid workload with and without the learned warm start (trains the network first)")
    ap.add_argument("--train-clouds", type=int, default=4)
    ap.add_argument("--train-steps", type=int, default=1500)
    ap.add_argument("--compare-precisions", action="store_true",
                    help="larger workload: time the float64, complex64 and bfloat16-refinement paths")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.workload != "mid" and args.impl == "ours":
        if args.compare_precisions:
            run_compare(args)
        else:
            run_scale(args)
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
