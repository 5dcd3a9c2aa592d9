"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bars: S-NFC pattern bit-exact; FP64 blocks and right-hand sides to 1e-10 relative; FP64 currents
to 1e-5 relative; RCS within 0.1 dB.  The complex64 path (FP32 kernel evaluation): each block to
1e-6 of the scale of the two self blocks it couples and 1e-3 of its own largest entry, right-hand
sides to 2e-6, RCS within 0.1 dB.  (For well separated wires the scalar-potential term of a block
is a second difference of four segment integrals that cancels to about (D/R)^2 of each, so FP32
rounding of the kernel is amplified in the block's own relative error but not on the scale of Z.)
"""
import math

import numpy as np
import pytest

import oracle as O
from gpu_helpers import K, assert_rcs_db, block_errors, run_gpu
from synth import (CONFIGS, Cloud, cloud_mid, cloud_small, cloud_uniform_cube, incidences_single_minus_z,
                   observations_phi_cut)

pytestmark = pytest.mark.gpu

C128, C64 = 0, 1
BLOCK_TOL = {C128: 1e-10, C64: 1e-3}
BLOCK_TOL_SCALED = {C128: 1e-12, C64: 1e-6}


def _mixed_cloud(nw=48, side=2.5, seed=31):
    """Tight cloud with every segment count 2..16 and near-touching wires (8-point rule)."""
    rng = np.random.default_rng(seed)
    c = cloud_uniform_cube(nw, side, seed=seed)
    c.nseg = (2 + np.arange(nw) % 15).astype(np.int32)
    c.lengths = rng.uniform(0.2, 0.7, nw)
    c.radii = rng.uniform(5e-4, 2e-3, nw)
    # two almost touching wires
    c.centres[1] = c.centres[0] + 0.03 * np.cross(c.dirs[0], [0.0, 0.0, 1.0]) / max(
        1e-9, np.linalg.norm(np.cross(c.dirs[0], [0.0, 0.0, 1.0])))
    return c


def _ties_cloud():
    rng = np.random.default_rng(21)
    nw = 150
    c = np.round(rng.uniform(-3, 3, size=(nw, 3)) * 4) / 4
    d = rng.standard_normal((nw, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return Cloud(c, d, np.full(nw, 0.4), np.full(nw, 1e-3), np.full(nw, 5, np.int32), "ties")


# ------------------------------------------------------------------------------------- a1 pattern
@pytest.mark.parametrize("case", ["small", "ties", "mixed", "single"])
def test_pattern_bit_exact(case):
    if case == "small":
        cl, r_c = cloud_small(), 3.0
    elif case == "ties":
        cl, r_c = _ties_cloud(), 1.5
    elif case == "mixed":
        cl, r_c = _mixed_cloud(), 0.9
    else:
        cl, r_c = cloud_uniform_cube(1, 1.0, seed=1), 2.0
    out = run_gpu(cl, K, r_c, C128, np.array([[0.0, 0.0, 0.0]]))
    ref = O.neighbour_pairs(cl.centres, r_c)
    assert np.array_equal(out["pattern"], ref)


def test_dense_mode_keeps_every_pair():
    cl = cloud_uniform_cube(30, 40.0, seed=3)
    out = run_gpu(cl, K, 0.0, C128, np.array([[0.0, 0.0, 0.0]]))
    assert out["stats"]["nb"] == 30 * 30


# ------------------------------------------------------------------------------------- a2/a3 fill
@pytest.mark.parametrize("prec", [C128, C64])
def test_blocks_match_oracle(prec):
    cl = _mixed_cloud()
    out = run_gpu(cl, K, 0.9, prec, np.array([[0.3, 0.2, 0.1]]))
    pairs = out["pattern"]
    near = [(p, q) for p, q in pairs if p != q and O.mutual_order(cl, p, q) == O.NQ_NEAR]
    assert len(near) > 0
    err, where = block_errors(out["ctx"], cl, K, pairs)
    assert err < BLOCK_TOL[prec], (err, where)
    err, where = block_errors(out["ctx"], cl, K, pairs, scaled=True)
    assert err < BLOCK_TOL_SCALED[prec], (err, where)


@pytest.mark.parametrize("prec", [C128, C64])
def test_self_blocks_all_segment_counts(prec):
    cl = cloud_uniform_cube(15, 60.0, seed=4)
    cl.nseg = np.arange(2, 17, dtype=np.int32)
    out = run_gpu(cl, K, 0.5, prec, np.array([[0.0, 0.0, 0.0]]))
    assert len(out["pattern"]) == 15  # isolated wires
    assert block_errors(out["ctx"], cl, K, out["pattern"])[0] < BLOCK_TOL[prec]


# ------------------------------------------------------------------------------------- a4 rhs
@pytest.mark.parametrize("prec", [C128, C64])
def test_rhs_matches_oracle(prec):
    cl = _mixed_cloud(seed=5)
    rng = np.random.default_rng(0)
    inc = np.stack([rng.uniform(0, math.pi, 7), rng.uniform(0, 2 * math.pi, 7), rng.uniform(0, math.pi, 7)], 1)
    out = run_gpu(cl, K, 0.9, prec, inc)
    ref = O.rhs(cl, K, inc)
    tol = 1e-12 if prec == C128 else 2e-6
    assert np.max(np.abs(out["rhs"] - ref)) / np.max(np.abs(ref)) < tol


# ------------------------------------------------------------------------------------- a5-a7 solve + RCS
def test_currents_and_rcs_fp64_vs_oracle_lu():
    cl = cloud_uniform_cube(80, 5.0, seed=41)
    inc = np.array([[0.0, 0.0, 0.0], [1.1, 0.7, 0.5], [2.5, 4.0, 1.2]])
    obs = observations_phi_cut(90)
    for r_c in (1.5, 0.0):
        out = run_gpu(cl, K, r_c, C128, inc, obs=obs, tol=1e-12, mono=True)
        Z = O.assemble(cl, K, r_c if r_c > 0 else None, sparse=False)
        X = O.solve_lu(Z, O.rhs(cl, K, inc))
        rel = np.linalg.norm(out["currents"] - X) / np.linalg.norm(X)
        assert rel < 1e-5, rel
        assert out["rc"] == 0 and out["stats"]["converged"] == 1
        s_ref = O.rcs_bistatic(cl, K, X, obs)
        assert np.max(np.abs(out["sigma"] - s_ref)) / np.max(s_ref) < 1e-8
        assert np.allclose(out["sigma_mono"], O.rcs_monostatic(cl, K, X, inc), rtol=1e-7, atol=1e-12)


@pytest.mark.parametrize("mode", ["dense", "sparse"])
def test_small_config_fp64_and_c64(mode):
    """The small workload (200 wires, N = 1400) in both precisions against the oracle."""
    cfg = CONFIGS["small"]
    cl = cloud_small()
    r_c = cfg["r_c"] if mode == "sparse" else 0.0
    inc, obs = cfg["inc"](), cfg["obs"]()
    Z = O.assemble(cl, K, r_c if mode == "sparse" else None, sparse=False)
    X = O.solve_lu(Z, O.rhs(cl, K, inc))
    s_ref = O.rcs_bistatic(cl, K, X, obs)[0, :, 0]
    g64 = run_gpu(cl, K, r_c, C128, inc, obs=obs, tol=1e-11)
    assert np.linalg.norm(g64["currents"] - X) / np.linalg.norm(X) < 1e-5
    assert_rcs_db(g64["sigma"][0, :, 0], s_ref, db=1e-4)
    g32 = run_gpu(cl, K, r_c, C64, inc, obs=obs, tol=1e-6)
    assert np.linalg.norm(g32["currents"] - X) / np.linalg.norm(X) < 1e-4
    assert_rcs_db(g32["sigma"][0, :, 0], s_ref, db=0.1)


def test_far_field_stateless_matches_oracle():
    import torch
    from paper_2410_03060_gb300 import swm

    cl = _mixed_cloud(seed=9)
    m, off = O.numbering(cl.nseg)
    rng = np.random.default_rng(2)
    cur = rng.standard_normal((3, off[-1])) + 1j * rng.standard_normal((3, off[-1]))
    obs = np.stack([rng.uniform(0, math.pi, 33), rng.uniform(0, 2 * math.pi, 33)], 1)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sig = torch.zeros((3, 33, 2), dtype=torch.float64, device="cuda")
    swm.swm_far_field(None, t(cl.centres), t(cl.dirs), t(cl.lengths), t(cl.nseg), t(off), K, t(cur), t(obs), sig)
    torch.cuda.synchronize()
    ref = np.transpose(O.rcs_from_far_field(O.far_field(cl, K, cur.T, _rhat(obs)), obs), (2, 0, 1))
    assert np.max(np.abs(sig.cpu().numpy() - ref)) / np.max(ref) < 1e-10


def test_far_field_stateless_refuses_host_memory():
    """The stateless far field takes device pointers only: the binding refuses host arrays, and the
    C entry point itself returns SWM_EINVAL when one of its pointers is host memory."""
    import ctypes as C

    import torch
    from paper_2410_03060_gb300 import swm

    cl = _mixed_cloud(seed=9)
    m, off = O.numbering(cl.nseg)
    cur = np.ones((1, off[-1]), dtype=np.complex128)
    obs = np.array([[0.3, 0.2]])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sig = torch.zeros((1, 1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        swm.swm_far_field(None, t(cl.centres), t(cl.dirs), t(cl.lengths), t(cl.nseg), t(off), K, cur, t(obs), sig)
    dev = [t(cl.centres), t(cl.dirs), t(cl.lengths), t(cl.nseg), t(off), t(cur), t(obs)]
    host_obs = np.ascontiguousarray(obs)
    lib = swm.load()
    for entry in ("swm_far_field", "swm_far_field_noalloc"):
        rc = getattr(lib, entry)(C.c_void_p(torch.cuda.current_stream().cuda_stream), cl.nw,
                                 *[C.c_void_p(a.data_ptr()) for a in dev[:5]], float(K), 1,
                                 C.c_void_p(dev[5].data_ptr()), 1, host_obs.ctypes.data_as(C.c_void_p),
                                 C.c_void_p(sig.data_ptr()))
        assert rc == swm.SWM_EINVAL
        assert "device memory" in lib.swm_stateless_error().decode()


def test_c64_far_field_many_chunks_matches_oracle():
    """The float32 far field where each pair's wire range is cut into more than 256 chunks (its
    reduction then takes several batches per lane): bistatic and monostatic RCS of the solved
    complex64 currents against the oracle's far field of the same currents."""
    cl = cloud_uniform_cube(6000, 40.0, seed=77)
    inc = np.array([[0.3, 0.2, 0.0], [2.0, 4.5, 1.0]])
    obs = np.array([[0.4, 0.1], [1.0, 2.0], [1.6, 3.3], [2.2, 4.4], [3.0, 5.9]])
    out = run_gpu(cl, K, 1.0, C64, inc, obs=obs, tol=1e-4, mono=True)
    try:
        X = out["currents"]
        ref = O.rcs_bistatic(cl, K, X, obs)
        assert np.max(np.abs(out["sigma"] - ref)) / np.max(ref) < 1e-4
        ref_m = O.rcs_monostatic(cl, K, X, inc)
        assert np.max(np.abs(out["sigma_mono"] - ref_m)) / np.max(ref_m) < 1e-4
    finally:
        from paper_2410_03060_gb300 import swm
        swm.swm_destroy(out["ctx"])


def test_mid_workload_at_full_size_sampled_parity():
    """The benchmark's workload at full size (10,000 wires, 51,397 unknowns) in its configuration:
    device inputs through swm_run, complex64, r_c 3, GMRES(50) to 1e-6, 720 observations.  Checked
    against the oracle: the pattern bit for bit, the right-hand side, 40 sampled blocks, the
    residual b - Z x of the GPU currents on 60 sampled block-rows of the oracle's Z (below 1e-4: the
    GMRES tolerance 1e-6 plus the complex64 fill error, about 1e-5 here), the RCS against the
    oracle's far field of the same currents, and the RCS against the same cloud run on the
    float64 path within 0.1 dB (the method's accuracy criterion)."""
    import torch
    from paper_2410_03060_gb300 import swm

    cl = cloud_mid(seed=1)
    r_c = 3.0
    inc, obs = incidences_single_minus_z(), observations_phi_cut(720)
    m, off = O.numbering(cl.nseg)
    N = int(off[-1])
    pairs_ref = O.neighbour_pairs(cl.centres, r_c)
    b_ref = O.rhs(cl, K, inc)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
           (cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)]
    sig = torch.zeros((1, len(obs), 2), dtype=torch.float64, device="cuda")
    ctx = swm.swm_create(0)
    try:
        sig64 = torch.zeros_like(sig)
        assert swm.swm_run(ctx, *dev, K, r_c, C128, inc, obs, sig64, 1e-6, 50, 1000) == 0
        assert swm.swm_run(ctx, *dev, K, r_c, C64, inc, obs, sig, 1e-6, 50, 1000) == 0
        torch.cuda.synchronize()
        sigma = sig.cpu().numpy()
        assert_rcs_db(sigma[0, :, 0], sig64.cpu().numpy()[0, :, 0], db=0.1)
        assert np.array_equal(swm.swm_get_pattern(ctx), pairs_ref)
        b_gpu = swm.swm_get_rhs(ctx).T
        assert np.max(np.abs(b_gpu - b_ref)) / np.max(np.abs(b_ref)) < 2e-6
        rng = np.random.default_rng(8)
        sample = pairs_ref[rng.choice(len(pairs_ref), 40, replace=False)]
        err, where = block_errors(ctx, cl, K, sample, scaled=True)
        assert err < BLOCK_TOL_SCALED[C64], (err, where)
        # the currents of the same built system (the solve is deterministic)
        cur = np.zeros((1, N), dtype=np.complex128)
        assert swm.swm_solve(ctx, inc, 1e-6, 50, 1000, cur) == 0
        X = cur.T
    finally:
        swm.swm_destroy(ctx)
    wires = rng.choice(cl.nw, 60, replace=False)
    r2 = b2 = 0.0
    for p in wires:
        rows = slice(int(off[p]), int(off[p + 1]))
        acc = b_ref[rows, 0].copy()
        for q in pairs_ref[pairs_ref[:, 0] == p, 1]:
            acc -= O.block(cl, K, int(p), int(q)) @ X[int(off[q]):int(off[q + 1]), 0]
        r2 += float(np.sum(np.abs(acc) ** 2))
        b2 += float(np.sum(np.abs(b_ref[rows, 0]) ** 2))
    assert math.sqrt(r2 / b2) < 1e-4, math.sqrt(r2 / b2)
    s_ref = O.rcs_bistatic(cl, K, X, obs)
    assert np.max(np.abs(sigma - s_ref)) / np.max(s_ref) < 1e-4
    assert_rcs_db(sigma[0, :, 0], s_ref[0, :, 0], db=0.1)


def _rhat(obs):
    th, ph = obs[:, 0], obs[:, 1]
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)


# ------------------------------------------------------------------------------------- units
def test_scaled_currents_convert_to_amperes_and_ohms():
    """The ABI returns jt, the solution of the paper's system multiplied by j omega mu0 (Sec. II-A,
    Eq. TW_EFIE_MOM); its header states the physical current as I = jt / (j omega mu0) =
    -j jt / (k eta0) and Z_phys = j k eta0 Z.  Checked on the GPU's own outputs: (1) the GPU's
    self block of a half-wave dipole, so converted, gives an input impedance (delta gap at the
    centre vertex) in the textbook band for a = 1e-3 wavelength; (2) the power the converted
    currents take from a plane wave of 1 V/m, sigma_ext = eta0 Re(I^H b), equals the power they
    scatter, (1/4 pi) times the integral of the GPU's bistatic RCS over the sphere (optical
    theorem for a lossless conductor), on a small dense cloud."""
    import json
    import os
    from paper_2410_03060_gb300 import swm
    from synth import cloud_single

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook_values.json")))
    band = g["halfwave_dipole_input_impedance_thin_ohm"]["band_radius_1e-3"]
    dip = cloud_single(0.5, 16)
    out = run_gpu(dip, K, 3.0, C128, np.array([[math.pi / 2, 0.0, 0.0]]))
    try:
        Zs = swm.swm_get_block(out["ctx"], 0, 0, 15, 15)
    finally:
        swm.swm_destroy(out["ctx"])
    zin = 1j * K * O.ETA0 / np.linalg.inv(Zs)[7, 7]
    assert band["R"][0] <= zin.real <= band["R"][1] and band["X"][0] <= zin.imag <= band["X"][1], zin

    cl = cloud_uniform_cube(6, 1.2, seed=41, length=0.47, nseg=8)
    inc = np.array([[0.6, 0.3, 0.4]])
    nt, nph = 32, 64
    xg, wg = np.polynomial.legendre.leggauss(nt)
    th = np.arccos(xg)
    obs = np.array([[t, 2 * math.pi * j / nph] for t in th for j in range(nph)])
    out = run_gpu(cl, K, 0.0, C128, inc, obs=obs, tol=1e-12)
    try:
        I_amp = -1j * out["currents"][:, 0] / (K * O.ETA0)
        sig_ext = O.ETA0 * float(np.real(np.vdot(I_amp, out["rhs"][:, 0])))
        s = out["sigma"][0].sum(axis=1).reshape(nt, nph)
        sig_sca = float(np.sum(wg[:, None] * s) * (2 * math.pi / nph)) / (4 * math.pi)
    finally:
        swm.swm_destroy(out["ctx"])
    assert sig_ext > 0
    assert abs(sig_ext - sig_sca) / sig_sca < 1e-3, (sig_ext, sig_sca)


# ------------------------------------------------------------------------------------- edge cases
def test_edge_single_wire_and_two_segment_wires():
    cl = cloud_uniform_cube(1, 1.0, seed=2, nseg=2)
    out = run_gpu(cl, K, 3.0, C128, np.array([[0.4, 0.0, 0.0]]), tol=1e-12)
    X = O.solve_lu(O.assemble(cl, K, None, sparse=False), O.rhs(cl, K, np.array([[0.4, 0.0, 0.0]])))
    assert np.allclose(out["currents"], X, rtol=1e-9)
    cl = cloud_uniform_cube(40, 3.0, seed=3, nseg=2)
    out = run_gpu(cl, K, 1.0, C128, np.array([[0.4, 0.0, 0.0]]), tol=1e-12)
    X = O.solve_lu(O.assemble(cl, K, 1.0, sparse=False), O.rhs(cl, K, np.array([[0.4, 0.0, 0.0]])))
    assert np.linalg.norm(out["currents"] - X) / np.linalg.norm(X) < 1e-8


def test_edge_isolated_limit_converges_at_once():
    cl = cloud_uniform_cube(50, 50.0, seed=6)
    out = run_gpu(cl, K, 1e-3, C128, np.array([[0.0, 0.0, 0.0]]), tol=1e-10)
    assert out["stats"]["nb"] == 50 and out["stats"]["iterations"] <= 1
    X = O.solve_lu(O.assemble(cl, K, 1e-3, sparse=False), O.rhs(cl, K, np.array([[0.0, 0.0, 0.0]])))
    assert np.allclose(out["currents"], X, rtol=1e-9, atol=1e-15)


def test_edge_restart_one_and_max_iter():
    cl = cloud_uniform_cube(60, 4.0, seed=7)
    inc = np.array([[0.0, 0.0, 0.0]])
    X = O.solve_lu(O.assemble(cl, K, 2.0, sparse=False), O.rhs(cl, K, inc))
    out = run_gpu(cl, K, 2.0, C128, inc, tol=1e-10, restart=1)
    assert np.linalg.norm(out["currents"] - X) / np.linalg.norm(X) < 1e-6
    out = run_gpu(cl, K, 2.0, C128, inc, tol=1e-14, max_iter=2)
    assert out["rc"] == 1 and out["stats"]["iterations"] == 2 and out["stats"]["converged"] == 0


def test_device_inputs_equal_host_inputs():
    cl = _mixed_cloud(seed=12)
    a = run_gpu(cl, K, 0.9, C128, np.array([[0.2, 0.3, 0.0]]))
    b = run_gpu(cl, K, 0.9, C128, np.array([[0.2, 0.3, 0.0]]), device_inputs=True)
    assert np.array_equal(a["currents"], b["currents"])


def test_pinned_host_buffers_read_and_written_in_place():
    """Page-locked host inputs are read by the ingest kernel in place and a page-locked RCS buffer is
    written in place (no staging copies); results equal those of pageable and device buffers."""
    import torch

    from paper_2410_03060_gb300 import swm

    cl = _mixed_cloud(seed=13)
    inc, obs = np.array([[0.2, 0.1, 0.3]]), observations_phi_cut(16)
    ref = run_gpu(cl, K, 0.9, C64, inc, obs=obs, tol=1e-5)
    swm.swm_destroy(ref["ctx"])
    pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
           for a in (cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)]
    sig = torch.zeros((1, len(obs), 2), dtype=torch.float64).pin_memory().numpy()
    ctx = swm.swm_create(0)
    try:
        swm.swm_set_cloud(ctx, *pin)
        swm.swm_build(ctx, K, 0.9, C64)
        swm.swm_solve(ctx, inc, 1e-5, 50, 3000)
        swm.swm_rcs_bistatic(ctx, obs, sig)
        assert np.array_equal(sig, ref["sigma"])
        sig[:] = 0.0
        swm.swm_run(ctx, *pin, K, 0.9, C64, inc, obs, sig, tol=1e-5, max_iter=3000)
        assert np.array_equal(sig, ref["sigma"])
    finally:
        swm.swm_destroy(ctx)


@pytest.mark.parametrize("prec", [C128, C64])
def test_run_equals_separate_calls(prec):
    """swm_run (cloud, build, solve, bistatic RCS in one call, fewer host synchronisations) gives
    bit-identical RCS and the same statistics as the four calls made in turn, on the same context
    and on a fresh one; an invalid cloud is still rejected before any work."""
    from paper_2410_03060_gb300 import swm

    cl = _mixed_cloud(seed=14)
    inc = np.array([[0.3, 0.1, 0.2]])
    obs = observations_phi_cut(24)
    tol = 1e-8 if prec == C128 else 1e-5
    ref = run_gpu(cl, K, 0.9, prec, inc, obs=obs, tol=tol, max_iter=500)
    assert ref["rc"] == 0
    try:
        for ctx in (ref["ctx"], swm.swm_create(0)):
            sig = np.zeros((1, len(obs), 2))
            rc = swm.swm_run(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg, K, 0.9, prec, inc, obs, sig,
                             tol=tol, max_iter=500)
            st = swm.swm_get_stats(ctx)
            assert rc == ref["rc"]
            assert np.array_equal(sig, ref["sigma"])
            for key in ("n", "nb", "iterations", "restarts", "converged", "rel_residual", "fill_evals", "nminv"):
                assert st[key] == ref["stats"][key], key
            if ctx is not ref["ctx"]:
                swm.swm_destroy(ctx)
        # monostatic form (no observation list): the RCS of swm_rcs_monostatic after the same solve
        incm = np.array([[0.3, 0.1, 0.2], [1.2, 2.0, 0.0], [2.9, 4.0, 1.0]])
        refm = run_gpu(cl, K, 0.9, prec, incm, tol=tol, max_iter=500, mono=True)
        try:
            ctx = swm.swm_create(0)
            sm = np.zeros((3, 2))
            rc = swm.swm_run(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg, K, 0.9, prec, incm, None, sm,
                             tol=tol, max_iter=500)
            assert rc == refm["rc"] and np.array_equal(sm, refm["sigma_mono"])
            swm.swm_destroy(ctx)
        finally:
            swm.swm_destroy(refm["ctx"])
        ctx = swm.swm_create(0)
        bad = cl.dirs.copy()
        bad[3] *= 1.5
        with pytest.raises(swm.SwmError):
            swm.swm_run(ctx, cl.centres, bad, cl.lengths, cl.radii, cl.nseg, K, 0.9, prec, inc, obs,
                        np.zeros((1, len(obs), 2)))
        swm.swm_destroy(ctx)
    finally:
        swm.swm_destroy(ref["ctx"])


def test_profiled_classes_do_not_change_results():
    """Profiling a kernel class times its launches on the context's stream (the self blocks and
    their inverses then leave the build's second stream): every class gives currents bit-identical
    to an unprofiled run, and repeated builds on one context agree too."""
    from paper_2410_03060_gb300 import swm

    cl = _mixed_cloud(seed=16)
    inc = np.array([[0.1, 0.4, 0.0]])
    N = int(np.sum(cl.nseg.astype(np.int64) - 1))
    ctx = swm.swm_create(0)
    try:
        swm.swm_set_cloud(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)
        ref = None
        for cls in ("none", "fill_self", "invert", "fill_mutual", "form_e", "pairs", "rhs", "gmres", "none"):
            swm.swm_profile(ctx, cls)
            swm.swm_build(ctx, K, 0.9, C64)
            cur = np.zeros((1, N), dtype=np.complex128)
            swm.swm_solve(ctx, inc, 1e-5, 50, 500, cur)
            if ref is None:
                ref = cur.copy()
            assert np.array_equal(cur, ref), cls
        swm.swm_profile(ctx, "none")
    finally:
        swm.swm_destroy(ctx)


def test_invalid_inputs_rejected():
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(5, 2.0, seed=1)
    ctx = swm.swm_create(0)
    bad = cl.dirs.copy()
    bad[2] *= 1.01
    with pytest.raises(swm.SwmError) as e:
        swm.swm_set_cloud(ctx, cl.centres, bad, cl.lengths, cl.radii, cl.nseg)
    assert "unit" in str(e.value)
    ns = cl.nseg.copy()
    ns[0] = 17
    with pytest.raises(swm.SwmError):
        swm.swm_set_cloud(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, ns)
    with pytest.raises(swm.SwmError):
        swm.swm_build(ctx, K, 1.0, 0)  # no cloud loaded
    swm.swm_set_cloud(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)
    with pytest.raises(swm.SwmError):
        swm.swm_solve(ctx, [[0.0, 0.0, 0.0]])  # not built
    with pytest.raises(swm.SwmError):
        swm.swm_build(ctx, -1.0, 1.0, 0)
    swm.swm_build(ctx, K, 1.0, 0)
    with pytest.raises(swm.SwmError):
        swm.swm_solve(ctx, [[0.0, 0.0, 0.0]], restart=0)
    swm.swm_destroy(ctx)


def test_split_step_path_matches_oracle(monkeypatch):
    """The large-system form of the GMRES step (streaming product + separate dots), forced on a
    small system, against the oracle's LU solution, for one and for several incidences (with 12 or
    more, the product reads the vectors incidence-minor, one lane per incidence)."""
    monkeypatch.setenv("SWM_SPLIT_ROWS", "0")
    cl = cloud_uniform_cube(80, 5.0, seed=43)
    obs = observations_phi_cut(60)
    g = np.random.default_rng(7)
    many = lambda n: np.stack([g.uniform(0, np.pi, n), g.uniform(0, 2 * np.pi, n), g.uniform(0, np.pi, n)], 1)
    # 1 incidence; 9 (blocks of 8 share E); 13 and 30 (incidence-minor product, 16 and 32 lanes)
    for inc in (np.array([[0.2, 0.1, 0.0]]), np.array([[0.0, 0.0, 0.0], [1.1, 0.7, 0.5], [2.5, 4.0, 1.2]] * 3),
                many(13), many(30)):
        for prec, tol in ((C128, 1e-5), (C64, 1e-3)):
            out = run_gpu(cl, K, 1.5, prec, inc, obs=obs, tol=1e-11 if prec == C128 else 1e-6)
            X = O.solve_lu(O.assemble(cl, K, 1.5, sparse=False), O.rhs(cl, K, inc))
            assert np.linalg.norm(out["currents"] - X) / np.linalg.norm(X) < tol
            s_ref = O.rcs_bistatic(cl, K, X, obs)
            for i in range(inc.shape[0]):
                assert_rcs_db(out["sigma"][i, :, 0], s_ref[i, :, 0], db=0.1)


@pytest.mark.parametrize("form", [4, 8, 16, 32, 64, 65, 67, 68, 69, 70, 71, 72, 73, 74, 75])
def test_every_product_form_matches_oracle(monkeypatch, form):
    """Each form of the many-incidence product, forced (SWM_PRODUCT_FORM) on the large-system GMRES
    step: 4/8/16 incidences per read of E, 32 the incidence-minor form, 64 and 65 the wire-tiled
    form (65: five CTAs per SM; 67: two incidences per thread, E of the tile in shared memory;
    68 and 69: the same with packed FP32x2 arithmetic, E expanded in shared memory, three CTAs
    per SM with a 48 KB budget and two with 96 KB; 70 and 71: packed, E and the column map read
    from global memory, three and four CTAs per SM; 72 and 73: the same in small CTAs of a few
    whole warps; 74: small CTAs with E and the column map staged by cp.async; 75: 74 over the wires sorted
    by loop length within windows).
    Clouds with every segment count 2..16 (wires of up to 15 rows, two row groups in the
    wire-tiled form) and ragged tiles, one dense (a tile's E exceeds the shared-memory budget, so
    the forms that stage it read it from global memory) and one sparse (it fits); 37 and 70
    incidences (one group of 37, two groups of 35 in the wire-tiled form); currents against the
    oracle's LU solution and the RCS within 0.1 dB."""
    from paper_2410_03060_gb300 import swm

    monkeypatch.setenv("SWM_SPLIT_ROWS", "0")
    monkeypatch.setenv("SWM_PRODUCT_FORM", str(form))
    obs = observations_phi_cut(24)
    g = np.random.default_rng(8)
    many = lambda n: np.stack([g.uniform(0, np.pi, n), g.uniform(0, 2 * np.pi, n), g.uniform(0, np.pi, n)], 1)
    for cl, n_inc in ((_mixed_cloud(nw=61, side=3.0, seed=45), 37), (_mixed_cloud(nw=61, side=3.0, seed=45), 70),
                      (_mixed_cloud(nw=150, side=9.0, seed=46), 37)):
        inc = many(n_inc)
        Z = O.assemble(cl, K, 1.2, sparse=False)
        X = O.solve_lu(Z, O.rhs(cl, K, inc))
        s_ref = O.rcs_bistatic(cl, K, X, obs)
        for prec, tol in ((C128, 1e-5), (C64, 1e-3)):
            out = run_gpu(cl, K, 1.2, prec, inc, obs=obs, tol=1e-11 if prec == C128 else 1e-6)
            try:
                assert out["stats"]["step_rhs_block"] == form
                assert np.linalg.norm(out["currents"] - X) / np.linalg.norm(X) < tol
                for i in range(n_inc):
                    assert_rcs_db(out["sigma"][i, :, 0], s_ref[i, :, 0], db=0.1)
            finally:
                swm.swm_destroy(out["ctx"])


def test_per_kernel_step_path_matches_oracle(monkeypatch):
    """With the persistent solve turned off, small systems run one launch per kernel of each GMRES
    step (fused product and first dots, second pass, finish); same check as above."""
    monkeypatch.setenv("SWM_PERSIST", "0")
    cl = cloud_uniform_cube(80, 5.0, seed=44)
    obs = observations_phi_cut(60)
    g = np.random.default_rng(7)
    many = lambda n: np.stack([g.uniform(0, np.pi, n), g.uniform(0, 2 * np.pi, n), g.uniform(0, np.pi, n)], 1)
    # 1 incidence; 9 (blocks of 8 share E); 13 and 30 (incidence-minor product, 16 and 32 lanes)
    for inc in (np.array([[0.2, 0.1, 0.0]]), np.array([[0.0, 0.0, 0.0], [1.1, 0.7, 0.5], [2.5, 4.0, 1.2]] * 3),
                many(13), many(30)):
        for prec, tol in ((C128, 1e-5), (C64, 1e-3)):
            out = run_gpu(cl, K, 1.5, prec, inc, obs=obs, tol=1e-11 if prec == C128 else 1e-6)
            X = O.solve_lu(O.assemble(cl, K, 1.5, sparse=False), O.rhs(cl, K, inc))
            assert np.linalg.norm(out["currents"] - X) / np.linalg.norm(X) < tol
            s_ref = O.rcs_bistatic(cl, K, X, obs)
            for i in range(inc.shape[0]):
                assert_rcs_db(out["sigma"][i, :, 0], s_ref[i, :, 0], db=0.1)


@pytest.mark.parametrize("n_inc", [1, 2, 8])
def test_persistent_solve_matches_oracle_and_launches_once(n_inc):
    """The persistent cooperative solve (default for small systems with at most 8 incidences):
    currents against the oracle's LU solution, several restart cycles (restart 5), and a single
    GMRES launch per solve besides the final block-diagonal product."""
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(150, 6.0, seed=45)
    rng = np.random.default_rng(9)
    inc = np.stack([rng.uniform(0, np.pi, n_inc), rng.uniform(0, 2 * np.pi, n_inc), rng.uniform(0, np.pi, n_inc)], 1)
    X = O.solve_lu(O.assemble(cl, K, 2.0, sparse=False), O.rhs(cl, K, inc))
    for prec, tol in ((C128, 1e-6), (C64, 1e-3)):
        out = run_gpu(cl, K, 2.0, prec, inc, tol=1e-12 if prec == C128 else 1e-6, restart=5)
        try:
            st = out["stats"]
            assert st["converged"] == 1 and st["restarts"] >= 2
            assert np.linalg.norm(out["currents"] - X) / np.linalg.norm(X) < tol
            ctx = out["ctx"]
            cur = np.zeros((n_inc, X.shape[0]), dtype=np.complex128)
            l0 = swm.swm_get_stats(ctx)["kernel_launches"]
            swm.swm_profile(ctx, "gmres")
            swm.swm_solve(ctx, inc, 1e-12 if prec == C128 else 1e-6, 5, 3000, cur)
            st2 = swm.swm_get_stats(ctx)
            swm.swm_profile(ctx, "none")
            assert st2["prof_launches"] == 1
            assert st2["iterations"] == st["iterations"]
            assert np.array_equal(cur.T, out["currents"])  # deterministic
        finally:
            swm.swm_destroy(out["ctx"])


def test_persistent_barrier_wait_runs_out_and_reports_etimeout(monkeypatch):
    """Failure detection without a GPU fault: with the test hook every grid barrier of the
    persistent solve waits for one CTA that does not exist, so each wait runs out after its 1 s
    limit, every CTA returns, and the solve reports SWM_ETIMEOUT; the GPU and a new context then
    solve normally."""
    import time

    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(60, 4.0, seed=47)
    inc = np.array([[0.3, 0.1, 0.0]])
    monkeypatch.setenv("SWM_TEST_BARRIER_EXTRA", "1")
    ctx = swm.swm_create(0)
    try:
        swm.swm_set_cloud(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)
        swm.swm_build(ctx, K, 2.0, C64)
        t0 = time.perf_counter()
        with pytest.raises(swm.SwmError) as e:
            swm.swm_solve(ctx, inc, 1e-6, 20, 100)
        dt = time.perf_counter() - t0
        assert e.value.code == swm.SWM_ETIMEOUT and "timed out" in str(e.value)
        assert 0.9 < dt < 30.0
    finally:
        swm.swm_destroy(ctx)
    monkeypatch.delenv("SWM_TEST_BARRIER_EXTRA")
    out = run_gpu(cl, K, 2.0, C64, inc, tol=1e-6)
    try:
        assert out["rc"] == 0 and out["stats"]["converged"] == 1
    finally:
        swm.swm_destroy(out["ctx"])


def test_contexts_on_concurrent_host_threads(monkeypatch):
    """Contexts driven from several host threads at once (each on its own stream, with systems of
    different sizes, so their kernels ask for different amounts of shared memory) give the same
    currents as when run one after the other.  The product form is fixed (its timed choice could
    differ under the contention of concurrent runs, and two forms add in different orders)."""
    import threading

    import torch

    from paper_2410_03060_gb300 import swm

    monkeypatch.setenv("SWM_PRODUCT_FORM", "8")
    # up to 150k unknowns: the fused step kernel then asks for more than 48 KB of shared memory
    clouds = [cloud_uniform_cube(n, (n / 0.02) ** (1 / 3), seed=90 + i)
              for i, n in enumerate((30000, 26000, 12000, 3000))]
    inc = np.stack([np.linspace(0.1, 3.0, 9), np.linspace(0.0, 5.0, 9), np.zeros(9)], 1)

    def solve(cl, ctx, out):
        swm.swm_set_cloud(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)
        swm.swm_build(ctx, K, 2.0, C64)
        cur = np.zeros((inc.shape[0], cl.n_unknowns), dtype=np.complex128)
        swm.swm_solve(ctx, inc, 1e-6, 20, 500, cur)
        out.append(cur)

    seq = []
    for cl in clouds:
        ctx = swm.swm_create(0)
        try:
            solve(cl, ctx, seq)
        finally:
            swm.swm_destroy(ctx)
    streams = [torch.cuda.Stream() for _ in clouds]
    ctxs = [swm.swm_create(0, stream=s.cuda_stream) for s in streams]
    outs = [[] for _ in clouds]
    errors = []

    def work(i):
        try:
            with torch.cuda.stream(streams[i]):
                for _ in range(3):
                    solve(clouds[i], ctxs[i], outs[i])
        except Exception as e:  # reported below: a thread's exception does not reach pytest
            errors.append(repr(e))

    try:
        th = [threading.Thread(target=work, args=(i,)) for i in range(len(clouds))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        torch.cuda.synchronize()
        assert not errors, errors
        for i in range(len(clouds)):
            for cur in outs[i]:
                assert np.linalg.norm(cur - seq[i]) <= 1e-12 * np.linalg.norm(seq[i])
    finally:
        for c in ctxs:
            swm.swm_destroy(c)
