"""GPU tests of the paper's GCR solver and of frequency sweeps that keep the S-NFC pattern.

GCR (Sec. II-B, after Eq. neardef) is checked against the oracle's LU solution and against the
oracle's own GCR (same iteration count: both minimise the residual over the same Krylov space).
A frequency sweep rebuilds at a new k with the same r_c: the pattern is kept, the values are
refilled, and the result equals a fresh build at that k.
"""
import math

import numpy as np
import pytest

import oracle as O
from gpu_helpers import K, assert_rcs_db
from synth import cloud_uniform_cube, observations_phi_cut

pytestmark = pytest.mark.gpu

C128, C64 = 0, 1


def _solve(ctx, swm, cl, inc, tol, restart, max_iter=3000):
    cur = np.zeros((inc.shape[0], cl.n_unknowns), dtype=np.complex128)
    rc = swm.swm_solve(ctx, inc, tol, restart, max_iter, cur)
    return cur.T.copy(), rc, swm.swm_get_stats(ctx)


def _ctx(cl, k, r_c, prec, solver="gmres"):
    from paper_2410_03060_gb300 import swm

    ctx = swm.swm_create(0)
    swm.swm_set_solver(ctx, solver)
    swm.swm_set_cloud(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)
    swm.swm_build(ctx, k, r_c, prec)
    return ctx


def test_gcr_currents_and_rcs_match_oracle_lu():
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(120, 5.0, seed=61)
    inc = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 0.4], [2.2, 4.1, 1.3]])
    obs = observations_phi_cut(72)
    X = O.solve_lu(O.assemble(cl, K, 2.0, sparse=False), O.rhs(cl, K, inc))
    s_ref = O.rcs_bistatic(cl, K, X, obs)
    for prec, tol, bound in ((C128, 1e-11, 1e-8), (C64, 1e-6, 1e-3)):
        ctx = _ctx(cl, K, 2.0, prec, "gcr")
        try:
            cur, rc, st = _solve(ctx, swm, cl, inc, tol, restart=6)
            assert rc == 0 and st["converged"] == 1 and st["restarts"] >= 2
            assert np.linalg.norm(cur - X) / np.linalg.norm(X) < bound
            sig = np.zeros((inc.shape[0], len(obs), 2))
            swm.swm_rcs_bistatic(ctx, obs, sig)
            for i in range(inc.shape[0]):
                assert_rcs_db(sig[i, :, 0], s_ref[i, :, 0], db=0.1)
        finally:
            swm.swm_destroy(ctx)


def test_gcr_iterations_match_oracle_gcr_and_gmres():
    """Without restarts GCR and GMRES minimise the same residual, so they stop at the same step;
    the oracle's GCR stops there too."""
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(100, 5.0, seed=62)
    inc = np.array([[0.7, 0.3, 0.2]])
    tol = 1e-8
    Z = O.assemble(cl, K, 2.0, sparse=True)
    b = O.rhs(cl, K, inc)[:, 0]
    m, off = O.numbering(cl.nseg)
    _, it_ref, _ = O.gcr(Z, b, O.block_jacobi(cl, K), off, tol=tol, restart=100, max_iter=100)
    its = {}
    for solver in ("gcr", "gmres"):
        ctx = _ctx(cl, K, 2.0, C128, solver)
        try:
            _, rc, st = _solve(ctx, swm, cl, inc, tol, restart=100)
            assert rc == 0
            its[solver] = st["iterations"]
        finally:
            swm.swm_destroy(ctx)
    assert abs(its["gcr"] - it_ref) <= 1 and abs(its["gmres"] - it_ref) <= 1


def test_gcr_not_converged_and_bad_solver():
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(60, 4.0, seed=63)
    ctx = _ctx(cl, K, 2.0, C64, "gcr")
    try:
        _, rc, st = _solve(ctx, swm, cl, np.array([[0.1, 0.2, 0.0]]), 1e-12, restart=3, max_iter=4)
        assert rc == swm.SWM_ENOTCONV and st["iterations"] == 4 and st["converged"] == 0
        with pytest.raises(swm.SwmError):
            swm.swm_set_solver(ctx, 7)
    finally:
        swm.swm_destroy(ctx)


def test_frequency_sweep_keeps_pattern_and_equals_fresh_builds():
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(150, 6.0, seed=64)
    inc = np.array([[0.0, 0.0, 0.0], [1.2, 0.5, 0.0]])
    ks = [0.8 * K, 1.1 * K, 1.3 * K]
    sweep = _ctx(cl, ks[0], 2.5, C128)
    try:
        for i, k in enumerate(ks):
            if i:
                swm.swm_build(sweep, k, 2.5, C128)
            st = swm.swm_get_stats(sweep)
            assert st["pattern_reused"] == (1 if i else 0)
            cur, rc, _ = _solve(sweep, swm, cl, inc, 1e-11, restart=50)
            fresh = _ctx(cl, k, 2.5, C128)
            try:
                cur_f, _, st_f = _solve(fresh, swm, cl, inc, 1e-11, restart=50)
                assert st_f["pattern_reused"] == 0
                assert np.array_equal(cur, cur_f)
            finally:
                swm.swm_destroy(fresh)
            X = O.solve_lu(O.assemble(cl, k, 2.5, sparse=False), O.rhs(cl, k, inc))
            assert np.linalg.norm(cur - X) / np.linalg.norm(X) < 1e-8
        # a new r_c rebuilds the pattern
        swm.swm_build(sweep, ks[0], 3.5, C128)
        assert swm.swm_get_stats(sweep)["pattern_reused"] == 0
    finally:
        swm.swm_destroy(sweep)


def test_frequency_sweep_resonance_of_half_wave_wire():
    """Orientation-averaged backscatter of a thin wire of length L, swept in frequency on one
    pattern, peaks where the wire is about half a wavelength long (Sec. III-C: resonance at
    f1 = c / (2 L)); at the peak it matches the oracle."""
    from paper_2410_03060_gb300 import swm
    from synth import cloud_single

    L = 0.5
    cl = cloud_single(length=L, nseg=8)
    th = np.linspace(0.0, math.pi, 37)
    inc = np.stack([th, np.zeros_like(th), np.zeros_like(th)], 1)
    w = np.sin(th)  # solid-angle weight of the elevation samples (the wire lies along z)
    fs = np.linspace(0.8, 1.2, 9)  # frequency / f1, with c = 1 and f1 = 1 / (2 L)
    ctx = _ctx(cl, 2 * math.pi * fs[0] / (2 * L), 3.0, C64)
    mean = []
    try:
        for i, f in enumerate(fs):
            k = 2 * math.pi * f / (2 * L)
            if i:
                swm.swm_build(ctx, k, 3.0, C64)
                assert swm.swm_get_stats(ctx)["pattern_reused"] == 1
            swm.swm_solve(ctx, inc, 1e-7, 30, 1000)
            sm = np.zeros((inc.shape[0], 2))
            swm.swm_rcs_monostatic(ctx, sm)
            lam = 2 * L / f
            mean.append(float(np.sum(w * sm[:, 0]) / np.sum(w)) / lam ** 2)
    finally:
        swm.swm_destroy(ctx)
    peak = fs[int(np.argmax(mean))]
    assert 0.85 <= peak <= 1.0, (peak, mean)
    assert mean[int(np.argmax(mean))] > 1.5 * min(mean[0], mean[-1])
    kp = 2 * math.pi * peak / (2 * L)
    Xr = O.solve_lu(O.assemble(cl, kp, 3.0, sparse=False), O.rhs(cl, kp, inc))
    sr = O.rcs_monostatic(cl, kp, Xr, inc)
    ctx = _ctx(cl, kp, 3.0, C64)
    try:
        swm.swm_solve(ctx, inc, 1e-7, 30, 1000)
        sm = np.zeros((inc.shape[0], 2))
        swm.swm_rcs_monostatic(ctx, sm)
        assert_rcs_db(sm[:, 0], sr[:, 0], db=0.1)
    finally:
        swm.swm_destroy(ctx)
