"""GPU tests of BiCGSTAB on the block-Jacobi right-preconditioned S-NFC system (Sec. II-B), the
short-recurrence solver beside GMRES and GCR.

Currents against the oracle's LU solution and bistatic RCS within 0.1 dB, for one incidence, 9
(wire-tiled product read in place) and 37 (incidence-minor copy, packed product, on a dense cloud
whose tiles exceed shared memory and a sparse one whose tiles fit) in float64 and complex64; the
float64 path's step count against the oracle's BiCGSTAB; the step limit; the identity operator
(one step); a start from the solution (no step).
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import K, assert_rcs_db
from synth import cloud_uniform_cube, observations_phi_cut

pytestmark = pytest.mark.gpu

C128, C64 = 0, 1


def _ctx(cl, r_c, prec):
    from paper_2410_03060_gb300 import swm

    ctx = swm.swm_create(0)
    swm.swm_set_solver(ctx, "bicgstab")
    swm.swm_set_cloud(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)
    swm.swm_build(ctx, K, r_c, prec)
    return ctx


def _solve(swm, ctx, cl, inc, tol, max_iter=2000):
    cur = np.zeros((inc.shape[0], cl.n_unknowns), dtype=np.complex128)
    rc = swm.swm_solve(ctx, inc, tol, 50, max_iter, cur)
    return cur.T.copy(), rc, swm.swm_get_stats(ctx)


def _many(n, seed):
    g = np.random.default_rng(seed)
    return np.stack([g.uniform(0, np.pi, n), g.uniform(0, 2 * np.pi, n), g.uniform(0, np.pi, n)], 1)


@pytest.mark.parametrize("n_inc,form,major", [(1, 0, 0), (9, 0, 0), (9, 0, 1), (37, 68, 0), (37, 69, 0), (37, 70, 0),
                                               (37, 71, 0), (37, 71, 1), (37, 68, 1),
                                               (37, 72, 0), (37, 73, 0), (37, 73, 1),
                                               (37, 74, 0), (37, 75, 0), (37, 75, 1)])
def test_bicgstab_currents_and_rcs_match_oracle_lu(monkeypatch, n_inc, form, major):
    """form: the packed product's shape forced (68/69: E staged in shared memory, three or two CTAs
    per SM; 70/71: E read from global memory, three or four CTAs per SM; 72/73: the same in small
    CTAs), 0 the default; major: the
    complex64 vectors kept incidence-major (SWM_BICGSTAB_MAJOR) instead of incidence-minor."""
    from paper_2410_03060_gb300 import swm

    if form:
        monkeypatch.setenv("SWM_PRODUCT_FORM", str(form))
    if major:
        monkeypatch.setenv("SWM_BICGSTAB_MAJOR", "1")

    obs = observations_phi_cut(48)
    cases = [(cloud_uniform_cube(120, 5.0, seed=61), 2.0)]
    if n_inc == 37:
        cases.append((cloud_uniform_cube(150, 9.0, seed=46), 1.2))
    inc = _many(n_inc, 11 + n_inc)
    for cl, r_c in cases:
        X = O.solve_lu(O.assemble(cl, K, r_c, sparse=False), O.rhs(cl, K, inc))
        s_ref = O.rcs_bistatic(cl, K, X, obs)
        for prec, tol, bound in ((C128, 1e-11, 1e-8), (C64, 1e-6, 1e-3)):
            ctx = _ctx(cl, r_c, prec)
            try:
                cur, rc, st = _solve(swm, ctx, cl, inc, tol)
                assert rc == swm.SWM_OK and st["converged"] == 1
                if form and prec == C64:
                    assert st["step_rhs_block"] == form
                assert st["rel_residual"] <= tol
                assert np.linalg.norm(cur - X) / np.linalg.norm(X) < bound
                sig = np.zeros((n_inc, len(obs), 2))
                swm.swm_rcs_bistatic(ctx, obs, sig)
                for i in range(n_inc):
                    assert_rcs_db(sig[i, :, 0], s_ref[i, :, 0], db=0.1)
            finally:
                swm.swm_destroy(ctx)


def test_bicgstab_steps_match_oracle_bicgstab():
    """Float64 path and the oracle take the same steps up to rounding: the same count, one more or
    one fewer where a residual lands on the tolerance."""
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(100, 5.0, seed=62)
    inc = np.array([[0.7, 0.3, 0.2]])
    Z = O.assemble(cl, K, 2.0, sparse=True)
    b = O.rhs(cl, K, inc)[:, 0]
    m, off = O.numbering(cl.nseg)
    for tol in (1e-4, 1e-8):
        _, it_ref, _ = O.bicgstab(Z, b, O.block_jacobi(cl, K), off, tol=tol)
        ctx = _ctx(cl, 2.0, C128)
        try:
            _, rc, st = _solve(swm, ctx, cl, inc, tol)
            assert rc == swm.SWM_OK
            assert abs(st["iterations"] - it_ref) <= 1, (st["iterations"], it_ref)
        finally:
            swm.swm_destroy(ctx)


def test_bicgstab_step_limit_identity_and_start_at_solution():
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(100, 5.0, seed=63)
    inc = _many(3, 5)
    X = O.solve_lu(O.assemble(cl, K, 2.0, sparse=False), O.rhs(cl, K, inc))
    ctx = _ctx(cl, 2.0, C128)
    try:
        # two steps are not enough for 1e-12
        _, rc, st = _solve(swm, ctx, cl, inc, 1e-12, max_iter=2)
        assert rc == swm.SWM_ENOTCONV and st["iterations"] == 2 and st["converged"] == 0
        # from the LU solution: the first true residual already meets tol
        cur = np.zeros((inc.shape[0], cl.n_unknowns), dtype=np.complex128)
        rc = swm.swm_solve_guess(ctx, inc, X.T.copy(), 1e-9, 50, 100, cur)
        st = swm.swm_get_stats(ctx)
        assert rc == swm.SWM_OK and st["iterations"] == 0
        assert np.linalg.norm(cur.T - X) / np.linalg.norm(X) < 1e-12
    finally:
        swm.swm_destroy(ctx)
    # wires farther apart than r_c: Z is block-diagonal and the preconditioned operator the identity
    far = cloud_uniform_cube(30, 40.0, seed=64)
    d = np.linalg.norm(far.centres[:, None] - far.centres[None], axis=2)
    r_c = 0.5 * d[np.triu_indices(far.nw, 1)].min()
    Xf = O.solve_lu(O.assemble(far, K, r_c, sparse=False), O.rhs(far, K, inc))
    for prec, bound in ((C128, 1e-12), (C64, 1e-5)):
        ctx = _ctx(far, r_c, prec)
        try:
            cur, rc, st = _solve(swm, ctx, far, inc, 1e-10 if prec == C128 else 1e-5)
            assert rc == swm.SWM_OK and st["iterations"] == 1
            assert np.linalg.norm(cur - Xf) / np.linalg.norm(Xf) < bound
        finally:
            swm.swm_destroy(ctx)


def test_sorted_product_over_several_order_windows(monkeypatch):
    """Form 75 takes the wires in an order sorted within windows of 4096 wires; a cloud of 9,000
    wires spans two full windows and a ragged one.  Its complex64 currents and RCS against the
    float64 path on the same cloud (no oracle LU at 45,000 unknowns), and against form 73 (the
    cell order): both forms solve the same system, so their currents agree to the tolerance."""
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(9000, 39.0, seed=65)
    inc = _many(37, 66)
    obs = observations_phi_cut(24)

    def run(prec, tol, form=None):
        if form:
            monkeypatch.setenv("SWM_PRODUCT_FORM", str(form))
        else:
            monkeypatch.delenv("SWM_PRODUCT_FORM", raising=False)
        ctx = _ctx(cl, 2.0, prec)
        try:
            cur, rc, st = _solve(swm, ctx, cl, inc, tol)
            assert rc == swm.SWM_OK and st["converged"] == 1
            if form:
                assert st["step_rhs_block"] == form
            sig = np.zeros((inc.shape[0], len(obs), 2))
            swm.swm_rcs_bistatic(ctx, obs, sig)
            return cur, sig
        finally:
            swm.swm_destroy(ctx)

    X64, s64 = run(C128, 1e-10)
    X73, _ = run(C64, 1e-6, 73)
    X75, s75 = run(C64, 1e-6, 75)
    assert np.linalg.norm(X75 - X64) / np.linalg.norm(X64) < 1e-4
    assert np.linalg.norm(X75 - X73) / np.linalg.norm(X64) < 1e-4
    for i in range(inc.shape[0]):
        assert_rcs_db(s75[i, :, 0], s64[i, :, 0], db=0.1)
