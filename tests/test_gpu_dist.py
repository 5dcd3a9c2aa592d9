"""The partitioned solve on the GPU: each rank a context holding its owned and halo wires, the
product, preconditioner, right-hand sides, Gram-Schmidt vector algebra and far-field components in
the library's kernels (swm_apply, swm_precond_apply, swm_rhs, swm_vec_*, swm_far_components).
Ranks run as host threads on one device with their own contexts; they exchange host arrays
between launches only (no kernel waits on another rank).  Against the single-context solve
(swm_solve, FP64 path) and the oracle's LU solution."""
import math
import threading

import numpy as np
import pytest

import oracle as O
from paper_2410_03060_gb300 import dist
from synth import cloud_uniform_cube, observations_phi_cut

pytestmark = pytest.mark.gpu
K = 2.0 * math.pi


def _ranks(n, fn):
    import torch

    comms = dist.ThreadComm.group(n)
    out, err = [None] * n, []

    def go(r):
        try:
            torch.cuda.set_device(0)
            out[r] = fn(comms[r])
        except Exception as e:
            err.append(e)
            comms[r].sh.barrier.abort()

    th = [threading.Thread(target=go, args=(r,)) for r in range(n)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if err:
        raise err[0]
    return out


def _global(cl, parts):
    m, off = O.numbering(cl.nseg)
    X = np.full((int(off[-1]), parts[0][0].shape[0]), np.nan + 0j)
    for x, wires in parts:
        pos = 0
        for w in wires:
            X[off[w]:off[w + 1], :] = x[:, pos:pos + m[w]].T
            pos += m[w]
    return X


def test_building_blocks_match_the_oracle():
    """swm_apply = Z M^-1 x, swm_precond_apply = M^-1 y, swm_rhs = b, and the vector algebra, on
    one context, against the oracle's assembled matrices (float64)."""
    import torch
    import scipy.sparse as sp
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(50, 4.0, seed=61)
    r_c = 1.5
    m, off = O.numbering(cl.nseg)
    N = int(off[-1])
    ctx = swm.swm_create(0)
    try:
        swm.swm_set_cloud(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)
        swm.swm_build(ctx, K, r_c, swm.SWM_C128)
        g = np.random.default_rng(3)
        x = g.standard_normal((3, N)) + 1j * g.standard_normal((3, N))
        Z = O.assemble(cl, K, r_c, sparse=True)
        Minv = sp.block_diag([sp.csr_matrix(B) for B in O.block_jacobi(cl, K)], format="csr")
        y = np.zeros_like(x)
        swm.swm_apply(ctx, x, y)
        ref = (Z @ (Minv @ x.T)).T
        assert np.max(np.abs(y - ref)) / np.max(np.abs(ref)) < 1e-12
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        swm.swm_apply(ctx, xd, yd)
        assert np.max(np.abs(yd.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 1e-12
        z = np.zeros_like(x)
        swm.swm_precond_apply(ctx, x, z)
        assert np.max(np.abs(z - (Minv @ x.T).T)) / np.max(np.abs(z)) < 1e-12
        inc = np.array([[0.2, 0.4, 0.1], [1.5, 3.0, 0.7]])
        b = np.zeros((2, N), dtype=np.complex128)
        swm.swm_rhs(ctx, inc, b)
        assert np.max(np.abs(b - O.rhs(cl, K, inc).T)) / np.max(np.abs(b)) < 1e-12
        Vb = torch.from_numpy(np.stack([x, 2 * x[::-1].copy(), x * 1j])).cuda().contiguous()
        w = torch.from_numpy(x[::-1].copy()).cuda()
        d = swm.swm_vec_dots(ctx, Vb, 2, w)
        Vh = Vb.cpu().numpy()
        assert np.allclose(d, np.einsum("irn,rn->ir", np.conj(Vh[:2]), w.cpu().numpy()), rtol=1e-12)
        coef = np.array([[1 + 2j, 0.5, -1j], [0.25j, 2.0, 1.0]])
        v = w.clone()
        swm.swm_vec_axpy(ctx, Vb, 2, coef, v)
        assert np.allclose(v.cpu().numpy(), w.cpu().numpy() - np.einsum("ir,irn->rn", coef, Vh[:2]), rtol=1e-12)
        out = torch.empty_like(w)
        swm.swm_vec_scale(ctx, np.array([2.0, -1.0, 0.5]), w, out)
        assert np.allclose(out.cpu().numpy(), np.array([2.0, -1.0, 0.5])[:, None] * w.cpu().numpy(), rtol=1e-15)
    finally:
        swm.swm_destroy(ctx)


@pytest.mark.parametrize("n_ranks", [1, 2, 3])
def test_partitioned_solve_on_thread_ranks_matches_single_context(n_ranks):
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(90, 6.0, seed=62)
    r_c = 1.5
    inc = np.array([[0.3, 0.2, 0.0], [2.0, 4.0, 1.0], [1.1, 0.5, 0.3]])
    obs = observations_phi_cut(16)
    res = _ranks(n_ranks, lambda comm: dist.solve_partitioned(comm, cl.centres, cl.dirs, cl.lengths, cl.radii,
                                                               cl.nseg, K, r_c, inc, obs, tol=1e-12, restart=30))
    X = _global(cl, [(r[0], r[1]) for r in res])
    assert not np.isnan(X).any()
    ctx = swm.swm_create(0)
    try:
        swm.swm_set_cloud(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)
        swm.swm_build(ctx, K, r_c, swm.SWM_C128)
        cur = np.zeros((3, cl.n_unknowns), dtype=np.complex128)
        swm.swm_solve(ctx, inc, 1e-12, 30, 1000, cur)
        sig = np.zeros((3, len(obs), 2))
        swm.swm_rcs_bistatic(ctx, obs, sig)
    finally:
        swm.swm_destroy(ctx)
    assert np.linalg.norm(X - cur.T) / np.linalg.norm(cur) < 1e-10
    X_lu = O.solve_lu(O.assemble(cl, K, r_c, sparse=False), O.rhs(cl, K, inc))
    assert np.linalg.norm(X - X_lu) / np.linalg.norm(X_lu) < 1e-10
    for r in res:
        assert np.allclose(r[2], sig, rtol=1e-9, atol=1e-14)


def test_block_gmres_snapshots_match_lu():
    """Block GMRES (one Krylov space per snapshot for all its incidences) in the library's kernels
    on three snapshots of the batching statistics (uniform cube at 0.005 wires per cubic wavelength,
    lengths U[0.3, 0.6], r_c 3) with 20 monostatic incidences each: currents against the oracle's
    LU solution for every incidence (complex128 path) and the RCS within 0.1 dB."""
    from gpu_helpers import assert_rcs_db
    from synth import cloud_batching_snapshot, incidences_monostatic

    inc = incidences_monostatic(20)
    obs = observations_phi_cut(12)
    for i, nw in ((0, 150), (1, 220), (2, 300)):
        cl = cloud_batching_snapshot(i, nw=nw)
        res = _ranks(1, lambda comm: dist.solve_partitioned(comm, cl.centres, cl.dirs, cl.lengths, cl.radii,
                                                            cl.nseg, K, 3.0, inc, obs, tol=1e-11, restart=8,
                                                            block=True))
        X = _global(cl, [(res[0][0], res[0][1])])
        X_lu = O.solve_lu(O.assemble(cl, K, 3.0, sparse=False), O.rhs(cl, K, inc))
        err = np.linalg.norm(X - X_lu, axis=0) / np.linalg.norm(X_lu, axis=0)
        assert err.max() < 1e-8, err.max()
        s_ref = O.rcs_bistatic(cl, K, X_lu, obs)
        for r in range(20):
            assert_rcs_db(res[0][2][r, :, 0], s_ref[r, :, 0], db=0.1)
