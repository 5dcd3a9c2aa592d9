"""Shared helpers for the GPU parity tests: run the CUDA path through the C ABI, compare RCS."""
import math

import numpy as np

K = 2.0 * math.pi


def run_gpu(cloud, k, r_c, prec, inc, obs=None, tol=1e-10, restart=50, max_iter=3000, mono=False,
            device_inputs=False):
    """Full CUDA path through the binding: returns dict(currents, sigma, sigma_mono, stats, ctx)."""
    from paper_2410_03060_gb300 import swm

    ctx = swm.swm_create(0)
    try:
        if device_inputs:
            import torch
            args = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
                    (cloud.centres, cloud.dirs, cloud.lengths, cloud.radii, cloud.nseg)]
        else:
            args = [cloud.centres, cloud.dirs, cloud.lengths, cloud.radii, cloud.nseg]
        swm.swm_set_cloud(ctx, *args)
        swm.swm_build(ctx, k, r_c, prec)
        inc = np.atleast_2d(inc)
        N = int(np.sum(cloud.nseg.astype(np.int64) - 1))
        cur = np.zeros((inc.shape[0], N), dtype=np.complex128)
        rc = swm.swm_solve(ctx, inc, tol, restart, max_iter, cur)
        out = {"rc": rc, "currents": cur.T.copy(), "stats": swm.swm_get_stats(ctx)}
        if obs is not None:
            sig = np.zeros((inc.shape[0], len(obs), 2))
            swm.swm_rcs_bistatic(ctx, obs, sig)
            out["sigma"] = sig
        if mono:
            sm = np.zeros((inc.shape[0], 2))
            swm.swm_rcs_monostatic(ctx, sm)
            out["sigma_mono"] = sm
        out["rhs"] = swm.swm_get_rhs(ctx).T.copy()
        out["pattern"] = swm.swm_get_pattern(ctx)
        out["ctx"] = ctx
        return out
    except Exception:
        swm.swm_destroy(ctx)
        raise


def block_errors(ctx, cloud, k, pairs, scaled=False):
    """Worst block error over the given blocks: max |Z_gpu - Z_oracle| / max |Z_oracle| per block,
    or, with ``scaled``, divided instead by sqrt(max|Z_pp| max|Z_qq|), the scale of the two self
    blocks the block couples.  Returns (worst, (p, q) of the worst block)."""
    import oracle as O
    from paper_2410_03060_gb300 import swm

    worst, where = 0.0, None
    m = cloud.nseg - 1
    diag = {}

    def dmax(p):
        if p not in diag:
            diag[p] = float(np.max(np.abs(O.self_block(cloud, k, p))))
        return diag[p]
    for p, q in pairs:
        p, q = int(p), int(q)
        zg = swm.swm_get_block(ctx, p, q, int(m[p]), int(m[q]))
        zo = O.block(cloud, k, p, q)
        scale = math.sqrt(dmax(p) * dmax(q)) if scaled else float(np.max(np.abs(zo)))
        e = float(np.max(np.abs(zg - zo)) / scale)
        if e > worst:
            worst, where = e, (p, q)
    return worst, where


def assert_rcs_db(s_gpu, s_ref, db=0.1, floor_db=30.0):
    """RCS agreement: |10 log10(s_gpu / s_ref)| <= db wherever s_ref is within floor_db of its
    maximum, and aggregate relative L2 error <= 10^(db/10) - 1."""
    s_gpu = np.asarray(s_gpu, dtype=np.float64).ravel()
    s_ref = np.asarray(s_ref, dtype=np.float64).ravel()
    keep = s_ref >= s_ref.max() * 10 ** (-floor_db / 10)
    err_db = np.abs(10 * np.log10(s_gpu[keep] / s_ref[keep]))
    assert err_db.max() <= db, f"max RCS error {err_db.max():.4g} dB"
    rel = np.linalg.norm(s_gpu - s_ref) / np.linalg.norm(s_ref)
    assert rel <= 10 ** (db / 10) - 1, f"aggregate RCS error {rel:.4g}"
    return err_db.max(), rel
