"""GPU tests of the learned warm start: the network's forward pass, loss and gradient against the
float64 oracle (oracle/learned.py), training on solver currents, and what the trained network
gains over the isolated-wire guess and over a cold start on clouds it has not seen."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.learned as NL
from gpu_helpers import K
from synth import cloud_uniform_cube
from synth.netinit import init_params

pytestmark = pytest.mark.gpu

C128, C64 = 0, 1


def _ctx(cl, r_c, prec):
    from paper_2410_03060_gb300 import swm

    ctx = swm.swm_create(0)
    swm.swm_set_cloud(ctx, cl.centres, cl.dirs, cl.lengths, cl.radii, cl.nseg)
    swm.swm_build(ctx, K, r_c, prec)
    return ctx


def _scaled_params(seed):
    p = init_params(seed).astype(np.float64)
    o = 0
    for li, (i, n) in enumerate(NL.LAYERS):  # undo the small initial scale of the last layers
        if li in (2, 5):
            p[o:o + i * n] *= 100.0
        o += i * n + n
    return p.astype(np.float32)


def test_forward_loss_and_gradient_match_oracle():
    from paper_2410_03060_gb300 import swm

    assert swm.swm_net_num_params() == init_params(0).size
    cl = cloud_uniform_cube(60, 5.0, seed=81)
    r_c = 2.0
    inc = np.array([[0.3, 0.5, 0.1], [1.2, 2.0, 0.7], [2.5, 4.0, 1.3]])
    p32 = _scaled_params(5)
    ctx = _ctx(cl, r_c, C128)
    net = swm.swm_net_create(0)
    try:
        swm.swm_net_set_params(net, p32)
        assert np.array_equal(swm.swm_net_get_params(net), p32)
        x0 = swm.swm_net_predict(net, ctx, inc).T
        nbr = NL.neighbour_lists(cl, r_c)
        Xe, Xs = NL.features(cl, K, inc, r_c, nbr)
        xi = NL.isolated_currents(cl, K, inc)
        x0o, _ = NL.forward(p32.astype(np.float64), cl, K, inc, Xe, Xs, xi, nbr)
        assert np.linalg.norm(x0 - x0o) / np.linalg.norm(x0o - xi) < 1e-4  # the correction itself
        Xt = O.solve_lu(O.assemble(cl, K, r_c, sparse=False), O.rhs(cl, K, inc))
        lg, gg = swm.swm_net_train_step(net, ctx, inc, Xt.T.copy(), 0.0, want_grad=True)
        lo, go, _ = NL.loss_and_grad(p32.astype(np.float64), cl, K, inc, Xe, Xs, xi, Xt, nbr)
        assert abs(lg - lo) <= 1e-5 * lo
        o = 0
        for i, n in NL.LAYERS:
            a, b = gg[o:o + i * n + n], go[o:o + i * n + n]
            assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b)
            o += i * n + n
        # lr = 0 leaves the parameters alone; lr > 0 moves them
        assert np.array_equal(swm.swm_net_get_params(net), p32)
        swm.swm_net_train_step(net, ctx, inc, Xt.T.copy(), 1e-3)
        assert not np.array_equal(swm.swm_net_get_params(net), p32)
    finally:
        swm.swm_net_destroy(net)
        swm.swm_destroy(ctx)


def _incidences(n, seed):
    g = np.random.default_rng(seed)
    return np.stack([np.arccos(g.uniform(-1, 1, n)), g.uniform(0, 2 * math.pi, n), g.uniform(0, math.pi, n)], 1)


def _dataset(seed, nw=1200, dens=0.1, n_inc=8):
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(nw, (nw / dens) ** (1 / 3), seed=seed)
    ctx = _ctx(cl, 3.0, C64)
    inc = _incidences(n_inc, seed + 7)
    X = np.zeros((n_inc, cl.n_unknowns), dtype=np.complex128)
    swm.swm_solve(ctx, inc, 1e-8, 50, 2000, X)
    return cl, ctx, X, inc


def test_trained_network_beats_isolated_guess_and_cold_start_on_unseen_clouds():
    from paper_2410_03060_gb300 import swm

    train = [_dataset(300 + s) for s in range(4)]
    test = [_dataset(400 + s) for s in range(2)]
    net = swm.swm_net_create(0)
    try:
        swm.swm_net_set_params(net, init_params(0))
        iso = [swm.swm_net_train_step(net, t[1], t[3], t[2], 0.0)[0] for t in test]
        for it in range(800):
            cl, ctx, X, inc = train[it % len(train)]
            swm.swm_net_train_step(net, ctx, inc, X, 3e-4)
        learned = [swm.swm_net_train_step(net, t[1], t[3], t[2], 0.0)[0] for t in test]
        # the prediction error on clouds the network never saw, against the isolated-wire guess
        assert all(l < 0.6 * i for l, i in zip(learned, iso)), (learned, iso)
        for cl, ctx, X, inc in test:
            swm.swm_solve(ctx, inc, 1e-6, 50, 2000)
            cold = swm.swm_get_stats(ctx)["iterations"]
            x0 = swm.swm_net_predict(net, ctx, inc)
            cur = np.zeros_like(X)
            assert swm.swm_solve_guess(ctx, inc, x0, 1e-6, 50, 2000, cur) == 0
            st = swm.swm_get_stats(ctx)
            assert st["converged"] == 1 and st["iterations"] <= cold
            # same answer as the cold solve, to the tolerance
            assert np.linalg.norm(cur - X) / np.linalg.norm(X) < 1e-4
    finally:
        swm.swm_net_destroy(net)
        for t in train + test:
            swm.swm_destroy(t[1])


def test_solve_from_guess_all_paths(monkeypatch):
    """Starting from the exact solution every solver path stops at once; from a perturbed one it
    converges to the same currents (tolerance relative to |b|)."""
    from paper_2410_03060_gb300 import swm

    cl = cloud_uniform_cube(100, 5.0, seed=82)
    inc = np.array([[0.2, 0.3, 0.0], [1.0, 1.0, 0.5]])
    X = O.solve_lu(O.assemble(cl, K, 2.0, sparse=False), O.rhs(cl, K, inc)).T.copy()
    for path in ("persistent", "per_kernel", "gcr", "bf16"):
        monkeypatch.setenv("SWM_PERSIST", "0" if path == "per_kernel" else "1")
        prec = {"bf16": 2}.get(path, C128)
        ctx = _ctx(cl, 2.0, prec)
        try:
            if path == "gcr":
                swm.swm_set_solver(ctx, "gcr")
            tol = 1e-4 if prec == 2 else 1e-10  # bfloat16 path: complex64 blocks, so a looser tol
            cur = np.zeros_like(X)
            swm.swm_solve_guess(ctx, inc, X, tol, 50, 500, cur)
            assert swm.swm_get_stats(ctx)["iterations"] == 0
            rng = np.random.default_rng(3)
            x0 = X * (1 + 0.05 * rng.standard_normal(X.shape))
            swm.swm_solve_guess(ctx, inc, x0, tol, 50, 500, cur)
            st = swm.swm_get_stats(ctx)
            assert st["converged"] == 1 and st["iterations"] > 0
            assert np.linalg.norm(cur - X) / np.linalg.norm(X) < (1e-3 if prec == 2 else 1e-8)
        finally:
            swm.swm_destroy(ctx)
