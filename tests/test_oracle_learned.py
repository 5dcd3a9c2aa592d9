"""Pins of the warm-start network's oracle (oracle/learned.py): the hand-derived backward pass
against central finite differences, rotation invariance of the features and of the prediction,
the neighbour lists against a k-d tree query, and the untrained network's identity limit."""
import math

import numpy as np

import oracle as O
import oracle.learned as NL
from synth import cloud_uniform_cube
from synth.netinit import init_params, n_params

K = 2.0 * math.pi


def _case(seed=5, nw=12, side=3.0, r_c=2.0):
    cl = cloud_uniform_cube(nw, side, seed=seed)
    inc = np.array([[0.3, 0.5, 0.1], [1.2, 2.0, 0.7]])
    nbr = NL.neighbour_lists(cl, r_c)
    Xe, Xs = NL.features(cl, K, inc, r_c, nbr)
    return cl, inc, nbr, Xe, Xs


def test_param_count_and_layout():
    assert n_params() == sum(i * o + o for i, o in NL.LAYERS) == 93720
    Ws = NL.unpack(init_params(0))
    assert [w.shape for w, _ in Ws] == [(i, o) for i, o in NL.LAYERS]


def test_backward_matches_central_differences():
    cl, inc, nbr, Xe, Xs = _case()
    xi = NL.isolated_currents(cl, K, inc)
    rng = np.random.default_rng(1)
    params = init_params(3).astype(np.float64)
    params *= 1.0
    o = 0
    for li, (i, n) in enumerate(NL.LAYERS):  # undo the small initial scale of the two last layers
        if li in (2, 5):
            params[o:o + i * n] *= 100.0
        o += i * n + n
    xt = xi + 0.1 * np.abs(xi).mean() * (rng.standard_normal(xi.shape) + 1j * rng.standard_normal(xi.shape))
    L, g, _ = NL.loss_and_grad(params, cl, K, inc, Xe, Xs, xi, xt, nbr)
    # a few entries of every weight matrix and bias vector
    o, idx = 0, []
    for i, n in NL.LAYERS:
        idx += list(o + rng.choice(i * n, 4, replace=False)) + list(o + i * n + rng.choice(n, 2, replace=False))
        o += i * n + n
    for j in idx:
        h = 1e-6 * max(1.0, abs(params[j]))
        pp = params.copy()
        pp[j] += h
        Lp = NL.loss_and_grad(pp, cl, K, inc, Xe, Xs, xi, xt, nbr)[0]
        pp[j] -= 2 * h
        Lm = NL.loss_and_grad(pp, cl, K, inc, Xe, Xs, xi, xt, nbr)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[j]) <= 1e-5 * (abs(fd) + abs(g[j])) + 1e-9, (j, fd, g[j])


def _rotate(cl, inc, Rm):
    from synth.clouds import Cloud

    c2 = Cloud(centres=cl.centres @ Rm.T, dirs=cl.dirs @ Rm.T, lengths=cl.lengths, radii=cl.radii, nseg=cl.nseg,
               name=cl.name)
    u, _, e = O.incidence_frames(inc)
    u2, e2 = u @ Rm.T, e @ Rm.T
    th = np.arccos(np.clip(u2[:, 2], -1, 1))
    ph = np.arctan2(u2[:, 1], u2[:, 0])
    th_hat = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], 1)
    ph_hat = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], 1)
    psi = np.arctan2(np.sum(e2 * ph_hat, 1), np.sum(e2 * th_hat, 1))
    return c2, np.stack([th, ph, psi], 1)


def test_features_and_prediction_are_rotation_invariant():
    cl, inc, nbr, Xe, Xs = _case(seed=7)
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    cl2, inc2 = _rotate(cl, inc, Q)
    nbr2 = NL.neighbour_lists(cl2, 2.0)
    assert np.array_equal(nbr, nbr2)
    Xe2, Xs2 = NL.features(cl2, K, inc2, 2.0, nbr2)
    assert np.allclose(Xe, Xe2, atol=1e-10) and np.allclose(Xs, Xs2, atol=1e-12)
    params = init_params(2).astype(np.float64) * 5.0
    x0, _ = NL.forward(params, cl, K, inc, Xe, Xs, NL.isolated_currents(cl, K, inc), nbr)
    x02, _ = NL.forward(params, cl2, K, inc2, Xe2, Xs2, NL.isolated_currents(cl2, K, inc2), nbr2)
    assert np.allclose(x0, x02, rtol=1e-8, atol=1e-12 * np.abs(x0).max())


def test_neighbour_lists_match_kdtree_query():
    from scipy.spatial import cKDTree

    cl = cloud_uniform_cube(300, 8.0, seed=9)
    nbr = NL.neighbour_lists(cl, 2.0)
    tree = cKDTree(cl.centres)
    for p in range(cl.nw):
        cand = [q for q in tree.query_ball_point(cl.centres[p], 2.0 * (1 + 1e-12)) if q != p]
        d2 = np.sum((cl.centres[cand] - cl.centres[p]) ** 2, 1)
        keep = [q for _, q in sorted(zip(d2, cand))][:NL.K_NBR]
        got = [q for q in nbr[p] if q >= 0]
        assert got == keep


def test_mode_amplitudes_reproduce_sine_shaped_currents():
    """The amplitudes are the discrete sine transform of the isolated currents: a current made of
    the three modes is recovered exactly (times the wire's incident phase)."""
    cl, inc, nbr, Xe, Xs = _case(seed=13)
    m, off = O.numbering(cl.nseg)
    _, khat, _ = O.incidence_frames(inc)
    rng = np.random.default_rng(2)
    want = rng.standard_normal((2, cl.nw, 3)) + 1j * rng.standard_normal((2, cl.nw, 3))
    x = np.zeros((int(off[-1]), 2), dtype=complex)
    for r in range(2):
        for p in range(cl.nw):
            i = np.arange(1, cl.nseg[p])[:, None]
            phi = np.sin(np.arange(1, 4)[None, :] * np.pi * i / cl.nseg[p])
            x[off[p]:off[p + 1], r] = np.exp(-1j * K * (khat[r] @ cl.centres[p])) * (phi @ want[r, p])
    a = NL.amplitudes(cl, K, inc, x)
    assert np.allclose(a, want, rtol=1e-12, atol=1e-12)


def test_untrained_output_layer_zero_gives_isolated_currents():
    cl, inc, nbr, Xe, Xs = _case(seed=11)
    params = init_params(0).astype(np.float64)
    o = 0
    for li, (i, n) in enumerate(NL.LAYERS):  # zero the last layer of both MLPs: no correction
        if li in (2, 5):
            params[o:o + i * n + n] = 0.0
        o += i * n + n
    xi = NL.isolated_currents(cl, K, inc)
    x0, _ = NL.forward(params, cl, K, inc, Xe, Xs, xi, nbr)
    assert np.array_equal(x0, xi)
    # the isolated currents solve the block-diagonal part of the system exactly
    Z = O.assemble(cl, K, None, sparse=False)
    m, off = O.numbering(cl.nseg)
    b = O.rhs(cl, K, inc)
    for p in range(cl.nw):
        sl = slice(off[p], off[p + 1])
        assert np.allclose(Z[sl, sl] @ xi[sl], b[sl], rtol=1e-10, atol=1e-14)
