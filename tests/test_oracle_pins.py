"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test checks one part of the oracle against a closed form, adaptive quadrature, brute force,
a symmetry of the physics or a textbook value, chosen so that a plausible slip (a dropped term, a
wrong sign or index, a transposed operand, a wrong factor) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad, quad_vec

import oracle as O
from synth import Cloud, cloud_single, cloud_uniform_cube

K = 2.0 * math.pi
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook_values.json")))
pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def _cloud(centres, dirs, lengths, nseg, radius=1e-3):
    centres = np.asarray(centres, dtype=np.float64)
    dirs = np.asarray(dirs, dtype=np.float64)
    dirs = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    n = len(centres)
    return Cloud(centres, dirs, np.asarray(lengths, dtype=np.float64), np.full(n, radius),
                 np.asarray(nseg, dtype=np.int32), "pin")


# ----------------------------------------------------------------------------- building blocks
def test_convolution_polynomials_match_direct_integration():
    shapes = {O.RISE: lambda x: x, O.FALL: lambda x: 1.0 - x}
    for a in (O.RISE, O.FALL):
        for b in (O.RISE, O.FALL):
            for w in (-0.93, -0.5, -0.1, 0.0, 0.2, 0.61, 0.99):
                lo, hi = max(0.0, w), min(1.0, 1.0 + w)
                ref = quad(lambda x: shapes[a](x) * shapes[b](x - w), lo, hi, epsabs=1e-15)[0]
                half = 0 if w < 0 else 1
                assert abs(O.convolution_poly(a, b, half)(w) - ref) < 1e-14


def test_static_antiderivatives_by_quadrature():
    for alpha in (0.016, 0.3):
        for n in range(4):
            for (t0, t1) in ((-1.0, 0.0), (0.0, 1.0), (1.0, 2.0), (-2.0, -1.0)):
                ref = quad(lambda t: t ** n / math.sqrt(t * t + alpha * alpha), t0, t1,
                           points=[0.0] if t0 < 0 < t1 else None, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
                got = O.static_antiderivative(n, t1, alpha) - O.static_antiderivative(n, t0, alpha)
                assert abs(got - ref) < 1e-11 * max(1.0, abs(ref))


def _adaptive_pair(k, fun_R, D1, D2):
    """int_0^1 int_0^1 phi_a(x) phi_b(y) G(R(x, y)) dy dx * D1 D2 by nested adaptive quadrature,
    returned as I[a, b]."""
    def inner(x, y_break):
        def f(y):
            G = O.green(k, fun_R(x, y))
            pa, pb = (x, 1.0 - x), (y, 1.0 - y)
            v = np.array([pa[i] * pb[j] * G for i in (0, 1) for j in (0, 1)])
            return np.concatenate([v.real, v.imag])
        pts = [y_break(x)] if y_break is not None and 0.0 < y_break(x) < 1.0 else None
        return quad_vec(f, 0.0, 1.0, points=pts, epsabs=1e-14, epsrel=1e-11, limit=400)[0]
    return inner


def test_self_integrals_match_2d_adaptive_quadrature():
    """Same-wire segment pairs: the 1-D reduction, the convolution weights, the static closed form
    and the Gauss rule for the rest together reproduce the 2-D integral."""
    D, a = 0.5 / 8, 1e-3
    for delta in (0, 1, -1, 2, -3):
        R = lambda x, y: math.sqrt((D * (delta + x - y)) ** 2 + a * a)
        inner = _adaptive_pair(K, R, D, D)
        outer = quad_vec(lambda x: inner(x, lambda xx: xx + delta), 0.0, 1.0, epsabs=1e-14, epsrel=1e-10,
                         limit=400)[0]
        ref = ((outer[:4] + 1j * outer[4:]) * D * D).reshape(2, 2)
        got = O.self_offset_integrals(K, D, a, delta)
        hi = O.self_offset_integrals(K, D, a, delta, nq=64)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(hi - ref)) / scale < 1e-9, delta
        # the 8-point rule's own error (the smooth remainder has a kink rounded over a/D)
        assert np.max(np.abs(got - ref)) / scale < 1e-6, delta


def test_mutual_integrals_match_adaptive_quadrature():
    """Segment pairs on different wires: the far rule (4 points) and the near rule (8 points) are
    within their stated error of adaptive quadrature, and a high-order rule converges to it."""
    rng = np.random.default_rng(5)
    for trial in range(3):
        tp, tq = rng.standard_normal(3), rng.standard_normal(3)
        tp /= np.linalg.norm(tp)
        tq /= np.linalg.norm(tq)
        dist = (0.35, 0.12, 0.05)[trial]  # >= D (far rule), ~1.7 D and ~0.7 D (near rule)
        n = rng.standard_normal(3)
        n -= (n @ tp) * tp
        n /= np.linalg.norm(n)
        cl = _cloud([[0, 0, 0], dist * n + 0.02 * tp], [tp, tq], [0.5, 0.45], [7, 6])
        u, v = 3, 2
        Dp, Dq = 0.5 / 7, 0.45 / 6

        def R(x, y):
            rp = cl.centres[0] + (-0.25 + (u + x) * Dp) * cl.dirs[0]
            rq = cl.centres[1] + (-0.225 + (v + y) * Dq) * cl.dirs[1]
            d = rp - rq
            return math.sqrt(d @ d + 1e-6)
        inner = _adaptive_pair(K, R, Dp, Dq)
        outer = quad_vec(lambda x: inner(x, None), 0.0, 1.0, epsabs=1e-14, epsrel=1e-10)[0]
        ref = ((outer[:4] + 1j * outer[4:]) * Dp * Dq).reshape(2, 2)
        nq = O.mutual_order(cl, 0, 1)
        got = O.mutual_segment_integrals(cl, K, 0, 1)[u, v]
        hi = O.mutual_segment_integrals(cl, K, 0, 1, nq=24)[u, v]
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(hi - ref)) / scale < 1e-9
        tol = 3e-5 if nq == O.NQ_FAR else 5e-4
        assert np.max(np.abs(got - ref)) / scale < tol, (trial, nq)


def test_segment_distance_brute_force():
    rng = np.random.default_rng(11)
    for _ in range(40):
        cp, cq = rng.uniform(-0.4, 0.4, 3), rng.uniform(-0.4, 0.4, 3)
        tp, tq = rng.standard_normal(3), rng.standard_normal(3)
        tp /= np.linalg.norm(tp)
        tq /= np.linalg.norm(tq)
        if _ % 5 == 0:
            tq = tp.copy()  # parallel wires
        Lp, Lq = rng.uniform(0.3, 0.6, 2)
        s = np.linspace(-Lp / 2, Lp / 2, 801)
        sq = np.linspace(-Lq / 2, Lq / 2, 801)
        P = cp[None, :] + s[:, None] * tp[None, :]
        Q = cq[None, :] + sq[:, None] * tq[None, :]
        d2 = ((P[:, None, :] - Q[None, :, :]) ** 2).sum(-1)
        brute = math.sqrt(d2.min())
        got = O.segment_distance(cp, tp, Lp, cq, tq, Lq)
        assert got <= brute + 1e-12
        assert brute - got < 2e-3 * max(Lp, Lq) / 800 * 4 + 1e-9


def test_triangle_fourier_transform_by_quadrature():
    for D in (0.0625, 0.1):
        for beta in (0.0, 1e-9, 2.3, -7.1, 40.0):
            f = lambda x: (1 - abs(x) / D) * np.exp(1j * beta * x)
            re = quad(lambda x: f(x).real, -D, D, points=[0.0], epsabs=1e-15)[0]
            im = quad(lambda x: f(x).imag, -D, D, points=[0.0], epsabs=1e-15)[0]
            assert abs(O.triangle_ft(beta, D) - (re + 1j * im)) < 1e-14


def test_rhs_and_far_field_by_segment_quadrature():
    """b_n = int Lambda_n t.E_inc and the far-field radiation vector, integrated numerically with
    64 Gauss points per segment, equal the closed forms."""
    cl = cloud_uniform_cube(3, 2.0, seed=2)
    inc = np.array([[0.3, 1.1, 0.4], [2.0, -0.5, 0.0]])
    u, khat, e = O.incidence_frames(inc)
    b = O.rhs(cl, K, inc)
    xg, wg = O.gauss_legendre_01(64)
    m, off = O.numbering(cl.nseg)
    rhat = np.array([[0.2, -0.7, 0.3]])
    rhat /= np.linalg.norm(rhat)
    cur = np.random.default_rng(0).standard_normal((off[-1], 2)) + 0j
    F_ref = np.zeros((1, 3, 2), dtype=complex)
    for p in range(cl.nw):
        ns, L = int(cl.nseg[p]), cl.lengths[p]
        D = L / ns
        for i in range(1, ns):
            si = -L / 2 + i * D
            s = np.concatenate([si - D + D * xg, si + D * xg])
            w = np.concatenate([D * wg, D * wg])
            lam = 1.0 - np.abs(s - si) / D
            r = cl.centres[p][None, :] + s[:, None] * cl.dirs[p][None, :]
            for ii in range(2):
                Einc = e[ii][None, :] * np.exp(-1j * K * (r @ khat[ii]))[:, None]
                ref = np.sum(w * lam * (Einc @ cl.dirs[p]))
                assert abs(b[off[p] + i - 1, ii] - ref) < 1e-13
                F_ref[0, :, ii] += cur[off[p] + i - 1, ii] * np.sum(w * lam * np.exp(1j * K * (r @ rhat[0]))) * cl.dirs[p]
    F = O.far_field(cl, K, cur, rhat)
    assert np.max(np.abs(F - F_ref)) < 1e-12


def test_incidence_frame_is_right_handed_and_matches_minus_z_case():
    u, khat, e = O.incidence_frames(np.array([[0.0, 0.0, 0.0]]))
    assert np.allclose(khat[0], [0, 0, -1]) and np.allclose(e[0], [1, 0, 0])
    rng = np.random.default_rng(3)
    inc = np.stack([rng.uniform(0, math.pi, 20), rng.uniform(0, 2 * math.pi, 20), rng.uniform(0, math.pi, 20)], 1)
    u, khat, e = O.incidence_frames(inc)
    assert np.allclose(np.sum(e * khat, 1), 0.0) and np.allclose(np.linalg.norm(e, axis=1), 1.0)


# ----------------------------------------------------------------------------- dipole (textbook)
def _dipole_zin(L, ns, a=1e-3):
    cl = cloud_single(L, ns, radius=a)
    Z = O.self_block(cl, K, 0)
    c = ns // 2 - 1  # centre vertex
    return 1j * K * O.ETA0 / np.linalg.inv(Z)[c, c]


def test_halfwave_dipole_input_impedance_band_and_convergence():
    g = GOLDEN["halfwave_dipole_input_impedance_thin_ohm"]["band_radius_1e-3"]
    z16, z32 = _dipole_zin(0.5, 16), _dipole_zin(0.5, 32)
    for z in (z16, z32):
        assert g["R"][0] <= z.real <= g["R"][1] and g["X"][0] <= z.imag <= g["X"][1], z
    assert abs(z32.real - z16.real) / z32.real < 0.03
    # a thinner wire moves toward the infinitely thin value 73 + j42.5
    zthin = _dipole_zin(0.5, 32, a=1e-5)
    assert abs(zthin.real - 73.1) < abs(z32.real - 73.1)
    # resonance (X = 0) below half a wavelength
    assert _dipole_zin(0.46, 16).imag < 0 < _dipole_zin(0.49, 16).imag


def test_resonant_dipole_broadside_rcs():
    g = GOLDEN["resonant_dipole_broadside_rcs_lambda2"]
    inc = np.array([[math.pi / 2, 0.0, 0.0]])  # arrival along +x, E along -z (wire axis)
    best = 0.0
    for L in np.linspace(0.45, 0.5, 11):
        cl = cloud_single(L, 16)
        X, _ = O.solve(cl, K, inc)
        best = max(best, O.rcs_monostatic(cl, K, X, inc)[0, 0])
    assert abs(best - g["value"]) / g["value"] < g["rtol"], best
    # crossed polarisation on a wire along z is zero
    cl = cloud_single(0.48, 16)
    X, _ = O.solve(cl, K, inc)
    assert O.rcs_monostatic(cl, K, X, inc)[0, 1] < 1e-20


@pytest.mark.slow
def test_marcus_mean_rcs_of_random_resonant_wire():
    """Orientation average of the co-polarised backscatter of one resonant half-wave wire, the
    single-chaff limit of the averaged cloud RCS (Sec. III-B)."""
    g = GOLDEN["marcus_random_halfwave_mean_rcs_lambda2"]
    inc = np.array([[0.0, 0.0, 0.0]])
    xt, wt = np.polynomial.legendre.leggauss(12)
    nph = 12
    acc = 0.0
    for ct, w in zip(xt, wt):
        st = math.sqrt(1 - ct * ct)
        for j in range(nph):
            ph = 2 * math.pi * j / nph
            cl = cloud_single(0.475, 12, direction=(st * math.cos(ph), st * math.sin(ph), ct))
            X, _ = O.solve(cl, K, inc)
            acc += w * O.rcs_monostatic(cl, K, X, inc)[0, 0] / nph
    mean = acc / 2.0
    assert abs(mean - g["value"]) / g["value"] < g["rtol"], mean


# ----------------------------------------------------------------------------- whole-matrix symmetries
def _tiny_cloud(seed=7, nw=12, side=1.5):
    return cloud_uniform_cube(nw, side, seed=seed)


def test_reciprocity_Z_symmetric():
    cl = _tiny_cloud()
    Z = O.assemble(cl, K, None, mirror=False, sparse=False)
    assert np.max(np.abs(Z - Z.T)) / np.max(np.abs(Z)) < 1e-13


def test_translation_invariance_of_Z_and_rcs():
    cl = _tiny_cloud(seed=8)
    sh = Cloud(cl.centres + np.array([3.7, -11.2, 5.5]), cl.dirs, cl.lengths, cl.radii, cl.nseg)
    Z1 = O.assemble(cl, K, None, sparse=False)
    Z2 = O.assemble(sh, K, None, sparse=False)
    assert np.max(np.abs(Z1 - Z2)) / np.max(np.abs(Z1)) < 1e-11
    inc = np.array([[0.4, 0.9, 0.0]])
    obs = np.array([[1.0, 0.3], [2.2, 4.0]])
    s1 = O.rcs_bistatic(cl, K, O.solve_lu(Z1, O.rhs(cl, K, inc)), obs)
    s2 = O.rcs_bistatic(sh, K, O.solve_lu(Z2, O.rhs(sh, K, inc)), obs)
    assert np.allclose(s1, s2, rtol=1e-9)


def test_rotation_covariance_of_far_field():
    cl = _tiny_cloud(seed=9, nw=8)
    th, ax = 0.7, np.array([0.3, -0.5, 0.8])
    ax /= np.linalg.norm(ax)
    Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rm = np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * Kx @ Kx
    rot = Cloud(cl.centres @ Rm.T, cl.dirs @ Rm.T, cl.lengths, cl.radii, cl.nseg)
    inc = np.array([[0.9, 0.2, 0.0]])
    u, khat, e = O.incidence_frames(inc)
    # the rotated problem: incidence rotated with the cloud; build its (theta, phi, psi)
    u2 = Rm @ u[0]
    th2, ph2 = math.acos(u2[2]), math.atan2(u2[1], u2[0])
    _, _, e2 = O.incidence_frames(np.array([[th2, ph2, 0.0]]))
    th_hat2 = e2[0]
    ph_hat2 = np.cross(u2, th_hat2)
    er = Rm @ e[0]
    psi2 = math.atan2(er @ ph_hat2, er @ th_hat2)
    inc2 = np.array([[th2, ph2, psi2]])
    X1, _ = O.solve(cl, K, inc)
    X2, _ = O.solve(rot, K, inc2)
    rhat = np.array([[0.1, 0.8, -0.3]])
    rhat /= np.linalg.norm(rhat)
    F1 = O.far_field(cl, K, X1, rhat)[0, :, 0]
    F2 = O.far_field(rot, K, X2, (Rm @ rhat[0])[None, :])[0, :, 0]
    assert np.allclose(Rm @ F1, F2, rtol=1e-9, atol=1e-12 * np.abs(F1).max())


def test_wire_direction_flip_reverses_current_and_keeps_rcs():
    cl = _tiny_cloud(seed=10, nw=6)
    fl = Cloud(cl.centres.copy(), cl.dirs.copy(), cl.lengths, cl.radii, cl.nseg)
    fl.dirs[2] *= -1.0
    inc = np.array([[0.5, 1.0, 0.3]])
    obs = np.array([[1.2, 0.4], [0.3, 3.0]])
    X1, _ = O.solve(cl, K, inc)
    X2, _ = O.solve(fl, K, inc)
    m, off = O.numbering(cl.nseg)
    a, b = off[2], off[3]
    assert np.allclose(X2[a:b, 0], -X1[a:b, 0][::-1], rtol=1e-9)
    assert np.allclose(O.rcs_bistatic(cl, K, X1, obs), O.rcs_bistatic(fl, K, X2, obs), rtol=1e-9)


def test_bistatic_reciprocity_exact_for_symmetric_Z():
    cl = _tiny_cloud(seed=12, nw=10, side=3.0)
    for r_c in (None, 1.2):
        Z = O.assemble(cl, K, r_c, sparse=False)
        inc_a = np.array([[0.7, 0.4, 0.3]])
        obs = np.array([1.9, 2.5])
        ua, _, ea = O.incidence_frames(inc_a)
        # forward: arrive from u_a, observe at r, receive theta_hat(r)
        r = np.array([math.sin(obs[0]) * math.cos(obs[1]), math.sin(obs[0]) * math.sin(obs[1]), math.cos(obs[0])])
        inc_b = np.array([[obs[0], obs[1], 0.0]])
        _, _, eb = O.incidence_frames(inc_b)
        Xa = O.solve_lu(Z, O.rhs(cl, K, inc_a))
        amp_ab = eb[0] @ O.far_field(cl, K, Xa, r[None, :])[0, :, 0]
        # reverse: arrive from r with polarisation theta_hat(r), observe at u_a, receive e_a
        Xb = O.solve_lu(Z, O.rhs(cl, K, inc_b))
        amp_ba = ea[0] @ O.far_field(cl, K, Xb, ua)[0, :, 0]
        assert abs(amp_ab - amp_ba) < 1e-10 * abs(amp_ab)


def test_optical_theorem_dense():
    """Lossless PEC: extinction (forward amplitude) equals the scattered power integrated over
    the sphere, to quadrature error and the O((ka)^2) of the reduced kernel."""
    cl = cloud_uniform_cube(5, 1.2, seed=13, length=(0.4, 0.55))
    inc = np.array([[0.6, 0.8, 0.5]])
    X, _ = O.solve(cl, K, inc)
    b = O.rhs(cl, K, inc)
    sig_ext = np.imag(np.vdot(b[:, 0], X[:, 0])) / K
    _, khat, e = O.incidence_frames(inc)
    fwd = np.imag(e[0] @ O.far_field(cl, K, X, khat)[0, :, 0]) / K
    assert abs(sig_ext - fwd) < 1e-12 * abs(sig_ext)
    nth, nph = 48, 96
    xt, wt = np.polynomial.legendre.leggauss(nth)
    TH, PH = np.meshgrid(np.arccos(xt), np.arange(nph) * 2 * math.pi / nph, indexing="ij")
    s = O.rcs_bistatic(cl, K, X, np.stack([TH.ravel(), PH.ravel()], 1))[0]
    sig_sca = np.sum(wt[:, None] * (s[:, 0] + s[:, 1]).reshape(nth, nph)) * (2 * math.pi / nph) / (4 * math.pi)
    assert sig_ext > 0
    assert abs(sig_ext - sig_sca) / sig_sca < 1e-3, (sig_ext, sig_sca)


# ----------------------------------------------------------------------------- sparsification and solvers
def test_neighbour_pairs_brute_force_with_exact_ties():
    rng = np.random.default_rng(21)
    c = np.round(rng.uniform(-3, 3, size=(60, 3)) * 4) / 4  # quarter-grid points: many exact ties
    r_c = 1.5
    got = {tuple(x) for x in O.neighbour_pairs(c, r_c)}
    ref = set()
    for p in range(len(c)):
        for q in range(len(c)):
            d = c[p] - c[q]
            if d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= r_c * r_c:
                ref.add((p, q))
    assert got == ref
    ties = [(p, q) for (p, q) in ref if abs(np.sum((c[p] - c[q]) ** 2) - r_c * r_c) == 0.0]
    assert len(ties) > 0  # the inclusive test is exercised


def test_neighbour_pairs_kdtree_branch_on_a_lattice_with_exact_ties():
    """Clouds above PAIRS_BRUTE_MAX wires take the k-d tree branch of the pair search (Eq. neardef):
    checked against an independent enumeration on an integer lattice.  The centres are distinct
    lattice sites scaled by 1/4 (exact in binary), so every squared distance is exact and the pairs
    at exactly r_c (offsets of squared length 9 lattice units, e.g. (3,0,0) and (2,2,1)) must be
    kept; the reference looks each site's lattice offsets of squared length <= 9 up in a table."""
    rng = np.random.default_rng(23)
    side = 36
    nw = O.PAIRS_BRUTE_MAX + 1500
    sites = rng.choice(side ** 3, size=nw, replace=False)
    ijk = np.stack([sites // (side * side), (sites // side) % side, sites % side], axis=1)
    c = ijk.astype(np.float64) * 0.25
    r_c = 0.75  # 3 lattice units
    got = O.neighbour_pairs(c, r_c)
    assert nw > O.PAIRS_BRUTE_MAX
    where = {tuple(v): i for i, v in enumerate(ijk.tolist())}
    offs = [(a, b, d) for a in range(-3, 4) for b in range(-3, 4) for d in range(-3, 4) if a * a + b * b + d * d <= 9]
    ref = []
    for p, (i, j, k) in enumerate(ijk.tolist()):
        for a, b, d in offs:
            q = where.get((i + a, j + b, k + d))
            if q is not None:
                ref.append((p, q))
    ref = np.array(sorted(ref), dtype=np.int64)
    assert got.shape == ref.shape and np.array_equal(got, ref)
    d2 = np.sum((ijk[got[:, 0]] - ijk[got[:, 1]]) ** 2, axis=1)
    assert np.count_nonzero(d2 == 9) > 1000  # the inclusive test is exercised many times


def test_block_jacobi_inverts_each_wires_self_block():
    """block_jacobi (the block-diagonal preconditioner named after Eq. neardef) holds, for every
    wire p of a cloud with mixed segment counts, the inverse of the diagonal block of the assembled
    Z at that wire's unknowns: Z[off_p:off_p+1, off_p:off_p+1] M_p = I.  With r_c below every
    pair distance, Z is block-diagonal, so the right-preconditioned operator Z M^-1 is the identity
    and GMRES converges to the LU solution in a single iteration."""
    rng = np.random.default_rng(24)
    nw = 9
    centres = rng.uniform(-2.0, 2.0, size=(nw, 3))
    dirs = rng.standard_normal((nw, 3))
    lengths = rng.uniform(0.3, 0.6, size=nw)
    nseg = np.array([2, 3, 4, 5, 6, 7, 8, 11, 16], dtype=np.int32)
    cl = _cloud(centres, dirs, lengths, nseg)
    m, off = O.numbering(cl.nseg)
    Z = O.assemble(cl, K, None, sparse=False)
    Mi = O.block_jacobi(cl, K)
    assert len(Mi) == nw
    for p in range(nw):
        a, b = off[p], off[p + 1]
        assert Mi[p].shape == (m[p], m[p])
        I = np.eye(m[p])
        assert np.max(np.abs(Z[a:b, a:b] @ Mi[p] - I)) < 1e-10
        assert np.max(np.abs(Mi[p] @ Z[a:b, a:b] - I)) < 1e-10
    dmin = min(np.linalg.norm(centres[p] - centres[q]) for p in range(nw) for q in range(p))
    Zb = O.assemble(cl, K, 0.5 * dmin, sparse=True)
    b = O.rhs(cl, K, np.array([[0.4, 0.7, 0.2]]))[:, 0]
    x, it, rel = O.gmres(Zb, b, Mi, off, tol=1e-12, restart=10)
    assert it == 1 and rel <= 1e-12
    x_lu = O.solve_lu(Zb.toarray(), b)
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-12


def test_sparse_equals_dense_when_rc_covers_cloud():
    cl = _tiny_cloud(seed=14, nw=10)
    Zd = O.assemble(cl, K, None, sparse=False)
    Zs = O.assemble(cl, K, 10.0, sparse=True).toarray()
    assert np.array_equal(Zd, Zs)


def test_isolated_limit_each_wire_alone():
    cl = cloud_uniform_cube(8, 30.0, seed=15)
    inc = np.array([[0.3, 0.2, 0.0]])
    X, _ = O.solve(cl, K, inc, r_c=1e-3, method="lu")
    m, off = O.numbering(cl.nseg)
    b = O.rhs(cl, K, inc)
    for p in range(cl.nw):
        xp = np.linalg.solve(O.self_block(cl, K, p), b[off[p]:off[p + 1], 0])
        assert np.allclose(X[off[p]:off[p + 1], 0], xp, rtol=1e-12)


def test_gmres_matches_lu_and_stops_at_tolerance():
    cl = cloud_uniform_cube(40, 4.0, seed=16)
    inc = np.array([[0.0, 0.0, 0.0]])
    Z = O.assemble(cl, K, 2.0, sparse=True)
    b = O.rhs(cl, K, inc)[:, 0]
    x_lu = O.solve_lu(Z, b)
    m, off = O.numbering(cl.nseg)
    Mi = O.block_jacobi(cl, K)
    x, it, rel = O.gmres(Z, b, Mi, off, tol=1e-12, restart=10)
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-10
    assert np.linalg.norm(b - Z @ x) / np.linalg.norm(b) < 1e-11
    x6, it6, rel6 = O.gmres(Z, b, Mi, off, tol=1e-6, restart=50)
    assert rel6 <= 1e-6 and np.linalg.norm(b - Z @ x6) / np.linalg.norm(b) < 2e-6 and 0 < it6 < it
    # a restart length of 1 still converges (more slowly) to the same answer
    x1, it1, _ = O.gmres(Z, b, Mi, off, tol=1e-10, restart=1, max_iter=2000)
    assert np.linalg.norm(x1 - x_lu) / np.linalg.norm(x_lu) < 1e-8


def test_gcr_matches_lu_and_restarts():
    """The paper's solver (GCR, Sec. II-B) reaches the LU solution, with and without restarts."""
    cl = cloud_uniform_cube(40, 4.0, seed=16)
    inc = np.array([[0.0, 0.0, 0.0]])
    Z = O.assemble(cl, K, 2.0, sparse=True)
    b = O.rhs(cl, K, inc)[:, 0]
    x_lu = O.solve_lu(Z, b)
    m, off = O.numbering(cl.nseg)
    Mi = O.block_jacobi(cl, K)
    for restart in (50, 4, 1):
        x, it, rel = O.gcr(Z, b, Mi, off, tol=1e-12, restart=restart, max_iter=3000)
        assert rel <= 1e-12
        assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-9
        assert np.linalg.norm(b - Z @ x) / np.linalg.norm(b) < 1e-11


def test_bicgstab_matches_lu_and_terminates_on_two_eigenvalues():
    """BiCGSTAB (the short-recurrence solver of the block-diagonally preconditioned system of
    Sec. II-B): the LU solution of a cloud's sparsified system; one iteration when the
    right-preconditioned operator is the identity (Z block-diagonal, exact block inverses); and at
    most two iterations on an operator with two distinct eigenvalues (its residual polynomial of
    degree two vanishes on both)."""
    cl = cloud_uniform_cube(40, 4.0, seed=16)
    inc = np.array([[0.0, 0.0, 0.0]])
    Z = O.assemble(cl, K, 2.0, sparse=True)
    b = O.rhs(cl, K, inc)[:, 0]
    x_lu = O.solve_lu(Z, b)
    m, off = O.numbering(cl.nseg)
    Mi = O.block_jacobi(cl, K)
    x, it, rel = O.bicgstab(Z, b, Mi, off, tol=1e-12)
    assert rel <= 1e-12 and it > 1
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-10
    assert np.linalg.norm(b - Z @ x) / np.linalg.norm(b) < 1e-11
    # tolerance 1e-6: the true residual is below it, in fewer iterations
    x6, it6, rel6 = O.bicgstab(Z, b, Mi, off, tol=1e-6)
    assert np.linalg.norm(b - Z @ x6) / np.linalg.norm(b) <= 1e-6 and it6 < it
    # identity operator: Z block-diagonal (r_c below every pair distance), M^-1 its exact inverse
    d = np.linalg.norm(cl.centres[:, None] - cl.centres[None], axis=2)
    dmin = d[np.triu_indices(cl.nw, 1)].min()
    Zb = O.assemble(cl, K, 0.5 * dmin, sparse=True)
    xb, itb, relb = O.bicgstab(Zb, b, Mi, off, tol=1e-12)
    assert itb == 1 and relb < 1e-12
    assert np.linalg.norm(xb - O.solve_lu(Zb.toarray(), b)) / np.linalg.norm(xb) < 1e-12
    # two distinct eigenvalues, no preconditioner (1 x 1 identity blocks)
    rng = np.random.default_rng(5)
    n = 12
    V = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 4 * np.eye(n)
    D = np.where(np.arange(n) % 2 == 0, 1.5 + 0.5j, -0.7 + 2.0j)
    A = V @ np.diag(D) @ np.linalg.inv(V)
    rhs2 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ones = [np.eye(1)] * n
    x2, it2, rel2 = O.bicgstab(A, rhs2, ones, np.arange(n + 1), tol=1e-10)
    assert it2 <= 2 and rel2 <= 1e-10
    assert np.linalg.norm(x2 - np.linalg.solve(A, rhs2)) / np.linalg.norm(x2) < 1e-9


def test_bicgstab_first_step_is_galerkin_then_minimal_residual():
    """One BiCGSTAB iteration from zero is the BiCG step (the new residual s = b - alpha A b is
    orthogonal to the shadow residual b) followed by the one-dimensional minimal-residual step
    (r = s - omega A s of least norm): both conditions solved independently (the orthogonality
    by its scalar equation, the least-norm step by numpy's least squares) give the oracle's first
    iterate."""
    rng = np.random.default_rng(6)
    n = 15
    A = np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ones = [np.eye(1)] * n
    x1, it1, _ = O.bicgstab(A, b, ones, np.arange(n + 1), tol=1e-300, max_iter=1)
    assert it1 == 1
    Ab = A @ b
    alpha = (b.conj() @ b) / (b.conj() @ Ab)
    s = b - alpha * Ab
    assert abs(b.conj() @ s) < 1e-12 * np.linalg.norm(b) ** 2
    t = A @ s
    omega = np.linalg.lstsq(t[:, None], s, rcond=None)[0][0]
    r1 = s - omega * t
    assert np.linalg.norm(b - A @ x1 - r1) < 1e-12 * np.linalg.norm(b)
    assert np.linalg.norm(x1 - (alpha * b + omega * s)) < 1e-12 * np.linalg.norm(x1)


def test_gcr_residual_is_the_krylov_least_squares_minimum():
    """After k steps (no restart) the GCR iterate is x_k = M^-1 z_k with z_k minimising
    |b - A M^-1 z| over the Krylov space K_k(A M^-1, b): checked against that definition solved by
    least squares on an explicit, orthonormalised Krylov basis (iterate and residual); GMRES's
    residual estimates are the same numbers."""
    cl = cloud_uniform_cube(30, 4.0, seed=21)
    inc = np.array([[0.4, 1.0, 0.3]])
    Z = O.assemble(cl, K, 2.0, sparse=False)
    b = O.rhs(cl, K, inc)[:, 0]
    m, off = O.numbering(cl.nseg)
    Mi = O.block_jacobi(cl, K)
    N = b.shape[0]
    Mfull = np.zeros((N, N), dtype=complex)
    for p, B in enumerate(Mi):
        Mfull[off[p]:off[p + 1], off[p]:off[p + 1]] = B
    Ap = Z @ Mfull
    kmax = 8
    hist_gcr, hist_gmres = [], []
    O.gcr(Z, b, Mi, off, tol=1e-300, restart=kmax, max_iter=kmax, history=hist_gcr)
    O.gmres(Z, b, Mi, off, tol=1e-300, restart=kmax, max_iter=kmax, history=hist_gmres)
    basis = []
    v = b.copy()
    for k in range(1, kmax + 1):
        for u in basis:  # orthonormal basis of span{b, A'b, ..., A'^(k-1) b}
            v = v - np.vdot(u, v) * u
        basis.append(v / np.linalg.norm(v))
        Kb = np.stack(basis, 1)
        c = np.linalg.lstsq(Ap @ Kb, b, rcond=None)[0]
        rmin = np.linalg.norm(b - Ap @ (Kb @ c)) / np.linalg.norm(b)
        assert abs(hist_gcr[k - 1] - rmin) <= 1e-9 * max(rmin, 1e-3)
        assert abs(hist_gmres[k - 1] - rmin) <= 1e-9 * max(rmin, 1e-3)
        xk, _, _ = O.gcr(Z, b, Mi, off, tol=1e-300, restart=kmax, max_iter=k)
        x_ls = Mfull @ (Kb @ c)
        assert np.linalg.norm(xk - x_ls) <= 1e-8 * np.linalg.norm(x_ls)
        v = Ap @ basis[-1]
    assert hist_gcr[-1] < hist_gcr[0] < 1.0


def test_rcs_error_shrinks_as_rc_grows():
    """Sparsified RCS approaches the entire-coupling RCS as the coupling radius grows (Sec. III-B)."""
    cl = cloud_uniform_cube(60, 5.0, seed=17, length=0.475, nseg=8)
    inc = np.array([[0.0, 0.0, 0.0]])
    obs = np.stack([np.full(36, math.pi / 2), np.arange(36) * 10 * math.pi / 180], 1)
    Xd, _ = O.solve(cl, K, inc)
    sd = O.rcs_bistatic(cl, K, Xd, obs)[0, :, 0]
    errs = []
    for r_c in (0.5, 2.0, 4.0, 6.0):
        Xs, _ = O.solve(cl, K, inc, r_c=r_c)
        ss = O.rcs_bistatic(cl, K, Xs, obs)[0, :, 0]
        errs.append(np.linalg.norm(ss - sd) / np.linalg.norm(sd))
    assert errs[0] > errs[2] and errs[1] > errs[3] and errs[3] < 0.05, errs
