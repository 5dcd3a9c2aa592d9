"""Plain FP64 restatement of the thin-wire EFIE method of moments with S-NFC sparsification.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Citations name the paper's sections and
equations (arXiv 2410.03060).

Notation (Sec. II-A).  Wire p has centre c_p, unit direction t_p, length L_p, radius a_p and n_s
segments of length D_p = L_p / n_s.  Its vertices sit at s_i = -L_p/2 + i D_p, i = 0..n_s; the two
end vertices carry no unknown, so the wire has m_p = n_s - 1 rooftop unknowns, one per interior
vertex i = 1..n_s-1 (Eq. "current_expression" and its footnote).  Unknowns are numbered wire by
wire: n(p, i) = off_p + (i - 1).

Scaled system.  Galerkin testing of the EFIE (Eq. "TW_EFIE_MOM", Eqs. (4)-(8)) gives the paper's
Z_paper j = v with v_m = -(j / (w mu0)) int Lambda_m t_m . E_inc.  Writing Z_paper = Z and
multiplying both sides by j w mu0 gives the system this module solves,

    Z jt = b,   b_m = int Lambda_m(s) t_m . E_inc(r(s)) ds,
    Z_mn = (t_m . t_n) int int Lambda_m Lambda_n G  -  (1/k^2) int int Lambda_m' Lambda_n' G,

where Lambda' is the derivative along the wire and G = exp(-j k R) / (4 pi R) with the reduced
thin-wire distance R = sqrt(|r - r'|^2 + a^2).  The physical current is jt / (j w mu0); radar cross
sections do not depend on that factor.  Time convention exp(+j w t) (Sec. I).

Quadrature rule (the paper names only "analytic singularity extraction" and "Gaussian quadrature"
after Eq. (8)); this is the reading both the oracle and the CUDA library follow:
  * different wires: tensor Gauss-Legendre with NQ_FAR = 4 points per segment, or NQ_NEAR = 8 when
    the two wires (as finite line segments) come closer than the longer of their segment lengths;
  * same wire: the double integral over two segments depends only on s - s', so it is reduced
    exactly to a 1-D integral against the convolution of the two linear shape functions, which is
    integrated with SELF_NQ = 8 Gauss-Legendre points on each of its two halves; when the segments
    coincide or touch, the static part 1/(4 pi R) is integrated in closed form and only the smooth
    remainder (exp(-j k R) - 1)/(4 pi R) uses the Gauss rule;
  * radius in mutual terms: a^2 = (a_p^2 + a_q^2) / 2, which keeps Z symmetric.
"""
from __future__ import annotations

import functools
import math

import numpy as np

FOUR_PI = 4.0 * math.pi
ETA0 = 376.730313668  # free-space impedance (ohm) = mu0 * c
NQ_FAR = 4
NQ_NEAR = 8
PAIRS_BRUTE_MAX = 20000  # clouds up to this size test every pair; larger ones take k-d tree candidates
SELF_NQ = 8
RISE, FALL = 0, 1

__all__ = [
    "FOUR_PI", "ETA0", "NQ_FAR", "NQ_NEAR", "PAIRS_BRUTE_MAX", "SELF_NQ", "RISE", "FALL",
    "gauss_legendre_01", "numbering", "vertex_positions", "green",
    "segment_distance", "mutual_order", "mutual_segment_integrals",
    "convolution_poly", "static_antiderivative", "self_offset_integrals", "self_segment_integrals",
    "assemble_block", "mutual_block", "self_block", "block",
    "neighbour_pairs", "block_pattern", "assemble", "block_jacobi",
    "incidence_frames", "triangle_ft", "rhs", "far_field", "rcs_from_far_field",
    "rcs_bistatic", "rcs_monostatic", "solve_lu", "gmres", "gcr", "bicgstab", "solve",
]


# --------------------------------------------------------------------------- quadrature nodes
def gauss_legendre_01(n: int):
    """n-point Gauss-Legendre nodes and weights on [0, 1] (library Legendre roots, mapped)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


# --------------------------------------------------------------------------- discretisation
def numbering(nseg):
    """Unknowns per wire m_p = n_s - 1 and wire offsets off (length nw + 1) of the global index
    n(p, i) = off_p + i - 1 (Sec. II-A, Eq. current_expression and footnote)."""
    m = np.asarray(nseg, dtype=np.int64) - 1
    off = np.zeros(len(m) + 1, dtype=np.int64)
    off[1:] = np.cumsum(m)
    return m, off


def vertex_positions(L: float, ns: int) -> np.ndarray:
    """Arc-length positions s_i = -L/2 + i L/n_s of the n_s + 1 vertices of a wire."""
    return -0.5 * L + np.arange(ns + 1) * (L / ns)


def green(k: float, R):
    """Free-space scalar Green's function exp(-j k R) / (4 pi R) (after Eq. (8))."""
    return np.exp(-1j * k * R) / (FOUR_PI * R)


# --------------------------------------------------------------------------- mutual (different wires)
def segment_distance(cp, tp, Lp, cq, tq, Lq) -> float:
    """Shortest distance between the finite segments c_p + s t_p (|s| <= L_p/2) and
    c_q + s' t_q (|s'| <= L_q/2).  The squared distance is a convex quadratic in (s, s'); its
    minimum over the rectangle is the interior stationary point when that lies inside, else the
    best of the four edges, each minimised by clamping the 1-D optimum."""
    cp, tp, cq, tq = (np.asarray(v, dtype=np.float64) for v in (cp, tp, cq, tq))
    D = cp - cq
    b = float(tp @ tq)
    dp = float(D @ tp)
    dq = float(D @ tq)
    hp, hq = 0.5 * Lp, 0.5 * Lq

    def dist2(s, sq):
        v = D + s * tp - sq * tq
        return float(v @ v)

    cands = []
    det = 1.0 - b * b
    if det > 1e-12:
        s = (b * dq - dp) / det
        sq = (dq - b * dp) / det
        if abs(s) <= hp and abs(sq) <= hq:
            cands.append(dist2(s, sq))
    for s in (-hp, hp):
        sq = min(max(dq + b * s, -hq), hq)
        cands.append(dist2(s, sq))
    for sq in (-hq, hq):
        s = min(max(b * sq - dp, -hp), hp)
        cands.append(dist2(s, sq))
    return math.sqrt(min(cands))


def mutual_order(cloud, p: int, q: int) -> int:
    """Gauss points per segment for the block of wires p != q: NQ_NEAR when the wires come closer
    than the longer segment length, NQ_FAR otherwise."""
    Dp = cloud.lengths[p] / cloud.nseg[p]
    Dq = cloud.lengths[q] / cloud.nseg[q]
    d = segment_distance(cloud.centres[p], cloud.dirs[p], cloud.lengths[p],
                         cloud.centres[q], cloud.dirs[q], cloud.lengths[q])
    return NQ_NEAR if d < max(Dp, Dq) else NQ_FAR


def mutual_segment_integrals(cloud, k: float, p: int, q: int, nq: int | None = None) -> np.ndarray:
    """I[u, v, a, b] = int_{seg u of p} int_{seg v of q} phi_a(s) phi_b(s') G(R) ds' ds for every
    segment pair, by tensor Gauss-Legendre (Eqs. (5)-(8)).  phi_RISE rises from 0 to 1 along the
    segment, phi_FALL falls from 1 to 0."""
    if nq is None:
        nq = mutual_order(cloud, p, q)
    xg, wg = gauss_legendre_01(nq)
    nsp, nsq = int(cloud.nseg[p]), int(cloud.nseg[q])
    Lp, Lq = cloud.lengths[p], cloud.lengths[q]
    Dp, Dq = Lp / nsp, Lq / nsq
    a2 = 0.5 * (cloud.radii[p] ** 2 + cloud.radii[q] ** 2)
    sp = -0.5 * Lp + (np.arange(nsp)[:, None] + xg[None, :]) * Dp  # (nsp, nq)
    sq = -0.5 * Lq + (np.arange(nsq)[:, None] + xg[None, :]) * Dq  # (nsq, nq)
    rp = cloud.centres[p] + sp[..., None] * cloud.dirs[p]  # (nsp, nq, 3)
    rq = cloud.centres[q] + sq[..., None] * cloud.dirs[q]  # (nsq, nq, 3)
    d = rp[:, :, None, None, :] - rq[None, None, :, :, :]
    R = np.sqrt(np.sum(d * d, axis=-1) + a2)  # (nsp, nq, nsq, nq)
    G = green(k, R)
    shape = np.stack([xg, 1.0 - xg])  # (2, nq): rise, fall
    I = np.einsum("ugvh,ag,bh,g,h->uvab", G, shape, shape, wg, wg)
    return I * (Dp * Dq)


# --------------------------------------------------------------------------- self (same wire)
# Convolution of the unit-segment shapes, C_xy(w) = int x^i (x - w)^j dx over x, x - w in [0, 1],
# as polynomial coefficients in w (lowest power first), on w in [-1, 0] and on w in [0, 1].
_CONV_MONOMIAL = {
    # (i, j): (coefficients on [-1, 0], coefficients on [0, 1])
    (0, 0): ([1.0, 1.0], [1.0, -1.0]),
    (1, 0): ([0.5, 1.0, 0.5], [0.5, 0.0, -0.5]),
    (0, 1): ([0.5, 0.0, -0.5], [0.5, -1.0, 0.5]),
    (1, 1): ([1.0 / 3.0, 0.5, 0.0, -1.0 / 6.0], [1.0 / 3.0, -0.5, 0.0, 1.0 / 6.0]),
}


@functools.lru_cache(maxsize=None)
def _conv_coeffs(a: int, b: int, half: int) -> tuple:
    """Coefficients (in w, lowest power first) of W_ab on the given half."""
    P = np.polynomial.Polynomial
    mono = {key: P(val[half]) for key, val in _CONV_MONOMIAL.items()}
    if a == RISE and b == RISE:
        W = mono[(1, 1)]
    elif a == RISE and b == FALL:  # x (1 - (x - w))
        W = mono[(1, 0)] - mono[(1, 1)]
    elif a == FALL and b == RISE:  # (1 - x)(x - w)
        W = mono[(0, 1)] - mono[(1, 1)]
    else:
        W = mono[(0, 0)] - mono[(1, 0)] - mono[(0, 1)] + mono[(1, 1)]
    return tuple(W.coef)


def convolution_poly(a: int, b: int, half: int) -> np.polynomial.Polynomial:
    """W_ab(w) = int_0^1 phi_a(x) phi_b(x - w) dx on half 0 (w in [-1, 0]) or half 1 (w in [0, 1]),
    with phi_RISE(x) = x and phi_FALL(x) = 1 - x."""
    return np.polynomial.Polynomial(_conv_coeffs(a, b, half))


@functools.lru_cache(maxsize=None)
def _conv_coeffs_in_t(a: int, b: int, half: int, delta: int) -> tuple:
    """Coefficients of W_ab(t - delta) as a polynomial in t = delta + w."""
    return tuple(convolution_poly(a, b, half)(np.polynomial.Polynomial([-float(delta), 1.0])).coef)


def static_antiderivative(n: int, t, alpha):
    """Antiderivative of t^n / sqrt(t^2 + alpha^2), n = 0..3."""
    t = np.asarray(t, dtype=np.float64)
    r = np.sqrt(t * t + alpha * alpha)
    if n == 0:
        return np.arcsinh(t / alpha)
    if n == 1:
        return r
    if n == 2:
        return 0.5 * (t * r - alpha * alpha * np.arcsinh(t / alpha))
    if n == 3:
        return (t * t - 2.0 * alpha * alpha) * r / 3.0
    raise ValueError(n)


def self_offset_integrals(k: float, D: float, a: float, delta: int, nq: int = SELF_NQ) -> np.ndarray:
    """I[a, b] for two segments of one wire whose indices differ by delta = u - v.

    With s = s_u + D x and s' = s_v + D y, s - s' = D (delta + w) with w = x - y, so
    I_ab = D^2 int_{-1}^{1} W_ab(w) G(R(w)) dw, R(w) = sqrt(D^2 (delta + w)^2 + a^2).
    For |delta| <= 1 the part 1/(4 pi R) is integrated exactly (in t = delta + w the integrand is
    a cubic over sqrt(t^2 + (a/D)^2)) and the rest by Gauss-Legendre on each half."""
    polyval = np.polynomial.polynomial.polyval
    xg, wg = gauss_legendre_01(nq)
    alpha = a / D
    out = np.zeros((2, 2), dtype=np.complex128)
    for half, (w0, w1) in enumerate(((-1.0, 0.0), (0.0, 1.0))):
        w = w0 + (w1 - w0) * xg
        ww = (w1 - w0) * wg
        R = np.sqrt((D * (delta + w)) ** 2 + a * a)
        if abs(delta) <= 1:
            kern = (np.exp(-1j * k * R) - 1.0) / (FOUR_PI * R)
            prim = [static_antiderivative(n, w1 + delta, alpha) - static_antiderivative(n, w0 + delta, alpha)
                    for n in range(4)]
        else:
            kern = green(k, R)
        for aa in (RISE, FALL):
            for bb in (RISE, FALL):
                val = np.sum(ww * polyval(w, _conv_coeffs(aa, bb, half)) * kern)
                if abs(delta) <= 1:
                    # static part: int W(t - delta) / (4 pi D sqrt(t^2 + alpha^2)) dt
                    ct = _conv_coeffs_in_t(aa, bb, half, int(delta))
                    val = val + sum(c * prim[n] for n, c in enumerate(ct)) / (FOUR_PI * D)
                out[aa, bb] += val
    return out * (D * D)


def self_segment_integrals(cloud, k: float, p: int) -> np.ndarray:
    """I[u, v, a, b] for all segment pairs of wire p with itself."""
    ns = int(cloud.nseg[p])
    D = cloud.lengths[p] / ns
    a = cloud.radii[p]
    table = {d: self_offset_integrals(k, D, a, d) for d in range(-(ns - 1), ns)}
    I = np.zeros((ns, ns, 2, 2), dtype=np.complex128)
    for u in range(ns):
        for v in range(ns):
            I[u, v] = table[u - v]
    return I


# --------------------------------------------------------------------------- block assembly
def assemble_block(I: np.ndarray, tpq: float, Dp: float, Dq: float, k: float) -> np.ndarray:
    """Z block from segment-pair integrals (Eqs. (5)-(8)).  Basis i (1..m) of a wire rises on
    segment i-1 (slope +1/D) and falls on segment i (slope -1/D)."""
    nsp, nsq = I.shape[0], I.shape[1]
    mp, mq = nsp - 1, nsq - 1
    IG = I.sum(axis=(2, 3))
    Z = np.zeros((mp, mq), dtype=np.complex128)
    for i in range(1, nsp):
        for (u, sa, sgn_a) in ((i - 1, RISE, 1.0), (i, FALL, -1.0)):
            for j in range(1, nsq):
                for (v, sb, sgn_b) in ((j - 1, RISE, 1.0), (j, FALL, -1.0)):
                    Z[i - 1, j - 1] += (tpq * I[u, v, sa, sb]
                                        - (sgn_a * sgn_b / (Dp * Dq * k * k)) * IG[u, v])
    return Z


def mutual_block(cloud, k: float, p: int, q: int, nq: int | None = None) -> np.ndarray:
    I = mutual_segment_integrals(cloud, k, p, q, nq)
    tpq = float(cloud.dirs[p] @ cloud.dirs[q])
    return assemble_block(I, tpq, cloud.lengths[p] / cloud.nseg[p], cloud.lengths[q] / cloud.nseg[q], k)


def self_block(cloud, k: float, p: int) -> np.ndarray:
    I = self_segment_integrals(cloud, k, p)
    D = cloud.lengths[p] / cloud.nseg[p]
    return assemble_block(I, 1.0, D, D, k)


def block(cloud, k: float, p: int, q: int) -> np.ndarray:
    """Z_pq, the m_p x m_q block coupling the unknowns of wire p (tested) and wire q (source)."""
    return self_block(cloud, k, p) if p == q else mutual_block(cloud, k, p, q)


# --------------------------------------------------------------------------- sparsification (Sec. II-B)
def neighbour_pairs(centres: np.ndarray, r_c: float) -> np.ndarray:
    """All ordered pairs (p, q), p == q included, whose centroid distance is at most r_c
    (Eq. "neardef": the block is kept iff d(Omega_p, Omega_q) <= d_c).  The squared distance is
    formed as (dx*dx + dy*dy) + dz*dz in float64 and compared with r_c*r_c.  Sorted by (p, q)."""
    c = np.ascontiguousarray(centres, dtype=np.float64)
    nw = c.shape[0]
    rc2 = r_c * r_c
    out = []
    if nw <= PAIRS_BRUTE_MAX:
        cand_rows = None
    else:
        from scipy.spatial import cKDTree  # library range search proposes candidates only
        tree = cKDTree(c)
        cand_rows = tree.query_ball_point(c, r_c * (1.0 + 1e-9) + 1e-12)
    chunk = 256
    for p0 in range(0, nw, chunk):
        p1 = min(nw, p0 + chunk)
        if cand_rows is None:
            dx = c[p0:p1, None, 0] - c[None, :, 0]
            dy = c[p0:p1, None, 1] - c[None, :, 1]
            dz = c[p0:p1, None, 2] - c[None, :, 2]
            d2 = dx * dx + dy * dy + dz * dz
            pi, qi = np.nonzero(d2 <= rc2)
            out.append(np.stack([pi + p0, qi], axis=1))
        else:
            for p in range(p0, p1):
                qs = np.asarray(sorted(cand_rows[p]), dtype=np.int64)
                dx = c[p, 0] - c[qs, 0]
                dy = c[p, 1] - c[qs, 1]
                dz = c[p, 2] - c[qs, 2]
                d2 = dx * dx + dy * dy + dz * dz
                qs = qs[d2 <= rc2]
                out.append(np.stack([np.full(len(qs), p), qs], axis=1))
    pairs = np.concatenate(out, axis=0) if out else np.zeros((0, 2), dtype=np.int64)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    return pairs[order].astype(np.int64)


def block_pattern(cloud, r_c: float | None) -> np.ndarray:
    """Kept blocks: every pair in dense mode (r_c is None), else the S-NFC pairs."""
    nw = cloud.nw
    if r_c is None:
        p, q = np.meshgrid(np.arange(nw), np.arange(nw), indexing="ij")
        return np.stack([p.ravel(), q.ravel()], axis=1).astype(np.int64)
    return neighbour_pairs(cloud.centres, r_c)


def assemble(cloud, k: float, r_c: float | None = None, mirror: bool = False, sparse: bool | None = None):
    """Assemble Z (Eq. TW_EFIE_MOM, sparsified by Eq. neardef when r_c is given).  With
    ``mirror`` the block (q, p) is taken as the transpose of (p, q) instead of being integrated
    again.  Returns a dense array (``sparse`` False) or a scipy CSR matrix."""
    import scipy.sparse as sp

    m, off = numbering(cloud.nseg)
    N = int(off[-1])
    pairs = block_pattern(cloud, r_c)
    if sparse is None:
        sparse = r_c is not None
    cache = {}
    rows, cols, vals = [], [], []
    for p, q in pairs:
        p, q = int(p), int(q)
        if mirror and p > q and (q, p) in cache:
            Zb = cache.pop((q, p)).T
        else:
            Zb = block(cloud, k, p, q)
            if mirror and p < q:
                cache[(p, q)] = Zb
        ri = off[p] + np.arange(m[p])
        ci = off[q] + np.arange(m[q])
        rr, cc = np.meshgrid(ri, ci, indexing="ij")
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        vals.append(Zb.ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    Z = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
    return Z if sparse else Z.toarray()


def block_jacobi(cloud, k: float):
    """Inverses of the self blocks Z_pp (the block-diagonal preconditioner named after Eq. neardef)."""
    return [np.linalg.inv(self_block(cloud, k, p)) for p in range(cloud.nw)]


# --------------------------------------------------------------------------- excitation and far field
def incidence_frames(inc: np.ndarray):
    """For rows (theta, phi, psi): arrival direction u, propagation k_hat = -u, and the polarisation
    e = cos(psi) theta_hat + sin(psi) phi_hat of the spherical frame at (theta, phi)."""
    inc = np.atleast_2d(np.asarray(inc, dtype=np.float64))
    th, ph, psi = inc[:, 0], inc[:, 1], inc[:, 2]
    u = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    th_hat = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], axis=1)
    ph_hat = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], axis=1)
    e = np.cos(psi)[:, None] * th_hat + np.sin(psi)[:, None] * ph_hat
    return u, -u, e


def triangle_ft(beta, D):
    """int_{-D}^{D} (1 - |x|/D) exp(j beta x) dx = D sinc^2(beta D / 2), sinc(z) = sin(z)/z."""
    z = 0.5 * np.asarray(beta, dtype=np.float64) * D
    with np.errstate(invalid="ignore", divide="ignore"):
        s = np.where(np.abs(z) < 1e-8, 1.0 - z * z / 6.0, np.sin(z) / np.where(z == 0, 1.0, z))
    return D * s * s


def rhs(cloud, k: float, inc: np.ndarray) -> np.ndarray:
    """b[n, i] = int Lambda_n(s) t_n . E_inc,i(r(s)) ds for plane waves E = e exp(-j k k_hat . r)
    (Eq. (4) without its -j/(w mu0) factor), in closed form."""
    _, khat, e = incidence_frames(inc)
    m, off = numbering(cloud.nseg)
    b = np.zeros((int(off[-1]), khat.shape[0]), dtype=np.complex128)
    for p in range(cloud.nw):
        ns = int(cloud.nseg[p])
        L = cloud.lengths[p]
        D = L / ns
        s = vertex_positions(L, ns)[1:-1]  # interior vertices
        kt = khat @ cloud.dirs[p]  # (n_inc,)
        et = e @ cloud.dirs[p]
        phase_c = np.exp(-1j * k * (khat @ cloud.centres[p]))
        vals = (et * phase_c * triangle_ft(-k * kt, D))[None, :] * np.exp(-1j * k * s[:, None] * kt[None, :])
        b[off[p]:off[p + 1], :] = vals
    return b


def far_field(cloud, k: float, currents: np.ndarray, rhat: np.ndarray) -> np.ndarray:
    """F[o, :, i] = sum_n j_n,i t_n int Lambda_n(s) exp(+j k rhat_o . r(s)) ds, the radiation
    vector of the currents; the scattered field is E_s = -exp(-j k r) F_perp / (4 pi r)."""
    currents = np.atleast_2d(currents.T).T if currents.ndim == 1 else currents
    rhat = np.atleast_2d(rhat)
    m, off = numbering(cloud.nseg)
    F = np.zeros((rhat.shape[0], 3, currents.shape[1]), dtype=np.complex128)
    for p in range(cloud.nw):
        ns = int(cloud.nseg[p])
        L = cloud.lengths[p]
        D = L / ns
        s = vertex_positions(L, ns)[1:-1]
        rt = rhat @ cloud.dirs[p]  # (n_obs,)
        f = (np.exp(1j * k * (rhat @ cloud.centres[p])) * triangle_ft(k * rt, D))[:, None] \
            * np.exp(1j * k * rt[:, None] * s[None, :])  # (n_obs, m)
        Sp = f @ currents[off[p]:off[p + 1], :]  # (n_obs, n_inc)
        F += Sp[:, None, :] * cloud.dirs[p][None, :, None]
    return F


def rcs_from_far_field(F: np.ndarray, obs: np.ndarray) -> np.ndarray:
    """sigma = |e_s . F|^2 / (4 pi) for e_s = theta_hat and phi_hat at each observation (theta, phi);
    returns (n_obs, 2, n_inc) with [.., 0, ..] theta-received and [.., 1, ..] phi-received."""
    obs = np.atleast_2d(obs)
    th, ph = obs[:, 0], obs[:, 1]
    th_hat = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], axis=1)
    ph_hat = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], axis=1)
    Ft = np.einsum("oc,oci->oi", th_hat, F)
    Fp = np.einsum("oc,oci->oi", ph_hat, F)
    return np.stack([np.abs(Ft) ** 2, np.abs(Fp) ** 2], axis=1) / FOUR_PI


def rcs_bistatic(cloud, k, currents, obs):
    """Bistatic RCS (Sec. III-A): returns (n_inc, n_obs, 2), theta- and phi-received, in lambda^2
    units when the wavelength is 1."""
    obs = np.atleast_2d(obs)
    th, ph = obs[:, 0], obs[:, 1]
    rhat = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    F = far_field(cloud, k, currents, rhat)
    return np.transpose(rcs_from_far_field(F, obs), (2, 0, 1))


def rcs_monostatic(cloud, k, currents, inc):
    """Monostatic RCS (Sec. III-B): observation along each incidence's arrival direction;
    returns (n_inc, 2)."""
    inc = np.atleast_2d(inc)
    out = np.zeros((inc.shape[0], 2))
    for i in range(inc.shape[0]):
        s = rcs_bistatic(cloud, k, currents[:, i:i + 1], inc[i:i + 1, :2])
        out[i] = s[0, 0]
    return out


# --------------------------------------------------------------------------- solvers
def solve_lu(Z, b):
    """Direct solve (the 'entire coupling (LU)' reference of Sec. III)."""
    Zd = Z.toarray() if hasattr(Z, "toarray") else Z
    return np.linalg.solve(Zd, b)


def gmres(A, b: np.ndarray, Minv_blocks, off, tol: float = 1e-6, restart: int = 50,
          max_iter: int = 1000, x0=None, history=None):
    """Restarted GMRES with right block-Jacobi preconditioning, modified Gram-Schmidt and complex
    Givens rotations, in float64.  Solves A x = b for one right-hand side.  The paper uses GCR
    with a block-diagonal preconditioner (after Eq. neardef); GMRES minimises the same residual
    over the same Krylov space and reaches the same solution to tolerance.
    Returns (x, iterations, relative residual estimate); ``history`` (a list) receives the
    residual estimate after every iteration."""
    b = np.asarray(b, dtype=np.complex128)
    N = b.shape[0]

    def Minv(v):
        z = np.empty_like(v)
        for p, Mi in enumerate(Minv_blocks):
            z[off[p]:off[p + 1]] = Mi @ v[off[p]:off[p + 1]]
        return z

    x = np.zeros(N, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    rel = 1.0
    while True:
        r = b - A @ x
        beta = np.linalg.norm(r)
        rel = beta / bnorm
        if rel <= tol or it >= max_iter:
            return x, it, rel
        V = np.zeros((restart + 1, N), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        jlast = -1
        for j in range(restart):
            w = A @ Minv(V[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):  # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a_, b_ = H[j, j], H[j + 1, j]
            nu = math.hypot(abs(a_), abs(b_))
            if abs(a_) == 0.0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a_) / nu
                sn[j] = (a_ / abs(a_)) * np.conj(b_) / nu
            H[j, j] = cs[j] * a_ + sn[j] * b_
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            jlast = j
            rel = abs(g[j + 1]) / bnorm
            if history is not None:
                history.append(rel)
            if rel <= tol or it >= max_iter or H[j, j] == 0.0:
                break
        n = jlast + 1
        y = np.zeros(n, dtype=np.complex128)
        for i in range(n - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:n] @ y[i + 1:n]) / H[i, i]
        x = x + Minv(V[:n].T @ y)


def gcr(A, b: np.ndarray, Minv_blocks, off, tol: float = 1e-6, restart: int = 50,
        max_iter: int = 1000, x0=None, history=None):
    """Restarted GCR, the Krylov method the paper names (Sec. II-B, after Eq. neardef), with right
    block-Jacobi preconditioning, in float64, for one right-hand side of A x = b.

    Each step takes the search direction p = M^-1 r from the current residual and its image
    q = A p, makes q orthogonal to the earlier images q_i (modified Gram-Schmidt, with the same
    combination applied to p so that q = A p still holds), scales both so |q| = 1, and then moves
    x along p by the coefficient alpha = q^H r that removes the q-component of the residual:
    x += alpha p, r -= alpha q.  After k steps r is the smallest residual over the Krylov space of
    dimension k, as in GMRES.  Every ``restart`` steps the bases are dropped and r is recomputed
    as b - A x.  Returns (x, iterations, relative residual); ``history`` receives |r|/|b| after
    every step."""
    b = np.asarray(b, dtype=np.complex128)
    N = b.shape[0]

    def Minv(v):
        z = np.empty_like(v)
        for p, Mi in enumerate(Minv_blocks):
            z[off[p]:off[p + 1]] = Mi @ v[off[p]:off[p + 1]]
        return z

    x = np.zeros(N, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    while True:
        r = b - A @ x
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol or it >= max_iter:
            return x, it, rel
        P, Q = [], []
        for _ in range(restart):
            p = Minv(r)
            q = A @ p
            for pi, qi in zip(P, Q):
                beta = np.vdot(qi, q)
                q = q - beta * qi
                p = p - beta * pi
            nq = np.linalg.norm(q)
            if nq == 0.0:
                break
            q, p = q / nq, p / nq
            alpha = np.vdot(q, r)
            x = x + alpha * p
            r = r - alpha * q
            P.append(p)
            Q.append(q)
            it += 1
            rel = np.linalg.norm(r) / bnorm
            if history is not None:
                history.append(rel)
            if rel <= tol or it >= max_iter:
                break


def bicgstab(A, b: np.ndarray, Minv_blocks, off, tol: float = 1e-6, max_iter: int = 1000, x0=None,
             history=None):
    """BiCGSTAB (van der Vorst, SIAM J. Sci. Stat. Comput. 13 (1992) 631) with right block-Jacobi
    preconditioning, in float64, for one right-hand side of A x = b: a short-recurrence Krylov
    solver for the block-diagonally preconditioned system of Sec. II-B, whose cost per step is two
    products and a fixed number of vector operations (no basis is stored).

    On the right-preconditioned system (A M^-1) y = b, x = M^-1 y, starting from y = 0, r = b and
    the shadow residual rh = r; each iteration (two products):
        rho = rh^H r,  beta = (rho / rho_prev) (alpha / omega),  p = r + beta (p - omega v),
        v = A M^-1 p,  alpha = rho / (rh^H v),  s = r - alpha v,
        t = A M^-1 s,  omega = (t^H s) / (t^H t),  y += alpha p + omega s,  r = s - omega t.
    The iteration stops when the recursive residual |r| <= tol |b|; the true residual b - A x is
    then formed, and if it still exceeds tol |b| (the recursion drifted) the method restarts from
    it with rh = r.  A breakdown (rho, rh^H v or t^H t equal to zero) restarts the same way.
    Returns (x, iterations, true relative residual); ``history`` receives |r|/|b| after every
    iteration."""
    b = np.asarray(b, dtype=np.complex128)
    N = b.shape[0]

    def Minv(v):
        z = np.empty_like(v)
        for p, Mi in enumerate(Minv_blocks):
            z[off[p]:off[p + 1]] = Mi @ v[off[p]:off[p + 1]]
        return z

    def op(v):
        return A @ Minv(v)

    bnorm = np.linalg.norm(b)
    x = np.zeros(N, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    if bnorm == 0.0:
        return x, 0, 0.0
    y = np.zeros(N, dtype=np.complex128)  # x = x_start + M^-1 y
    x_start = x.copy()
    it = 0
    while True:
        r = b - A @ (x_start + Minv(y))
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol or it >= max_iter:
            return x_start + Minv(y), it, rel
        rh = r.copy()
        rho_prev = alpha = omega = 1.0 + 0.0j
        p = np.zeros(N, dtype=np.complex128)
        v = np.zeros(N, dtype=np.complex128)
        while it < max_iter:
            rho = np.vdot(rh, r)
            if rho == 0.0:
                break
            beta = (rho / rho_prev) * (alpha / omega)
            p = r + beta * (p - omega * v)
            v = op(p)
            rv = np.vdot(rh, v)
            if rv == 0.0:
                break
            alpha = rho / rv
            s = r - alpha * v
            t = op(s)
            tt = np.vdot(t, t).real
            if tt == 0.0:
                y = y + alpha * p
                it += 1
                break
            omega = np.vdot(t, s) / tt
            y = y + alpha * p + omega * s
            r = s - omega * t
            rho_prev = rho
            it += 1
            rel = np.linalg.norm(r) / bnorm
            if history is not None:
                history.append(rel)
            if rel <= tol or omega == 0.0:
                break


def solve(cloud, k: float, inc: np.ndarray, r_c: float | None = None, method: str = "lu",
          tol: float = 1e-6, restart: int = 50, max_iter: int = 1000):
    """Currents jt (N x n_inc) of Z jt = b for each incidence.  ``method`` 'lu', 'gmres', 'gcr' or
    'bicgstab'."""
    Z = assemble(cloud, k, r_c, sparse=(method != "lu"))
    b = rhs(cloud, k, inc)
    if method == "lu":
        return solve_lu(Z, b), {"iterations": 0}
    m, off = numbering(cloud.nseg)
    Mi = block_jacobi(cloud, k)
    X = np.zeros_like(b)
    its = []
    for i in range(b.shape[1]):
        if method == "bicgstab":
            X[:, i], it, rel = bicgstab(Z, b[:, i], Mi, off, tol, max_iter)
        else:
            krylov = gcr if method == "gcr" else gmres
            X[:, i], it, rel = krylov(Z, b[:, i], Mi, off, tol, restart, max_iter)
        its.append(it)
    return X, {"iterations": its}
