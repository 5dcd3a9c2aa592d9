"""Plain FP64 restatement of the warm-start network (TEST INFRASTRUCTURE ONLY).

The network maps each wire's neighbourhood to a correction of its isolated-wire current, which
then serves as the initial guess of the Krylov solve.  The paper has no such part; this is the
reading the CUDA library implements (csrc/learned.cu), written here a second time, slowly, for the
parity tests.  Everything is a function of rotation-invariant quantities in the wire's own frame,
so the prediction does not change when the cloud and the incidences are rotated together.

Per wire p and incidence (k_hat, e):
  modes: phi_k(i) = sin(k pi (i+1) / n_s), k = 1..3, on the wire's unknowns i = 0..n_s-2;
  isolated amplitudes: a_p,k = (2 / n_s) sum_i x_iso_{p,i} phi_k(i) exp(+j k k_hat.c_p) (the mode
      content of x_iso = Z_pp^-1 b_p with the wire's incident phase removed);
  neighbours: the up to 16 wires q != p with |c_q - c_p| <= r_c, nearest first (ties: lower index);
  neighbour features (16): z/r_c, rho/r_c, t_p.t_q, t_q.d/r_c, L_q/lambda, L_p/lambda, e.t_p,
      k_hat.t_p, e.t_q, k_hat.t_q, cos(k k_hat.d), sin(k k_hat.d), cos(kR), sin(kR), 1/(1+kR), 1
      with d = c_q - c_p, R = |d|, z = d.t_p, rho = sqrt(R^2 - z^2); empty slots are all zero;
  self features (8): e.t_p, k_hat.t_p, L_p/lambda, (number of neighbours)/16, (e.t_p)(k_hat.t_p),
      (k_hat.t_p)^2, 0, 0;
  coupling C_pq = W3 s(W2 s(W1 f_q + b1) + b2) + b3  (s = SiLU, x sigmoid(x)): 18 values, a complex
      3 x 3 matrix (real parts row-major, then imaginary parts);
  h = sum over present slots of C_pq a_q exp(-j k k_hat.d)   (neighbour amplitudes in p's phase);
  output   o = W6 s(W5 s(W4 [Re h, Im h, self, Re a_p, Im a_p] + b4) + b5) + b6 (6 values);
  c_k = h_k + o_k (complex; o as (re, im) pairs);
  x0_{p,i} = x_iso_{p,i} + exp(-j k k_hat.c_p) sum_k c_k phi_k(i).
The correction is linear in the neighbours' isolated currents, as the first-order coupling
-Z_pp^-1 sum_q Z_pq x_iso_q is; the network learns the coupling matrices from the geometry.
Loss: sum |x0 - x_true|^2 / sum |x_true|^2 over wires, unknowns and incidences.
"""
import numpy as np

from .mom import block_jacobi, incidence_frames, numbering, rhs

K_NBR = 16
F_E = 16
F_S = 8
H_MSG = 18
N_MODES = 3
F_OUT_IN = 2 * N_MODES + F_S + 2 * N_MODES  # [Re h, Im h, self, Re a_p, Im a_p]
LAYERS = [(16, 128), (128, 128), (128, 18), (20, 256), (256, 256), (256, 6)]

__all__ = ["K_NBR", "F_E", "F_S", "LAYERS", "unpack", "neighbour_lists", "features", "isolated_currents",
           "amplitudes", "forward", "loss_and_grad"]


def unpack(params):
    """Flat parameter vector -> [(W, b), ...] (views, float64)."""
    p = np.asarray(params, dtype=np.float64)
    out, o = [], 0
    for i, n in LAYERS:
        W = p[o:o + i * n].reshape(i, n)
        o += i * n
        b = p[o:o + n]
        o += n
        out.append((W, b))
    assert o == p.size
    return out


def neighbour_lists(cloud, r_c):
    """Up to K_NBR neighbours q != p with |c_q - c_p| <= r_c, nearest first (ties: lower index);
    -1 pads.  Distances squared formed as (dx^2 + dy^2) + dz^2."""
    c = cloud.centres
    nw = cloud.nw
    out = -np.ones((nw, K_NBR), dtype=np.int64)
    for p in range(nw):
        d = c - c[p]
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        cand = [(d2[q], q) for q in range(nw) if q != p and d2[q] <= r_c * r_c]
        cand.sort()
        for s, (_, q) in enumerate(cand[:K_NBR]):
            out[p, s] = q
    return out


def features(cloud, k, inc, r_c, nbr):
    """Neighbour features Xe (n_inc, nw, K_NBR, F_E) and self features Xs (n_inc, nw, F_S)."""
    _, khat, e = incidence_frames(inc)
    lam = 2.0 * np.pi / k
    ni, nw = khat.shape[0], cloud.nw
    Xe = np.zeros((ni, nw, K_NBR, F_E))
    Xs = np.zeros((ni, nw, F_S))
    t, c, L = cloud.dirs, cloud.centres, cloud.lengths
    for r in range(ni):
        for p in range(nw):
            cnt = 0
            for s in range(K_NBR):
                q = nbr[p, s]
                if q < 0:
                    continue
                cnt += 1
                d = c[q] - c[p]
                R = np.sqrt(d @ d)
                z = d @ t[p]
                rho = np.sqrt(max(R * R - z * z, 0.0))
                ph = k * (khat[r] @ d)
                Xe[r, p, s] = [z / r_c, rho / r_c, t[p] @ t[q], (t[q] @ d) / r_c, L[q] / lam, L[p] / lam,
                               e[r] @ t[p], khat[r] @ t[p], e[r] @ t[q], khat[r] @ t[q], np.cos(ph), np.sin(ph),
                               np.cos(k * R), np.sin(k * R), 1.0 / (1.0 + k * R), 1.0]
            a, b_ = e[r] @ t[p], khat[r] @ t[p]
            Xs[r, p] = [a, b_, L[p] / lam, cnt / K_NBR, a * b_, b_ * b_, 0.0, 0.0]
    return Xe, Xs


def isolated_currents(cloud, k, inc):
    """x_iso = Z_pp^-1 b_p wire by wire, (N, n_inc)."""
    b = rhs(cloud, k, inc)
    m, off = numbering(cloud.nseg)
    Mi = block_jacobi(cloud, k)
    x = np.zeros_like(b)
    for p in range(cloud.nw):
        x[off[p]:off[p + 1]] = Mi[p] @ b[off[p]:off[p + 1]]
    return x


def _silu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return z * s, s


def _modes(cloud):
    """Per wire, the (m_p, N_MODES) matrix sin((k+1) pi (i+1) / n_s)."""
    out = []
    for p in range(cloud.nw):
        ns = int(cloud.nseg[p])
        i = np.arange(1, ns)[:, None]
        kk = np.arange(1, N_MODES + 1)[None, :]
        out.append(np.sin(kk * np.pi * i / ns))
    return out


def amplitudes(cloud, k, inc, x_iso):
    """a (n_inc, nw, 3): mode content of x_iso with each wire's incident phase removed."""
    _, khat, _ = incidence_frames(inc)
    m, off = numbering(cloud.nseg)
    modes = _modes(cloud)
    ni = khat.shape[0]
    a = np.zeros((ni, cloud.nw, N_MODES), dtype=np.complex128)
    for r in range(ni):
        for p in range(cloud.nw):
            ph = np.exp(1j * k * (khat[r] @ cloud.centres[p]))
            a[r, p] = (2.0 / cloud.nseg[p]) * (modes[p].T @ x_iso[off[p]:off[p + 1], r]) * ph
    return a


def forward(params, cloud, k, inc, Xe, Xs, x_iso, nbr):
    """Initial guess x0 (N, n_inc) and the intermediate values backward needs."""
    Ws = unpack(params)
    _, khat, _ = incidence_frames(inc)
    ni, nw = Xe.shape[0], Xe.shape[1]
    pres = Xe[..., F_E - 1]  # 1 for a present slot
    a0 = Xe.reshape(-1, F_E)
    z1 = a0 @ Ws[0][0] + Ws[0][1]
    a1, s1 = _silu(z1)
    z2 = a1 @ Ws[1][0] + Ws[1][1]
    a2, s2 = _silu(z2)
    Cf = (a2 @ Ws[2][0] + Ws[2][1]).reshape(ni, nw, K_NBR, H_MSG)
    Cm = Cf[..., :9].reshape(ni, nw, K_NBR, 3, 3) + 1j * Cf[..., 9:].reshape(ni, nw, K_NBR, 3, 3)
    amp = amplitudes(cloud, k, inc, x_iso)
    # neighbour amplitudes in p's phase: a_q exp(-j k k_hat.d), exp(-j phi) from the features
    rel = np.zeros((ni, nw, K_NBR, N_MODES), dtype=np.complex128)
    for r in range(ni):
        for p in range(nw):
            for s in range(K_NBR):
                q = nbr[p, s]
                if q >= 0:
                    rel[r, p, s] = amp[r, q] * (Xe[r, p, s, 10] - 1j * Xe[r, p, s, 11])
    h = np.einsum("rpskl,rpsl->rpk", Cm * pres[..., None, None], rel)
    u0 = np.concatenate([h.real, h.imag, Xs, amp.real, amp.imag], axis=2).reshape(-1, F_OUT_IN)
    z4 = u0 @ Ws[3][0] + Ws[3][1]
    u1, s4 = _silu(z4)
    z5 = u1 @ Ws[4][0] + Ws[4][1]
    u2, s5 = _silu(z5)
    o = (u2 @ Ws[5][0] + Ws[5][1]).reshape(ni, nw, 2 * N_MODES)
    cmode = h + o[..., 0::2] + 1j * o[..., 1::2]
    m, off = numbering(cloud.nseg)
    modes = _modes(cloud)
    x0 = np.array(x_iso, dtype=np.complex128, copy=True)
    phase = np.exp(-1j * k * (cloud.centres @ khat.T))  # (nw, n_inc)
    for r in range(ni):
        for p in range(nw):
            x0[off[p]:off[p + 1], r] += phase[p, r] * (modes[p] @ cmode[r, p])
    cache = dict(Ws=Ws, a0=a0, a1=a1, s1=s1, z1=z1, a2=a2, s2=s2, z2=z2, pres=pres, rel=rel, u0=u0, u1=u1, s4=s4,
                 z4=z4, u2=u2, s5=s5, z5=z5, phase=phase, modes=modes, off=off, ni=ni, nw=nw)
    return x0, cache


def _silu_back(dy, z, s):
    return dy * (s * (1.0 + z * (1.0 - s)))


def loss_and_grad(params, cloud, k, inc, Xe, Xs, x_iso, x_true, nbr):
    """Normalised squared error of x0 and its gradient with respect to the flat parameters."""
    x0, c = forward(params, cloud, k, inc, Xe, Xs, x_iso, nbr)
    scale = 1.0 / np.sum(np.abs(x_true) ** 2)
    res = x0 - x_true
    loss = float(np.sum(np.abs(res) ** 2) * scale)
    ni, nw, off, Ws = c["ni"], c["nw"], c["off"], c["Ws"]
    # dL/do: o = (Re c_k, Im c_k); x0 = ... + phase * sum_k c_k mode_k
    do = np.zeros((ni, nw, 2 * N_MODES))
    for r in range(ni):
        for p in range(nw):
            g = 2.0 * scale * np.conj(c["phase"][p, r]) * (c["modes"][p].T @ res[off[p]:off[p + 1], r])
            do[r, p, 0::2] = g.real
            do[r, p, 1::2] = g.imag
    do = do.reshape(-1, 2 * N_MODES)
    grads = [None] * 6
    grads[5] = (c["u2"].T @ do, do.sum(0))
    du2 = do @ Ws[5][0].T
    dz5 = _silu_back(du2, c["z5"], c["s5"])
    grads[4] = (c["u1"].T @ dz5, dz5.sum(0))
    du1 = dz5 @ Ws[4][0].T
    dz4 = _silu_back(du1, c["z4"], c["s4"])
    grads[3] = (c["u0"].T @ dz4, dz4.sum(0))
    du0 = (dz4 @ Ws[3][0].T).reshape(ni, nw, F_OUT_IN)
    # h enters both the output MLP and, directly, c: dL/dh = dL/dc + dL/du0[Re h, Im h]
    dh = (do.reshape(ni, nw, 2 * N_MODES)[..., 0::2] + du0[..., :N_MODES]) + \
        1j * (do.reshape(ni, nw, 2 * N_MODES)[..., 1::2] + du0[..., N_MODES:2 * N_MODES])
    # h_k = sum_s pres sum_l C_kl rel_l and dL = Re(conj(dh_k) dh_k-change) with dh = dL/dRe h + j dL/dIm h,
    # so dL/dRe C_kl = Re(conj(dh_k) rel_l) and dL/dIm C_kl = -Im(conj(dh_k) rel_l)
    g = np.conj(dh)[:, :, None, :, None] * c["rel"][:, :, :, None, :] * c["pres"][..., None, None]
    dmsg = np.concatenate([g.real.reshape(ni, nw, K_NBR, 9), -g.imag.reshape(ni, nw, K_NBR, 9)],
                          axis=3).reshape(-1, H_MSG)
    grads[2] = (c["a2"].T @ dmsg, dmsg.sum(0))
    da2 = dmsg @ Ws[2][0].T
    dz2 = _silu_back(da2, c["z2"], c["s2"])
    grads[1] = (c["a1"].T @ dz2, dz2.sum(0))
    da1 = dz2 @ Ws[1][0].T
    dz1 = _silu_back(da1, c["z1"], c["s1"])
    grads[0] = (c["a0"].T @ dz1, dz1.sum(0))
    flat = np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])
    return loss, flat, x0
