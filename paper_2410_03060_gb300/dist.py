"""One wire cloud split over ranks: spatial partition, halo plan, communicator and the restarted
GMRES that runs on it.

The S-NFC system keeps only the blocks of wire pairs whose centroids are within r_c (Sec. II-B,
Eq. neardef), so the rows of the right-preconditioned operator A = Z M^-1 = I + E that belong to a
set of wires need the current vector on those wires and on the wires within r_c of them (the
halo) and nothing else.  A rank owns a contiguous range of wires in Morton order of their r_c
cells, holds its own wires and a read-only copy of its halo's geometry (enough to fill its rows of
Z and the halo's self blocks), and per product receives the halo's current values from their
owners: one point-to-point exchange with the ranks that own a halo wire.  The Krylov method needs
the inner products summed over the ranks (one all-reduce per Gram-Schmidt pass) and the far field
summed over the ranks (one all-reduce of the received components, Sec. III-A).

Everything here is host logic: the partition and the exchange plan are computed identically on
every rank from the full list of centres, the communicator moves host arrays, and the numerical
work goes through an ``ops`` object -- :class:`SwmOps` runs it in the library's kernels through
the C ABI (device vectors), one context per rank.  The Hessenberg least-squares problem of GMRES
(at most restart + 1 by restart per incidence) is solved on the host by Givens rotations.
"""
from __future__ import annotations

import math
import threading

import numpy as np


# ------------------------------------------------------------------------------------ partition
def _spread_bits(v: np.ndarray) -> np.ndarray:
    """Insert two zero bits between the low 21 bits of v (Morton interleave helper)."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_order(centres: np.ndarray, cell: float) -> np.ndarray:
    """Wire indices sorted by the Morton code of their cell (cells of side ``cell`` from the
    bounding box corner), ties by index."""
    c = np.asarray(centres, dtype=np.float64)
    ijk = np.floor((c - c.min(axis=0)) / cell).astype(np.int64)
    code = _spread_bits(ijk[:, 0]) | (_spread_bits(ijk[:, 1]) << np.uint64(1)) | (_spread_bits(ijk[:, 2]) << np.uint64(2))
    return np.lexsort((np.arange(len(c)), code))


def partition(centres: np.ndarray, nseg: np.ndarray, n_ranks: int, r_c: float) -> np.ndarray:
    """Owner rank of every wire: contiguous ranges of the Morton order with about equal numbers of
    unknowns (n_s - 1 per wire)."""
    order = morton_order(centres, r_c)
    m = np.asarray(nseg, dtype=np.int64)[order] - 1
    cum = np.cumsum(m)
    total = int(cum[-1]) if len(cum) else 0
    owner = np.empty(len(order), dtype=np.int64)
    # wire i of the order goes to the rank whose share of the unknowns its first unknown falls in
    first = cum - m
    owner[order] = np.minimum(n_ranks - 1, (first * n_ranks) // max(1, total))
    return owner


def within(centres: np.ndarray, a: np.ndarray, b: np.ndarray, r_c: float) -> np.ndarray:
    """Pairs (a[i], b[i]) whose centroid distance is at most r_c, the squared distance formed as
    (dx*dx + dy*dy) + dz*dz (the form the library's pair search uses)."""
    d = centres[a] - centres[b]
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2] <= r_c * r_c


class Plan:
    """The wires of one rank and its halo exchange, computed from the full cloud.

    ``wires``: global ids of the local wires, the owned ones first (ascending), then the halo
    (ascending).  ``n_own_wires``, ``n_own`` (owned unknowns), ``n_loc`` (local unknowns).
    ``recv[s]``: local unknown positions (in the halo part) filled from rank s, in the order rank s
    sends them; ``send[s]``: local unknown positions of owned unknowns sent to rank s."""

    def __init__(self, centres, nseg, owner, rank, r_c):
        from scipy.spatial import cKDTree  # candidate neighbours only; the test above decides

        centres = np.asarray(centres, dtype=np.float64)
        nseg = np.asarray(nseg)
        self.rank, self.size = int(rank), int(owner.max()) + 1 if len(owner) else 1
        tree = cKDTree(centres)
        halos = []
        for s in range(self.size):
            own = np.nonzero(owner == s)[0]
            cand = tree.query_ball_point(centres[own], r_c * (1.0 + 1e-9) + 1e-12)
            pa = np.repeat(own, [len(c) for c in cand])
            pb = np.concatenate([np.asarray(c, dtype=np.int64) for c in cand]) if len(cand) else np.zeros(0, np.int64)
            keep = (owner[pb] != s) & within(centres, pa, pb, r_c)
            halos.append(np.unique(pb[keep]))
        own = np.nonzero(owner == rank)[0]
        halo = halos[rank]
        self.wires = np.concatenate([own, halo]).astype(np.int64)
        self.n_own_wires = len(own)
        m = nseg[self.wires].astype(np.int64) - 1
        self.off = np.zeros(len(self.wires) + 1, dtype=np.int64)
        self.off[1:] = np.cumsum(m)
        self.n_own = int(self.off[self.n_own_wires])
        self.n_loc = int(self.off[-1])
        pos = {int(w): i for i, w in enumerate(self.wires)}

        def unknowns(local_ids):
            return np.concatenate([np.arange(self.off[i], self.off[i + 1]) for i in local_ids]) \
                if len(local_ids) else np.zeros(0, dtype=np.int64)

        self.recv, self.send = {}, {}
        for s in range(self.size):
            if s == rank:
                continue
            need = halo[owner[halo] == s]  # ascending global ids
            if len(need):
                self.recv[s] = unknowns([pos[int(w)] for w in need])
            give = halos[s][owner[halos[s]] == rank]  # ascending global ids, as rank s receives them
            if len(give):
                self.send[s] = unknowns([pos[int(w)] for w in give])


# ------------------------------------------------------------------------------------ communicators
class Comm:
    """What the solver needs from the ranks: sums and a point-to-point exchange of host arrays."""

    rank = 0
    size = 1

    def allreduce_sum(self, a: np.ndarray) -> np.ndarray:
        raise NotImplementedError

    def exchange(self, sends: dict, recv_sizes: dict) -> dict:
        """Send sends[s] (a complex array) to rank s for every key and receive recv_sizes[s]
        complex values from every rank s in recv_sizes; returns {s: received flat array}."""
        raise NotImplementedError


class LocalComm(Comm):
    """A single rank: sums are the identity and nothing is exchanged."""

    def allreduce_sum(self, a):
        return np.array(a, copy=True)

    def exchange(self, sends, recv_sizes=None):
        if sends or recv_sizes:
            raise ValueError("a single rank has no peers")
        return {}


class TorchComm(Comm):
    """torch.distributed (gloo or NCCL) with host staging: sums by all_reduce, the halo by
    point-to-point isend/irecv with the peers only."""

    def __init__(self):
        import torch.distributed as dist

        self.dist = dist
        self.rank = dist.get_rank()
        self.size = dist.get_world_size()
        self.backend = dist.get_backend()

    def _t(self, a):
        import torch

        t = torch.from_numpy(np.ascontiguousarray(a))
        return t.cuda() if self.backend == "nccl" else t

    def allreduce_sum(self, a):
        a = np.asarray(a)
        if np.iscomplexobj(a):
            flat = np.ascontiguousarray(a).view(np.float64)
            t = self._t(flat)
            self.dist.all_reduce(t)
            return t.cpu().numpy().view(np.complex128).reshape(a.shape)
        t = self._t(np.asarray(a, dtype=np.float64))
        self.dist.all_reduce(t)
        return t.cpu().numpy().reshape(a.shape)

    def exchange(self, sends, recv_sizes=None):
        import torch

        reqs, bufs = [], {}
        for s, n in (recv_sizes or {}).items():
            buf = torch.empty(2 * n, dtype=torch.float64, device="cuda" if self.backend == "nccl" else "cpu")
            bufs[s] = buf
            reqs.append(self.dist.irecv(buf, src=s))
        for s, a in sends.items():
            reqs.append(self.dist.isend(self._t(np.ascontiguousarray(a, dtype=np.complex128).view(np.float64)), dst=s))
        for r in reqs:
            r.wait()
        return {s: b.cpu().numpy().view(np.complex128) for s, b in bufs.items()}


class ThreadComm(Comm):
    """Ranks as host threads of one process (tests, or several contexts on one device).  Only host
    arrays move between the threads; no kernel of one rank waits on another rank's."""

    class _Shared:
        def __init__(self, size):
            self.size = size
            self.barrier = threading.Barrier(size)
            self.slots = [None] * size
            self.mail = {}

    def __init__(self, shared, rank):
        self.sh = shared
        self.rank = rank
        self.size = shared.size

    @classmethod
    def group(cls, size):
        sh = cls._Shared(size)
        return [cls(sh, r) for r in range(size)]

    def allreduce_sum(self, a):
        a = np.asarray(a)
        self.sh.slots[self.rank] = np.array(a, copy=True)
        self.sh.barrier.wait()
        out = self.sh.slots[0].copy()
        for r in range(1, self.size):
            out = out + self.sh.slots[r]  # same order on every rank
        self.sh.barrier.wait()
        return out

    def exchange(self, sends, recv_sizes=None):
        for s, a in sends.items():
            self.sh.mail[(self.rank, s)] = np.array(a, copy=True)
        self.sh.barrier.wait()
        got = {s: self.sh.mail[(s, self.rank)] for s in (recv_sizes or {})}
        self.sh.barrier.wait()
        for s in sends:
            self.sh.mail.pop((self.rank, s), None)
        self.sh.barrier.wait()
        return got


def _exchange(comm, plan, sends, n_rhs):
    """Halo exchange of one vector: complex values, n_rhs x (unknowns) per peer."""
    if isinstance(comm, LocalComm):
        return {}
    sizes = {s: n_rhs * len(idx) for s, idx in plan.recv.items()}
    return comm.exchange(sends, sizes)


# ------------------------------------------------------------------------------------ GMRES
def dist_gmres(ops, comm, plan, b_own, tol=1e-6, restart=50, max_iter=1000, history=None):
    """Restarted GMRES, right block-Jacobi preconditioned (Sec. II-B), on the owned rows of every
    rank: y with A y = b, A = I + E; classical Gram-Schmidt with a second pass (inner products
    summed over the ranks), Givens rotations of each incidence's Hessenberg column on the host.
    ``b_own``: the ops' vector of the owned right-hand sides (n_rhs x n_own).  Returns (y_own,
    iterations, relative residuals of the last restart's true residual)."""
    R = ops.n_rhs
    bn = np.sqrt(comm.allreduce_sum(ops.norms2(b_own)))
    bn = np.where(bn > 0, bn, 1.0)
    y = ops.zeros()
    it = 0
    rel = np.ones(R)

    def product(v_own):
        sends = {s: ops.take(v_own, idx) for s, idx in plan.send.items()}
        got = _exchange(comm, plan, sends, R)
        return ops.apply(v_own, {s: (plan.recv[s], vals) for s, vals in got.items()})

    while True:
        r = ops.sub(b_own, product(y))
        rn = np.sqrt(comm.allreduce_sum(ops.norms2(r)))
        rel = rn / bn
        if history is not None:
            history.append(rel.copy())
        active = rel > tol
        if not active.any() or it >= max_iter:
            return y, it, rel
        beta = np.where(active, rn, 0.0)
        Vb = ops.basis(restart + 1)  # restart + 1 vectors of n_rhs x n_own
        ops.put(Vb, 0, ops.scale(r, np.where(active, 1.0 / np.where(rn > 0, rn, 1.0), 0.0)))
        H = np.zeros((restart + 1, restart, R), dtype=np.complex128)
        cs = np.zeros((restart, R))
        sn = np.zeros((restart, R), dtype=np.complex128)
        g = np.zeros((restart + 1, R), dtype=np.complex128)
        g[0] = beta
        jlast = np.zeros(R, dtype=np.int64)
        j = 0
        while j < restart and it < max_iter and active.any():
            w = product(ops.get(Vb, j))
            h = comm.allreduce_sum(ops.dots(Vb, j + 1, w))  # (j + 1) x R
            w = ops.axpy(Vb, j + 1, h, w)
            h2 = comm.allreduce_sum(ops.dots(Vb, j + 1, w))
            w = ops.axpy(Vb, j + 1, h2, w)
            h = h + h2
            nrm = np.sqrt(comm.allreduce_sum(ops.norms2(w)))
            col = np.zeros((j + 2, R), dtype=np.complex128)
            col[:j + 1] = h
            col[j + 1] = nrm
            for i in range(j):  # earlier rotations
                a, b = col[i].copy(), col[i + 1].copy()
                col[i] = cs[i] * a + sn[i] * b
                col[i + 1] = -np.conj(sn[i]) * a + cs[i] * b
            a = col[j]
            aa = np.abs(a)
            nu = np.sqrt(aa * aa + nrm * nrm)
            safe_nu = np.where(nu > 0, nu, 1.0)
            c = np.where(aa > 0, aa / safe_nu, 0.0)
            s = np.where(aa > 0, (a / np.where(aa > 0, aa, 1.0)) * nrm / safe_nu, 1.0 + 0j)
            cs[j], sn[j] = c, s
            col[j] = c * a + s * nrm
            col[j + 1] = 0.0
            H[:j + 2, j] = np.where(active, col, 0.0)
            gj = g[j].copy()
            g[j + 1] = np.where(active, -np.conj(s) * gj, g[j + 1])
            g[j] = np.where(active, c * gj, g[j])
            jlast = np.where(active, j + 1, jlast)
            est = np.abs(g[j + 1]) / bn
            it += 1
            j += 1
            active = active & (est > tol) & (nrm > 0)
            if j < restart:
                ops.put(Vb, j, ops.scale(w, np.where(nrm > 0, 1.0 / np.where(nrm > 0, nrm, 1.0), 0.0)))
        # y += sum_i c_i V_i, c from the triangular system of each incidence's rotated columns
        coef = np.zeros((j, R), dtype=np.complex128)
        for q in range(R):
            k = int(jlast[q])
            if k == 0:
                continue
            coef[:k, q] = np.linalg.solve(np.triu(H[:k, :k, q]), g[:k, q])
        if j > 0:
            y = ops.axpy(Vb, j, -coef, y)


def _block_qr(ops, comm, W):
    """W = V Rf with V orthonormal (columns = the block's vectors) by Cholesky QR twice: the Gram
    matrix is summed over the ranks, its Cholesky factor inverted on the host (at most a few tens
    of columns).  Returns (V, Rf) or (None, None) when the block is numerically rank deficient."""
    Rf = np.eye(ops.n_rhs, dtype=np.complex128)
    V = W
    for _ in range(2):
        G = comm.allreduce_sum(ops.gram(ops.as_basis(V), 1, V))  # G[a, b] = V_a^H V_b
        G = 0.5 * (G + G.conj().T)
        try:
            L = np.linalg.cholesky(G)
        except np.linalg.LinAlgError:
            return None, None
        Rk = L.conj().T  # V = Vn Rk
        if np.min(np.abs(np.diag(Rk))) <= 1e-13 * np.max(np.abs(np.diag(Rk))):
            return None, None
        V = ops.gemm(ops.as_basis(V), 1, -np.linalg.inv(Rk), ops.zeros())  # 0 - V (-Rk^-1)
        Rf = Rk @ Rf
    return V, Rf


def dist_block_gmres(ops, comm, plan, b_own, tol=1e-6, restart=10, max_iter=1000, history=None):
    """Restarted block GMRES (one Krylov space shared by all n_rhs right-hand sides of ``ops``),
    right block-Jacobi preconditioned like :func:`dist_gmres`: block Arnoldi with classical block
    Gram-Schmidt and a second pass (block inner products summed over the ranks), Cholesky QR twice
    for each new block, and the block Hessenberg least-squares problem solved on the host.  Every
    right-hand side stops at the first cycle boundary after all of them meet tol (their columns
    share the space).  Returns (y_own, block iterations, relative residuals)."""
    R = ops.n_rhs
    bn = np.sqrt(comm.allreduce_sum(ops.norms2(b_own)))
    bn = np.where(bn > 0, bn, 1.0)
    y = ops.zeros()
    it = 0

    def product(v_own):
        sends = {s: ops.take(v_own, idx) for s, idx in plan.send.items()}
        got = _exchange(comm, plan, sends, R)
        return ops.apply(v_own, {s: (plan.recv[s], vals) for s, vals in got.items()})

    while True:
        r = ops.sub(b_own, product(y))
        rn = np.sqrt(comm.allreduce_sum(ops.norms2(r)))
        rel = rn / bn
        if history is not None:
            history.append(rel.copy())
        if not (rel > tol).any() or it >= max_iter:
            return y, it, rel
        V0, beta = _block_qr(ops, comm, r)
        if V0 is None:
            return y, it, rel
        Vb = ops.basis(restart + 1)
        ops.put(Vb, 0, V0)
        H = np.zeros(((restart + 1) * R, restart * R), dtype=np.complex128)
        rhs = np.zeros(((restart + 1) * R, R), dtype=np.complex128)
        rhs[:R] = beta
        Z, j = None, 0
        while j < restart and it < max_iter:
            W = product(ops.get(Vb, j))
            h = comm.allreduce_sum(ops.gram(Vb, j + 1, W))  # ((j+1) R) x R
            W = ops.gemm(Vb, j + 1, h, W)
            h2 = comm.allreduce_sum(ops.gram(Vb, j + 1, W))
            W = ops.gemm(Vb, j + 1, h2, W)
            H[:(j + 1) * R, j * R:(j + 1) * R] = h + h2
            Vn, Rn = _block_qr(ops, comm, W)
            if Vn is None:  # the block space stopped growing: solve with what there is
                j += 1
                it += 1
                Z = np.linalg.lstsq(H[:(j + 1) * R, :j * R], rhs[:(j + 1) * R], rcond=None)[0]
                break
            H[(j + 1) * R:(j + 2) * R, j * R:(j + 1) * R] = Rn
            j += 1
            it += 1
            Hj = H[:(j + 1) * R, :j * R]
            Z = np.linalg.lstsq(Hj, rhs[:(j + 1) * R], rcond=None)[0]
            est = np.linalg.norm(rhs[:(j + 1) * R] - Hj @ Z, axis=0) / bn
            if j < restart:
                ops.put(Vb, j, Vn)
            if not (est > tol).any():
                break
        if Z is not None and j > 0:
            # y += sum over blocks i of V_i Z_i, Z_i the rows i R .. (i+1) R of Z
            y = ops.gemm(Vb, j, -Z[:j * R], y)


# ------------------------------------------------------------------------------------ device ops
class SwmOps:
    """The numerical steps of :func:`dist_gmres` on one rank, in the library's kernels: a context
    holding the rank's wires (owned then halo) built with its S-NFC rows; vectors are CUDA complex128
    tensors (n_rhs x unknowns), inner products and updates by swm_vec_*, the product by swm_apply,
    the preconditioner by swm_precond_apply, right-hand sides by swm_rhs, far-field components by
    swm_far_components."""

    def __init__(self, ctx, plan, n_rhs):
        import torch

        self.torch = torch
        self.ctx, self.plan, self.n_rhs = ctx, plan, n_rhs

    def _lib(self):
        from . import swm
        return swm

    def zeros(self):
        return self.torch.zeros((self.n_rhs, self.plan.n_own), dtype=self.torch.complex128, device="cuda")

    def basis(self, k):
        return self.torch.zeros((k, self.n_rhs, self.plan.n_own), dtype=self.torch.complex128, device="cuda")

    def put(self, Vb, j, v):
        Vb[j].copy_(v)

    def get(self, Vb, j):
        return Vb[j]

    def take(self, v, idx):
        return v[:, self.torch.from_numpy(idx).cuda()].cpu().numpy()

    def apply(self, v_own, halo):
        torch = self.torch
        x = torch.zeros((self.n_rhs, self.plan.n_loc), dtype=torch.complex128, device="cuda")
        x[:, :self.plan.n_own] = v_own
        for _, (pos, vals) in halo.items():
            x[:, torch.from_numpy(pos).cuda()] = torch.from_numpy(np.asarray(vals).reshape(self.n_rhs, -1)).cuda()
        y = torch.empty_like(x)
        self._lib().swm_apply(self.ctx, x, y)
        return y[:, :self.plan.n_own].contiguous()

    def sub(self, a, b):
        out = a.clone()
        self._lib().swm_vec_axpy(self.ctx, b.unsqueeze(0), 1, np.ones((1, self.n_rhs), dtype=np.complex128), out)
        return out

    def norms2(self, v):
        return np.real(self._lib().swm_vec_dots(self.ctx, v.unsqueeze(0), 1, v)[0])

    def dots(self, Vb, k, w):
        return self._lib().swm_vec_dots(self.ctx, Vb, k, w)

    def axpy(self, Vb, k, coef, v):
        out = v.clone()
        self._lib().swm_vec_axpy(self.ctx, Vb, k, coef, out)
        return out

    def scale(self, v, a):
        out = self.torch.empty_like(v)
        self._lib().swm_vec_scale(self.ctx, np.asarray(a, dtype=np.float64), v, out)
        return out

    def as_basis(self, v):
        return v.unsqueeze(0)

    def gram(self, Vb, k, w):
        """((k n_rhs) x n_rhs) inner products of every basis vector of the first k blocks with
        every vector of w."""
        return self._lib().swm_vec_gram(self.ctx, Vb, k, w)

    def gemm(self, Vb, k, C, w):
        """w - (first k blocks of Vb) C, C of (k n_rhs) x n_rhs."""
        out = w.clone()
        self._lib().swm_vec_gemm(self.ctx, Vb, k, C, out)
        return out


def gather_rhs_own(ops, inc):
    """Owned rows of the right-hand sides (Eq. (4)) of the rank's wires."""
    from . import swm

    torch = ops.torch
    b = torch.zeros((ops.n_rhs, ops.plan.n_loc), dtype=torch.complex128, device="cuda")
    swm.swm_rhs(ops.ctx, inc, b)
    return b[:, :ops.plan.n_own].contiguous()


def currents_own(ops, y_own):
    """x = M^-1 y on the owned wires (the self blocks do not couple wires)."""
    from . import swm

    torch = ops.torch
    yl = torch.zeros((ops.n_rhs, ops.plan.n_loc), dtype=torch.complex128, device="cuda")
    yl[:, :ops.plan.n_own] = y_own
    xl = torch.empty_like(yl)
    swm.swm_precond_apply(ops.ctx, yl, xl)
    return xl[:, :ops.plan.n_own].contiguous()


def solve_partitioned(comm, centres, dirs, lengths, radii, nseg, k, r_c, inc, obs, tol=1e-6, restart=50,
                      max_iter=1000, device=0, block=False):
    """One rank's share of the whole path on a cloud split over ``comm``: partition (every rank the
    same), its context with owned and halo wires, build, distributed GMRES, x = M^-1 y, and the
    bistatic RCS from the far-field components summed over the ranks; with ``block`` the solve is
    block GMRES over all incidences.  Returns (x_own (n_rhs x n_own, numpy), global ids of the owned
    wires, sigma (n_rhs x n_obs x 2), iterations)."""
    import torch

    from . import swm

    owner = partition(centres, nseg, comm.size, r_c)
    plan = Plan(centres, nseg, owner, comm.rank, r_c)
    w = plan.wires
    ctx = swm.swm_create(device)
    try:
        dev = [torch.from_numpy(np.ascontiguousarray(a[w])).cuda() for a in (centres, dirs, lengths, radii, nseg)]
        swm.swm_set_cloud(ctx, *dev)
        swm.swm_build(ctx, k, r_c, swm.SWM_C128)
        inc = np.atleast_2d(np.asarray(inc, dtype=np.float64))
        ops = SwmOps(ctx, plan, inc.shape[0])
        b = gather_rhs_own(ops, inc)
        y, it, rel = (dist_block_gmres if block else dist_gmres)(ops, comm, plan, b, tol, restart, max_iter)
        x = currents_own(ops, y)
        no = plan.n_own_wires
        off = torch.from_numpy(plan.off[:no + 1].copy()).cuda()
        obs = np.atleast_2d(np.asarray(obs, dtype=np.float64))
        comp = torch.zeros((inc.shape[0], obs.shape[0], 2), dtype=torch.complex128, device="cuda")
        if no > 0:
            swm.swm_far_components(None, dev[0][:no].contiguous(), dev[1][:no].contiguous(),
                                   dev[2][:no].contiguous(), dev[4][:no].contiguous(), off, k, x,
                                   torch.from_numpy(obs).cuda(), comp)
        comp = comm.allreduce_sum(comp.cpu().numpy())
        sigma = np.abs(comp) ** 2 / (4.0 * math.pi)
        return x.cpu().numpy(), w[:no].copy(), sigma, it
    finally:
        swm.swm_destroy(ctx)
