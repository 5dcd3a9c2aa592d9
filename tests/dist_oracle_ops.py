"""Test helper: the local numerical steps of the partitioned solve computed by the FP64 oracle on the
CPU, so that the host logic of paper_2410_03060_gb300.dist (partition, halo plan, exchange,
all-reduce, GMRES) runs on gloo or thread ranks without a GPU.  Test infrastructure only."""
import math

import numpy as np
import scipy.sparse as sp

import oracle as O


class OracleOps:
    """One rank's wires (owned then halo, ``plan.wires``): A = Z M^-1 of the local wires assembled
    by the oracle (the owned rows are complete: every wire within r_c of an owned wire is local),
    vectors as numpy n_rhs x n arrays."""

    def __init__(self, cloud, plan, k, r_c, n_rhs):
        self.plan, self.n_rhs, self.k = plan, n_rhs, k
        self.local = cloud.subset(plan.wires)
        Z = O.assemble(self.local, k, r_c, sparse=True)
        Mi = O.block_jacobi(self.local, k)
        self.Minv = sp.block_diag([sp.csr_matrix(B) for B in Mi], format="csr")
        self.A = (Z @ self.Minv).tocsr()

    def zeros(self):
        return np.zeros((self.n_rhs, self.plan.n_own), dtype=np.complex128)

    def basis(self, k):
        return np.zeros((k, self.n_rhs, self.plan.n_own), dtype=np.complex128)

    def put(self, Vb, j, v):
        Vb[j] = v

    def get(self, Vb, j):
        return Vb[j]

    def take(self, v, idx):
        return v[:, idx]

    def apply(self, v_own, halo):
        x = np.zeros((self.n_rhs, self.plan.n_loc), dtype=np.complex128)
        x[:, :self.plan.n_own] = v_own
        for _, (pos, vals) in halo.items():
            x[:, pos] = np.asarray(vals).reshape(self.n_rhs, -1)
        return (self.A @ x.T).T[:, :self.plan.n_own].copy()

    def sub(self, a, b):
        return a - b

    def norms2(self, v):
        return np.sum(np.abs(v) ** 2, axis=1)

    def dots(self, Vb, k, w):
        return np.einsum("irn,rn->ir", np.conj(Vb[:k]), w)

    def axpy(self, Vb, k, coef, v):
        return v - np.einsum("ir,irn->rn", coef, Vb[:k])

    def scale(self, v, a):
        return np.asarray(a)[:, None] * v

    def as_basis(self, v):
        return v[None]

    def gram(self, Vb, k, w):
        Q = Vb[:k].reshape(-1, Vb.shape[-1])
        return np.conj(Q) @ w.T

    def gemm(self, Vb, k, C, w):
        Q = Vb[:k].reshape(-1, Vb.shape[-1])
        return w - (Q.T @ C).T

    def rhs_own(self, inc):
        return O.rhs(self.local, self.k, inc).T[:, :self.plan.n_own].copy()

    def currents_own(self, y_own):
        y = np.zeros((self.n_rhs, self.plan.n_loc), dtype=np.complex128)
        y[:, :self.plan.n_own] = y_own
        return (self.Minv @ y.T).T[:, :self.plan.n_own].copy()

    def far_components(self, x_own, obs):
        """theta_hat . F and phi_hat . F of the owned wires' currents, n_rhs x n_obs x 2."""
        own = self.local.subset(np.arange(self.plan.n_own_wires))
        th, ph = obs[:, 0], obs[:, 1]
        rhat = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
        F = O.far_field(own, self.k, x_own.T, rhat)  # (n_obs, 3, n_rhs)
        th_hat = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], axis=1)
        ph_hat = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], axis=1)
        Ft = np.einsum("oc,oci->io", th_hat, F)
        Fp = np.einsum("oc,oci->io", ph_hat, F)
        return np.stack([Ft, Fp], axis=2)


def run_rank(comm, cloud, k, r_c, inc, obs, tol, restart, max_iter=500, block=False):
    """One rank's whole partitioned solve with oracle operators: (global wire ids owned, currents
    n_rhs x n_own, sigma n_rhs x n_obs x 2, iterations)."""
    from paper_2410_03060_gb300 import dist

    owner = dist.partition(cloud.centres, cloud.nseg, comm.size, r_c)
    plan = dist.Plan(cloud.centres, cloud.nseg, owner, comm.rank, r_c)
    ops = OracleOps(cloud, plan, k, r_c, inc.shape[0])
    b = ops.rhs_own(inc)
    solver = dist.dist_block_gmres if block else dist.dist_gmres
    y, it, rel = solver(ops, comm, plan, b, tol, restart, max_iter)
    x = ops.currents_own(y)
    comp = comm.allreduce_sum(ops.far_components(x, obs))
    sigma = np.abs(comp) ** 2 / (4.0 * math.pi)
    return plan.wires[:plan.n_own_wires].copy(), x, sigma, it


def to_global(cloud, parts):
    """Currents in the cloud's unknown order (N x n_rhs) from the ranks' (wires, x_own) parts."""
    m, off = O.numbering(cloud.nseg)
    n_rhs = parts[0][1].shape[0]
    X = np.full((int(off[-1]), n_rhs), np.nan + 0j)
    for wires, x in parts:
        pos = 0
        for w in wires:
            X[off[w]:off[w + 1], :] = x[:, pos:pos + m[w]].T
            pos += m[w]
    return X
