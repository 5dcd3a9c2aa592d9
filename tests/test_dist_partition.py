"""One cloud split over ranks on the CPU (Sec. II-B: S-NFC couples wires within r_c only): the
partition and halo plan, and the partitioned GMRES with its halo exchange and all-reduces on
thread ranks and on two gloo processes, its local steps computed by the FP64 oracle.  The
currents and RCS of 2 and 3 ranks equal the 1-rank ones to 1e-10 and the oracle's LU solution."""
import math
import os
import socket
import threading

import numpy as np
import pytest

import oracle as O
from dist_oracle_ops import run_rank, to_global
from paper_2410_03060_gb300 import dist
from synth import cloud_uniform_cube, observations_phi_cut

K = 2.0 * math.pi


def _cloud():
    return cloud_uniform_cube(70, 5.0, seed=51)


def test_partition_covers_every_wire_and_halo_is_exact():
    cl = cloud_uniform_cube(400, 12.0, seed=52)
    r_c = 2.0
    for n in (1, 2, 3, 5):
        owner = dist.partition(cl.centres, cl.nseg, n, r_c)
        assert set(np.unique(owner)) == set(range(n))
        m = cl.nseg.astype(np.int64) - 1
        share = np.array([m[owner == r].sum() for r in range(n)])
        assert share.max() - share.min() <= 2 * m.max()  # balanced by unknowns
        pairs = O.neighbour_pairs(cl.centres, r_c)
        for r in range(n):
            plan = dist.Plan(cl.centres, cl.nseg, owner, r, r_c)
            own = set(np.nonzero(owner == r)[0].tolist())
            assert set(plan.wires[:plan.n_own_wires].tolist()) == own
            # the halo is exactly the other ranks' partners of owned wires (brute-force pairs)
            want = {int(q) for p, q in pairs if int(p) in own and int(q) not in own}
            assert set(plan.wires[plan.n_own_wires:].tolist()) == want
    # what rank r sends to s is what s expects from r, in the same order
    owner = dist.partition(cl.centres, cl.nseg, 3, r_c)
    plans = [dist.Plan(cl.centres, cl.nseg, owner, r, r_c) for r in range(3)]
    m, off = O.numbering(cl.nseg)
    for r in range(3):
        for s, idx in plans[r].send.items():
            sent = np.concatenate([np.arange(off[w], off[w + 1]) for w in plans[r].wires])[idx]
            recv = np.concatenate([np.arange(off[w], off[w + 1]) for w in plans[s].wires])[plans[s].recv[r]]
            assert np.array_equal(sent, recv)


def _threads(n, fn):
    comms = dist.ThreadComm.group(n)
    out = [None] * n
    err = []

    def go(r):
        try:
            out[r] = fn(comms[r])
        except Exception as e:  # surfaced below
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


def test_partitioned_gmres_on_thread_ranks_matches_one_rank_and_lu():
    cl = _cloud()
    r_c = 1.5
    inc = np.array([[0.3, 0.2, 0.0], [2.0, 4.0, 1.0]])
    obs = observations_phi_cut(20)
    one = run_rank(dist.LocalComm(), cl, K, r_c, inc, obs, 1e-12, 30)
    X1 = to_global(cl, [one[:2]])
    Z = O.assemble(cl, K, r_c, sparse=False)
    X_lu = O.solve_lu(Z, O.rhs(cl, K, inc))
    assert np.linalg.norm(X1 - X_lu) / np.linalg.norm(X_lu) < 1e-10
    s_ref = np.transpose(O.rcs_bistatic(cl, K, X_lu, obs), (0, 1, 2))
    for n in (2, 3):
        res = _threads(n, lambda comm: run_rank(comm, cl, K, r_c, inc, obs, 1e-12, 30))
        Xn = to_global(cl, [r[:2] for r in res])
        assert not np.isnan(Xn).any()
        assert np.linalg.norm(Xn - X1) / np.linalg.norm(X1) < 1e-10
        assert res[0][3] == one[3]  # same iteration count
        for r in res:
            assert np.allclose(r[2], one[2], rtol=1e-9, atol=1e-14)
            assert np.allclose(r[2], s_ref, rtol=1e-8, atol=1e-14)


def test_partitioned_gmres_with_restarts_and_an_empty_rank():
    """Restarts inside the partitioned solve, and more ranks than the cloud has Morton ranges for
    some of them: a rank may own few wires or have no halo."""
    cl = cloud_uniform_cube(12, 6.0, seed=53)
    r_c = 1.2
    inc = np.array([[1.0, 0.5, 0.0]])
    obs = observations_phi_cut(8)
    one = run_rank(dist.LocalComm(), cl, K, r_c, inc, obs, 1e-11, 3)
    res = _threads(4, lambda comm: run_rank(comm, cl, K, r_c, inc, obs, 1e-11, 3))
    Xn = to_global(cl, [r[:2] for r in res])
    X1 = to_global(cl, [one[:2]])
    assert np.linalg.norm(Xn - X1) / np.linalg.norm(X1) < 1e-10


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _gloo_worker(rank, world, port, out):
    import torch.distributed as tdist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    cl = _cloud()
    inc = np.array([[0.3, 0.2, 0.0], [2.0, 4.0, 1.0]])
    obs = observations_phi_cut(20)
    wires, x, sigma, it = run_rank(dist.TorchComm(), cl, K, 1.5, inc, obs, 1e-12, 30)
    out[rank] = (wires, x, sigma, it)
    tdist.barrier()
    tdist.destroy_process_group()


def test_partitioned_gmres_on_two_gloo_ranks():
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_gloo_worker, args=(world, port, out), nprocs=world, join=True)
    cl = _cloud()
    inc = np.array([[0.3, 0.2, 0.0], [2.0, 4.0, 1.0]])
    obs = observations_phi_cut(20)
    one = run_rank(dist.LocalComm(), cl, K, 1.5, inc, obs, 1e-12, 30)
    X1 = to_global(cl, [one[:2]])
    X2 = to_global(cl, [out[0][:2], out[1][:2]])
    assert np.linalg.norm(X2 - X1) / np.linalg.norm(X1) < 1e-10
    assert np.allclose(out[0][2], one[2], rtol=1e-9, atol=1e-14)
    assert np.array_equal(out[0][2], out[1][2])  # every rank holds the same RCS


def test_block_gmres_one_and_two_ranks_match_lu():
    """Restarted block GMRES (one Krylov space shared by the incidences), on one rank and split
    over two thread ranks, against the oracle's LU solution; with several restart cycles."""
    cl = _cloud()
    r_c = 1.5
    g = np.random.default_rng(9)
    inc = np.stack([g.uniform(0, np.pi, 6), g.uniform(0, 2 * np.pi, 6), g.uniform(0, np.pi, 6)], 1)
    obs = observations_phi_cut(12)
    X_lu = O.solve_lu(O.assemble(cl, K, r_c, sparse=False), O.rhs(cl, K, inc))
    one = run_rank(dist.LocalComm(), cl, K, r_c, inc, obs, 1e-11, 4, block=True)
    X1 = to_global(cl, [one[:2]])
    assert np.linalg.norm(X1 - X_lu) / np.linalg.norm(X_lu) < 1e-9
    res = _threads(2, lambda comm: run_rank(comm, cl, K, r_c, inc, obs, 1e-11, 4, block=True))
    X2 = to_global(cl, [r[:2] for r in res])
    assert np.linalg.norm(X2 - X1) / np.linalg.norm(X1) < 1e-9
    # the block space contains every incidence's own Krylov space: no more block iterations than
    # the independent GMRES needs
    ind = run_rank(dist.LocalComm(), cl, K, r_c, inc, obs, 1e-11, 4)
    assert one[3] <= ind[3]
