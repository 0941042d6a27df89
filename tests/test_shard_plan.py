"""The row-sharded partition plan (Sec. 3.3) on the CPU: its invariants in one
process, then a world_size-2 gloo run in which each rank keeps only its rows,
exchanges its halo through the plan's messages, computes its rows of y = A x
and its Galerkin contribution P_ext^T A_ext P_ext from a gathered P_oth, and
the contributions are reduced (Sec. 4.8's exchanges, as collectives).  The
local arithmetic here is scipy on the host; the results must equal the
unsharded oracle."""
import os
import socket

import numpy as np
import pytest
import scipy.sparse as sp
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle.galerkin import galerkin
from paper_2606_24748_gb300 import bamg as B

from oracle_cases import hierarchy


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def fine_problem():
    h = hierarchy(8)
    return h.levels[0].A, h.levels[0].P


def starts_for(n, nparts):
    return np.array([round(k * n / nparts) for k in range(nparts + 1)], dtype=np.int64)


def local_to_global(halo, p, starts):
    n, g, _ = halo.info(p)
    ghosts, _ = halo.ghosts(p)
    return np.concatenate([np.arange(starts[p], starts[p] + n), ghosts]).astype(np.int64)


@pytest.mark.parametrize("nparts", [1, 2, 3, 7])
def test_plan_covers_every_block_once_with_consistent_halos(nparts):
    A, _ = fine_problem()
    starts = starts_for(A.nbr, nparts)
    halo = B.Halo(A.rowptr, A.colidx, starts)
    try:
        seen = np.zeros(A.nnzb, dtype=int)
        for p in range(nparts):
            n, g, nb = halo.info(p)
            assert n == starts[p + 1] - starts[p]
            rp, ci, src = halo.pattern(p)
            l2g = local_to_global(halo, p, starts)
            ghosts, owner = halo.ghosts(p)
            assert np.all(np.diff(ghosts) > 0)
            assert np.all((ghosts < starts[p]) | (ghosts >= starts[p + 1]))
            assert np.all(starts[owner] <= ghosts) and np.all(ghosts < starts[owner + 1])
            for i in range(n):
                row = slice(rp[i], rp[i + 1])
                assert np.all(np.diff(ci[row]) > 0)                   # ascending local columns
                gsrc = src[row]
                assert np.all(A.block_rows()[gsrc] == starts[p] + i)  # each block from its own row
                assert np.array_equal(A.colidx[gsrc], l2g[ci[row]])   # local column maps to the global one
            seen[src] += 1
            # the messages into p are exactly its ghosts, grouped by owner in ghost order
            recv = np.concatenate([halo.sends(q, p) + starts[q] for q in range(nparts)]) if g else []
            assert np.array_equal(np.asarray(recv, dtype=np.int64), ghosts)
            assert len(halo.sends(p, p)) == 0
        assert np.all(seen == 1)
    finally:
        halo.close()


def test_plan_rejects_bad_ranges():
    A, _ = fine_problem()
    with pytest.raises(B.BamgError):
        B.Halo(A.rowptr, A.colidx, [0, 10, 5, A.nbr])
    with pytest.raises(B.BamgError):
        B.Halo(A.rowptr, A.colidx, [0, A.nbr - 1])


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, P = fine_problem()
        bs, bsp, nc = A.bs_r, P.bs_c, P.nbc
        starts = starts_for(A.nbr, world)
        halo = B.Halo(A.rowptr, A.colidx, starts)
        n, g, _ = halo.info(rank)
        rp, ci, src = halo.pattern(rank)
        ghosts, owner = halo.ghosts(rank)
        r0 = starts[rank]
        # this rank's data only: its rows of A, its entries of x, its rows of P
        rng = np.random.default_rng(42)
        x_all = rng.standard_normal(A.nbr * bs)          # every rank draws the same vector ...
        x_own = x_all[r0 * bs:(r0 + n) * bs].copy()      # ... and keeps its own entries
        vals = A.vals[src]
        # halo exchange: send what the other rank needs, receive the ghosts
        peer = 1 - rank
        send_rows = halo.sends(rank, peer)
        send = torch.from_numpy(x_own.reshape(n, bs)[send_rows].reshape(-1).copy())
        recv = torch.empty(len(halo.sends(peer, rank)) * bs, dtype=torch.float64)
        reqs = [dist.isend(send, peer), dist.irecv(recv, peer)]
        for r in reqs:
            r.wait()
        assert len(recv) == g * bs and np.all(owner == peer)
        x_ext = np.concatenate([x_own, recv.numpy()])
        Aloc = sp.bsr_matrix((vals, ci, rp), shape=(n * bs, (n + g) * bs)).tocsr()
        y_own = Aloc @ x_ext
        # P_oth: the ghost rows of P, from their owner (as block rows of
        # pattern + values, one object message each way)
        def p_rows(rows):
            return [(P.colidx[P.rowptr[i]:P.rowptr[i + 1]].copy(), P.vals[P.rowptr[i]:P.rowptr[i + 1]].copy())
                    for i in rows]
        mine = p_rows(starts[rank] + halo.sends(rank, peer))
        box = [None, None]
        dist.all_gather_object(box, mine)
        poth = box[peer]
        own_rows = p_rows(range(r0, r0 + n))
        Pext = sp.lil_matrix(((n + g) * bs, nc * bsp))
        for k, (cols, blocks) in enumerate(own_rows + poth):
            for c, blk in zip(cols, blocks):
                Pext[k * bs:(k + 1) * bs, c * bsp:(c + 1) * bsp] = blk
        Pext = Pext.tocsr()
        Aext = sp.vstack([Aloc, sp.csr_matrix((g * bs, (n + g) * bs))]).tocsr()
        C = (Pext.T @ (Aext @ Pext)).toarray()
        # off-process reduce of the coarse contributions (here all of them: a sum)
        Ct = torch.from_numpy(C)
        dist.all_reduce(Ct)
        ys = [None, None]
        dist.all_gather_object(ys, y_own)
        if rank == 0:
            out["y"] = np.concatenate(ys)
            out["Ac"] = Ct.numpy()
            out["x"] = x_all
        halo.close()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_spmv_and_galerkin_product():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    A, P = fine_problem()
    y_ref = A.scalar() @ out["x"]
    assert np.linalg.norm(out["y"] - y_ref) <= 1e-13 * np.linalg.norm(y_ref)
    Ac_ref = galerkin(A, P).dense()
    assert np.linalg.norm(out["Ac"] - Ac_ref) <= 1e-12 * np.linalg.norm(Ac_ref)
