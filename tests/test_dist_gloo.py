"""Host-side bookkeeping of the slab-decomposed solve with two processes
(gloo on 127.0.0.1): the library's partition and block sizes, the documented
block layouts (phase 0 [zl][k_y][j], phase 1 [zl][y][j]) and the package's
all-to-all (exchange_dist) move every labelled value of the doubled-grid
half spectrum to the rank that owns it, for an even and an uneven split."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _label(z, ky, kx):
    return z * 1_000_000.0 + ky * 1000.0 + kx + 0.5


def _rank(rank, world, port, N, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import paper_2405_02603_gb300 as fsp
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        z0, z1, c0, c1 = fsp.dist_partition(N, world, rank)
        parts = [fsp.dist_partition(N, world, r) for r in range(world)]
        # phase 0: this rank's z-slab of W2, labelled by global (z, k_y, k_x)
        send = []
        for p in range(world):
            pc0, pc1 = parts[p][2], parts[p][3]
            blk = np.array([_label(z, ky, pc0 + j) for z in range(z0, z1) for ky in range(2 * N)
                            for j in range(pc1 - pc0)])
            assert blk.size == fsp.dist_block_elems(N, world, rank, 0, p, True)
            send.append(torch.from_numpy(blk))
        recv = [torch.zeros(fsp.dist_block_elems(N, world, rank, 0, p, False), dtype=torch.float64)
                for p in range(world)]
        fsp.exchange_dist(send, recv)
        w = c1 - c0
        V = np.zeros((N, 2 * N, w))
        for p in range(world):
            pz0, pz1 = parts[p][0], parts[p][1]
            V[pz0:pz1] = recv[p].numpy().reshape(pz1 - pz0, 2 * N, w)
        want = np.array([[[_label(z, ky, c0 + j) for j in range(w)] for ky in range(2 * N)] for z in range(N)])
        ok0 = bool(np.array_equal(V, want))
        # phase 1: U[z][y][j] of this rank's columns, labelled (z, y, k_x)
        send = []
        for p in range(world):
            pz0, pz1 = parts[p][0], parts[p][1]
            blk = np.array([_label(z, y, c0 + j) for z in range(pz0, pz1) for y in range(N) for j in range(w)])
            assert blk.size == fsp.dist_block_elems(N, world, rank, 1, p, True)
            send.append(torch.from_numpy(blk))
        recv = [torch.zeros(fsp.dist_block_elems(N, world, rank, 1, p, False), dtype=torch.float64)
                for p in range(world)]
        fsp.exchange_dist(send, recv)
        W1 = np.zeros((z1 - z0, N, N + 1))
        for p in range(world):
            pc0, pc1 = parts[p][2], parts[p][3]
            W1[:, :, pc0:pc1] = recv[p].numpy().reshape(z1 - z0, N, pc1 - pc0)
        want = np.array([[[_label(z, y, kx) for kx in range(N + 1)] for y in range(N)] for z in range(z0, z1)])
        q.put((rank, ok0, bool(np.array_equal(W1, want))))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("N", [6, 7])
def test_slab_exchange_bookkeeping_two_ranks(N):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, N, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, True, True), (1, True, True)]


def test_partition_and_block_sizes_host_only():
    sys.path.insert(0, ROOT)
    import paper_2405_02603_gb300 as fsp
    for N, R in ((8, 1), (8, 3), (9, 4), (256, 8), (5, 5)):
        parts = [fsp.dist_partition(N, R, r) for r in range(R)]
        assert parts[0][0] == 0 and parts[-1][1] == N and parts[0][2] == 0 and parts[-1][3] == N + 1
        for a, b in zip(parts, parts[1:]):
            assert a[1] == b[0] and a[3] == b[2]
        assert all(p[1] > p[0] and p[3] > p[2] for p in parts)
        for ph in (0, 1):
            tot = 0
            for r in range(R):
                for p in range(R):
                    n = fsp.dist_block_elems(N, R, r, ph, p, True)
                    assert n == fsp.dist_block_elems(N, R, p, ph, r, False)
                    tot += n
            assert tot == (2 * N * N * (N + 1) if ph == 0 else N * N * (N + 1))
    with pytest.raises(fsp.FspError):
        fsp.dist_partition(4, 5, 0)
    with pytest.raises(fsp.FspError):
        fsp.dist_block_elems(8, 2, 0, 2, 1, True)
