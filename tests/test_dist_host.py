"""Host side of the row-partitioned solve (Sec. 3.1, Eq. 4-5), without a GPU: the row
partition, the halo of a rank (pc_dist_halo, the library's host routine), and the
request / halo exchange protocol between ranks over gloo (two and three ranks on CPU),
checked against the columns each rank's rows really reference."""
import datetime
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ds():
    from paper_2008_00409_gb300 import build
    build.build()
    from paper_2008_00409_gb300 import dist
    return dist


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def random_pattern(V, seed, far=0.02):
    """A symmetric block pattern like a cloth's: grid neighbours within a band plus a few
    far couplings (contacts), diagonal included, columns sorted."""
    rng = np.random.default_rng(seed)
    side = int(np.sqrt(V)) or 1
    pairs = {(i, i) for i in range(V)}
    for i in range(V):
        for d in (1, side, side + 1):
            if i + d < V:
                pairs |= {(i, i + d), (i + d, i)}
    for _ in range(int(far * V)):
        a, b = rng.integers(0, V, 2)
        pairs |= {(int(a), int(b)), (int(b), int(a))}
    pairs = sorted(pairs)
    rp = np.zeros(V + 1, np.int32)
    for r, _ in pairs:
        rp[r + 1] += 1
    return np.cumsum(rp).astype(np.int32), np.array([c for _, c in pairs], np.int32)


def test_partition_is_balanced_and_tile_aligned(ds):
    rp, ci = random_pattern(4000, 1)
    for n in (1, 2, 3, 5, 8):
        rs = ds.partition(4000, n, rp)
        assert rs[0] == 0 and rs[-1] == 4000 and np.all(np.diff(rs) >= 0)
        assert np.all(rs[1:-1] % 32 == 0)
        blocks = np.diff(rp[rs])
        assert blocks.max() - blocks.min() <= 2 * 32 * 8  # within two tiles of rows
    rs = ds.partition(1000, 4)
    assert list(rs) == [0, 256, 512, 736, 1000]


def test_halo_is_sorted_distinct_and_counted_by_owner(ds):
    rng = np.random.default_rng(3)
    rs = np.array([0, 96, 320, 480, 600], np.int32)
    for rank in range(4):
        own = np.arange(rs[rank], rs[rank + 1])
        others = np.setdiff1d(np.arange(600), own)
        remote = rng.choice(others, 300)
        h, counts = ds.halo(rs, rank, remote)
        want = np.unique(remote)
        np.testing.assert_array_equal(h, want)
        owner = np.searchsorted(rs, want, side="right") - 1
        np.testing.assert_array_equal(counts, np.bincount(owner, minlength=4))
        assert counts[rank] == 0
    with pytest.raises(Exception):
        ds.halo(rs, 1, np.array([100], np.int32))   # a row of rank 1 itself
    with pytest.raises(Exception):
        ds.halo(rs, 1, np.array([600], np.int32))   # out of range
    h, counts = ds.halo(rs, 2, np.zeros(0, np.int32))
    assert len(h) == 0 and counts.sum() == 0


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2008_00409_gb300 import dist as ds
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=300))
    V = 1500
    rp, ci = random_pattern(V, 7)
    rs = ds.partition(V, world, rp)
    r0, r1 = rs[rank], rs[rank + 1]
    cols = ci[rp[r0]: rp[r1]]
    remote = cols[(cols < r0) | (cols >= r1)]
    halo, counts = ds.halo(rs, rank, remote)
    comm = ds.HostComm()
    # 1. request counts: 8 bytes to each peer
    W = world
    one = [0 if j == rank else 8 for j in range(W)]
    off = [8 * j for j in range(W)]
    send = torch.from_numpy(counts.astype(np.int64)).view(torch.uint8)
    recv = torch.zeros(8 * W, dtype=torch.uint8)
    comm.exchange(send, off, one, recv, off, one)
    want_from_me = recv.view(torch.int64).numpy().copy()
    want_from_me[rank] = 0
    # 2. the requested rows themselves
    start = np.concatenate([[0], np.cumsum(counts)])
    sstart = np.concatenate([[0], np.cumsum(want_from_me)])
    req = torch.zeros(4 * int(sstart[-1]), dtype=torch.uint8)
    comm.exchange(torch.from_numpy(halo.astype(np.int32)).view(torch.uint8), [4 * int(s) for s in start[:-1]],
                  [4 * int(c) for c in counts], req, [4 * int(s) for s in sstart[:-1]],
                  [4 * int(c) for c in want_from_me])
    requested = req.view(torch.int32).numpy().copy()
    # 3. a vector's halo: each rank sends x[requested] (x_i = 10 i + rank-independent)
    x = (10.0 * np.arange(r0, r1)).astype(np.float32)
    sendx = torch.from_numpy(x[requested - r0]).view(torch.uint8)
    recvx = torch.zeros(4 * len(halo), dtype=torch.uint8)
    comm.exchange(sendx, [4 * int(s) for s in sstart[:-1]], [4 * int(c) for c in want_from_me], recvx,
                  [4 * int(s) for s in start[:-1]], [4 * int(c) for c in counts])
    got = recvx.view(torch.float32).numpy().copy()
    # 4. all-reduce of the ranks' partial sums
    t = torch.tensor([float(rank + 1), float(len(halo))], dtype=torch.float64)
    comm.allreduce(t)
    out[rank] = (rs, halo, requested, got, t.numpy().copy(), want_from_me)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_request_and_halo_exchange_over_gloo(ds, world):
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    V = 1500
    rp, ci = random_pattern(V, 7)
    rs = out[0][0]
    total_halo = sum(len(out[r][1]) for r in range(world))
    for r in range(world):
        _, halo, requested, got, sums, want = out[r]
        r0, r1 = rs[r], rs[r + 1]
        # brute force: the remote columns rank r's rows reference
        cols = ci[rp[r0]: rp[r1]]
        np.testing.assert_array_equal(halo, np.unique(cols[(cols < r0) | (cols >= r1)]))
        # the halo values arrived from their owners
        np.testing.assert_array_equal(got, (10.0 * halo).astype(np.float32))
        # the rows rank r was asked for are the rows of r that other ranks reference
        asked = np.sort(requested)
        expect = []
        for q in range(world):
            if q != r:
                qc = ci[rp[rs[q]]: rp[rs[q + 1]]]
                expect.append(np.unique(qc[(qc >= r0) & (qc < r1)]))
        np.testing.assert_array_equal(asked, np.sort(np.concatenate(expect)))
        assert sums[0] == world * (world + 1) / 2 and sums[1] == total_halo
