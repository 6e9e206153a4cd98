"""Multi-rank host logic on CPU (gloo, world size 2): column sharding covers
every column exactly once with balanced particle counts, the benchmark's
per-rank share of the batched columns (dist.shard_state) reassembles into the
whole batch, and the timing reduction takes the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, offs, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2206_14061_gb300 import workloads as W
    from paper_2206_14061_gb300.dist import max_over_ranks, shard_columns, shard_state
    c0, c1 = shard_columns(offs, rank, world)
    t = max_over_ranks(10.0 + rank)
    counts = torch.tensor([offs[c1] - offs[c0], c0, c1], dtype=torch.int64)
    gathered = [torch.zeros(3, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(gathered, counts)
    # the benchmark's sharding of the batched columns (smaller batch): each
    # rank's x values and per-column mu_s, gathered on rank 0
    wl = W.columns(ncol=16, n_lo=300, n_hi=1500)
    sh = shard_state(wl.state, wl.column_offsets, rank, world, wl.mu_s_col)
    parts = [None] * world
    dist.all_gather_object(parts, (sh["state"]["x"], sh["offsets"], sh["per_column"],
                                   sh["c0"], sh["c1"]))
    if rank == 0:
        out.put((t, [g.tolist() for g in gathered], parts))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_columns_and_max_over_ranks_gloo():
    from paper_2206_14061_gb300 import workloads as W
    rng = np.random.default_rng(0)
    sizes = np.round(np.exp(rng.uniform(np.log(2000), np.log(64000), 256))).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, offs, q)) for r in range(2)]
    for p in procs:
        p.start()
    t, parts, shards = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert t == 11.0
    (n0, a0, b0), (n1, a1, b1) = parts
    assert a0 == 0 and b0 == a1 and b1 == 256
    assert n0 + n1 == offs[-1]
    assert abs(n0 - n1) <= sizes.max()
    # the shards of the batched workload cover it exactly once, in order
    wl = W.columns(ncol=16, n_lo=300, n_hi=1500)
    assert np.array_equal(np.concatenate([s[0] for s in shards]), wl.state["x"])
    assert np.array_equal(np.concatenate([s[2] for s in shards]), wl.mu_s_col)
    assert shards[0][3] == 0 and shards[0][4] == shards[1][3] and shards[1][4] == 16
    for x, lo, _, c0, c1 in shards:
        assert lo[0] == 0 and lo[-1] == x.size and len(lo) == c1 - c0 + 1
        assert np.array_equal(np.diff(lo), np.diff(wl.column_offsets)[c0:c1])


def test_shard_columns_edge_cases():
    from paper_2206_14061_gb300.dist import local_offsets, shard_columns
    offs = np.array([0, 5, 5, 12, 20])
    got = [shard_columns(offs, r, 3) for r in range(3)]
    assert got[0][0] == 0 and got[-1][1] == 4
    for (a, b), (c, d) in zip(got, got[1:]):
        assert b == c
    assert list(local_offsets(offs, 1, 3)) == [0, 0, 7]
    with pytest.raises(ValueError):
        shard_columns(offs, 3, 3)
