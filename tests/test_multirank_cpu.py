"""The multi-process path on CPU (gloo, world size 2): a genotype range split
across ranks, each rank's sorted histogram gathered and merged on the host
with jatam_hist_merge, equals the histogram of the whole range.  Classification
on each rank is done by the oracle here (no GPU in this test); the merge and
the range split are the library's own host logic."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def shard(first, count, rank, world):
    lo = first + count * rank // world
    hi = first + count * (rank + 1) // world
    return lo, hi - lo


def _to_lib_hist(h):
    from paper_2205_15311_gb300 import binding as J
    out = np.zeros(h.shape[0], J.HIST_DTYPE)
    for f in ("cls", "shape_hash", "size", "count", "min_id"):
        out[f] = h[f]
    return out


def _worker(rank, world, port, first, count, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_2205_15311_gb300 import binding as J
    n, c, L, k, seed = 2, 8, 12, 6, 2
    lo, cnt = shard(first, count, rank, world)
    res, _ = O.enumerate_space(n, c, L, k, seed, lo, cnt, nthreads=1)
    mine = _to_lib_hist(O.histogram(res, np.arange(lo, lo + cnt, dtype=np.uint64)))
    gathered = [None] * world
    dist.all_gather_object(gathered, mine.tobytes())
    merged = np.zeros(0, J.HIST_DTYPE)
    for raw in gathered:
        merged = J.merge_histograms(merged, np.frombuffer(raw, J.HIST_DTYPE))
    if rank == 0:
        q.put(merged.tobytes())
    dist.barrier()
    dist.destroy_process_group()


def test_range_split_and_host_merge_two_ranks():
    from oracle import oracle as O
    from paper_2205_15311_gb300 import binding as J
    from paper_2205_15311_gb300 import build as B
    B.build()
    O.build()
    first, count, world = 5 << 18, 6001, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, first, count, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged = np.frombuffer(q.get(timeout=120), J.HIST_DTYPE)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res, _ = O.enumerate_space(2, 8, 12, 6, 2, first, count)
    whole = _to_lib_hist(O.histogram(res, np.arange(first, first + count, dtype=np.uint64)))
    assert np.array_equal(merged, whole)


def test_shards_cover_the_range_exactly():
    for count in (0, 1, 7, 1000, 16777216):
        for world in (1, 2, 3, 8):
            spans = [shard(11, count, r, world) for r in range(world)]
            assert sum(c for _, c in spans) == count
            pos = 11
            for lo, c in spans:
                assert lo == pos
                pos += c
