"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every comparison is exact: classes, deciding replicates, sizes and shape hashes
are integers, and the histogram rows (class, hash, size, count, smallest id)
must match row for row.
"""
import hashlib
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2205_15311_gb300 import binding as J  # noqa: E402
from paper_2205_15311_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


def _dev_enumerate(n, c, L, k, seed, first, count, sampled=False, hist_cap=1 << 16, c4_hash=False):
    out = torch.full((max(count, 1) * 8,), 0xEE, dtype=torch.uint8, device="cuda")  # poisoned
    hist = torch.empty(hist_cap * 32, dtype=torch.uint8, device="cuda")
    hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
    J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out, hist=hist, hist_len=hlen,
                      hist_cap=hist_cap, sync=True, c4_hash=c4_hash)
    m = int(hlen.item())
    return J.results_view(out)[:count], J.hist_view(hist, min(m, hist_cap)), m


def _oracle_hist(res, ids):
    return O.histogram(res, ids)


def _hist_rows(h):
    return [(int(r["cls"]), int(r["shape_hash"]), int(r["size"]), int(r["count"]), int(r["min_id"])) for r in h]


def test_philox_matches_oracle():
    rng = np.random.default_rng(1)
    rec = rng.integers(0, 1 << 32, size=(4096, 6), dtype=np.uint64).astype(np.uint32)
    rec[0] = 0
    rec[1] = 0xFFFFFFFF
    out = np.zeros((4096, 4), np.uint32)
    J.philox(rec, out)
    for i in range(0, 4096, 37):
        assert out[i].tolist() == O.philox(rec[i, :4].tolist(), rec[i, 4:].tolist())
    dev_in = torch.from_numpy(rec.view(np.int32)).cuda()
    dev_out = torch.zeros((4096, 4), dtype=torch.int32, device="cuda")
    J.philox(dev_in, dev_out)
    torch.cuda.synchronize()
    assert np.array_equal(dev_out.cpu().numpy().view(np.uint32), out)


def test_s24_full_space_matches_oracle_and_golden():
    n, c, L, k, seed, first, count, _ = W.WORKLOADS["s24_full"]
    res, hist, m = _dev_enumerate(n, c, L, k, seed, first, count)
    ref, _ = O.enumerate_space(n, c, L, k, seed, first, count)
    assert np.array_equal(res, ref)
    gold = json.load(open(os.path.join(GOLDEN, "c1_summary.json")))
    assert hashlib.sha256(res.tobytes()).hexdigest() == gold["results_sha256"]
    want = _oracle_hist(ref, np.arange(count, dtype=np.uint64))
    assert m == len(want)
    assert _hist_rows(hist) == _hist_rows(want)


def _golden_hist(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#"):
            continue
        rows.append(tuple(int(v) for v in line.split()))
    return rows


def test_s28_full_space_matches_golden():
    """All 8^8 genotypes of S_{2,8}: the SHA-256 of the 134 MB result array and
    the histogram equal what the oracle wrote (tests/golden/make_golden.py)."""
    n, c, L, k, seed, first, count, _ = W.WORKLOADS["s28_full"]
    res, hist, m = _dev_enumerate(n, c, L, k, seed, first, count)
    gold = json.load(open(os.path.join(GOLDEN, "c2_summary.json")))
    assert np.bincount(res["cls"], minlength=4).tolist() == gold["class_counts"]
    assert hashlib.sha256(res.tobytes()).hexdigest() == gold["results_sha256"]
    assert _hist_rows(hist) == _golden_hist("c2_histogram.txt")
    # spot-check against the oracle run one genotype at a time
    rng = np.random.default_rng(7)
    for g in rng.integers(0, count, size=300):
        r = O.classify(n, c, L, k, seed, O.decode(int(g), n, c), int(g))
        assert (r["cls"], r["decided_rep"], r["size"], r["shape_hash"]) == tuple(res[int(g)].tolist())


def test_s38_sample_slice_matches_oracle():
    n, c, L, k, seed, _, _, _ = W.WORKLOADS["s38_sample"]
    first, count = 12345, (1 << 16) + 77
    res, hist, m = _dev_enumerate(n, c, L, k, seed, first, count, sampled=True)
    ref, _ = O.enumerate_space(n, c, L, k, seed, first, count, sampled=True)
    assert np.array_equal(res, ref)
    ids = np.array([O.sample_genotype(first + i, n, c, seed) for i in range(count)], np.uint64)
    assert _hist_rows(hist) == _hist_rows(_oracle_hist(ref, ids))


@pytest.mark.parametrize("case", ["s24_full", "s28_slice", "s38_sample", "s28_large"])
def test_c4_hash_variant_matches_oracle(case):
    """The rotation-only hash of Section 2.5: every field but the hash equals
    the default run, the hashes equal the oracle's C4 hashes, and chiral pairs
    now land in different histogram rows."""
    if case == "s24_full":
        n, c, L, k, seed, first, count, _ = W.WORKLOADS["s24_full"]
        sampled = False
    elif case == "s28_slice":
        n, c, L, k, seed, sampled = 2, 8, 16, 20, 2, False
        first, count = 5 * (1 << 20) + 3, 40000
    elif case == "s28_large":  # the call's crop table and the heavy-first list at scale
        n, c, L, k, seed, sampled = 2, 8, 16, 20, 2, False
        first, count = 9 << 20, 1 << 20
    else:
        n, c, L, k, seed, _, _, _ = W.WORKLOADS["s38_sample"]
        first, count, sampled = 777, 40000, True
    res, hist, m = _dev_enumerate(n, c, L, k, seed, first, count, sampled=sampled, c4_hash=True)
    base, _, m8 = _dev_enumerate(n, c, L, k, seed, first, count, sampled=sampled)
    with O.hash_mode(True):
        ref, _ = O.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled)
    assert np.array_equal(res, ref)
    for f in ("cls", "decided_rep", "size"):
        assert np.array_equal(res[f], base[f])
    if sampled:
        ids = np.array([O.sample_genotype(first + i, n, c, seed) for i in range(count)], np.uint64)
    else:
        ids = np.arange(first, first + count, dtype=np.uint64)
    with O.hash_mode(True):
        want = _oracle_hist(ref, ids)
    assert _hist_rows(hist) == _hist_rows(want)
    assert m >= m8  # a free shape splits into at most two one-sided shapes


@pytest.mark.parametrize("L", [1, 2, 3, 5, 8, 9, 16, 19, 31, 32])
def test_grid_sizes_including_ragged_ones(L):
    n, c, k, seed = 2, 8, 7, 11
    first, count = 3 * (1 << 20) + 5, 3001
    res, hist, m = _dev_enumerate(n, c, L, k, seed, first, count)
    ref, _ = O.enumerate_space(n, c, L, k, seed, first, count)
    assert np.array_equal(res, ref)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_few_replicates_match_oracle(k):
    """k = 1 (replicate 0 alone decides) to 3: the shortcuts that end a genotype
    after replicate 0 (forced path, closed or dominated final shape) and the
    steric comparison of later replicates at their smallest counts."""
    n, c, L, seed = 2, 8, 16, 9
    first, count = 5 << 20, 200000
    res, hist, m = _dev_enumerate(n, c, L, k, seed, first, count)
    ref, _ = O.enumerate_space(n, c, L, k, seed, first, count)
    assert np.array_equal(res, ref)
    if k == 1:
        assert not np.any(ref["cls"] == O.ND_STERIC)


@pytest.mark.parametrize("count", [0, 1, 31, 32, 33, 1000])
def test_ragged_counts(count):
    n, c, L, k, seed = 2, 8, 16, 20, 2
    first = (1 << 24) - count  # ends exactly at the end of the space
    res, hist, m = _dev_enumerate(n, c, L, k, seed, first, count)
    ref, _ = O.enumerate_space(n, c, L, k, seed, first, count)
    assert np.array_equal(res, ref)
    assert m == len(_oracle_hist(ref, np.arange(first, first + count, dtype=np.uint64)))


def _mixed_run(colours, shapes, ids=None, per_shape=False, hist_cap=1 << 14):
    N = colours.shape[0]
    dc = torch.from_numpy(colours).cuda()
    ds = torch.from_numpy(shapes).cuda()
    di = None if ids is None else torch.from_numpy(ids.view(np.int64)).cuda()
    out = torch.full((N * 8,), 0xEE, dtype=torch.uint8, device="cuda")  # poisoned: every result must be written
    hist = torch.empty(hist_cap * 32, dtype=torch.uint8, device="cuda")
    hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
    J.classify_batch(dc, seed=4, shapes=ds, stream_ids=di, out=out, hist=hist, hist_len=hlen, hist_cap=hist_cap,
                     sync=True, per_shape=per_shape)
    m = int(hlen.item())
    return J.results_view(out), J.hist_view(hist, m)


def test_mixed_records_match_oracle():
    """Mixed n, c, L, k in one persistent launch, with several CTA plans, and as
    per-size fixed launches: all equal the oracle."""
    colours, shapes = W.mixed_records(20000, seed=4)
    ids = np.arange(20000, dtype=np.uint64) * np.uint64(7919) + np.uint64(5)
    ref, _ = O.classify_batch(colours, shapes=shapes, seed=4, ids=ids)
    want_hist = _hist_rows(_oracle_hist(ref, ids))
    old_plan = J.get_mixed_plan()
    try:
        for plan in ((2, 4, 2), (1, 0, 0), (1, 2, 1), (1, 0, 5), (4, 2, 2)):
            J.set_mixed_plan(*plan)
            res, hist = _mixed_run(colours, shapes, ids)
            assert np.array_equal(res, ref), plan
            assert _hist_rows(hist) == want_hist
        for bad in ((0, 1, 3), (0, 0, 8), (3, 3, 3)):
            with pytest.raises(J.JatamError):
                J.set_mixed_plan(*bad)
    finally:
        J.set_mixed_plan(*old_plan)
    res, hist = _mixed_run(colours, shapes, ids, per_shape=True)
    assert np.array_equal(res, ref)
    assert _hist_rows(hist) == want_hist


def test_mixed_1e6_matches_golden():
    """A million mixed-size tile sets: SHA-256 of the results equals the oracle's."""
    gold = json.load(open(os.path.join(GOLDEN, "c4s_summary.json")))
    colours, shapes = W.mixed_records(1_000_000, seed=4)
    assert hashlib.sha256(colours.tobytes() + shapes.tobytes()).hexdigest() == gold["inputs_sha256"]
    for per_shape in (False, True):
        res, hist = _mixed_run(colours, shapes, per_shape=per_shape)
        assert np.bincount(res["cls"], minlength=4).tolist() == gold["class_counts"]
        assert hashlib.sha256(res.tobytes()).hexdigest() == gold["results_sha256"]
        assert len(hist) == gold["distinct_keys"]


def test_uniform_records_all_tile_counts():
    rng = np.random.default_rng(3)
    for n, c, L in ((1, 8, 16), (4, 8, 16), (3, 6, 12), (4, 2, 32), (2, 1, 5)):
        N = 4000
        colours = np.zeros((N, 16), np.uint8)
        colours[:, : 4 * n] = rng.integers(0, c, size=(N, 4 * n))
        out = np.zeros(N, J.RESULT_DTYPE)
        J.classify_batch(colours, n=n, c=c, L=L, k=9, seed=99, out=out)
        ref, _ = O.classify_batch(colours, n=n, c=c, L=L, k=9, seed=99)
        assert np.array_equal(out, ref), (n, c, L)


def test_host_buffers_equal_device_buffers():
    n, c, L, k, seed = 3, 8, 32, 20, 3
    first, count = 1 << 30, 5000
    out = np.zeros(count, J.RESULT_DTYPE)
    hist = np.zeros(4096, J.HIST_DTYPE)
    hlen = np.zeros(1, np.uint32)
    J.enumerate_space(n, c, L, k, seed, first, count, sampled=True, out=out, hist=hist, hist_len=hlen, hist_cap=4096)
    res, dh, m = _dev_enumerate(n, c, L, k, seed, first, count, sampled=True)
    assert np.array_equal(out, res)
    assert int(hlen[0]) == m and np.array_equal(hist[:m], dh)


def test_pinned_host_buffers_pipelined_equal_device_buffers():
    """Calls whose results go to page-locked host memory and that hold at least
    2^23 items run in pieces (of at least 2^22, up to 8) whose copies overlap
    the next piece's work; the results, the histogram and the fitness values
    equal the one-pass device call."""
    n, c, L, k, seed = 3, 8, 16, 20, 3
    first, count = 1 << 30, (1 << 24) + 4_000_001  # a ragged last piece
    res, dh, m = _dev_enumerate(n, c, L, k, seed, first, count, sampled=True)
    out = torch.full((count * 8,), 0xEE, dtype=torch.uint8, pin_memory=True)
    hist = np.zeros(1 << 16, J.HIST_DTYPE)
    hlen = np.zeros(1, np.uint32)
    J.enumerate_space(n, c, L, k, seed, first, count, sampled=True, out=out, hist=hist, hist_len=hlen,
                      hist_cap=1 << 16)
    assert np.array_equal(J.results_view(out), res)
    assert int(hlen[0]) == m and np.array_equal(hist[:m], dh)
    # a genome batch: staged inputs, fitness and results in page-locked memory
    g = W.random_genomes(1 << 24, 3, 8, seed=17)
    gd = torch.from_numpy(g.view(np.int64)).cuda()
    fd = torch.empty(g.shape[0], dtype=torch.int32, device="cuda")
    od = torch.empty(g.shape[0] * 8, dtype=torch.uint8, device="cuda")
    J.evaluate_genomes(gd, fd, n=3, c=8, L=16, k=20, seed=5, out=od, sync=True)
    gh = torch.from_numpy(g.view(np.int64)).pin_memory()
    fh = torch.empty(g.shape[0], dtype=torch.int32, pin_memory=True)
    oh = torch.empty(g.shape[0] * 8, dtype=torch.uint8, pin_memory=True)
    J.evaluate_genomes(gh, fh, n=3, c=8, L=16, k=20, seed=5, out=oh, sync=True)
    assert torch.equal(fh, fd.cpu()) and torch.equal(oh, od.cpu())


def test_pinned_windowed_pipelined_equal_device_buffers():
    """A call that grows in the 16 x 16 window first (L = 32, at least 2^23
    items) with results to page-locked memory runs its pieces side by side on
    two streams, their sizes falling geometrically, each with its own
    escalation list: results and histogram equal the one-pass device call."""
    n, c, L, k, seed = 3, 8, 32, 20, 3
    first, count = 5 << 26, (1 << 23) + 12_345
    res, dh, m = _dev_enumerate(n, c, L, k, seed, first, count, sampled=True)
    out = torch.full((count * 8,), 0xEE, dtype=torch.uint8, pin_memory=True)
    hist = np.zeros(1 << 16, J.HIST_DTYPE)
    hlen = np.zeros(1, np.uint32)
    J.enumerate_space(n, c, L, k, seed, first, count, sampled=True, out=out, hist=hist, hist_len=hlen,
                      hist_cap=1 << 16)
    assert np.array_equal(J.results_view(out), res)
    assert int(hlen[0]) == m and np.array_equal(hist[:m], dh)
    assert (res["cls"] == 3).any() and (res["size"] > 12).any()  # unbounded genotypes and large shapes


def test_pinned_records_with_ids_pipelined_equal_device_buffers():
    """Explicit records of mixed shape with stream ids, results and histogram to
    page-locked memory: the pieces offset the colours, the shapes and the ids."""
    N = (1 << 24) + 5
    colours, shapes = W.mixed_records(N, seed=6)
    ids = W.splitmix64(6, N, 99)
    dc, ds = torch.from_numpy(colours).cuda(), torch.from_numpy(shapes).cuda()
    di = torch.from_numpy(ids.view(np.int64)).cuda()
    od = torch.empty(N * 8, dtype=torch.uint8, device="cuda")
    hd = torch.empty((1 << 16) * 32, dtype=torch.uint8, device="cuda")
    ld = torch.zeros(1, dtype=torch.int32, device="cuda")
    J.classify_batch(dc, seed=4, shapes=ds, stream_ids=di, out=od, hist=hd, hist_len=ld, hist_cap=1 << 16,
                     sync=True)
    oh = torch.empty(N * 8, dtype=torch.uint8, pin_memory=True)
    hh = np.zeros(1 << 16, J.HIST_DTYPE)
    lh = np.zeros(1, np.uint32)
    J.classify_batch(torch.from_numpy(colours).pin_memory(), seed=4, shapes=torch.from_numpy(shapes).pin_memory(),
                     stream_ids=torch.from_numpy(ids.view(np.int64)).pin_memory(), out=oh, hist=hh, hist_len=lh,
                     hist_cap=1 << 16)
    assert torch.equal(oh, od.cpu())
    m = int(ld.item())
    assert int(lh[0]) == m and np.array_equal(hh[:m], J.hist_view(hd, m))


def test_hist_capacity_too_small_reports_length():
    n, c, L, k, seed = 2, 8, 16, 20, 2
    hist = np.zeros(3, J.HIST_DTYPE)
    hlen = np.zeros(1, np.uint32)
    with pytest.raises(J.JatamError) as e:
        J.enumerate_space(n, c, L, k, seed, 0, 1 << 20, hist=hist, hist_len=hlen, hist_cap=3)
    assert e.value.code == J.JATAM_EINVAL and int(hlen[0]) > 3


def test_ga_evaluate_fitness():
    n, c, L, k, seed = 3, 8, 16, 20, 5
    g = W.random_genomes(30000, n, c, seed=5)
    fit = np.zeros(30000, np.int32)
    out = np.zeros(30000, J.RESULT_DTYPE)
    J.evaluate_genomes(g, fit, n=n, c=c, L=L, k=k, seed=seed, out=out)
    for i in range(0, 30000, 97):
        r = O.classify(n, c, L, k, seed, O.decode(int(g[i]), n, c), int(g[i]))
        assert tuple(out[i].tolist()) == (r["cls"], r["decided_rep"], r["size"], r["shape_hash"])
        assert fit[i] == (r["size"] if r["cls"] == O.DET_BOUNDED else 0)
    # same genotype, same stream id: identical to the enumeration of that index
    res, _, _ = _dev_enumerate(n, c, L, k, seed, int(g[0]), 1)
    assert tuple(res[0].tolist()) == tuple(out[0].tolist())


def test_large_genome_batch_matches_oracle():
    """2^20 random genomes of S_{2,8}: a call large enough that the pre-filter
    hands out the genotypes with two or more frontier sites first; every result
    equals the oracle's (stream id = the genome)."""
    n, c, L, k, seed = 2, 8, 16, 20, 5
    g = W.random_genomes(1 << 20, n, c, seed=23)
    cols = np.zeros((g.shape[0], 16), np.uint8)
    for m in range(4 * n):
        cols[:, m] = ((g >> np.uint64(3 * (4 * n - 1 - m))) & np.uint64(7)).astype(np.uint8)
    ref, _ = O.classify_batch(cols, n=n, c=c, L=L, k=k, seed=seed, ids=g)
    dg = torch.from_numpy(g.view(np.int64)).cuda()
    fit = torch.empty(g.shape[0], dtype=torch.int32, device="cuda")
    out = torch.full((g.shape[0] * 8,), 0xEE, dtype=torch.uint8, device="cuda")
    J.evaluate_genomes(dg, fit, n=n, c=c, L=L, k=k, seed=seed, out=out, sync=True)
    assert np.array_equal(J.results_view(out), ref)


def test_argument_errors():
    with pytest.raises(J.JatamError) as e:
        J.enumerate_space(5, 8, 16, 20, 2, 0, 10, out=np.zeros(10, J.RESULT_DTYPE))
    assert e.value.code == J.JATAM_EUNSUPPORTED
    with pytest.raises(J.JatamError) as e:
        J.enumerate_space(2, 6, 16, 20, 2, 0, 10, out=np.zeros(10, J.RESULT_DTYPE))
    assert e.value.code == J.JATAM_EINVAL
    with pytest.raises(J.JatamError) as e:
        J.enumerate_space(2, 8, 16, 20, 2, (1 << 24) - 5, 10, out=np.zeros(10, J.RESULT_DTYPE))
    assert e.value.code == J.JATAM_EINVAL
    bad = np.zeros((4, 16), np.uint8)
    bad[2, 3] = 9  # colour >= c
    out = np.zeros(4, J.RESULT_DTYPE)
    with pytest.raises(J.JatamError) as e:
        J.classify_batch(bad, n=2, c=8, L=16, k=4, seed=1, out=out)
    assert e.value.code == J.JATAM_EINVAL and out["cls"][2] == 255
    # the error was consumed: the next call is clean
    J.classify_batch(bad[:2], n=2, c=8, L=16, k=4, seed=1, out=out[:2])


def test_s38_sample_2e20_matches_golden():
    """2^20 genotypes sampled from S_{3,8} on the 32 x 32 grid: SHA-256 of the
    results and the histogram equal what the oracle wrote."""
    n, c, L, k, seed, _, _, _ = W.WORKLOADS["s38_sample"]
    res, hist, m = _dev_enumerate(n, c, L, k, seed, 0, 1 << 20, sampled=True)
    gold = json.load(open(os.path.join(GOLDEN, "c3s_summary.json")))
    assert np.bincount(res["cls"], minlength=4).tolist() == gold["class_counts"]
    assert hashlib.sha256(res.tobytes()).hexdigest() == gold["results_sha256"]
    assert _hist_rows(hist) == _golden_hist("c3s_histogram.txt")


def test_results_do_not_depend_on_the_launch_shape():
    """The draws depend only on (genotype, replicate, step): every launch shape
    gives bit-identical results; jatam_autotune picks one of them."""
    n, c, L, k, seed = 2, 8, 16, 20, 2
    first, count = 5 << 20, 200000
    base, hbase, _ = _dev_enumerate(n, c, L, k, seed, first, count)
    try:
        for warps, stop in ((1, 1), (2, 32), (4, 8), (6, 3)):
            J.set_tuning(n, c, L, warps, stop)
            assert J.get_tuning(n, c, L) == (warps, stop)
            res, hist, _ = _dev_enumerate(n, c, L, k, seed, first, count)
            assert np.array_equal(res, base)
            assert np.array_equal(hist, hbase)
        J.autotune([{"n": n, "c": c, "L": L, "k": k, "seed": seed}])
        w, s = J.get_tuning(n, c, L)
        assert 1 <= w <= 6 and 1 <= s <= 32
        res, _, _ = _dev_enumerate(n, c, L, k, seed, first, count)
        assert np.array_equal(res, base)
    finally:
        J.set_tuning(n, c, L, 0, 8)  # back to the defaults


def test_graph_replay_equals_direct_launches():
    """JATAM_GRAPH: the first call captures the kernel sequence, later calls with
    the same arguments replay it; results equal the direct launches."""
    n, c, L, k, seed = 3, 8, 32, 20, 3
    first, count = 777, 50000
    base, hbase, _ = _dev_enumerate(n, c, L, k, seed, first, count, sampled=True)
    out = torch.empty(count * 8, dtype=torch.uint8, device="cuda")
    hist = torch.empty((1 << 16) * 32, dtype=torch.uint8, device="cuda")
    hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(3):
        out.zero_()
        J.enumerate_space(n, c, L, k, seed, first, count, sampled=True, out=out, hist=hist, hist_len=hlen,
                          hist_cap=1 << 16, sync=True, graph=True)
        assert np.array_equal(J.results_view(out)[:count], base)
        assert np.array_equal(J.hist_view(hist, int(hlen.item())), hbase)
    colours, shapes = W.mixed_records(30000, seed=4)
    ref, _ = _mixed_run(colours, shapes)
    dc, ds = torch.from_numpy(colours).cuda(), torch.from_numpy(shapes).cuda()
    o2 = torch.empty(30000 * 8, dtype=torch.uint8, device="cuda")
    for per_shape in (False, True, False):
        o2.zero_()
        J.classify_batch(dc, seed=4, shapes=ds, out=o2, sync=True, per_shape=per_shape, graph=True)
        assert np.array_equal(J.results_view(o2), ref)
    g = torch.from_numpy(W.random_genomes(8192, 3, 8, seed=5).view(np.int64)).cuda()
    f1 = torch.empty(8192, dtype=torch.int32, device="cuda")
    f2 = torch.empty(8192, dtype=torch.int32, device="cuda")
    J.evaluate_genomes(g, f1, n=3, c=8, L=16, k=20, seed=5, sync=True)
    for _ in range(2):
        f2.zero_()
        J.evaluate_genomes(g, f2, n=3, c=8, L=16, k=20, seed=5, sync=True, graph=True)
        assert torch.equal(f1, f2)


from certificates import closed as _closed, dominated as _dominated  # noqa: E402


def test_work_counters_count_the_executed_process():
    """jatam_profile(2) counts exactly the placements the kernel performs: every
    replicate of every genotype the pre-filter left, except that a DET genotype
    whose replicate 0 was forced (a single frontier site at every draw), closed
    or dominated stops after replicate 0 (each fixes the outcome of all
    replicates)."""
    n, c, L, k, seed = 2, 8, 16, 20, 2
    genomes = W.random_genomes(3000, n, c, seed=21)  # stream id = the genome itself
    want = {"placements": 0, "seeds": 0, "genotypes": 0}
    ref = []
    for g in genomes.tolist():
        col = O.decode(g, n, c)
        r = O.classify(n, c, L, k, seed, col, g, want_grid=True, trace_rep=0)
        ref.append((r["cls"], r["decided_rep"], r["size"], r["shape_hash"]))
        at_seed = r["placements"] == 0 and r["decided_rep"] == 0 and r["cls"] in (1, 3)
        lone = r["cls"] == 0 and r["size"] == 1
        if at_seed or lone:
            continue
        want["genotypes"] += 1
        if r["cls"] == 0 and (all(t[0] <= 1 for t in r["trace"]) or _closed(list(col), n, c, r["grid"])
                              or _dominated(list(col), n, c, r["grid"])):
            want["placements"] += r["size"] - 1
            want["seeds"] += 1
        else:
            want["placements"] += r["placements"]
            want["seeds"] += min(r["decided_rep"] + 1, k)
    dg = torch.from_numpy(genomes.view(np.int64)).cuda()
    out = torch.full((len(genomes) * 8,), 0xEE, dtype=torch.uint8, device="cuda")
    fit = torch.empty(len(genomes), dtype=torch.int32, device="cuda")
    J.jatam_profile(2)
    try:
        J.evaluate_genomes(dg, fit, n=n, c=c, L=L, k=k, seed=seed, out=out, sync=True)
        got = J.work_counters()
    finally:
        J.jatam_profile(0)
    res = J.results_view(out)
    assert [tuple(x) for x in res.tolist()] == ref
    assert {key: got[key] for key in want} == want
    assert got["lane_slots"] % 32 == 0 and got["lane_slots"] >= got["placements"] + got["seeds"]


@pytest.mark.parametrize("n,c,L,k,seed,count", [(2, 4, 16, 10, 1, 1 << 16), (2, 8, 16, 20, 2, 300000),
                                                (3, 4, 8, 6, 5, 200000), (2, 8, 16, 20, 2, 1 << 20)])
def test_orbit_mode_matches_oracle(n, c, L, k, seed, count):
    """JATAM_ORBITS: every genotype gets its orbit representative's result
    (classified with the representative as stream id), equal to the oracle's
    orbit mode; the histogram counts every genotype under its representative's
    stream id."""
    res, hist, m = _dev_enumerate_orbits(n, c, L, k, seed, count)
    want, reps = O.enumerate_orbits(n, c, L, k, seed, count)
    assert np.array_equal(res, want)
    assert _hist_rows(hist) == _hist_rows(_oracle_hist(want, reps))


def _dev_enumerate_orbits(n, c, L, k, seed, count, hist_cap=1 << 16):
    out = torch.full((count * 8,), 0xEE, dtype=torch.uint8, device="cuda")
    hist = torch.empty(hist_cap * 32, dtype=torch.uint8, device="cuda")
    hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
    J.enumerate_space(n, c, L, k, seed, 0, count, out=out, hist=hist, hist_len=hlen, hist_cap=hist_cap, sync=True,
                      orbits=True)
    m = int(hlen.item())
    return J.results_view(out)[:count], J.hist_view(hist, min(m, hist_cap)), m


def test_orbit_mode_rejects_ranges_not_starting_at_zero():
    out = torch.empty(16 * 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(J.JatamError) as e:
        J.enumerate_space(2, 8, 16, 20, 2, 5, 16, out=out, sync=True, orbits=True)
    assert e.value.code == J.JATAM_EINVAL


@pytest.mark.parametrize("case", ["s24_full", "s28_slice", "s38_sample_L32", "s28_large"])
def test_movelist_process_matches_oracle(case):
    """JATAM_LIFO: the movelist process of Section 2.4 (stack of frontier sites,
    new sites pushed in a drawn order, the top one placed) equals the oracle's
    movelist process, results and histogram."""
    if case == "s24_full":
        n, c, L, k, seed, first, count, _ = W.WORKLOADS["s24_full"]
        sampled = False
    elif case == "s28_slice":
        n, c, L, k, seed, sampled = 2, 8, 16, 20, 2, False
        first, count = 7 * (1 << 20) + 11, 30000
    elif case == "s28_large":  # large enough for the heavy-first list
        n, c, L, k, seed, sampled = 2, 8, 16, 20, 2, False
        first, count = 3 << 20, 1 << 20
    else:
        n, c, L, k, seed, _, _, _ = W.WORKLOADS["s38_sample"]
        first, count, sampled = 4242, 20000, True
    out = torch.full((count * 8,), 0xEE, dtype=torch.uint8, device="cuda")
    hist = torch.empty((1 << 16) * 32, dtype=torch.uint8, device="cuda")
    hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
    J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out, hist=hist, hist_len=hlen,
                      hist_cap=1 << 16, sync=True, lifo=True)
    res = J.results_view(out)[:count]
    with O.process_mode(True):
        ref, _ = O.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled)
    assert np.array_equal(res, ref)
    if sampled:
        ids = np.array([O.sample_genotype(first + i, n, c, seed) for i in range(count)], np.uint64)
    else:
        ids = np.arange(first, first + count, dtype=np.uint64)
    m = int(hlen.item())
    assert _hist_rows(J.hist_view(hist, m)) == _hist_rows(_oracle_hist(ref, ids))
    # a different process: some results differ from the row-major one
    plain, _ = O.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled)
    assert not np.array_equal(plain, ref)
