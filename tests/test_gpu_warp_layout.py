"""One genotype per warp (lattice rows in lanes, in registers) against the
oracle and against one genotype per lane: per-genotype results, histograms and
the shape side table must be identical, on 32 x 32 and ragged lattices of
17 to 32, few and many replicates, every tile count and colour count."""
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


class layout:
    """Set the layout of the (n, c, L) key for the duration of a block."""

    def __init__(self, n, c, L, per_warp):
        self.key = (n, c, L)
        self.per_warp = per_warp

    def __enter__(self):
        J.set_genotypes_per_warp(*self.key, self.per_warp)
        assert J.get_genotypes_per_warp(*self.key) == self.per_warp

    def __exit__(self, *exc):
        J.set_genotypes_per_warp(*self.key, 0)


def _run(n, c, L, k, seed, first, count, sampled, per_warp, cap=1 << 14, c4_hash=False):
    with layout(n, c, L, per_warp):
        out = torch.full((count * 8,), 0xEE, dtype=torch.uint8, device="cuda")
        hist = torch.empty(cap * 32, dtype=torch.uint8, device="cuda")
        hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
        J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out, hist=hist, hist_len=hlen,
                          hist_cap=cap, sync=True, c4_hash=c4_hash)
        shapes = None if c4_hash else J.last_shapes()
    rows = [tuple(int(v) for v in r) for r in J.hist_view(hist, int(hlen.item())).tolist()]
    return J.results_view(out)[:count].copy(), rows, shapes


def _same_shapes(a, b):
    (ea, ca), (eb, cb) = a, b
    assert ca == 0 and cb == 0
    assert ea.tobytes() == eb.tobytes()


@pytest.mark.parametrize("case", [
    (3, 8, 32, 20, 3, 777, 40000, True),     # S_{3,8} sample, the 32 x 32 workload
    (2, 8, 32, 20, 2, 5 << 20, 40000, False),
    (2, 8, 19, 8, 2, 3 << 20, 40000, False),  # the paper's 19 x 19, k = 8
    (3, 8, 17, 3, 5, 0, 30000, True),
    (4, 8, 25, 2, 9, 0, 20000, True),
    (2, 4, 31, 1, 1, 0, 1 << 16, False),
    (1, 8, 24, 5, 4, 0, 4096, False),
])
def test_warp_layout_matches_oracle_and_lane_layout(case):
    n, c, L, k, seed, first, count, sampled = case
    got, hist_w, shapes_w = _run(n, c, L, k, seed, first, count, sampled, 1)
    ref, _ = O.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled)
    assert np.array_equal(got, ref)
    lane, hist_l, shapes_l = _run(n, c, L, k, seed, first, count, sampled, 32)
    assert np.array_equal(lane, ref)
    assert hist_w == hist_l
    _same_shapes(shapes_w, shapes_l)


def test_warp_layout_c4_hash_matches_oracle():
    n, c, L, k, seed, first, count = 3, 8, 32, 20, 3, 4242, 30000
    got, _, _ = _run(n, c, L, k, seed, first, count, True, 1, c4_hash=True)
    with O.hash_mode(True):
        ref, _ = O.enumerate_space(n, c, L, k, seed, first, count, sampled=True)
    assert np.array_equal(got, ref)


def test_warp_layout_records_of_every_tile_and_colour_count():
    rng = np.random.default_rng(17)
    for n, c, L in ((1, 8, 32), (2, 6, 29), (3, 4, 32), (4, 8, 20), (4, 2, 32), (2, 1, 18)):
        N = 6000
        colours = np.zeros((N, 16), np.uint8)
        colours[:, : 4 * n] = rng.integers(0, c, size=(N, 4 * n))
        ref, _ = O.classify_batch(colours, n=n, c=c, L=L, k=7, seed=99)
        with layout(n, c, L, 1):
            out = np.zeros(N, J.RESULT_DTYPE)
            J.classify_batch(colours, n=n, c=c, L=L, k=7, seed=99, out=out)
        assert np.array_equal(out, ref), (n, c, L)


def test_warp_layout_2e20_sample_matches_golden():
    """The 2^20 S_{3,8} golden with one genotype per warp (the heavy-first list
    is used at this size)."""
    n, c, L, k, seed, _, _, _ = W.WORKLOADS["s38_sample"]
    got, rows, shapes = _run(n, c, L, k, seed, 0, 1 << 20, True, 1, cap=1 << 16)
    gold = json.load(open(os.path.join(GOLDEN, "c3s_summary.json")))
    assert hashlib.sha256(got.tobytes()).hexdigest() == gold["results_sha256"]
    want = [tuple(int(v) for v in line.split()) for line in open(os.path.join(GOLDEN, "c3s_histogram.txt"))
            if not line.startswith("#")]
    assert [(r[0], r[1], r[2], r[4], r[5]) for r in rows] == want
    assert shapes[1] == 0


def test_work_counters_and_autotune_cover_the_warp_layout():
    """jatam_autotune times both layouts of a 32 x 32 key and keeps one; the
    results do not change with the choice."""
    n, c, L, k, seed = 3, 8, 32, 20, 3
    J.autotune([{"n": n, "c": c, "L": L, "k": k, "seed": seed, "sampled": True}])
    choice = J.get_genotypes_per_warp(n, c, L)
    assert choice in (1, 32)
    got, _, _ = _run(n, c, L, k, seed, 99, 20000, True, choice)
    ref, _ = O.enumerate_space(n, c, L, k, seed, 99, 20000, sampled=True)
    assert np.array_equal(got, ref)
    J.set_genotypes_per_warp(n, c, L, 0)
