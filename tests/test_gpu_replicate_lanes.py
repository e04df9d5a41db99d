"""Replicate lanes (one genotype per warp, lane r growing replicate r of the
k independent assemblies of Section 2.4 side by side, the first deciding
replicate taken afterwards) against the oracle, and against the kernel that
grows one genotype per lane, replicate after replicate.  The cases cover every
tile count, ragged and degenerate lattices (L = 1, 2, 9), k from 1 to 32, the
sampled, genome and record inputs, the rotation-only hash, and the histogram
with its exact side table of shapes."""
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
    J.set_replicate_lanes(0)


def _hist_rows(h):
    return [(int(r["cls"]), int(r["shape_hash"]), int(r["size"]), int(r["count"]), int(r["min_id"])) for r in h]


def _enumerate(mode, n, c, L, k, seed, first, count, sampled=False, c4=False):
    J.set_replicate_lanes(mode)
    cap = 1 << 12
    out = torch.full((count * 8,), 0xEE, dtype=torch.uint8, device="cuda")
    hist = torch.empty(cap * 32, dtype=torch.uint8, device="cuda")
    hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
    J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out, hist=hist, hist_len=hlen,
                      hist_cap=cap, sync=True, c4_hash=c4)
    res = J.results_view(out).copy()
    rows = _hist_rows(J.hist_view(hist, int(hlen.item())))
    shapes = None
    if not c4:
        entries, collisions = J.last_shapes()
        assert collisions == 0
        shapes = {int(e["shape_hash"]): J.shape_bitmap(e) for e in entries}
    return res, rows, shapes


CASES = [  # n, c, L, k, seed, first, count, sampled
    (1, 8, 16, 20, 4, 0, 4096, False),
    (2, 8, 16, 20, 2, 5 << 20, 1 << 14, False),
    (2, 8, 9, 32, 7, 123456, 5000, False),
    (2, 8, 1, 3, 3, 0, 4096, False),
    (2, 8, 2, 5, 3, 77, 3000, False),
    (2, 4, 13, 1, 5, 1000, 3000, False),
    (3, 8, 16, 20, 3, 0, 1 << 13, True),
    (4, 4, 12, 7, 11, 0, 3000, True),
]


@pytest.mark.parametrize("case", CASES)
def test_replicate_lanes_match_oracle(case):
    n, c, L, k, seed, first, count, sampled = case
    with O.shape_table() as T:
        ref, _ = O.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled)
    ids = (O.sample_genotypes(first, count, n, c, seed) if sampled
           else np.arange(first, first + count, dtype=np.uint64))
    want_rows = _hist_rows(O.histogram(ref, ids))
    for mode in (2, 1):  # replicate lanes, then one genotype per lane
        res, rows, shapes = _enumerate(mode, n, c, L, k, seed, first, count, sampled)
        assert np.array_equal(res, ref), mode
        assert rows == want_rows, mode
        assert sorted(shapes) == sorted(T.forms), mode
        for key, bm in shapes.items():
            assert np.array_equal(bm, T.forms[key]), (mode, key)


def test_all_of_s24_matches_golden_with_replicate_lanes():
    """All 65,536 genotypes of S_{2,4} (L = 16, k = 10): the oracle's stored digest."""
    n, c, L, k, seed, first, count, _ = W.WORKLOADS["s24_full"]
    res, _, _ = _enumerate(2, n, c, L, k, seed, first, count)
    gold = json.load(open(os.path.join(GOLDEN, "c1_summary.json")))
    assert hashlib.sha256(res.tobytes()).hexdigest() == gold["results_sha256"]


def test_rotation_only_hash_and_genomes_with_replicate_lanes():
    n, c, L, k, seed = 3, 8, 16, 20, 9
    res2, rows2, _ = _enumerate(2, 2, 8, 16, 20, 2, 7 << 20, 1 << 13, c4=True)
    ref, _ = O.enumerate_space(2, 8, 16, 20, 2, 7 << 20, 1 << 13)
    assert np.array_equal(res2["cls"], ref["cls"]) and np.array_equal(res2["decided_rep"], ref["decided_rep"])
    res1, rows1, _ = _enumerate(1, 2, 8, 16, 20, 2, 7 << 20, 1 << 13, c4=True)
    assert np.array_equal(res1, res2) and rows1 == rows2
    # genomes (the GA's fitness call) of a random and of an evolved-looking population
    genomes = W.random_genomes(4096, n, c, seed=seed)
    fits = []
    for mode in (2, 1):
        J.set_replicate_lanes(mode)
        g = torch.from_numpy(genomes.view(np.int64)).cuda()
        fit = torch.empty(4096, dtype=torch.int32, device="cuda")
        J.evaluate_genomes(g, fit, n=n, c=c, L=L, k=k, seed=seed, sync=True)
        fits.append(fit.cpu().numpy())
    want = np.array([O.classify(n, c, L, k, seed, O.decode(int(x), n, c), int(x)) for x in genomes[:512].tolist()],
                    dtype=object)
    want_fit = np.array([r["size"] if r["cls"] == 0 else 0 for r in want])
    assert np.array_equal(fits[0], fits[1])
    assert np.array_equal(fits[0][:512], want_fit)
