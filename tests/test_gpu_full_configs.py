"""Full-size parity of the two largest workloads with the oracle's stored values
(tests/golden/make_golden.py, which calls only oracle/):

  * 2^28 genotypes sampled uniformly from S_{3,8} (three tile types, eight
    colours: the space of Section 3.3), 32 x 32 grid, 20 replicates, seed 3:
    SHA-256 of the 2 GiB result array (and of each 2^24 chunk, to locate a
    difference), class counts, every histogram row, and the largest
    deterministic bounded shapes found;
  * 10^7 explicit tile sets of mixed n, c, L, k (seed 4), in one persistent
    launch, in one CUDA-graph replay of it, and as per-size fixed launches.

Every comparison is exact."""
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


def _golden_hist(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        if not line.startswith("#"):
            rows.append(tuple(int(v) for v in line.split()))
    return rows


def _hist_rows(h):
    return [(int(r["cls"]), int(r["shape_hash"]), int(r["size"]), int(r["count"]), int(r["min_id"])) for r in h]


def largest_det(rows, top):
    """The DET keys with the most tiles (ties: more genotypes first, then hash)."""
    det = sorted((r for r in rows if r[0] == 0), key=lambda r: (-r[2], -r[3], r[1]))
    return [(r[2], r[1], r[3], r[4]) for r in det[:top]]


def test_s38_all_2e28_sampled_genotypes_match_golden():
    n, c, L, k, seed, first, count, sampled = W.WORKLOADS["s38_sample"]
    gold = json.load(open(os.path.join(GOLDEN, "c3_summary.json")))
    assert gold["workload"]["count"] == count and gold["workload"]["L"] == L and gold["workload"]["k"] == k
    cap = 1 << 16
    out = torch.full((count * 8,), 0xEE, dtype=torch.uint8, device="cuda")  # poisoned, 2 GiB
    hist = torch.empty(cap * 32, dtype=torch.uint8, device="cuda")
    hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
    J.enumerate_space(n, c, L, k, seed, first, count, sampled=True, out=out, hist=hist, hist_len=hlen,
                      hist_cap=cap, sync=True)
    m = int(hlen.item())
    rows = _hist_rows(J.hist_view(hist, m))
    assert rows == _golden_hist("c3_histogram.txt")
    sha = hashlib.sha256()
    counts = np.zeros(4, np.int64)
    chunk = gold["chunk"]
    for i, lo in enumerate(range(0, count, chunk)):
        part = out[lo * 8:(lo + chunk) * 8].cpu().numpy()
        b = part.tobytes()
        assert hashlib.sha256(b).hexdigest() == gold["chunk_sha256"][i], f"chunk {i}"
        sha.update(b)
        counts += np.bincount(part.view(J.RESULT_DTYPE)["cls"], minlength=4)
    assert sha.hexdigest() == gold["results_sha256"]
    assert counts.tolist() == gold["class_counts"]
    # the largest deterministic bounded shapes found, as the oracle reported them, with their
    # canonical forms in the call's side table of shapes (and no hash naming two forms)
    largest = json.load(open(os.path.join(GOLDEN, "c3_largest.json")))
    want = [(e["size"], e["shape_hash"], e["count"], e["min_id"]) for e in largest]
    assert largest_det(rows, len(want)) == want
    entries, collisions = J.last_shapes()
    assert collisions == 0
    forms = {int(e["shape_hash"]): J.shape_bitmap(e) for e in entries}
    assert sorted(forms) == sorted({r[1] for r in rows if r[0] in (0, 2)})
    for e in largest:
        bm = np.array([[1 if ch == "#" else 0 for ch in row] for row in e["canonical"]], np.uint8)
        assert np.array_equal(forms[e["shape_hash"]], bm), e["shape_hash"]
    # a few genotypes re-classified one at a time by the oracle
    res = J.results_view(out)
    rng = np.random.default_rng(11)
    for i in rng.integers(0, count, size=64).tolist():
        g = O.sample_genotype(i, n, c, seed)
        r = O.classify(n, c, L, k, seed, O.decode(g, n, c), g)
        assert (r["cls"], r["decided_rep"], r["size"], r["shape_hash"]) == tuple(res[i].tolist())


def _mixed(colours, shapes, per_shape, graph=False, hist_cap=1 << 14):
    N = colours.shape[0]
    out = torch.full((N * 8,), 0xEE, dtype=torch.uint8, device="cuda")
    hist = torch.empty(hist_cap * 32, dtype=torch.uint8, device="cuda")
    hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
    J.classify_batch(colours, seed=4, shapes=shapes, out=out, hist=hist, hist_len=hlen, hist_cap=hist_cap,
                     sync=True, per_shape=per_shape, graph=graph)
    return J.results_view(out), _hist_rows(J.hist_view(hist, int(hlen.item())))


def test_mixed_1e7_records_match_golden():
    gold = json.load(open(os.path.join(GOLDEN, "c4_summary.json")))
    colours, shapes = W.mixed_records(10_000_000, seed=4)
    assert hashlib.sha256(colours.tobytes() + shapes.tobytes()).hexdigest() == gold["inputs_sha256"]
    dc = torch.from_numpy(colours).cuda()
    ds = torch.from_numpy(shapes).cuda()
    want_hist = _golden_hist("c4_histogram.txt")
    for per_shape, graph in ((False, False), (False, True), (False, True), (True, False)):
        res, rows = _mixed(dc, ds, per_shape, graph)
        assert np.bincount(res["cls"], minlength=4).tolist() == gold["class_counts"], (per_shape, graph)
        assert hashlib.sha256(res.tobytes()).hexdigest() == gold["results_sha256"], (per_shape, graph)
        assert rows == want_hist, (per_shape, graph)


def test_s28_at_the_papers_settings_matches_the_oracle_counts():
    """All of S_{2,8} at the paper's 19 x 19 grid, k = 8, with its rotation-only
    hash (Section 2.5): the class counts equal the oracle's (the counts set
    beside Section 3.1's remarks), and no shape has both deterministic and
    sterically non-deterministic genotypes under these readings."""
    facts = json.load(open(os.path.join(GOLDEN, "s28_paper_facts.json")))
    w = facts["workload"]
    n, c, L, k, seed, count = w["n"], w["c"], w["L"], w["k"], w["seed"], w["count"]
    cap = 1 << 12
    out = torch.empty(count * 8, dtype=torch.uint8, device="cuda")
    hist = torch.empty(cap * 32, dtype=torch.uint8, device="cuda")
    hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
    J.enumerate_space(n, c, L, k, seed, 0, count, out=out, hist=hist, hist_len=hlen, hist_cap=cap, sync=True,
                      c4_hash=True)
    cls = J.results_view(out)["cls"]
    got = np.bincount(cls, minlength=4).tolist()
    want = facts["class_counts"]
    assert got == [want["det_bounded"], want["nd_local"], want["nd_steric"], want["unbounded"]]
    rows = _hist_rows(J.hist_view(hist, int(hlen.item())))
    det = {r[1] for r in rows if r[0] == 0}
    steric = {r[1] for r in rows if r[0] == 2}
    assert len(det & steric) == facts["shapes_with_det_and_nd_steric_genotypes"]["count"]


def test_window_on_a_ragged_lattice_matches_the_oracle():
    """A call large enough for the 16 x 16 window (2^23 genotypes of S_{2,8} on
    a 25 x 25 lattice, 5 replicates): every result and histogram row equals the
    oracle's, items that leave the window included."""
    n, c, L, k, seed, first, count = 2, 8, 25, 5, 9, 1 << 23, 1 << 23
    cap = 1 << 12
    out = torch.full((count * 8,), 0xEE, dtype=torch.uint8, device="cuda")
    hist = torch.empty(cap * 32, dtype=torch.uint8, device="cuda")
    hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
    J.enumerate_space(n, c, L, k, seed, first, count, out=out, hist=hist, hist_len=hlen, hist_cap=cap, sync=True)
    ref, _ = O.enumerate_space(n, c, L, k, seed, first, count)
    assert np.array_equal(J.results_view(out), ref)
    ids = np.arange(first, first + count, dtype=np.uint64)
    assert _hist_rows(J.hist_view(hist, int(hlen.item()))) == _hist_rows(O.histogram(ref, ids))
    assert J.last_shapes()[1] == 0


def test_window_on_the_first_2e24_sampled_genotypes_matches_golden():
    """The first 2^24 of the S_{3,8} sample through the window: the chunk digest
    the oracle stored."""
    n, c, L, k, seed, _, _, _ = W.WORKLOADS["s38_sample"]
    gold = json.load(open(os.path.join(GOLDEN, "c3_summary.json")))
    count = gold["chunk"]
    out = torch.empty(count * 8, dtype=torch.uint8, device="cuda")
    J.enumerate_space(n, c, L, k, seed, 0, count, sampled=True, out=out, sync=True)
    assert hashlib.sha256(out.cpu().numpy().tobytes()).hexdigest() == gold["chunk_sha256"][0]
