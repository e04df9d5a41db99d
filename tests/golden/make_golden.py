"""Write the stored expected values under tests/golden/ -- calls only oracle/.

    python tests/golden/make_golden.py [c1] [c2] [c3s] [c3] [c4s] [c4] [facts]

For each workload it runs the CPU oracle and stores:
  * the SHA-256 of the per-genotype result array (8 bytes per genotype:
    class u8, decided replicate u8, size u16, shape hash u32, little endian),
  * the per-class genotype counts and the total number of placements,
  * the phenotype histogram (class, shape hash, size, count, smallest id).
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402

# (name, n, c, L, k, seed, first, count, sampled)
WORKLOADS = {
    # S_{2,4} in full: 4^8 genotypes, 16 x 16 grid, 10 replicates, seed 1
    "c1": (2, 4, 16, 10, 1, 0, 1 << 16, False),
    # S_{2,8} in full: 8^8 genotypes, 16 x 16 grid, 20 replicates, seed 2
    "c2": (2, 8, 16, 20, 2, 0, 1 << 24, False),
    # a 2^20-genotype uniform sample of S_{3,8}, 32 x 32 grid, 20 replicates, seed 3
    "c3s": (3, 8, 32, 20, 3, 0, 1 << 20, True),
}


def write_mixed(name, count, seed, histogram_file=False):
    """Explicit mixed-size tile sets from the seeded input generator (its
    SplitMix64 streams are the inputs; every result comes from the oracle)."""
    from paper_2205_15311_gb300 import workloads as WL  # input generator only
    colours, shapes = WL.mixed_records(count, seed=seed)
    t0 = time.time()
    res, placements = O.classify_batch(colours, shapes=shapes, seed=seed)
    dt = time.time() - t0
    hist = O.histogram(res, np.arange(count, dtype=np.uint64))
    meta = {
        "workload": {"mixed_records": count, "seed": seed},
        "inputs_sha256": hashlib.sha256(colours.tobytes() + shapes.tobytes()).hexdigest(),
        "results_sha256": hashlib.sha256(res.tobytes()).hexdigest(),
        "class_counts": np.bincount(res["cls"], minlength=4).tolist(),
        "placements": int(placements),
        "distinct_keys": int(hist.shape[0]),
        "oracle_seconds": round(dt, 1),
        "collisions": int(O.size_collisions(res).size),
    }
    with open(os.path.join(HERE, f"{name}_summary.json"), "w") as f:
        json.dump(meta, f, indent=1)
        f.write("\n")
    if histogram_file:
        with open(os.path.join(HERE, f"{name}_histogram.txt"), "w") as f:
            f.write("# cls shape_hash size count min_id\n")
            for h in hist:
                f.write(f"{int(h['cls'])} {int(h['shape_hash'])} {int(h['size'])} {int(h['count'])} "
                        f"{int(h['min_id'])}\n")
    print(name, meta, flush=True)


def largest_shapes(rows, n, c, L, k, seed, top=12):
    """The largest deterministic bounded shapes of a histogram: (size, hash,
    count, smallest id) of the DET keys with the most tiles, each with the
    canonical bitmap of its smallest genotype's replicate-0 shape as text rows
    ('#' occupied), from the oracle."""
    det = sorted((r for r in rows if r[0] == O.DET_BOUNDED), key=lambda r: (-r[2], -r[3], r[1]))[:top]
    out = []
    for cls, h, size, count, min_id in det:
        r = O.classify(n, c, L, k, seed, O.decode(min_id, n, c), min_id, want_grid=True)
        cells = [(x, y) for y in range(L) for x in range(L) if r["grid"][y, x] >= 0]
        bm = O.canonical(cells)
        assert r["cls"] == cls and r["shape_hash"] == h and len(cells) == size
        out.append({"size": size, "shape_hash": h, "count": count, "min_id": min_id,
                    "canonical": ["".join("#" if v else "." for v in row) for row in bm]})
    return out


def write_sampled_chunked(name, n, c, L, k, seed, count, chunk):
    """A sampled workload too large to hold at once: classified in chunks of
    `chunk` indices; the SHA-256 covers the whole result array (and one digest
    per chunk is kept), the histogram is merged over the chunks."""
    sha = hashlib.sha256()
    chunk_sha, cls_counts, placements, keys = [], np.zeros(4, np.int64), 0, {}
    t0 = time.time()
    for first in range(0, count, chunk):
        m = min(chunk, count - first)
        res, pl = O.enumerate_space(n, c, L, k, seed, first, m, sampled=True)
        placements += int(pl)
        b = res.tobytes()
        sha.update(b)
        chunk_sha.append(hashlib.sha256(b).hexdigest())
        cls_counts += np.bincount(res["cls"], minlength=4)
        ids = O.sample_genotypes(first, m, n, c, seed)
        sizes = {}
        for kk in O.size_collisions(res).tolist():
            sizes[kk] = True
        for h in O.histogram(res, ids):
            key = (int(h["cls"]), int(h["shape_hash"]))
            cur = keys.get(key)
            sz, cnt, mid = int(h["size"]), int(h["count"]), int(h["min_id"])
            if cur is None:
                keys[key] = [sz, sz, cnt, mid]
            else:
                cur[0], cur[1] = max(cur[0], sz), min(cur[1], sz)
                cur[2] += cnt
                cur[3] = min(cur[3], mid)
        print(name, first + m, "of", count, round(time.time() - t0, 1), "s", flush=True)
    dt = time.time() - t0
    rows = [(kk[0], kk[1], v[0], v[2], v[3]) for kk, v in sorted(keys.items())]
    collisions = sum(1 for v in keys.values() if v[0] != v[1])
    meta = {
        "workload": {"n": n, "c": c, "L": L, "k": k, "seed": seed, "first": 0, "count": count,
                     "sampled": True},
        "results_sha256": sha.hexdigest(),
        "chunk": chunk,
        "chunk_sha256": chunk_sha,
        "class_counts": cls_counts.tolist(),
        "placements": int(placements),
        "distinct_keys": len(rows),
        "oracle_seconds": round(dt, 1),
        "oracle_threads": O.default_threads(),
        "collisions": int(collisions),
    }
    with open(os.path.join(HERE, f"{name}_summary.json"), "w") as f:
        json.dump(meta, f, indent=1)
        f.write("\n")
    with open(os.path.join(HERE, f"{name}_histogram.txt"), "w") as f:
        f.write("# cls shape_hash size count min_id\n")
        for r in rows:
            f.write(" ".join(str(v) for v in r) + "\n")
    with open(os.path.join(HERE, f"{name}_largest.json"), "w") as f:
        json.dump(largest_shapes(rows, n, c, L, k, seed), f, indent=1)
        f.write("\n")
    print(name, meta, flush=True)


def write_paper_facts():
    """Section 3.1's two remarks on S_{2,8} at the paper's own settings (19 x 19
    grid, k = 8 replicates, the rotation-only hash of Section 2.5), set beside
    this model's counts: the ratio of sterically non-deterministic to unbounded
    genotypes, and which shapes have both deterministic and sterically
    non-deterministic genotypes.  Local ambiguity is split by the oracle's
    diagnostic into its trivial kind (one neighbour offers two tuples) and its
    first-order steric kind (two neighbours disagree), which Section 2.4
    detects with one check."""
    n, c, L, k, seed = 2, 8, 19, 8, 2
    count = 1 << 24
    t0 = time.time()
    with O.hash_mode(True), O.nd_detail():
        res, placements = O.enumerate_space(n, c, L, k, seed, 0, count)
    dt = time.time() - t0
    cls = res["cls"]
    counts = np.bincount(cls, minlength=4).tolist()
    nd = cls == O.ND_LOCAL
    kinds = np.bincount(res["size"][nd], minlength=3).tolist()
    det_keys = set(res["shape_hash"][cls == O.DET_BOUNDED].tolist())
    steric_keys = set(res["shape_hash"][cls == O.ND_STERIC].tolist())
    shared = sorted(det_keys & steric_keys)
    shared_sizes = sorted({int(res["size"][(cls == O.DET_BOUNDED) & (res["shape_hash"] == h)][0]) for h in shared})
    meta = {
        "workload": {"n": n, "c": c, "L": L, "k": k, "seed": seed, "count": count, "hash": "C4 (Section 2.5)"},
        "class_counts": {"det_bounded": counts[0], "nd_local": counts[1], "nd_steric": counts[2],
                         "unbounded": counts[3]},
        "nd_local_kinds": {"trivial": kinds[1], "first_order_steric": kinds[2]},
        "steric_to_unbounded": {
            "higher_order_only": round(counts[2] / counts[3], 4),
            "with_first_order": round((counts[2] + kinds[2]) / counts[3], 4),
            "paper": 2.2},
        "shapes_with_det_and_nd_steric_genotypes": {"count": len(shared), "sizes": shared_sizes,
                                                    "paper": "only the 12-mer"},
        "placements": int(placements),
        "oracle_seconds": round(dt, 1),
    }
    with open(os.path.join(HERE, "s28_paper_facts.json"), "w") as f:
        json.dump(meta, f, indent=1)
        f.write("\n")
    print(meta, flush=True)


def write(name):
    if name == "facts":
        return write_paper_facts()
    if name == "c4s":
        return write_mixed(name, 1_000_000, 4)
    if name == "c4":
        return write_mixed(name, 10_000_000, 4, histogram_file=True)
    if name == "c3":
        # all 2^28 sampled genotypes of S_{3,8}, 32 x 32 grid, 20 replicates, seed 3
        return write_sampled_chunked("c3", 3, 8, 32, 20, 3, 1 << 28, 1 << 24)
    if name == "c3chk":
        # the chunked writer on the first 2^20 (must reproduce c3s exactly)
        return write_sampled_chunked("c3chk", 3, 8, 32, 20, 3, 1 << 20, 1 << 18)
    n, c, L, k, seed, first, count, sampled = WORKLOADS[name]
    t0 = time.time()
    res, placements = O.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled)
    dt = time.time() - t0
    ids = (np.array([O.sample_genotype(i, n, c, seed) for i in range(first, first + count)], np.uint64)
           if sampled else None)
    digest = hashlib.sha256(res.tobytes()).hexdigest()
    hist = O.histogram(res, ids if ids is not None else (None if sampled else np.arange(first, first + count,
                                                                                          dtype=np.uint64)))
    meta = {
        "workload": {"n": n, "c": c, "L": L, "k": k, "seed": seed, "first": first, "count": count,
                     "sampled": sampled},
        "results_sha256": digest,
        "class_counts": np.bincount(res["cls"], minlength=4).tolist(),
        "placements": int(placements),
        "distinct_keys": int(hist.shape[0]),
        "oracle_seconds": round(dt, 1),
        "collisions": int(O.size_collisions(res).size),
    }
    with open(os.path.join(HERE, f"{name}_summary.json"), "w") as f:
        json.dump(meta, f, indent=1)
        f.write("\n")
    with open(os.path.join(HERE, f"{name}_histogram.txt"), "w") as f:
        f.write("# cls shape_hash size count min_id\n")
        for h in hist:
            f.write(f"{int(h['cls'])} {int(h['shape_hash'])} {int(h['size'])} {int(h['count'])} {int(h['min_id'])}\n")
    print(name, meta, flush=True)


if __name__ == "__main__":
    for nm in sys.argv[1:] or ["c1", "c2"]:
        write(nm)
