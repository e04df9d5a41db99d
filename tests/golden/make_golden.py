"""Write the stored expected values under tests/golden/ -- calls only oracle/.

    python tests/golden/make_golden.py [c1] [c2] [c3]

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


def write_mixed(name, count, seed):
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
    print(name, meta, flush=True)


def write(name):
    if name == "c4s":
        return write_mixed(name, 1_000_000, 4)
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
