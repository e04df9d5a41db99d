"""Seeded synthetic workloads (input generators only -- none of the method's
arithmetic lives here).

The paper's workloads are the genotype spaces themselves (Section 2.1 and
Section 3): S_{2,8} (two tile types, eight colours, 8^8 genotypes) classified
in full, and a large slice of S_{3,8} (three tile types, 8^12 genotypes).  No
dataset is involved; a workload is fixed by (n, c, L, k, seed, index range).
"""
from __future__ import annotations

import numpy as np

# name -> (n, c, L, k, seed, first, count, sampled)
WORKLOADS = {
    # S_{2,4} in full: 4^8 = 65,536 genotypes, 16 x 16 grid, k = 10, seed 1
    "s24_full": (2, 4, 16, 10, 1, 0, 1 << 16, False),
    # S_{2,8} in full: 8^8 = 16,777,216 genotypes, 16 x 16 grid, k = 20, seed 2
    "s28_full": (2, 8, 16, 20, 2, 0, 1 << 24, False),
    # S_{2,8} with the paper's own settings: 19 x 19 grid, k = 8
    "s28_paper": (2, 8, 19, 8, 2, 0, 1 << 24, False),
    # 2^28 genotypes sampled uniformly from S_{3,8} (8^12), 32 x 32 grid, k = 20, seed 3
    "s38_sample": (3, 8, 32, 20, 3, 0, 1 << 28, True),
}


def splitmix64(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """count words of SplitMix64 (Steele, Lea, Flood 2014) started from
    seed + stream * 2^32: a version-stable generator for synthetic inputs."""
    with np.errstate(over="ignore"):
        x = np.uint64((seed + (stream << 32)) & 0xFFFFFFFFFFFFFFFF) + \
            np.arange(1, count + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
        z = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _below(words: np.ndarray, bound) -> np.ndarray:
    """Map 64-bit words to [0, bound) by the high 32 bits times bound."""
    hi = (words >> np.uint64(32)).astype(np.uint64)
    return ((hi * np.asarray(bound, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)


def mixed_records(count: int, seed: int = 4):
    """Explicit tile sets of mixed size: n uniform in {2, 3, 4}, c in {4, 6, 8},
    L in {8, 16, 32}, k in {10, 20}, every colour uniform in [0, c).  Drawn from
    SplitMix64 streams of `seed`.  Returns (colours [count][16] u8, shapes
    [count][4] u8 = (n, c, L, k))."""
    n = (2 + _below(splitmix64(seed, count, 0), 3)).astype(np.uint8)
    c = np.array([4, 6, 8], np.uint8)[_below(splitmix64(seed, count, 1), 3)]
    L = np.array([8, 16, 32], np.uint8)[_below(splitmix64(seed, count, 2), 3)]
    k = np.array([10, 20], np.uint8)[_below(splitmix64(seed, count, 3), 2)]
    colours = np.zeros((count, 16), np.uint8)
    for e in range(16):
        colours[:, e] = _below(splitmix64(seed, count, 4 + e), c.astype(np.uint64)).astype(np.uint8)
    colours[np.arange(16)[None, :] >= 4 * n[:, None]] = 0
    shapes = np.stack([n, c, L, k], axis=1).astype(np.uint8)
    return np.ascontiguousarray(colours), np.ascontiguousarray(shapes)


def random_genomes(count: int, n: int, c: int, seed: int):
    """Uniform packed genomes of S_{n,c} (SplitMix64 stream of `seed`)."""
    bits = 4 * n * (int(c).bit_length() - 1)
    g = splitmix64(seed, count, 100)
    if bits < 64:
        g &= np.uint64((1 << bits) - 1)
    return g
