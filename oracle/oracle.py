"""CPU oracle for the JaTAM classification path -- TEST INFRASTRUCTURE.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this module.  It wraps ``jatam_oracle.c`` (plain C, compiled with gcc
by :func:`build`) through ctypes and adds the histogram of Section 2.6 of the
paper ("Exploiting CPU and GPU concurrently": count how often each shape hash
occurs) as a plain numpy group-by.  It never loads the CUDA library and the
CUDA library never loads it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "jatam_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")

DET_BOUNDED, ND_LOCAL, ND_STERIC, UNBOUNDED = 0, 1, 2, 3
CLASS_NAMES = {DET_BOUNDED: "det_bounded", ND_LOCAL: "nd_local", ND_STERIC: "nd_steric", UNBOUNDED: "unbounded"}

RESULT_DTYPE = np.dtype([("cls", "u1"), ("decided_rep", "u1"), ("size", "<u2"), ("shape_hash", "<u4")])


class _Result(ctypes.Structure):
    _fields_ = [("cls", ctypes.c_uint8), ("decided_rep", ctypes.c_uint8), ("size", ctypes.c_uint16),
                ("shape_hash", ctypes.c_uint32)]


class _Trace(ctypes.Structure):
    _fields_ = [("nfront", ctypes.c_int32), ("u", ctypes.c_uint32), ("index", ctypes.c_int32),
                ("x", ctypes.c_int32), ("y", ctypes.c_int32), ("tuple", ctypes.c_int32)]


class _GA(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("c", ctypes.c_int), ("selection", ctypes.c_int), ("tournament", ctypes.c_int),
                ("crossover", ctypes.c_int), ("crossover_threshold", ctypes.c_uint32),
                ("mutation_thresholds", ctypes.c_uint32 * 4), ("seed", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11 + pthreads) into oracle/_build."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-Wall", "-fPIC", "-shared", "-pthread", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            i32p = ctypes.POINTER(ctypes.c_int32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_philox4x32_10.restype = None
            L.orc_oaat.argtypes = [u8p, ctypes.c_uint64]
            L.orc_oaat.restype = ctypes.c_uint32
            L.orc_bind.argtypes = [ctypes.c_int, ctypes.c_int]
            L.orc_bind.restype = ctypes.c_int
            L.orc_decode.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, u8p]
            L.orc_decode.restype = ctypes.c_int
            L.orc_sample_genotype.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_uint64]
            L.orc_sample_genotype.restype = ctypes.c_uint64
            L.orc_sample_genotypes.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_uint64, ctypes.c_void_p]
            L.orc_sample_genotypes.restype = None
            L.orc_shape_table_begin.argtypes = []
            L.orc_shape_table_begin.restype = ctypes.c_int
            L.orc_shape_table_end.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int), u64p, u64p]
            L.orc_shape_table_end.restype = ctypes.c_int
            L.orc_shape_table_add.argtypes = [ctypes.c_uint32, u8p, ctypes.c_int, ctypes.c_int]
            L.orc_shape_table_add.restype = None
            L.orc_set_nd_detail.argtypes = [ctypes.c_int]
            L.orc_set_nd_detail.restype = None
            L.orc_canonical.argtypes = [i32p, i32p, ctypes.c_int, u8p, i32p, i32p]
            L.orc_canonical.restype = ctypes.c_int
            L.orc_shape_hash.argtypes = [u8p, ctypes.c_int, ctypes.c_int]
            L.orc_shape_hash.restype = ctypes.c_uint32
            L.orc_classify_ex.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                          u8p, ctypes.c_uint64, ctypes.POINTER(_Result), u64p, i32p, ctypes.c_int,
                                          ctypes.POINTER(_Trace), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            L.orc_classify_ex.restype = ctypes.c_int
            L.orc_enumerate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                        ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int,
                                        u64p]
            L.orc_enumerate.restype = ctypes.c_int
            L.orc_classify_batch.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p,
                                             ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int, u64p]
            L.orc_classify_batch.restype = ctypes.c_int
            L.orc_ga_breed.argtypes = [ctypes.POINTER(_GA), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_void_p]
            L.orc_ga_breed.restype = ctypes.c_int
            L.orc_poisson_thresholds.argtypes = [ctypes.c_double, u32p]
            L.orc_poisson_thresholds.restype = ctypes.c_int
            L.orc_roulette_pick.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]
            L.orc_roulette_pick.restype = ctypes.c_uint64
            L.orc_c4_hash.argtypes = [i32p, i32p, ctypes.c_int]
            L.orc_c4_hash.restype = ctypes.c_uint32
            L.orc_set_hash_mode.argtypes = [ctypes.c_int]
            L.orc_set_hash_mode.restype = None
            L.orc_colour_automorphism_count.argtypes = [ctypes.c_int]
            L.orc_colour_automorphism_count.restype = ctypes.c_int
            L.orc_orbit_rep.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
            L.orc_orbit_rep.restype = ctypes.c_uint64
            L.orc_orbit_reps.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_uint64)]
            L.orc_orbit_reps.restype = ctypes.c_int
            L.orc_set_process.argtypes = [ctypes.c_int]
            L.orc_set_process.restype = None
            L.orc_lifo_permutation.argtypes = [ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            L.orc_lifo_permutation.restype = None
            L.orc_hamming.argtypes = [ctypes.c_uint64]
            L.orc_hamming.restype = ctypes.c_int
            _lib = L
    return _lib


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# primitives
# ---------------------------------------------------------------------------
def philox(ctr, key):
    """Philox4x32-10 of one counter (4 x u32) under one key (2 x u32)."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def oaat(data: bytes) -> int:
    buf = np.frombuffer(bytes(data), dtype=np.uint8).copy() if len(data) else np.zeros(1, np.uint8)
    return int(lib().orc_oaat(_u8(buf), len(data)))


def bind(a: int, b: int) -> bool:
    return bool(lib().orc_bind(int(a), int(b)))


def decode(g: int, n: int, c: int) -> np.ndarray:
    col = np.zeros(16, np.uint8)
    rc = lib().orc_decode(int(g), int(n), int(c), _u8(col))
    if rc != 0:
        raise ValueError("c must be a power of two and 1 <= n <= 4")
    return col


def sample_genotype(i: int, n: int, c: int, seed: int) -> int:
    return int(lib().orc_sample_genotype(int(i), int(n), int(c), int(seed)))


def sample_genotypes(first: int, count: int, n: int, c: int, seed: int) -> np.ndarray:
    """The sampled genotypes of indices first .. first+count-1."""
    out = np.zeros(int(count), np.uint64)
    lib().orc_sample_genotypes(int(first), int(count), int(n), int(c), int(seed), out.ctypes.data)
    return out


def canonical(cells):
    """Canonical bitmap (h x w uint8 array) of a set of (x, y) cells."""
    cells = list(cells)
    m = len(cells)
    xs = np.array([c[0] for c in cells] or [0], np.int32)
    ys = np.array([c[1] for c in cells] or [0], np.int32)
    out = np.zeros(65 * 65, np.uint8)
    h = ctypes.c_int32()
    w = ctypes.c_int32()
    rc = lib().orc_canonical(xs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             ys.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), m, _u8(out),
                             ctypes.byref(h), ctypes.byref(w))
    if rc != 0:
        raise ValueError("shape too large")
    return out[: h.value * w.value].reshape(h.value, w.value).copy()


def shape_hash(bitmap) -> int:
    bm = np.ascontiguousarray(bitmap, dtype=np.uint8)
    h, w = bm.shape if bm.size else (0, 0)
    flat = bm.reshape(-1) if bm.size else np.zeros(1, np.uint8)
    return int(lib().orc_shape_hash(_u8(flat), h, w))


# ---------------------------------------------------------------------------
# classification
# ---------------------------------------------------------------------------
def classify(n, c, L, k, seed, col, stream_id, *, want_grid=False, trace_rep=-1, trace_cap=4096):
    """Classify one genotype from its colours col[4t + e]; returns a dict."""
    colv = np.zeros(16, np.uint8)
    colv[: len(col)] = np.asarray(col, dtype=np.uint8)
    res = _Result()
    placements = ctypes.c_uint64(0)
    grid = np.full(L * L, -1, np.int32) if want_grid else None
    trace = (_Trace * trace_cap)() if trace_rep >= 0 else None
    tlen = ctypes.c_int(0)
    rc = lib().orc_classify_ex(int(n), int(c), int(L), int(k), int(seed), _u8(colv), int(stream_id),
                               ctypes.byref(res), ctypes.byref(placements),
                               grid.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if want_grid else None,
                               int(trace_rep), trace, int(trace_cap), ctypes.byref(tlen))
    if rc != 0:
        raise ValueError(f"oracle rejected the genotype (rc={rc})")
    out = {"cls": res.cls, "decided_rep": res.decided_rep, "size": res.size, "shape_hash": res.shape_hash,
           "placements": placements.value}
    if want_grid:
        out["grid"] = grid.reshape(L, L)
    if trace is not None:
        out["trace"] = [(t.nfront, t.u, t.index, t.x, t.y, t.tuple) for t in trace[: tlen.value]]
    return out


def enumerate_space(n, c, L, k, seed, first, count, *, sampled=False, nthreads=None):
    """Classify indices first .. first+count-1 of S_{n,c}; returns (results, placements)."""
    out = np.zeros(int(count), RESULT_DTYPE)
    pl = ctypes.c_uint64(0)
    rc = lib().orc_enumerate(int(n), int(c), int(L), int(k), int(seed), int(bool(sampled)), int(first), int(count),
                             out.ctypes.data, int(nthreads or default_threads()), ctypes.byref(pl))
    if rc != 0:
        raise ValueError(f"oracle enumerate failed (rc={rc})")
    return out, pl.value


def classify_batch(cols, *, shapes=None, n=0, c=0, L=0, k=0, seed=0, ids=None, nthreads=None):
    """Classify explicit colour records cols[N][16] (shapes[N][4] = n, c, L, k)."""
    cols = np.ascontiguousarray(cols, dtype=np.uint8).reshape(-1, 16)
    N = cols.shape[0]
    shp = None if shapes is None else np.ascontiguousarray(shapes, dtype=np.uint8).reshape(N, 4)
    idv = None if ids is None else np.ascontiguousarray(ids, dtype=np.uint64).reshape(N)
    out = np.zeros(N, RESULT_DTYPE)
    pl = ctypes.c_uint64(0)
    rc = lib().orc_classify_batch(cols.ctypes.data, None if shp is None else shp.ctypes.data, int(n), int(c),
                                  int(L), int(k), int(seed), None if idv is None else idv.ctypes.data, N,
                                  out.ctypes.data, int(nthreads or default_threads()), ctypes.byref(pl))
    if rc != 0:
        raise ValueError(f"oracle batch failed (rc={rc})")
    return out, pl.value


HIST_DTYPE = np.dtype([("cls", "<u4"), ("shape_hash", "<u4"), ("size", "<u4"), ("pad", "<u4"),
                       ("count", "<u8"), ("min_id", "<u8")])


def histogram(results, ids=None):
    """Phenotype histogram of per-genotype results: one row per distinct
    (class, shape hash), sorted by that key, with the count, the shape size and
    the smallest stream id that produced it."""
    res = np.asarray(results)
    if ids is None:
        ids = np.arange(res.shape[0], dtype=np.uint64)
    ids = np.asarray(ids, dtype=np.uint64)
    key = (res["cls"].astype(np.uint64) << np.uint64(32)) | res["shape_hash"].astype(np.uint64)
    order = np.lexsort((ids, key))
    ks = key[order]
    if ks.size == 0:
        return np.zeros(0, HIST_DTYPE)
    starts = np.flatnonzero(np.concatenate(([True], ks[1:] != ks[:-1])))
    counts = np.diff(np.concatenate((starts, [ks.size])))
    h = np.zeros(starts.size, HIST_DTYPE)
    h["cls"] = (ks[starts] >> np.uint64(32)).astype(np.uint32)
    h["shape_hash"] = (ks[starts] & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    h["size"] = res["size"][order][starts]
    h["count"] = counts
    h["min_id"] = ids[order][starts]
    return h


def size_collisions(results):
    """Keys whose genotypes disagree on the shape size (a detected hash collision)."""
    res = np.asarray(results)
    key = (res["cls"].astype(np.uint64) << np.uint64(32)) | res["shape_hash"].astype(np.uint64)
    pairs = np.unique(np.stack([key, res["size"].astype(np.uint64)], axis=1), axis=0)
    k, cnt = np.unique(pairs[:, 0], return_counts=True)
    return k[cnt > 1]


# ---------------------------------------------------------------------------
# genetic algorithm (Section 2.2; the paper's appendix on GA operators)
# ---------------------------------------------------------------------------
TOURNAMENT, ROULETTE = 0, 1
NO_CROSSOVER, ONE_POINT, UNIFORM = 0, 1, 2


def poisson_thresholds(rate: float):
    """floor(2^32 P(K <= j)), j = 0..3, K ~ Poisson(rate)."""
    out = (ctypes.c_uint32 * 4)()
    if lib().orc_poisson_thresholds(float(rate), out) != 0:
        raise ValueError("rate must be >= 0")
    return [int(v) for v in out]


def hamming(g: int) -> int:
    """The paper's Fujiyama test-bed fitness: the number of set bits."""
    return int(lib().orc_hamming(int(g)))


def ga_breed(parents, fitness, generation, *, n, c, seed, selection=TOURNAMENT, tournament=4,
             crossover=NO_CROSSOVER, crossover_threshold=0, mutation_thresholds=(0xFFFFFFFF,) * 4):
    """One generation: children from parents and their fitness values."""
    parents = np.ascontiguousarray(parents, dtype=np.uint64)
    fitness = np.ascontiguousarray(fitness, dtype=np.int32)
    N = parents.shape[0]
    g = _GA(n=n, c=c, selection=selection, tournament=tournament, crossover=crossover,
            crossover_threshold=crossover_threshold, seed=seed)
    for j in range(4):
        g.mutation_thresholds[j] = int(mutation_thresholds[j])
    children = np.zeros(N, np.uint64)
    rc = lib().orc_ga_breed(ctypes.byref(g), parents.ctypes.data, fitness.ctypes.data, N, int(generation),
                            children.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle ga_breed failed (rc={rc})")
    return children


def roulette_pick(weights, dart):
    """Index chosen by the cumulative search of the roulette wheel."""
    cs = np.cumsum(np.asarray(weights, dtype=np.uint64)).astype(np.uint64)
    return int(lib().orc_roulette_pick(cs.ctypes.data, cs.shape[0], int(dart)))


def c4_hash(cells) -> int:
    """The rotation-invariant hash variant of Section 2.5 (mirror images differ)."""
    cells = list(cells)
    xs = np.array([c[0] for c in cells] or [0], np.int32)
    ys = np.array([c[1] for c in cells] or [0], np.int32)
    return int(lib().orc_c4_hash(xs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 ys.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(cells)))


class shape_table:
    """Context manager: record the canonical form of every shape the
    classification calls inside it hash (the exact side table of Section
    2.5's hash).  After the block: `forms` maps each shape hash to its
    canonical form (h x w uint8 array) and `collisions` counts the forms that
    differed from the one already stored under their hash."""

    CAP = 1 << 16

    def __enter__(self):
        if lib().orc_shape_table_begin() != 0:
            raise MemoryError("oracle shape table")
        return self

    def add(self, hash_value, bitmap):
        """Store one form under a given hash, as the classification does."""
        bm = np.ascontiguousarray(bitmap, dtype=np.uint8)
        lib().orc_shape_table_add(int(hash_value), _u8(bm.reshape(-1)), bm.shape[0], bm.shape[1])

    def __exit__(self, *exc):
        hashes = np.zeros(self.CAP, np.uint32)
        hw = np.zeros(2 * self.CAP, np.int32)
        rows = np.zeros(32 * self.CAP, np.uint32)
        n = ctypes.c_int(0)
        col = ctypes.c_uint64(0)
        ovf = ctypes.c_uint64(0)
        lib().orc_shape_table_end(hashes.ctypes.data, hw.ctypes.data, rows.ctypes.data, self.CAP, ctypes.byref(n),
                                  ctypes.byref(col), ctypes.byref(ovf))
        self.collisions = int(col.value)
        self.overflow = int(ovf.value)
        self.forms = {}
        for i in range(min(n.value, self.CAP)):
            h, w = int(hw[2 * i]), int(hw[2 * i + 1])
            bm = np.array([[(int(rows[32 * i + y]) >> x) & 1 for x in range(w)] for y in range(h)], np.uint8)
            self.forms[int(hashes[i])] = bm.reshape(h, w)


class nd_detail:
    """Context manager (diagnostic): ND_LOCAL results carry in `size` the kind
    of ambiguity that decided them -- 1 when one neighbour alone offers two
    distinct tuples (trivial non-determinism), 2 when only different
    neighbours disagree (two arms meeting: first-order steric
    non-determinism, Section 2.4).  Classes and other fields are unchanged."""

    def __enter__(self):
        lib().orc_set_nd_detail(1)
        return self

    def __exit__(self, *exc):
        lib().orc_set_nd_detail(0)


class hash_mode:
    """Context manager: classify with the C4 hash variant (Section 2.5) instead
    of the canonical form under the 8 symmetries."""

    def __init__(self, c4: bool):
        self.c4 = bool(c4)

    def __enter__(self):
        lib().orc_set_hash_mode(int(self.c4))
        return self

    def __exit__(self, *exc):
        lib().orc_set_hash_mode(0)


# ---------------------------------------------------------------------------
# orbit mode (exact symmetries of the process)
# ---------------------------------------------------------------------------
def colour_automorphism_count(c) -> int:
    """Permutations of the c colours that preserve the binding matrix."""
    return int(lib().orc_colour_automorphism_count(int(c)))


def orbit_rep(g, n, c) -> int:
    """Smallest packed genotype of g's orbit under the colour permutations that
    preserve the binding matrix, turns of non-seed tiles and permutations of
    non-seed tiles (all of them applied)."""
    return int(lib().orc_orbit_rep(int(g), int(n), int(c)))


def orbit_reps(n, c, first, count):
    out = np.zeros(count, np.uint64)
    lib().orc_orbit_reps(int(n), int(c), int(first), int(count),
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


def enumerate_orbits(n, c, L, k, seed, count, *, nthreads=None):
    """The orbit mode of the enumeration over genotypes 0 .. count - 1: every
    genotype gets the result of classifying its orbit representative with the
    representative as stream id."""
    reps = orbit_reps(n, c, 0, count)
    uniq = np.unique(reps)
    cols = np.zeros((uniq.shape[0], 16), np.uint8)
    for i, g in enumerate(uniq.tolist()):
        cols[i, : 4 * n] = decode(g, n, c)[: 4 * n]
    res_u, _ = classify_batch(cols, n=n, c=c, L=L, k=k, seed=seed, ids=uniq, nthreads=nthreads)
    pos = np.searchsorted(uniq, reps)
    return res_u[pos], reps


# ---------------------------------------------------------------------------
# the movelist (LIFO) process of Section 2.4
# ---------------------------------------------------------------------------
class process_mode:
    """Context manager: classify with the movelist process (new frontier sites
    pushed on a stack in a drawn order, the top one placed) instead of the
    uniform draw over the row-major frontier."""

    def __init__(self, lifo: bool):
        self.lifo = bool(lifo)

    def __enter__(self):
        lib().orc_set_process(int(self.lifo))
        return self

    def __exit__(self, *exc):
        lib().orc_set_process(0)


def lifo_permutation(idx, m):
    """Push order of permutation number idx of m items (item pushed first ...)."""
    out = (ctypes.c_int * 4)()
    lib().orc_lifo_permutation(int(idx), int(m), out)
    return [out[i] for i in range(m)]
