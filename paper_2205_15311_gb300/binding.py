"""Thin ctypes binding of libjatam.so (include/jatam.h).

The functions named like the C ABI (``jatam_enumerate``, ``jatam_classify_batch``,
``ga_evaluate``, ``jatam_philox``, ``jatam_hist_merge``, ``jatam_shutdown``,
``jatam_last_error``) take raw addresses (ints) exactly as the C calls do.  The
helpers below them only marshal torch tensors or numpy arrays into those calls:
every step of the classification runs in the CUDA kernels of the library.
There is no CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB_PATH

JATAM_OK = 0
JATAM_EINVAL = -1
JATAM_ENOMEM = -2
JATAM_ECUDA = -3
JATAM_ETIMEOUT = -4
JATAM_EUNSUPPORTED = -5

DET_BOUNDED, ND_LOCAL, ND_STERIC, UNBOUNDED = 0, 1, 2, 3
JATAM_SAMPLED = 0x1
JATAM_SYNC = 0x2
JATAM_PER_SHAPE = 0x4
JATAM_GRAPH = 0x8
JATAM_C4_HASH = 0x10
JATAM_PERSISTENT = 0x20
JATAM_ORBITS = 0x40
JATAM_LIFO = 0x80
JATAM_NO_DEDUP = 0x100
JATAM_NOALLOC_MAX_COUNT = 1048576

RESULT_DTYPE = np.dtype([("cls", "u1"), ("decided_rep", "u1"), ("size", "<u2"), ("shape_hash", "<u4")])
HIST_DTYPE = np.dtype([("cls", "<u4"), ("shape_hash", "<u4"), ("size", "<u4"), ("flags", "<u4"),
                       ("count", "<u8"), ("min_id", "<u8")])


class jatam_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint8), ("c", ctypes.c_uint8), ("L", ctypes.c_uint8), ("k", ctypes.c_uint8),
                ("flags", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class jatam_ga_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint8), ("c", ctypes.c_uint8), ("selection", ctypes.c_uint8),
                ("tournament", ctypes.c_uint8), ("crossover", ctypes.c_uint8), ("reserved", ctypes.c_uint8 * 3),
                ("crossover_threshold", ctypes.c_uint32), ("mutation_thresholds", ctypes.c_uint32 * 4),
                ("seed", ctypes.c_uint64)]


TOURNAMENT, ROULETTE = 0, 1
NO_CROSSOVER, ONE_POINT, UNIFORM = 0, 1, 2
FITNESS_SHAPE, FITNESS_HAMMING = 0, 1


class JatamError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libjatam error {code}: {msg}")
        self.code = code


_lib = None
_VP = ctypes.c_void_p
_U64 = ctypes.c_uint64
_U32 = ctypes.c_uint32


def lib():
    """Load libjatam.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        L.jatam_enumerate.argtypes = [_VP, _U64, _U64, _VP, _VP, _U32, _VP, _VP]
        L.jatam_classify_batch.argtypes = [_VP, _VP, _VP, _VP, _U64, _VP, _VP, _U32, _VP, _VP]
        L.ga_evaluate.argtypes = [_VP, _VP, _U64, _VP, _VP, _VP]
        L.jatam_philox.argtypes = [_VP, _U64, _VP, _VP]
        L.jatam_hist_merge.argtypes = [_VP, _U32, _VP, _U32, _VP, _U32, _VP]
        for f in ("jatam_enumerate", "jatam_classify_batch", "ga_evaluate", "jatam_philox", "jatam_hist_merge"):
            getattr(L, f).restype = ctypes.c_int
        L.jatam_enumerate_noalloc.argtypes = [_VP, _U64, _U64, _VP, _VP]
        L.jatam_enumerate_noalloc.restype = ctypes.c_int
        L.jatam_last_shapes.argtypes = [_VP, _U32, ctypes.POINTER(_U32), ctypes.POINTER(_U32)]
        L.jatam_last_shapes.restype = ctypes.c_int
        L.jatam_set_genotypes_per_warp.argtypes = [_VP, ctypes.c_int]
        L.jatam_set_genotypes_per_warp.restype = ctypes.c_int
        L.jatam_get_genotypes_per_warp.argtypes = [_VP, ctypes.POINTER(ctypes.c_int)]
        L.jatam_get_genotypes_per_warp.restype = ctypes.c_int
        L.jatam_workspace_bytes.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        L.jatam_workspace_bytes.restype = ctypes.c_int
        L.jatam_mlp_create.argtypes = [_U64, ctypes.POINTER(_VP)]
        L.jatam_mlp_create.restype = ctypes.c_int
        L.jatam_mlp_destroy.argtypes = [_VP]
        L.jatam_mlp_destroy.restype = None
        L.jatam_mlp_set_params.argtypes = [_VP, _VP, _VP]
        L.jatam_mlp_set_params.restype = ctypes.c_int
        L.jatam_mlp_get_params.argtypes = [_VP, _VP, _VP]
        L.jatam_mlp_get_params.restype = ctypes.c_int
        L.jatam_mlp_train_step.argtypes = [_VP, _VP, _VP, _U64, ctypes.c_float, _VP, _VP, _VP]
        L.jatam_mlp_train_step.restype = ctypes.c_int
        L.jatam_mlp_predict.argtypes = [_VP, _VP, _U64, _VP, _VP]
        L.jatam_mlp_predict.restype = ctypes.c_int
        L.jatam_mlp_labels.argtypes = [_VP, _U64, _VP, _VP]
        L.jatam_mlp_labels.restype = ctypes.c_int
        L.jatam_embed_genomes.argtypes = [_VP, _U64, ctypes.c_int, ctypes.c_int, _VP, _VP]
        L.jatam_embed_genomes.restype = ctypes.c_int
        L.jatam_set_replicate_lanes.argtypes = [ctypes.c_int]
        L.jatam_set_replicate_lanes.restype = ctypes.c_int
        L.jatam_get_replicate_lanes.argtypes = []
        L.jatam_get_replicate_lanes.restype = ctypes.c_int
        L.jatam_select_top.argtypes = [_VP, _U64, _U64, _VP, _VP]
        L.jatam_select_top.restype = ctypes.c_int
        L.ga_run_screened.argtypes = [_VP, _VP, _U64, _U32, _U32, _VP, ctypes.c_float, _VP, _VP, _VP, _VP]
        L.ga_run_screened.restype = ctypes.c_int
        L.ga_breed.argtypes = [_VP, _VP, _VP, _U64, _U32, _VP, _VP]
        L.ga_breed.restype = ctypes.c_int
        L.ga_hamming.argtypes = [_VP, _U64, _VP, _VP]
        L.ga_hamming.restype = ctypes.c_int
        L.ga_poisson_thresholds.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_uint32)]
        L.ga_poisson_thresholds.restype = ctypes.c_int
        L.ga_run.argtypes = [_VP, _VP, ctypes.c_int, _U64, _U32, _VP, _VP, _VP, _VP]
        L.ga_run.restype = ctypes.c_int
        L.jatam_set_mixed_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.jatam_set_mixed_plan.restype = ctypes.c_int
        L.jatam_get_mixed_plan.argtypes = [ctypes.POINTER(ctypes.c_int)] * 3
        L.jatam_get_mixed_plan.restype = ctypes.c_int
        L.jatam_get_mixed_launch.argtypes = [ctypes.POINTER(ctypes.c_int)]
        L.jatam_get_mixed_launch.restype = ctypes.c_int
        L.jatam_autotune_batch.argtypes = [_VP, _VP, _U64, _U64, _VP]
        L.jatam_autotune_batch.restype = ctypes.c_int
        L.jatam_autotune.argtypes = [_VP, _U32, _VP]
        L.jatam_autotune.restype = ctypes.c_int
        L.jatam_set_tuning.argtypes = [_VP, ctypes.c_int, ctypes.c_int]
        L.jatam_set_tuning.restype = ctypes.c_int
        L.jatam_get_tuning.argtypes = [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.jatam_get_tuning.restype = ctypes.c_int
        L.jatam_profile.argtypes = [ctypes.c_int]
        L.jatam_profile.restype = ctypes.c_int
        L.jatam_kernel_ms.argtypes = [ctypes.POINTER(ctypes.c_float)]
        L.jatam_kernel_ms.restype = ctypes.c_int
        L.jatam_work_counters.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        L.jatam_work_counters.restype = ctypes.c_int
        L.jatam_shutdown.argtypes = []
        L.jatam_shutdown.restype = None
        L.jatam_last_error.argtypes = []
        L.jatam_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# the C ABI, one to one
# ---------------------------------------------------------------------------
def jatam_enumerate(cfg, first, count, out, hist, hist_cap, hist_len, stream):
    return lib().jatam_enumerate(cfg, first, count, out, hist, hist_cap, hist_len, stream)


def jatam_classify_batch(cfg, colours, shapes, stream_ids, N, out, hist, hist_cap, hist_len, stream):
    return lib().jatam_classify_batch(cfg, colours, shapes, stream_ids, N, out, hist, hist_cap, hist_len, stream)


def ga_evaluate(cfg, genomes, N, fitness, out, stream):
    return lib().ga_evaluate(cfg, genomes, N, fitness, out, stream)


def jatam_philox(inp, N, out, stream):
    return lib().jatam_philox(inp, N, out, stream)


def jatam_hist_merge(a, na, b, nb, out, cap, length):
    return lib().jatam_hist_merge(a, na, b, nb, out, cap, length)


def jatam_get_mixed_launch(per_shape):
    return lib().jatam_get_mixed_launch(per_shape)


def jatam_enumerate_noalloc(cfg, first, count, out, stream):
    return lib().jatam_enumerate_noalloc(cfg, first, count, out, stream)


def ga_breed(ga, parents, fitness, N, generation, children, stream):
    return lib().ga_breed(ga, parents, fitness, N, generation, children, stream)


def ga_hamming(genomes, N, fitness, stream):
    return lib().ga_hamming(genomes, N, fitness, stream)


def ga_poisson_thresholds(rate, thresholds):
    return lib().ga_poisson_thresholds(rate, thresholds)


def ga_run(ga, cls, fitness_kind, N, generations, population, best, total, stream):
    return lib().ga_run(ga, cls, fitness_kind, N, generations, population, best, total, stream)


def jatam_mlp_create(max_batch, net):
    return lib().jatam_mlp_create(max_batch, net)


def jatam_mlp_destroy(net):
    lib().jatam_mlp_destroy(net)


def jatam_mlp_set_params(net, params, stream):
    return lib().jatam_mlp_set_params(net, params, stream)


def jatam_mlp_get_params(net, params, stream):
    return lib().jatam_mlp_get_params(net, params, stream)


def jatam_mlp_train_step(net, genomes, labels, B, lr, loss, grads, stream):
    return lib().jatam_mlp_train_step(net, genomes, labels, B, lr, loss, grads, stream)


def jatam_mlp_predict(net, genomes, N, logits, stream):
    return lib().jatam_mlp_predict(net, genomes, N, logits, stream)


def jatam_mlp_labels(results, N, labels, stream):
    return lib().jatam_mlp_labels(results, N, labels, stream)


def jatam_embed_genomes(genomes, N, n, c, out, stream):
    return lib().jatam_embed_genomes(genomes, N, n, c, out, stream)


def jatam_set_replicate_lanes(mode):
    return lib().jatam_set_replicate_lanes(int(mode))


def jatam_get_replicate_lanes():
    return lib().jatam_get_replicate_lanes()


def set_replicate_lanes(mode):
    """0: replicate lanes for small calls (default), 1: never, 2: whenever eligible."""
    return check(jatam_set_replicate_lanes(mode))


def jatam_select_top(scores, n, keep, idx, stream):
    return lib().jatam_select_top(scores, n, keep, idx, stream)


def ga_run_screened(ga, cls, N, generations, ratio, net, online_lr, population, best, total, stream):
    return lib().ga_run_screened(ga, cls, N, generations, ratio, net, online_lr, population, best, total, stream)


def jatam_set_mixed_plan(w32, w16, w8):
    return lib().jatam_set_mixed_plan(w32, w16, w8)


def jatam_get_mixed_plan(w32, w16, w8):
    return lib().jatam_get_mixed_plan(w32, w16, w8)


def jatam_autotune_batch(colours, shapes, N, seed, stream):
    return lib().jatam_autotune_batch(colours, shapes, N, seed, stream)


def jatam_autotune(shapes, n_shapes, stream):
    return lib().jatam_autotune(shapes, n_shapes, stream)


def jatam_set_tuning(cfg, warps_per_cta, stop_at):
    return lib().jatam_set_tuning(cfg, warps_per_cta, stop_at)


def jatam_get_tuning(cfg, warps_per_cta, stop_at):
    return lib().jatam_get_tuning(cfg, warps_per_cta, stop_at)


def jatam_profile(enable):
    return lib().jatam_profile(int(enable))


def jatam_kernel_ms(ms):
    return lib().jatam_kernel_ms(ms)


def jatam_work_counters(counters):
    return lib().jatam_work_counters(counters)


def jatam_last_shapes(shapes, cap, length, collisions):
    return lib().jatam_last_shapes(shapes, cap, length, collisions)


def jatam_set_genotypes_per_warp(cfg, genotypes_per_warp):
    return lib().jatam_set_genotypes_per_warp(cfg, genotypes_per_warp)


def jatam_get_genotypes_per_warp(cfg, genotypes_per_warp):
    return lib().jatam_get_genotypes_per_warp(cfg, genotypes_per_warp)


def jatam_workspace_bytes(nbytes):
    return lib().jatam_workspace_bytes(nbytes)


def jatam_shutdown():
    lib().jatam_shutdown()


def jatam_last_error() -> str:
    return lib().jatam_last_error().decode()


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def make_config(n, c, L, k, seed, flags=0):
    return jatam_config(n=n, c=c, L=L, k=k, flags=flags, seed=seed & 0xFFFFFFFFFFFFFFFF)


def _addr(x):
    """Address of a torch tensor, numpy array or int (None -> 0)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def check(rc):
    if rc != JATAM_OK:
        raise JatamError(rc, jatam_last_error())
    return rc


def enumerate_space(n, c, L, k, seed, first, count, *, sampled=False, out=None, hist=None, hist_len=None,
                    hist_cap=0, stream=None, sync=False, graph=False, c4_hash=False, orbits=False, lifo=False):
    """jatam_enumerate on caller buffers (torch tensors or numpy arrays)."""
    cfg = make_config(n, c, L, k, seed, (JATAM_SAMPLED if sampled else 0) | (JATAM_SYNC if sync else 0)
                      | (JATAM_GRAPH if graph else 0) | (JATAM_C4_HASH if c4_hash else 0)
                      | (JATAM_ORBITS if orbits else 0) | (JATAM_LIFO if lifo else 0))
    return check(jatam_enumerate(ctypes.addressof(cfg), first, count, _addr(out), _addr(hist), hist_cap,
                                 _addr(hist_len), _stream_handle(stream)))


SHAPE_DTYPE = np.dtype([("shape_hash", "<u4"), ("h", "u1"), ("w", "u1"), ("size", "<u2"), ("rows", "<u4", (32,))])


def last_shapes(cap=1 << 14):
    """jatam_last_shapes: (entries as a SHAPE_DTYPE array sorted by hash, collisions)."""
    out = np.zeros(cap, SHAPE_DTYPE)
    n = _U32(0)
    col = _U32(0)
    check(jatam_last_shapes(out.ctypes.data, cap, ctypes.byref(n), ctypes.byref(col)))
    return out[: n.value], int(col.value)


def shape_bitmap(entry):
    """h x w uint8 array of one jatam_shape entry (column j of row i = bit j)."""
    h, w = int(entry["h"]), int(entry["w"])
    return np.array([[(int(entry["rows"][i]) >> j) & 1 for j in range(w)] for i in range(h)], np.uint8)


def set_genotypes_per_warp(n, c, L, genotypes_per_warp):
    """1: one genotype per warp (L > 16); 32: one per lane; 0: the default."""
    cfg = make_config(n, c, L, 1, 0)
    return check(jatam_set_genotypes_per_warp(ctypes.addressof(cfg), int(genotypes_per_warp)))


def get_genotypes_per_warp(n, c, L):
    cfg = make_config(n, c, L, 1, 0)
    v = ctypes.c_int(0)
    check(jatam_get_genotypes_per_warp(ctypes.addressof(cfg), ctypes.byref(v)))
    return int(v.value)


def workspace_bytes() -> int:
    """Device bytes the library's workspace holds on the current device (0: none)."""
    v = ctypes.c_uint64(0)
    check(jatam_workspace_bytes(ctypes.byref(v)))
    return int(v.value)


def enumerate_noalloc(n, c, L, k, seed, first, count, out, *, sampled=False, stream=None, sync=False,
                      c4_hash=False):
    """jatam_enumerate_noalloc into a device buffer `out` (no library allocation)."""
    cfg = make_config(n, c, L, k, seed, (JATAM_SAMPLED if sampled else 0) | (JATAM_SYNC if sync else 0)
                      | (JATAM_C4_HASH if c4_hash else 0))
    return check(jatam_enumerate_noalloc(ctypes.addressof(cfg), first, count, _addr(out), _stream_handle(stream)))


def classify_batch(colours, *, n=0, c=0, L=0, k=0, seed=0, shapes=None, stream_ids=None, out=None, hist=None,
                   hist_len=None, hist_cap=0, stream=None, sync=False, per_shape=None, graph=False):
    """per_shape: True -> per-size fixed launches, False -> the persistent launch,
    None -> the form jatam_autotune_batch found faster."""
    N = int(colours.shape[0])
    form = 0 if per_shape is None else (JATAM_PER_SHAPE if per_shape else JATAM_PERSISTENT)
    cfg = make_config(n, c, L, k, seed, (JATAM_SYNC if sync else 0) | form | (JATAM_GRAPH if graph else 0))
    return check(jatam_classify_batch(ctypes.addressof(cfg), _addr(colours), _addr(shapes), _addr(stream_ids), N,
                                      _addr(out), _addr(hist), hist_cap, _addr(hist_len), _stream_handle(stream)))


def evaluate_genomes(genomes, fitness, *, n, c, L, k, seed, out=None, stream=None, sync=False, graph=False,
                     dedup=True):
    cfg = make_config(n, c, L, k, seed, (JATAM_SYNC if sync else 0) | (JATAM_GRAPH if graph else 0) |
                      (0 if dedup else JATAM_NO_DEDUP))
    N = int(genomes.shape[0])
    return check(ga_evaluate(ctypes.addressof(cfg), _addr(genomes), N, _addr(fitness), _addr(out),
                             _stream_handle(stream)))


def philox(records, out, stream=None):
    """records: [N][6] uint32 (ctr0..3, key0, key1) -> out [N][4] uint32."""
    N = int(records.shape[0])
    return check(jatam_philox(_addr(records), N, _addr(out), _stream_handle(stream)))


def autotune(configs, stream=None):
    """configs: list of dicts with n, c, L, k, seed (and optional sampled)."""
    arr = (jatam_config * len(configs))()
    for i, d in enumerate(configs):
        arr[i] = make_config(d["n"], d["c"], d["L"], d["k"], d.get("seed", 0), JATAM_SAMPLED if d.get("sampled") else 0)
    return check(jatam_autotune(ctypes.addressof(arr), len(configs), _stream_handle(stream)))


def set_mixed_plan(w32, w16, w8):
    return check(jatam_set_mixed_plan(w32, w16, w8))


def get_mixed_plan():
    v = [ctypes.c_int(0) for _ in range(3)]
    check(jatam_get_mixed_plan(*[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def get_mixed_launch():
    """'per_shape' or 'persistent': the launch form of mixed batches without a flag."""
    v = ctypes.c_int(0)
    check(jatam_get_mixed_launch(ctypes.byref(v)))
    return "per_shape" if v.value else "persistent"


def autotune_batch(colours, shapes, seed, stream=None):
    N = int(colours.shape[0])
    return check(jatam_autotune_batch(_addr(colours), _addr(shapes), N, seed, _stream_handle(stream)))


def set_tuning(n, c, L, warps_per_cta, stop_at):
    cfg = make_config(n, c, L, 1, 0)
    return check(jatam_set_tuning(ctypes.addressof(cfg), warps_per_cta, stop_at))


def get_tuning(n, c, L):
    cfg = make_config(n, c, L, 1, 0)
    w, s = ctypes.c_int(0), ctypes.c_int(0)
    check(jatam_get_tuning(ctypes.addressof(cfg), ctypes.byref(w), ctypes.byref(s)))
    return w.value, s.value


def last_kernel_ms() -> float:
    """Duration of the last profiled classification kernel (jatam_profile(1) first)."""
    ms = ctypes.c_float(0.0)
    check(jatam_kernel_ms(ctypes.byref(ms)))
    return float(ms.value)


def work_counters():
    """Executed work of the last counted call (jatam_profile(2) first): drawn
    placements, seed placements, lane slots of the growth rounds, genotypes
    grown by warps."""
    c = (ctypes.c_uint64 * 4)()
    check(jatam_work_counters(c))
    return {"placements": int(c[0]), "seeds": int(c[1]), "lane_slots": int(c[2]), "genotypes": int(c[3])}


def merge_histograms(a, b):
    """Host merge of two sorted histograms (numpy HIST_DTYPE arrays)."""
    a = np.ascontiguousarray(a, HIST_DTYPE)
    b = np.ascontiguousarray(b, HIST_DTYPE)
    cap = a.shape[0] + b.shape[0]
    out = np.zeros(max(cap, 1), HIST_DTYPE)
    n = ctypes.c_uint32(0)
    check(jatam_hist_merge(_addr(a) if a.size else None, a.shape[0], _addr(b) if b.size else None, b.shape[0],
                           out.ctypes.data, cap, ctypes.addressof(n)))
    return out[: n.value].copy()


def results_view(t):
    """numpy structured view of a result buffer (torch uint8/int64 tensor or numpy)."""
    if hasattr(t, "cpu"):
        t = t.cpu().numpy()
    return np.ascontiguousarray(t).view(np.uint8).reshape(-1).view(RESULT_DTYPE)


def hist_view(t, length=None):
    if hasattr(t, "cpu"):
        t = t.cpu().numpy()
    h = np.ascontiguousarray(t).view(np.uint8).reshape(-1).view(HIST_DTYPE)
    return h if length is None else h[:length]


# ---------------------------------------------------------------------------
# genetic algorithm helpers
# ---------------------------------------------------------------------------
def poisson_thresholds(rate):
    t = (ctypes.c_uint32 * 4)()
    check(ga_poisson_thresholds(float(rate), t))
    return [int(v) for v in t]


def make_ga(n, c, seed, *, selection=TOURNAMENT, tournament=4, crossover=NO_CROSSOVER, crossover_threshold=0,
            mutation_thresholds=(0xFFFFFFFF,) * 4):
    g = jatam_ga_config(n=n, c=c, selection=selection, tournament=tournament, crossover=crossover,
                        crossover_threshold=crossover_threshold, seed=seed & 0xFFFFFFFFFFFFFFFF)
    for j in range(4):
        g.mutation_thresholds[j] = int(mutation_thresholds[j])
    return g


def breed(ga, parents, fitness, generation, children, stream=None):
    N = int(parents.shape[0])
    return check(ga_breed(ctypes.addressof(ga), _addr(parents), _addr(fitness), N, int(generation), _addr(children),
                          _stream_handle(stream)))


def hamming(genomes, fitness, stream=None):
    return check(ga_hamming(_addr(genomes), int(genomes.shape[0]), _addr(fitness), _stream_handle(stream)))


def run_ga(ga, population, generations, *, fitness_kind=FITNESS_SHAPE, L=16, k=20, seed=0, best=None, total=None,
           stream=None):
    cls = make_config(ga.n, ga.c, L, k, seed)
    return check(ga_run(ctypes.addressof(ga), ctypes.addressof(cls), int(fitness_kind), int(population.shape[0]),
                        int(generations), _addr(population), _addr(best), _addr(total), _stream_handle(stream)))


# ---------------------------------------------------------------------------
# surrogate network
# ---------------------------------------------------------------------------
MLP_NPARAM = 80392
MLP_SHAPES = (("W1", (48, 256)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 8)), ("b3", (8,)))


def flatten_params(p):
    return np.concatenate([np.asarray(p[k], np.float32).reshape(-1) for k, _ in MLP_SHAPES]).astype(np.float32)


def unflatten_params(v):
    out, o = {}, 0
    for k, shp in MLP_SHAPES:
        n = int(np.prod(shp))
        out[k] = np.asarray(v[o: o + n], np.float64).reshape(shp)
        o += n
    return out


class Surrogate:
    """Owner of a jatam_mlp handle (argument marshalling only)."""

    def __init__(self, max_batch):
        h = ctypes.c_void_p()
        check(jatam_mlp_create(int(max_batch), ctypes.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            jatam_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat, stream=None):
        flat = np.ascontiguousarray(flat, np.float32) if not hasattr(flat, "data_ptr") else flat
        check(jatam_mlp_set_params(self.h, _addr(flat), _stream_handle(stream)))

    def get_params(self, stream=None):
        out = np.zeros(MLP_NPARAM, np.float32)
        check(jatam_mlp_get_params(self.h, out.ctypes.data, _stream_handle(stream)))
        return out

    def train_step(self, genomes, labels, lr, grads=None, stream=None):
        loss = ctypes.c_float(0.0)
        check(jatam_mlp_train_step(self.h, _addr(genomes), _addr(labels), int(genomes.shape[0]), float(lr),
                                   ctypes.addressof(loss), _addr(grads), _stream_handle(stream)))
        return float(loss.value)

    def predict(self, genomes, logits, stream=None):
        check(jatam_mlp_predict(self.h, _addr(genomes), int(genomes.shape[0]), _addr(logits),
                                _stream_handle(stream)))


def labels_of(results, labels, stream=None):
    """Device results (uint8 view, 8 B per genotype) -> device class labels."""
    N = int(results.numel() // 8) if hasattr(results, "numel") else int(results.shape[0])
    return check(jatam_mlp_labels(_addr(results), N, _addr(labels), _stream_handle(stream)))


def select_top(scores, keep, idx, stream=None):
    """Device float32 scores [n] -> idx[0 .. keep) (device int64): indices of the
    keep largest, ties lower index first, in increasing order."""
    return check(jatam_select_top(_addr(scores), int(scores.shape[0]), int(keep), _addr(idx), _stream_handle(stream)))


def embed(genomes, n, c, out, stream=None):
    return check(jatam_embed_genomes(_addr(genomes), int(genomes.shape[0]), int(n), int(c), _addr(out),
                                     _stream_handle(stream)))


def run_ga_screened(ga, population, generations, ratio, net, *, online_lr=1e-3, L=16, k=20, seed=0, best=None,
                    total=None, stream=None):
    cls = make_config(ga.n, ga.c, L, k, seed)
    return check(ga_run_screened(ctypes.addressof(ga), ctypes.addressof(cls), int(population.shape[0]),
                                 int(generations), int(ratio), net.h, float(online_lr), _addr(population), _addr(best),
                                 _addr(total), _stream_handle(stream)))
