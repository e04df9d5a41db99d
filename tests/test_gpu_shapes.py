"""The exact side table of the shape hash (Section 2.5), GPU against oracle:
for every shape hash of a call's histogram, the canonical form the GPU stored
equals the oracle's, and both sides count zero collisions (no two distinct
canonical forms share a hash)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2205_15311_gb300 import binding as J  # noqa: E402
from paper_2205_15311_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


def _gpu_forms():
    entries, collisions = J.last_shapes()
    forms = {}
    for e in entries:
        bm = J.shape_bitmap(e)
        assert int(e["size"]) == int(bm.sum())
        forms[int(e["shape_hash"])] = bm
    return forms, collisions


def _compare(gpu, ocl, hist):
    forms, collisions = gpu
    assert collisions == 0 and ocl.collisions == 0 and ocl.overflow == 0
    shaped = sorted(set(int(r["shape_hash"]) for r in hist if int(r["cls"]) in (0, 2)))
    assert sorted(forms) == shaped == sorted(ocl.forms)
    for key in shaped:
        assert np.array_equal(forms[key], ocl.forms[key]), key


@pytest.mark.parametrize("case", ["s24_full", "s28_slice", "s38_sample"])
def test_enumeration_shape_table_matches_oracle(case):
    if case == "s24_full":
        n, c, L, k, seed, first, count, sampled = W.WORKLOADS["s24_full"]
    elif case == "s28_slice":  # large enough for the heavy-first list and the crop table
        n, c, L, k, seed, first, count, sampled = 2, 8, 16, 20, 2, 7 << 20, 1 << 20, False
    else:
        n, c, L, k, seed, first, count, sampled = 3, 8, 32, 20, 3, 1 << 22, 1 << 18, True
    cap = 1 << 14
    out = torch.empty(count * 8, dtype=torch.uint8, device="cuda")
    hist = torch.empty(cap * 32, dtype=torch.uint8, device="cuda")
    hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
    J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out, hist=hist, hist_len=hlen,
                      hist_cap=cap, sync=True)
    gpu = _gpu_forms()
    with O.shape_table() as T:
        ref, _ = O.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled)
    assert np.array_equal(J.results_view(out)[:count], ref)
    _compare(gpu, T, J.hist_view(hist, int(hlen.item())))


def test_mixed_batch_shape_table_matches_oracle():
    colours, shapes = W.mixed_records(1 << 18, seed=4)
    cap = 1 << 14
    for per_shape in (False, True):
        out = torch.empty((1 << 18) * 8, dtype=torch.uint8, device="cuda")
        hist = torch.empty(cap * 32, dtype=torch.uint8, device="cuda")
        hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
        J.classify_batch(torch.from_numpy(colours).cuda(), seed=4, shapes=torch.from_numpy(shapes).cuda(),
                         out=out, hist=hist, hist_len=hlen, hist_cap=cap, sync=True, per_shape=per_shape)
        gpu = _gpu_forms()
        with O.shape_table() as T:
            ref, _ = O.classify_batch(colours, shapes=shapes, seed=4)
        assert np.array_equal(J.results_view(out), ref)
        _compare(gpu, T, J.hist_view(hist, int(hlen.item())))


def test_pipelined_host_call_records_the_same_shapes():
    """A host-buffer call of 2^24 genotypes (pieces on two streams) records the
    same table as the single-pass device-buffer call."""
    n, c, L, k, seed, first, count, _ = W.WORKLOADS["s28_full"]
    cap = 1 << 12
    out = torch.empty(count * 8, dtype=torch.uint8, device="cuda")
    hist = torch.empty(cap * 32, dtype=torch.uint8, device="cuda")
    hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
    J.enumerate_space(n, c, L, k, seed, first, count, out=out, hist=hist, hist_len=hlen, hist_cap=cap, sync=True)
    single, col1 = _gpu_forms()
    out_h = torch.empty(count * 8, dtype=torch.uint8, pin_memory=True)
    hist_h = np.zeros(cap, J.HIST_DTYPE)
    hlen_h = np.zeros(1, np.uint32)
    J.enumerate_space(n, c, L, k, seed, first, count, out=out_h, hist=hist_h, hist_len=hlen_h, hist_cap=cap)
    piped, col2 = _gpu_forms()
    assert col1 == 0 and col2 == 0
    assert sorted(single) == sorted(piped)
    for key in single:
        assert np.array_equal(single[key], piped[key])
    # the C4 hash records nothing, and the readout says so
    J.enumerate_space(n, c, L, k, seed, 0, 4096, out=out, hist=hist, hist_len=hlen, hist_cap=cap, sync=True,
                      c4_hash=True)
    with pytest.raises(J.JatamError):
        J.last_shapes()
