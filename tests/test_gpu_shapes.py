"""The exact side table of the shape hash (Section 2.5), GPU against oracle:
for every shape hash of a call's histogram, the canonical form the GPU stored
equals the oracle's, and both sides count zero collisions (no two distinct
canonical forms share a hash)."""
import os

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


_NO_CROP_TABLE = r"""
import json, sys
import os

import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2205_15311_gb300 import binding as J
n, c, L, k, seed, first, count, sampled = json.loads(sys.argv[2])
out = torch.empty(count * 8, dtype=torch.uint8, device="cuda")
hist = torch.empty((1 << 12) * 32, dtype=torch.uint8, device="cuda")
hlen = torch.zeros(1, dtype=torch.int32, device="cuda")
J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out, hist=hist, hist_len=hlen,
                  hist_cap=1 << 12, sync=True)
entries, collisions = J.last_shapes()
np.save(sys.argv[3] + "/res.npy", J.results_view(out).copy())
np.save(sys.argv[3] + "/shapes.npy", entries)
print(json.dumps({"collisions": collisions}))
"""


@pytest.mark.parametrize("case", [(2, 8, 16, 20, 2, 11 << 20, 1 << 14, False),
                                  (3, 8, 32, 20, 3, 5 << 20, 1 << 14, True)])
def test_without_the_crop_table_every_form_reaches_the_side_table(case):
    """With the crop table switched off (JATAM_CROP_TABLE=0, a fresh process)
    every computed form goes through the spill list to the side table: the
    results and the table still equal the oracle's."""
    import json
    import subprocess
    import sys
    import tempfile
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, JATAM_CROP_TABLE="0")
    with tempfile.TemporaryDirectory() as tmp:
        p = subprocess.run([sys.executable, "-c", _NO_CROP_TABLE, root, json.dumps(list(case)), tmp], env=env,
                           capture_output=True, text=True, timeout=600)
        assert p.returncode == 0, p.stderr[-4000:]
        assert json.loads(p.stdout.strip().splitlines()[-1])["collisions"] == 0
        res = np.load(os.path.join(tmp, "res.npy"))
        entries = np.load(os.path.join(tmp, "shapes.npy"))
    n, c, L, k, seed, first, count, sampled = case
    with O.shape_table() as T:
        ref, _ = O.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled)
    assert np.array_equal(res.view(J.RESULT_DTYPE), ref)
    forms = {int(e["shape_hash"]): J.shape_bitmap(e) for e in entries.view(J.SHAPE_DTYPE)}
    assert sorted(forms) == sorted(T.forms)
    for key, bm in forms.items():
        assert np.array_equal(bm, T.forms[key])
