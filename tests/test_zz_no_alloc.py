"""jatam_enumerate_noalloc: the variant of jatam_enumerate for callers that may
not allocate device memory (an application that owns every byte of the GPU
through its own pool, or code where a cudaMalloc, or the device-wide
synchronisation of a cudaFree, is not allowed).  Its results must equal the
oracle's and jatam_enumerate's, call after call, while it uses only its fixed
scratch array.  This file is collected last so that a stop-at-first-failure
run has already run every other test."""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2205_15311_gb300 import binding as J  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (n, c, L, k, seed, first, count, sampled, c4_hash)
S28_SLICE = (2, 8, 16, 20, 2, 3 << 20, 200000, False, False)
# J.JATAM_NOALLOC_MAX_COUNT genotypes of S_{2,8}: on a GB300 (152 SMs, four
# 5-warp CTAs an SM) every lane takes at least 8 of them on average
# (8 x 608 x 160 = 778,240 < 2^20), so the pre-filter writes the heavy-first
# list (two or more frontier sites after the seed from the front, the others
# from the end of the region)
S28_MAX = (2, 8, 16, 20, 2, 5 << 20, 1 << 20, False, False)
S28_C4 = (2, 8, 16, 20, 2, 9 << 20, 300000, False, True)       # the rotation-only hash of Section 2.5
S38_SAMPLED = (3, 8, 32, 20, 3, 12345, 150001, True, False)     # sampled S_{3,8}, 32 x 32 grid


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


def _oracle(case):
    n, c, L, k, seed, first, count, sampled, c4 = case
    with O.hash_mode(c4):
        res, _ = O.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled)
    return res


def _enumerate(case):
    n, c, L, k, seed, first, count, sampled, c4 = case
    out = torch.empty(max(count, 1) * 8, dtype=torch.uint8, device="cuda")
    J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out, sync=True, c4_hash=c4)
    return J.results_view(out)[:count]


def _noalloc(case, out):
    n, c, L, k, seed, first, count, sampled, c4 = case
    J.enumerate_noalloc(n, c, L, k, seed, first, count, out, sampled=sampled, sync=True, c4_hash=c4)
    return J.results_view(out)[:count]


def test_noalloc_matches_the_oracle_on_two_calls_in_a_row():
    """Each case runs twice in a row through the shared scratch (the second
    call must clear what the first left); both calls equal the oracle."""
    for case in (S28_SLICE, S28_MAX, S28_C4):
        want = _oracle(case)
        for _ in range(2):
            out = torch.full((case[6] * 8,), 0xEE, dtype=torch.uint8, device="cuda")  # poisoned
            assert np.array_equal(_noalloc(case, out), want), case


def test_noalloc_matches_enumerate_on_two_calls_in_a_row():
    outs = []
    for case in (S28_SLICE, S38_SAMPLED):
        out = torch.zeros(case[6] * 8, dtype=torch.uint8, device="cuda")
        _noalloc(case, out)
        outs.append(out)
    # both calls in a row reused the same scratch; each must equal the allocating path
    for case, out in zip((S28_SLICE, S38_SAMPLED), outs):
        assert np.array_equal(J.results_view(out)[:case[6]], _enumerate(case))


_CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2205_15311_gb300 import binding as J
cases = json.loads(sys.argv[2])
torch.cuda.init()
outs = [torch.zeros(c[6] * 8, dtype=torch.uint8, device="cuda") for c in cases]
torch.cuda.synchronize()
def call(case, out):
    n, c, L, k, seed, first, count, sampled, c4 = case
    J.enumerate_noalloc(n, c, L, k, seed, first, count, out, sampled=sampled, sync=True, c4_hash=c4)
call(cases[0], outs[0])            # first call on the device: the one-time set-up
free0, _ = torch.cuda.mem_get_info()
ws0 = J.workspace_bytes()
for case, out in zip(cases, outs):
    call(case, out)
    call(case, out)
torch.cuda.synchronize()
free1, _ = torch.cuda.mem_get_info()
ws1 = J.workspace_bytes()
for i, out in enumerate(outs):
    np.save(f"{sys.argv[3]}/out{i}.npy", out.cpu().numpy())
print(json.dumps({"free0": free0, "free1": free1, "ws0": ws0, "ws1": ws1}))
"""


def test_noalloc_in_a_fresh_process_allocates_nothing():
    """A fresh process that only ever calls the allocation-free entry point:
    the library never creates its workspace, the free device memory does not
    change across the calls after the first (which loads the kernels), and
    the results equal the oracle's."""
    cases = [S28_SLICE, S28_MAX, S28_C4, S38_SAMPLED]
    with tempfile.TemporaryDirectory() as tmp:
        p = subprocess.run([sys.executable, "-c", _CHILD, ROOT, json.dumps(cases), tmp], capture_output=True,
                           text=True, timeout=600)
        assert p.returncode == 0, p.stderr[-4000:]
        rep = json.loads(p.stdout.strip().splitlines()[-1])
        assert rep["ws0"] == 0 and rep["ws1"] == 0, rep
        assert rep["free1"] == rep["free0"], rep
        for i, case in enumerate(cases):
            got = np.load(os.path.join(tmp, f"out{i}.npy")).view(J.RESULT_DTYPE)[:case[6]]
            if case is S38_SAMPLED:
                continue  # compared with jatam_enumerate above; the oracle covers the three S_{2,8} cases
            assert np.array_equal(got, _oracle(case)), case


def test_noalloc_rejects_counts_beyond_its_scratch():
    out = torch.zeros(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(J.JatamError) as e:
        J.enumerate_noalloc(2, 8, 16, 20, 2, 0, J.JATAM_NOALLOC_MAX_COUNT + 1, out)
    assert e.value.code == J.JATAM_EINVAL and "JATAM_NOALLOC_MAX_COUNT" in str(e.value)
    host = np.zeros(4, J.RESULT_DTYPE)
    with pytest.raises(J.JatamError):
        J.enumerate_noalloc(2, 8, 16, 20, 2, 0, 4, host)


def test_noalloc_rejects_another_devices_memory():
    """A buffer of another GPU would be written through a peer pointer: the
    call refuses it (only where a second device is visible)."""
    if torch.cuda.device_count() < 2:
        pytest.skip("one visible device")
    out = torch.zeros(64, dtype=torch.uint8, device="cuda:1")
    with torch.cuda.device(0):
        with pytest.raises(J.JatamError) as e:
            J.enumerate_noalloc(2, 8, 16, 20, 2, 0, 8, out)
    assert e.value.code == J.JATAM_EINVAL
