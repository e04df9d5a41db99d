"""jatam_enumerate_noalloc: the variant of jatam_enumerate for callers that may
not allocate device memory.  It must give exactly the results of
jatam_enumerate, call after call, while using only its fixed scratch array.
This file is collected last so that a stop-at-first-failure run has already
run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2205_15311_gb300 import binding as J  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


def _reference(n, c, L, k, seed, first, count, sampled=False):
    out = torch.empty(max(count, 1) * 8, dtype=torch.uint8, device="cuda")
    J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out, sync=True)
    return J.results_view(out)[:count]


def test_noalloc_matches_enumerate_on_two_calls_in_a_row():
    cases = [(2, 8, 16, 20, 2, 3 << 20, 200000, False),   # S_{2,8} slice, 16 x 16 grid
             (3, 8, 32, 20, 3, 12345, 150001, True)]      # sampled S_{3,8}, 32 x 32 grid
    outs = []
    for (n, c, L, k, seed, first, count, sampled) in cases:
        out = torch.zeros(count * 8, dtype=torch.uint8, device="cuda")
        J.enumerate_noalloc(n, c, L, k, seed, first, count, out, sampled=sampled, sync=True)
        outs.append(out)
    # both calls in a row reused the same scratch; each must equal the allocating path
    for (n, c, L, k, seed, first, count, sampled), out in zip(cases, outs):
        got = J.results_view(out)
        assert np.array_equal(got, _reference(n, c, L, k, seed, first, count, sampled))


def test_noalloc_rejects_counts_beyond_its_scratch():
    out = torch.zeros(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(J.JatamError) as e:
        J.enumerate_noalloc(2, 8, 16, 20, 2, 0, J.JATAM_NOALLOC_MAX_COUNT + 1, out)
    assert e.value.code == J.JATAM_EINVAL and "JATAM_NOALLOC_MAX_COUNT" in str(e.value)
    host = np.zeros(4, J.RESULT_DTYPE)
    with pytest.raises(J.JatamError):
        J.enumerate_noalloc(2, 8, 16, 20, 2, 0, 4, host)
