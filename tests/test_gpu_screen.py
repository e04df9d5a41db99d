"""The selection step of the network pre-screen (ga_run_screened): the indices
of the keep largest scores, ties broken by the lower index, in increasing
order -- element by element against numpy's stable sort on the same scores.
The cases have many equal scores (the threshold value repeated across the
warps' segments), the screening size of the GA configuration (65,536
candidates, keep 8,192) and odd counts around it, and the degenerate ends."""
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


def _want(scores, keep):
    order = np.argsort(-scores.astype(np.float64), kind="stable")  # descending, ties: lower index first
    return np.sort(order[:keep])


def _got(scores, keep):
    d = torch.from_numpy(scores).cuda()
    idx = torch.full((max(keep, 1),), -1, dtype=torch.int64, device="cuda")
    J.select_top(d, keep, idx)
    torch.cuda.synchronize()
    return idx[:keep].cpu().numpy()


@pytest.mark.parametrize("n,keep,levels", [(65536, 8192, 0), (65536 + 77, 8192, 0), (65536, 8192, 7),
                                           (65535, 8192, 0), (65533, 30000, 4), (8192, 2048, 3), (1000, 1, 0),
                                           (1000, 1000, 2), (33, 5, 1), (300000, 4096, 50), (5000, 0, 0)])
def test_select_top_matches_numpy(n, keep, levels):
    rng = np.random.default_rng(n + keep + levels)
    if levels:
        # few distinct values: long runs of equal scores around the threshold
        scores = rng.integers(0, levels + 1, size=n).astype(np.float32) / levels
    else:
        # probabilities, half of them lifted by one (the pre-screen's first occurrences)
        scores = rng.random(n, dtype=np.float32) + (rng.random(n) < 0.5).astype(np.float32)
    got = _got(scores, keep)
    assert np.array_equal(got, _want(scores, keep))
