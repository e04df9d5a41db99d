"""Genome batches with repeats (a GA population after selection holds many
copies of few genomes): every distinct genome is classified once and its
repeats copy the result -- exact, since a genome's result depends only on the
genome, which is also its stream id.  Results, fitness and histogram against
the oracle, item by item, on batches whose repeats sit before and after their
first occurrence, for one genotype per lane and for replicate lanes."""
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
    J.set_replicate_lanes(0)


def _batch(n_distinct, n, seed):
    rng = np.random.default_rng(seed)
    distinct = W.random_genomes(n_distinct, 3, 8, seed=seed)
    return distinct[rng.integers(0, n_distinct, size=n)]


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("n_distinct,n", [(300, 8192), (5000, 6000), (1, 4096)])
def test_repeated_genomes_match_oracle(mode, n_distinct, n):
    J.set_replicate_lanes(mode)
    n_, c, L, k, seed = 3, 8, 16, 20, 13
    genomes = _batch(n_distinct, n, seed=n_distinct + n)
    g = torch.from_numpy(genomes.view(np.int64)).cuda()
    fit = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    out = torch.full((n * 8,), 0xEE, dtype=torch.uint8, device="cuda")
    J.evaluate_genomes(g, fit, n=n_, c=c, L=L, k=k, seed=seed, out=out, sync=True)
    res = J.results_view(out)
    uniq = np.unique(genomes)
    ref = {}
    for x in uniq.tolist():
        r = O.classify(n_, c, L, k, seed, O.decode(int(x), n_, c), int(x))
        ref[x] = (r["cls"], r["decided_rep"], r["size"], r["shape_hash"])
    want = np.array([ref[int(x)] for x in genomes.tolist()])
    got = np.stack([res["cls"], res["decided_rep"], res["size"], res["shape_hash"]], axis=1).astype(np.int64)
    assert np.array_equal(got, want.astype(np.int64))
    want_fit = np.where(want[:, 0] == 0, want[:, 2], 0)
    assert np.array_equal(fit.cpu().numpy(), want_fit)
    # every genome classified (JATAM_NO_DEDUP): the same bytes
    fit2 = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    out2 = torch.full((n * 8,), 0xEE, dtype=torch.uint8, device="cuda")
    J.evaluate_genomes(g, fit2, n=n_, c=c, L=L, k=k, seed=seed, out=out2, sync=True, dedup=False)
    assert torch.equal(out, out2) and torch.equal(fit, fit2)


def test_repeated_genomes_in_graph_replays():
    """The repeat table is emptied by every call, so replays of one captured call
    (the GA's fitness call) and calls of other sizes in between see a clean table."""
    n_, c, L, k, seed = 3, 8, 16, 20, 17
    outs = []
    for n in (4096, 1000, 4096, 9000, 4096):
        genomes = _batch(200, n, seed=n)
        g = torch.from_numpy(genomes.view(np.int64)).cuda()
        fit = torch.empty(n, dtype=torch.int32, device="cuda")
        J.evaluate_genomes(g, fit, n=n_, c=c, L=L, k=k, seed=seed, sync=True, graph=True)
        fit2 = torch.empty(n, dtype=torch.int32, device="cuda")
        J.evaluate_genomes(g, fit2, n=n_, c=c, L=L, k=k, seed=seed, sync=True, dedup=False)
        assert torch.equal(fit, fit2), n
        if n == 4096:
            outs.append(fit.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
