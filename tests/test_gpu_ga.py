"""Parity of the GPU genetic algorithm (ga_breed, ga_hamming, ga_run) with the
oracle: children, fitness and per-generation statistics are integers and must
match exactly."""
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


CASES = [
    dict(selection=0, tournament=4, crossover=0, rate=0.01),
    dict(selection=0, tournament=1, crossover=1, rate=0.2),
    dict(selection=1, tournament=1, crossover=2, rate=0.05),
    dict(selection=1, tournament=1, crossover=1, rate=0.0),
    dict(selection=0, tournament=16, crossover=2, rate=1.5),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("n,c", [(3, 8), (2, 4), (4, 8)])
def test_breed_matches_oracle(case, n, c):
    N = 3001
    parents = W.random_genomes(N, n, c, seed=21)
    fitness = (np.arange(N) * 7919 % 97).astype(np.int32)
    fitness[::5] = 0
    thr = J.poisson_thresholds(case["rate"])
    ga = J.make_ga(n, c, 77, selection=case["selection"], tournament=case["tournament"],
                   crossover=case["crossover"], crossover_threshold=0xC0000000, mutation_thresholds=thr)
    for gen in (0, 5, (1 << 24) - 1):
        want = O.ga_breed(parents, fitness, gen, n=n, c=c, seed=77, selection=case["selection"],
                          tournament=case["tournament"], crossover=case["crossover"],
                          crossover_threshold=0xC0000000, mutation_thresholds=thr)
        host = np.zeros(N, np.uint64)
        J.breed(ga, parents, fitness, gen, host)
        assert np.array_equal(host, want)
        dp = torch.from_numpy(parents.view(np.int64)).cuda()
        df = torch.from_numpy(fitness).cuda()
        dc = torch.zeros(N, dtype=torch.int64, device="cuda")
        J.breed(ga, dp, df, gen, dc)
        torch.cuda.synchronize()
        assert np.array_equal(dc.cpu().numpy().view(np.uint64), want)


def test_hamming_fitness():
    g = W.random_genomes(10000, 3, 8, seed=2)
    f = np.zeros(10000, np.int32)
    J.hamming(g, f)
    assert np.array_equal(f, np.array([O.hamming(int(v)) for v in g], np.int32))


def _oracle_ga(pop, gens, fit_fn, **kw):
    best, total = [], []
    for gen in range(gens):
        f = fit_fn(pop)
        best.append(int(f.max()))
        total.append(int(f.sum()))
        pop = O.ga_breed(pop, f, gen, **kw)
    return pop, best, total


def test_ga_run_fujiyama_matches_oracle():
    """The paper's test bed: Hamming-weight fitness, population 512."""
    n, c, N, gens = 3, 8, 512, 40
    thr = J.poisson_thresholds(0.02)
    pop0 = W.random_genomes(N, n, c, seed=31)
    kw = dict(n=n, c=c, seed=5, selection=0, tournament=4, crossover=1, crossover_threshold=0x80000000,
              mutation_thresholds=thr)
    want_pop, want_best, want_total = _oracle_ga(pop0, gens, lambda p: np.array([O.hamming(int(v)) for v in p],
                                                                                np.int32), **kw)
    ga = J.make_ga(n, c, 5, selection=0, tournament=4, crossover=1, crossover_threshold=0x80000000,
                   mutation_thresholds=thr)
    pop = torch.from_numpy(pop0.view(np.int64).copy()).cuda()
    best = np.zeros(gens, np.int32)
    total = np.zeros(gens, np.int64)
    J.run_ga(ga, pop, gens, fitness_kind=J.FITNESS_HAMMING, best=best, total=total)
    assert best.tolist() == want_best and total.tolist() == want_total
    assert np.array_equal(pop.cpu().numpy().view(np.uint64), want_pop)
    assert want_best[-1] > want_best[0]  # selection on the single Fujiyama peak climbs


def test_ga_run_shape_fitness_matches_oracle():
    """Fitness = size of the deterministic bounded shape (S_{3,8}, 16 x 16, k = 20)."""
    n, c, N, gens, L, k, cseed = 3, 8, 256, 6, 16, 20, 7
    thr = J.poisson_thresholds(0.03)
    pop0 = W.random_genomes(N, n, c, seed=41)

    def fit(p):
        out = []
        for v in p:
            r = O.classify(n, c, L, k, cseed, O.decode(int(v), n, c), int(v))
            out.append(r["size"] if r["cls"] == O.DET_BOUNDED else 0)
        return np.array(out, np.int32)

    kw = dict(n=n, c=c, seed=9, selection=1, tournament=1, crossover=2, crossover_threshold=0x40000000,
              mutation_thresholds=thr)
    want_pop, want_best, want_total = _oracle_ga(pop0, gens, fit, **kw)
    ga = J.make_ga(n, c, 9, selection=1, tournament=1, crossover=2, crossover_threshold=0x40000000,
                   mutation_thresholds=thr)
    pop = torch.from_numpy(pop0.view(np.int64).copy()).cuda()
    best = torch.zeros(gens, dtype=torch.int32, device="cuda")
    total = torch.zeros(gens, dtype=torch.int64, device="cuda")
    J.run_ga(ga, pop, gens, fitness_kind=J.FITNESS_SHAPE, L=L, k=k, seed=cseed, best=best, total=total)
    torch.cuda.synchronize()
    assert best.cpu().tolist() == want_best and total.cpu().tolist() == want_total
    assert np.array_equal(pop.cpu().numpy().view(np.uint64), want_pop)


def test_screened_ga_reaches_the_best_shape_with_fewer_simulations():
    """The network as a pre-screen pays: at the same number
    of simulations, 5 generations of N = 2048 survivors (every survivor
    simulated by the plain classification) screened from 8 candidates each (the
    screen ratio of the GA configuration), the screened GA reaches a verified
    best fitness of 32 in more of 12 independent runs than the plain GA, and its
    mean verified best is higher.  (Over 32 runs on a GB300: 28 against 4, mean
    best 30.5 against 20.4; at a ratio of 4, 13 against 4 -- a margin that 12
    runs do not always show.)"""
    from paper_2205_15311_gb300 import surrogate as S
    dev = torch.device("cuda")
    genomes, labels = S.build_training_set(torch, dev, s28_sample=1 << 21, s38_sample=1 << 21)
    perm = torch.from_numpy(np.random.default_rng(1).permutation(genomes.shape[0])).to(dev)
    genomes, labels = genomes[perm].contiguous(), labels[perm].contiguous()
    net = J.Surrogate(max_batch=1 << 17)
    net.set_params(S.initial_params(0))
    S.train(torch, net, genomes, labels, steps=3000, batch=8192, lr=2e-3)
    trained = net.get_params()
    N, G, ratio = 2048, 5, 8
    thr = J.poisson_thresholds(0.03)
    best_plain, best_screened = [], []
    for sd in range(12):
        pop0 = W.random_genomes(N, 3, 8, seed=100 + sd)
        ga = J.make_ga(3, 8, 500 + sd, selection=J.TOURNAMENT, tournament=4, crossover=J.ONE_POINT,
                       crossover_threshold=0x80000000, mutation_thresholds=thr)
        for mode, out in (("plain", best_plain), ("screened", best_screened)):
            pop = torch.from_numpy(pop0.view(np.int64).copy()).to(dev)
            best = np.zeros(G, np.int32)
            if mode == "plain":
                J.run_ga(ga, pop, G, fitness_kind=J.FITNESS_SHAPE, L=16, k=20, seed=7, best=best)
            else:
                net.set_params(trained)  # every run starts from the same network
                J.run_ga_screened(ga, pop, G, ratio, net, online_lr=1e-3, L=16, k=20, seed=7, best=best)
            out.append(int(best.max()))
    net.close()
    reach_plain = sum(b >= 32 for b in best_plain)
    reach_screened = sum(b >= 32 for b in best_screened)
    print("best after 5 generations: plain", best_plain, "screened", best_screened)
    assert reach_screened >= reach_plain + 3
    assert np.mean(best_screened) > np.mean(best_plain) + 2


def test_host_histogram_staging_keeps_the_ga_buffers():
    """Staging a larger host histogram between two GA runs leaves the GA's own
    device buffers alone: the second run repeats the first exactly."""
    thr = J.poisson_thresholds(0.05)
    ga = J.make_ga(3, 8, 9, selection=J.TOURNAMENT, tournament=4, crossover=J.ONE_POINT,
                   crossover_threshold=0x80000000, mutation_thresholds=thr)
    pop0 = W.random_genomes(1024, 3, 8, seed=3)
    bests = []
    for i in range(2):
        pop = torch.from_numpy(pop0.view(np.int64).copy()).cuda()
        best = np.zeros(3, np.int32)
        J.run_ga(ga, pop, 3, fitness_kind=J.FITNESS_SHAPE, L=16, k=8, seed=2, best=best)
        bests.append((best.copy(), pop.cpu().numpy().copy()))
        # a host histogram with a capacity the workspace has not staged before
        out = torch.empty(4096 * 8, dtype=torch.uint8, device="cuda")
        hist = np.zeros(1 << (17 + i), J.HIST_DTYPE)
        hlen = np.zeros(1, np.uint32)
        J.enumerate_space(2, 8, 16, 20, 2, 0, 4096, out=out, hist=hist, hist_len=hlen, hist_cap=hist.shape[0])
    assert np.array_equal(bests[0][0], bests[1][0]) and np.array_equal(bests[0][1], bests[1][1])
