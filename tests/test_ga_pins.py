"""Pins of the oracle's genetic-algorithm step (Section 2.2 of the paper, its
appendix listings of the evolutionary operators, Section 3.2's Fujiyama
landscape) against facts fixed outside it: the paper's worked roulette
example, the Poisson distribution from scipy, and distributional properties
of selection, crossover and mutation.  No GPU needed."""
import numpy as np
import pytest

from oracle import oracle as O


def test_roulette_cumulative_search_paper_example():
    """Appendix "Tournament Selection in Haskell": weights 2, 3, 4, 1 and
    cut-off 10 select index 3 (the first running sum >= the cut-off).  A dart
    d in [0, total) corresponds to cut-off d + 1."""
    w = [2, 3, 4, 1]
    assert O.roulette_pick(w, 10 - 1) == 3
    # every cut-off 1..10: the first index whose running sum reaches it
    running = np.cumsum(w)
    for cutoff in range(1, 11):
        assert O.roulette_pick(w, cutoff - 1) == int(np.argmax(running >= cutoff))


def test_poisson_thresholds_match_scipy():
    stats = pytest.importorskip("scipy.stats")
    for rate in (0.0, 0.001, 0.01, 0.12, 0.5, 1.0, 3.0):
        t = O.poisson_thresholds(rate)
        for j in range(4):
            want = min(int(np.floor(stats.poisson.cdf(j, rate) * 2.0 ** 32)), 2 ** 32 - 1)
            assert abs(t[j] - want) <= 1, (rate, j)
        assert t == sorted(t)


def test_hamming_is_popcount():
    rng = np.random.default_rng(0)
    for g in rng.integers(0, 1 << 62, size=200, dtype=np.int64):
        assert O.hamming(int(g)) == bin(int(g)).count("1")


NONE = (0xFFFFFFFF,) * 4  # no mutation events (u >= 2^32 - 1 almost never; tested below)


def test_tournament_of_one_is_uniform_selection():
    N = 64
    parents = np.arange(N, dtype=np.uint64) << np.uint64(4)
    fitness = np.random.default_rng(1).integers(0, 100, size=N).astype(np.int32)
    counts = np.zeros(N)
    for gen in range(200):
        ch = O.ga_breed(parents, fitness, gen, n=2, c=8, seed=9, tournament=1, mutation_thresholds=NONE)
        counts += np.bincount((ch >> np.uint64(4)).astype(np.int64), minlength=N)
    expect = counts.sum() / N
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 120  # 63 degrees of freedom; p ~ 1e-5


def test_large_tournament_picks_the_fittest():
    N = 32
    parents = np.arange(N, dtype=np.uint64)
    fitness = np.zeros(N, np.int32)
    fitness[17] = 5
    ch = O.ga_breed(parents, fitness, 0, n=2, c=8, seed=3, tournament=16, mutation_thresholds=NONE)
    # with 16 draws out of 32 the fittest is drawn with probability 1 - (31/32)^16 ~ 0.4
    share = np.mean(ch == 17)
    assert 0.25 < share < 0.55
    ties = O.ga_breed(parents, np.zeros(N, np.int32), 0, n=2, c=8, seed=3, tournament=16, mutation_thresholds=NONE)
    # equal fitness: the earliest drawn wins, so the choice is still uniform
    assert len(set(ties.tolist())) > 10


def test_roulette_selects_in_proportion_to_fitness():
    N = 8
    parents = np.arange(N, dtype=np.uint64)
    fitness = np.array([0, 1, 2, 3, 4, 5, 6, 9], np.int32)
    counts = np.zeros(N)
    for gen in range(300):
        ch = O.ga_breed(np.tile(parents, 16), np.tile(fitness, 16), gen, n=2, c=8, seed=4, selection=O.ROULETTE,
                        mutation_thresholds=NONE)
        counts += np.bincount(ch.astype(np.int64), minlength=N)
    p = fitness / fitness.sum()
    assert counts[0] == 0
    expect = counts.sum() * p
    chi2 = ((counts[1:] - expect[1:]) ** 2 / expect[1:]).sum()
    assert chi2 < 30  # 6 degrees of freedom


def test_one_point_crossover_takes_a_prefix_and_a_suffix():
    n, c = 3, 8
    bits = 36
    ones = np.uint64((1 << bits) - 1)
    N = 4096
    # parent A all ones (fitness 1), parent B all zeros (fitness 0): tournament
    # picks A first whenever drawn; roulette with only A fit always picks A, so
    # use equal fitness and read which parent came first from the result
    parents = np.array([ones, 0] * (N // 2), dtype=np.uint64)
    fitness = np.ones(N, np.int32)
    ch = O.ga_breed(parents, fitness, 0, n=n, c=c, seed=11, tournament=1, crossover=O.ONE_POINT,
                    crossover_threshold=0xFFFFFFFF, mutation_thresholds=NONE)
    cuts = []
    for v in ch.tolist():
        if v in (0, int(ones)):
            continue  # both parents were the same genome
        low = v & -v if v else 0
        if v & 1:  # A below, B above: a low run of ones
            m = (~v) & ((1 << bits) - 1)
            cut = (m & -m).bit_length() - 1
            assert v == (1 << cut) - 1
        else:      # A above, B below: a high run of ones
            cut = low.bit_length() - 1
            assert v == ((1 << bits) - 1) & ~((1 << cut) - 1)
        cuts.append(cut)
    cuts = np.array(cuts)
    assert cuts.min() >= 1 and cuts.max() <= bits - 1
    assert len(set(cuts.tolist())) == bits - 1  # every cut point occurs


def test_uniform_crossover_mixes_bits_evenly():
    ones = np.uint64((1 << 36) - 1)
    N = 4096
    parents = np.array([ones, 0] * (N // 2), dtype=np.uint64)
    ch = O.ga_breed(parents, np.ones(N, np.int32), 0, n=3, c=8, seed=12, tournament=1, crossover=O.UNIFORM,
                    crossover_threshold=0xFFFFFFFF, mutation_thresholds=NONE)
    frac = np.mean([bin(int(v)).count("1") for v in ch]) / 36
    assert 0.47 < frac < 0.53


def test_crossover_threshold_zero_never_crosses():
    ones = np.uint64((1 << 36) - 1)
    parents = np.array([ones, 0] * 512, dtype=np.uint64)
    ch = O.ga_breed(parents, np.ones(1024, np.int32), 0, n=3, c=8, seed=13, tournament=1, crossover=O.ONE_POINT,
                    crossover_threshold=0, mutation_thresholds=NONE)
    assert set(ch.tolist()) <= {0, int(ones)}


def test_mutation_counts_follow_poisson_per_edge():
    """Each edge gets a Poisson number of events with mean `rate`; each flips
    one of the edge's 3 bits.  The flipped-bit count per child has mean
    12 rate (1 - cancellations), and only bits of one edge change per event."""
    n, c, rate, N = 3, 8, 0.05, 20000
    thr = O.poisson_thresholds(rate)
    parents = np.zeros(N, np.uint64)
    ch = O.ga_breed(parents, np.zeros(N, np.int32), 5, n=n, c=c, seed=14, tournament=1, mutation_thresholds=thr)
    flips = np.array([bin(int(v)).count("1") for v in ch])
    # events per child ~ Poisson(12 rate) = Poisson(0.6); two events on one bit cancel (rare)
    assert abs(flips.mean() - 12 * rate) < 0.03
    p0 = np.mean(flips == 0)
    assert abs(p0 - np.exp(-12 * rate)) < 0.02
    none = O.ga_breed(parents, np.zeros(N, np.int32), 5, n=n, c=c, seed=14, tournament=1, mutation_thresholds=NONE)
    assert not none.any()


def test_breed_draw_layout_rederived():
    """Every word a child consumes, re-derived from Triton's Philox with the
    documented layout -- word k of child i in generation g is word (k mod 4) of
    Philox4x32-10(ctr = (k >> 2, (2 << 24) | g, i_lo, i_hi), key = seed), in
    the order: selection of parent A (T words, or one roulette dart), of
    parent B, the crossover decision, two cut/mask words, one Poisson word per
    edge, four bit-choice words per edge -- and the operators applied by hand:
    selection (Section 2.2), one-point / uniform crossover and single-bit
    mutations of an edge (the appendix listings of the operators)."""
    from triton_philox import triton_philox

    n, c, b = 3, 8, 3
    bits = 4 * n * b
    N, gen, seed = 12, 7, 0x0123456789ABCDEF
    rng = np.random.default_rng(4)
    parents = rng.integers(0, 1 << bits, size=N, dtype=np.int64).astype(np.uint64)
    fitness = rng.integers(0, 20, size=N).astype(np.int32)
    fitness[[2, 5]] = 0
    thr = O.poisson_thresholds(0.7)  # many mutation events, up to the cap of 4
    configs = [(O.TOURNAMENT, 4, O.ONE_POINT), (O.ROULETTE, 1, O.UNIFORM), (O.TOURNAMENT, 2, O.NO_CROSSOVER)]
    for selection, T, crossover in configs:
        got = O.ga_breed(parents, fitness, gen, n=n, c=c, seed=seed, selection=selection, tournament=T,
                         crossover=crossover, crossover_threshold=1 << 31, mutation_thresholds=thr)
        K = 2 * T + 3 + 4 * n + 4 * 4 * n
        nblk = (K + 3) // 4
        for i in range(N):
            blocks = triton_philox([[q, (2 << 24) | gen, i, 0] for q in range(nblk)],
                                   [seed & 0xFFFFFFFF, seed >> 32])
            w = [blocks[k >> 2][k & 3] for k in range(K)]

            def select(k0):
                if selection == O.TOURNAMENT:
                    best = None
                    for j in range(T):
                        idx = (w[k0 + j] * N) >> 32
                        if best is None or fitness[idx] > fitness[best]:
                            best = idx
                    return best
                total = int(np.maximum(fitness, 0).sum())
                if total == 0:
                    return (w[k0] * N) >> 32
                dart = (w[k0] * total) >> 32
                return int(np.argmax(np.cumsum(np.maximum(fitness, 0)) > dart))

            a, bb = int(parents[select(0)]), int(parents[select(T)])
            child = a
            if crossover != O.NO_CROSSOVER and w[2 * T] < (1 << 31):
                if crossover == O.ONE_POINT:
                    cut = 1 + ((w[2 * T + 1] * (bits - 1)) >> 32)
                    low = (1 << cut) - 1
                else:
                    low = (w[2 * T + 2] << 32) | w[2 * T + 1]
                child = (a & ~low) | (bb & low)
            for e in range(4 * n):
                events = sum(1 for t in thr if w[2 * T + 3 + e] >= t)
                pos = b * (4 * (n - 1 - e // 4) + (3 - e % 4))
                for m in range(events):
                    child ^= 1 << (pos + ((w[2 * T + 3 + 4 * n + 4 * e + m] * b) >> 32))
            assert int(got[i]) == child & ((1 << bits) - 1), (selection, T, crossover, i)
