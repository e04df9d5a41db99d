"""Benchmark: genotypes classified per second on one GB300.

Workload: S_{2,8} in full -- all 8^8 = 16,777,216 two-tile genotypes, 16 x 16
grid, k = 20 replicate assemblies, Philox key 2 -- classified by
jatam_enumerate into per-genotype results (8 B each, 134 MB, larger than the
129 MB L2) plus the phenotype histogram.  One step = one such enumeration.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank classifies its own full copy of the
workload under its own Philox key (weak scaling, no collective on the data
path); rank 0 prints one JSON line with the whole-job rate.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "s28_full"
METRIC = "genotypes classified/s (1 GB300, bit-exact vs oracle) + % int/smem roofline"
UNIT = "genotypes/s"

# algorithmic integer operations per unit of work of the growth kernel: a drawn placement
# (Philox word 15, rank 1, site selection 10, placement 4, four neighbour re-evaluations 32),
# a replicate (seed placement and its four neighbours, compare), a genotype (decode, tuples,
# candidate masks, result), a cell of a shaped genotype (crop, 8 images, hash bytes)
OPS_PER_PLACEMENT = 62
OPS_PER_REPLICATE = 37
OPS_PER_GENOTYPE = 300
OPS_PER_SHAPED_CELL = 24
SOAK_S = 2.0  # seconds of back-to-back steps inside the clock record before the timed steps


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.t:
                self.t.join(timeout=2)

    def summary(self):
        """Median SM clock over the samples taken under load (GPU utilisation of
        at least 50 %; all samples if the field is unavailable), the maximum
        clock, and every throttle reason seen active."""
        sm, smax, util, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            try:
                util.append(float(p[9]) if len(p) > 9 else -1.0)
            except ValueError:
                util.append(-1.0)
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    "samples_under_load": 0}
        loaded = [c for c, u in zip(sm, util) if u >= 50.0]
        return {"sm_mhz": float(np.median(loaded if loaded else sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm), "samples_under_load": len(loaded)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def algorithmic_ops(res_cls, res_rep, res_size, k, placements):
    """Integer operations the method as stated needs for one pass over the
    workload: every replicate of every genotype simulated (the oracle's count)."""
    reps = np.where(res_rep >= k, k, res_rep.astype(np.int64) + 1).sum()
    shaped = (res_cls == 0) | (res_cls == 2)
    cells = res_size[shaped].astype(np.int64).sum()
    return (OPS_PER_PLACEMENT * placements + OPS_PER_REPLICATE * int(reps) + OPS_PER_GENOTYPE * res_cls.size
            + OPS_PER_SHAPED_CELL * int(cells))


def executed_ops(work, res_cls, res_size):
    """Integer operations of the work the growth kernel itself executed (its
    counters): drawn and seed placements, genotypes taken by warps, and the
    cells of the shapes it canonicalised (the pre-filter settles lone seeds)."""
    shaped = ((res_cls == 0) | (res_cls == 2)) & (res_size > 1)
    cells = res_size[shaped].astype(np.int64).sum()
    return (OPS_PER_PLACEMENT * work["placements"] + OPS_PER_REPLICATE * work["seeds"]
            + OPS_PER_GENOTYPE * work["genotypes"] + OPS_PER_SHAPED_CELL * int(cells))


def measured_traffic(kernel_file):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary,
    or None when the kernel source changed since those counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "classify_kernel_s28_full_traffic.md")
    try:
        text = open(path).read()
        src = open(kernel_file, "rb").read()
    except OSError:
        return None
    want = None
    traffic = None
    for line in text.splitlines():
        if line.startswith("kernel_source_sha256_prefix:"):
            want = line.split(":", 1)[1].strip()
        if line.startswith("traffic_bytes_per_launch:"):
            traffic = int(line.split(":", 1)[1].strip())
    if want is None or traffic is None or hashlib.sha256(src).hexdigest()[: len(want)] != want:
        return None
    return traffic


def measured_pipes(kernel_file):
    """ALU-pipe and issue utilisation of the dominant kernel from the committed
    ncu full capture (2^22 random S_{2,8} genomes), or None when the kernel
    source changed since."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "classify_kernel_s28_rand4M_ncu_full.md")
    try:
        text = open(path).read()
        src = open(kernel_file, "rb").read()
    except OSError:
        return None
    m = re.search(r"sha256 prefix ([0-9a-f]+)", text)
    alu = re.search(r"sm__pipe_alu_cycles_active\.avg\.pct_of_peak_sustained_active` \| ([0-9.]+) %", text)
    issue = re.search(r"smsp__issue_active\.avg\.pct_of_peak_sustained_active` \| ([0-9.]+) %", text)
    if not (m and alu and issue) or hashlib.sha256(src).hexdigest()[: len(m.group(1))] != m.group(1):
        return None
    return {"alu_pipe_active": round(float(alu.group(1)) / 100, 4), "issue_active": round(float(issue.group(1)) / 100, 4),
            "source": "profiles/classify_kernel_s28_rand4M_ncu_full.md"}


def cpu_sample_plan():
    """Stratified bounded sample of the workload for the oracle: 64 blocks of
    up to 65,536 consecutive genotypes spread evenly over the workload."""
    n, c, L, k, seed, first, count, sampled = WORKLOAD_SPEC()
    blocks = 64
    stride = count // blocks
    per = min(65536, stride)
    return [(first + b * stride, per) for b in range(blocks)]


def cpu_sample_text():
    n, c, L, k, seed, first, count, sampled = WORKLOAD_SPEC()
    per = cpu_sample_plan()[0][1]
    what = "sample indices" if sampled else "consecutive genotypes"
    return f"64 blocks of {per:,} {what} of S_{{{n},{c}}} spread evenly over the workload"


def WORKLOAD_SPEC():
    from paper_2205_15311_gb300 import workloads as W
    return W.WORKLOADS[WORKLOAD]


MIXED_COUNT = 10_000_000


def _timed_steps(torch, stream, flush, steps, fn, J=None):
    """Mean CUDA-event time of `steps` calls of fn on `stream`, a buffer larger
    than L2 written before each; with J, also the mean growth-kernel time of
    the profiling mode."""
    st = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    kms = []
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 255)
            st[i].record(stream)
            fn()
            en[i].record(stream)
        if J is not None:
            kms.append(J.last_kernel_ms())
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in zip(st, en)]))
    return ms, (float(np.mean(kms)) if kms else None)


def _collisions(J):
    """Shape hashes of the last call that named two distinct canonical forms
    (the exact side table; None if the call recorded no shapes)."""
    try:
        return J.last_shapes()[1]
    except J.JatamError:
        return None


def measure_mixed(torch, J, dev, steps, warmup):
    """Batched uneven workload: 10^7 explicit tile sets with n in {2,3,4},
    c in {4,6,8}, L in {8,16,32}, k in {10,20} (seed 4) in one persistent,
    graph-captured launch whose CTA plan the autotuner picks; the per-size
    fixed launches are timed beside it."""
    from paper_2205_15311_gb300 import workloads as W
    colours, shapes = W.mixed_records(MIXED_COUNT, seed=4)
    dc = torch.from_numpy(colours).to(dev)
    ds = torch.from_numpy(shapes).to(dev)
    out = torch.empty(MIXED_COUNT * 8, dtype=torch.uint8, device=dev)
    hist_cap = 1 << 16
    hist = torch.empty(hist_cap * 32, dtype=torch.uint8, device=dev)
    hlen = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    J.autotune_batch(dc, ds, 4, stream=stream)
    plan = J.get_mixed_plan()
    choice = J.get_mixed_launch()

    def call(per_shape, graph):
        J.classify_batch(dc, seed=4, shapes=ds, out=out, hist=hist, hist_len=hlen, hist_cap=hist_cap,
                         stream=stream, per_shape=per_shape, graph=graph)

    J.jatam_profile(1)
    res = {}
    for name, per_shape, graph in (("persistent_graph", False, True), ("per_size_fixed", True, False)):
        for _ in range(warmup):
            call(per_shape, graph)
        stream.synchronize()
        ms, kms = _timed_steps(torch, stream, flush, steps, lambda: call(per_shape, graph), J)
        res[name] = {"value": MIXED_COUNT / (ms / 1e3), "ms_per_step": round(ms, 4), "growth_kernels_ms": round(kms, 4)}
    J.jatam_profile(0)
    collisions = _collisions(J)
    # end to end through the C ABI: the records, their shapes and stream ids copied from page-locked host
    # memory, the results copied back (the call runs in pieces whose copies overlap the classification)
    ch = torch.from_numpy(colours).pin_memory()
    sh = torch.from_numpy(shapes).pin_memory()
    ids = torch.arange(MIXED_COUNT, dtype=torch.int64).pin_memory()
    out_h = torch.empty(MIXED_COUNT * 8, dtype=torch.uint8, pin_memory=True)
    hist_h = np.zeros(hist_cap, J.HIST_DTYPE)
    hlen_h = np.zeros(1, np.uint32)

    def call_host():
        J.classify_batch(ch, seed=4, shapes=sh, stream_ids=ids, out=out_h, hist=hist_h, hist_len=hlen_h,
                         hist_cap=hist_cap, stream=stream)

    call_host()
    e2e = []
    for i in range(steps):
        flush.fill_(i & 255)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        call_host()
        e2e.append(time.perf_counter() - t0)
    e2e_line = {"value": MIXED_COUNT / float(np.mean(e2e)), "unit": UNIT,
                "h2d_bytes_per_step": MIXED_COUNT * (16 + 4 + 8), "d2h_bytes_per_step": MIXED_COUNT * 8 +
                int(hlen_h[0]) * 32 + 8}
    return {"workload": "mixed: 10^7 tile sets, n in {2,3,4}, c in {4,6,8}, L in {8,16,32}, k in {10,20}, seed 4",
            "e2e": e2e_line, "shape_collisions": collisions,
            "unit": UNIT, "value": res["persistent_graph"]["value"], "steps": steps, "warmup": warmup,
            "persistent_graph": res["persistent_graph"], "per_size_fixed": res["per_size_fixed"],
            "plan_w32_w16_w8": list(plan), "autotuner_default_launch": "per_size" if choice else "persistent",
            "distinct_phenotypes": int(hlen.item())}


def mixed_arm(args, torch, J, dev):
    with ClockSampler(int(str(dev).split(":")[-1]) if ":" in str(dev) else 0) as clocks:
        m = measure_mixed(torch, J, dev, args.steps, args.warmup)
    line = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["persistent_graph"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": m, "e2e": None, "gpu_launches": 5 * args.steps, "roofline": None, "cpu_baseline": None,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_ga(torch, J, dev, seed=5, N=8192, G=500, ratio=8, train_steps=3000, seeds=(5, 1, 2, 3, 4, 6, 7, 8)):
    """The GA of the fifth configuration (n = 3, c = 8 genomes, population
    8192, 500 generations, per-edge mutation rate 0.01, tournament of 4, shape
    fitness at L = 16, k = 20; the configuration's seed 5 and seven more),
    plain and with the surrogate network as a pre-screen (trained first on
    labels the library's classification gives: S_{2,4} in full, a uniform
    sample of S_{2,8}, and a uniform sample of S_{3,8} at the GA's L and k).
    Every reported fitness is simulated.  Per seed and arm: the best verified
    fitness and the generation at which it was first reached; per arm: how
    many seeds reached the best fitness any run found, the median
    generations and simulations to it, and genomes simulated per second."""
    from paper_2205_15311_gb300 import surrogate as S
    from paper_2205_15311_gb300 import workloads as W
    genomes, labels = S.build_training_set(torch, dev, s28_sample=1 << 21, s38_sample=1 << 21)
    perm = torch.from_numpy(np.random.default_rng(seed).permutation(genomes.shape[0])).to(dev)
    genomes, labels = genomes[perm].contiguous(), labels[perm].contiguous()
    net = J.Surrogate(max_batch=max(N * ratio, 1 << 15))
    net.set_params(S.initial_params(seed))
    t0 = time.perf_counter()
    S.train(torch, net, genomes, labels, steps=train_steps, batch=8192, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    trained = net.get_params()
    thr = J.poisson_thresholds(0.01)
    runs = {"plain": {}, "screened": {}}
    for sd in seeds:
        ga = J.make_ga(3, 8, sd, selection=J.TOURNAMENT, tournament=4, crossover=J.NO_CROSSOVER,
                       mutation_thresholds=thr)
        pop0 = W.random_genomes(N, 3, 8, seed=sd)
        for mode in ("plain", "screened"):
            pop = torch.from_numpy(pop0.view(np.int64).copy()).to(dev)
            best = np.zeros(G, np.int32)
            net.set_params(trained)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            if mode == "plain":
                J.run_ga(ga, pop, G, fitness_kind=J.FITNESS_SHAPE, L=16, k=20, seed=sd, best=best)
            else:
                J.run_ga_screened(ga, pop, G, ratio, net, online_lr=1e-3, L=16, k=20, seed=sd, best=best)
            b.record()
            torch.cuda.synchronize()
            so_far = np.maximum.accumulate(best)
            top = int(so_far[-1])
            runs[mode][sd] = {"best": top, "generation_of_best": int(np.argmax(so_far >= top)),
                              "ms": round(a.elapsed_time(b), 1), "so_far": so_far}
    net.close()
    target = max(r["best"] for m in runs.values() for r in m.values())
    arms = {}
    for mode, per_seed in runs.items():
        gens = [int(np.argmax(r["so_far"] >= target)) for r in per_seed.values() if r["best"] >= target]
        ms = sum(r["ms"] for r in per_seed.values())
        arms[mode] = {
            "genomes_per_s": len(seeds) * N * G / (ms / 1e3),
            "seeds_reaching_target": f"{len(gens)} of {len(seeds)}",
            "median_generations_to_target": float(np.median(gens)) if gens else None,
            "median_simulations_to_target": float(np.median(gens)) * N + N if gens else None,
            "per_seed": {str(sd): {"best": r["best"], "generation_of_best": r["generation_of_best"], "ms": r["ms"]}
                         for sd, r in per_seed.items()},
        }
    return {"workload": f"ga: n=3 c=8, population {N}, {G} generations, per-edge mutation 0.01, tournament 4, "
                        f"shape fitness L=16 k=20, seeds {list(seeds)} (the configuration's seed first)",
            "unit": "genomes/s", "value": arms["plain"]["genomes_per_s"], "target_best_fitness": target,
            "surrogate": f"36-256-256-8 bf16, {train_steps} Adam steps of 8192 on S_{{2,4}} + 2M S_{{2,8}} + "
                         f"2M S_{{3,8}} labels ({train_s:.1f} s); screen ratio {ratio}, online lr 1e-3",
            "plain": arms["plain"], "screened": arms["screened"]}


def ga_arm(args, torch, J, dev):
    m = measure_ga(torch, J, dev)
    line = {
        "metric": "GA genomes simulated/s (every survivor classified; plain vs surrogate-screened)",
        "value": m["value"], "unit": "genomes/s", "n_gpus": 1, "steps": 500, "warmup": 0,
        "ms_per_step": 8192 / m["value"] * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic", "config": m,
        "e2e": None, "gpu_launches": None, "roofline": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_enumeration(torch, J, dev, name, steps, warmup, top_shapes=0):
    """One of the enumerated or sampled workloads, timed like the bench line;
    with top_shapes, the largest deterministic bounded shapes of its histogram
    (size, hash, genotypes, smallest genotype)."""
    from paper_2205_15311_gb300 import workloads as W
    n, c, L, k, seed, first, count, sampled = W.WORKLOADS[name]
    hist_cap = 1 << 16
    stream = torch.cuda.Stream(device=dev)
    out = torch.empty(count * 8, dtype=torch.uint8, device=dev)
    hist = torch.empty(hist_cap * 32, dtype=torch.uint8, device=dev)
    hlen = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def call():
        J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out, hist=hist, hist_len=hlen,
                          hist_cap=hist_cap, stream=stream)

    J.jatam_profile(1)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            call()
    stream.synchronize()
    ms, kms = _timed_steps(torch, stream, flush, steps, call, J)
    J.jatam_profile(0)
    m = int(hlen.item())
    r = {"workload": f"{name}: {'sampled' if sampled else 'all'} {count} genotypes of S_{{{n},{c}}}, "
                     f"L={L} k={k} seed={seed}", "unit": UNIT, "value": count / (ms / 1e3), "ms_per_step": round(ms, 4),
         "growth_kernels_ms": round(kms, 4), "steps": steps, "warmup": warmup, "distinct_phenotypes": m}
    r["shape_collisions"] = _collisions(J)
    # end to end through the C ABI: results and histogram to page-locked host memory
    out_h = torch.empty(count * 8, dtype=torch.uint8, pin_memory=True)
    hist_h = np.zeros(hist_cap, J.HIST_DTYPE)
    hlen_h = np.zeros(1, np.uint32)

    def call_host():
        J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out_h, hist=hist_h, hist_len=hlen_h,
                          hist_cap=hist_cap, stream=stream)

    call_host()
    e2e = []
    for i in range(steps):
        flush.fill_(i & 255)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        call_host()
        e2e.append(time.perf_counter() - t0)
    r["e2e"] = {"value": count / float(np.mean(e2e)), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": count * 8 + int(hlen_h[0]) * 32 + 8}
    del out_h
    if top_shapes:
        h = J.hist_view(hist, min(m, hist_cap))
        det = [x for x in h.tolist() if x[0] == 0]
        det.sort(key=lambda x: (-x[2], -x[4], x[1]))
        r["largest_det_shapes"] = [{"size": int(x[2]), "shape_hash": int(x[1]), "genotypes": int(x[4]),
                                    "min_genotype": int(x[5])} for x in det[:top_shapes]]
    del out
    return r


def measure_configs(torch, J, dev, steps, warmup):
    """The other configurations, measured in the same run as the bench line."""
    cfg = {}
    cfg["c1_s24_full"] = measure_enumeration(torch, J, dev, "s24_full", steps, warmup)
    cfg["c3_s38_sample"] = measure_enumeration(torch, J, dev, "s38_sample", steps, warmup, top_shapes=8)
    torch.cuda.empty_cache()
    cfg["c4_mixed"] = measure_mixed(torch, J, dev, steps, warmup)
    torch.cuda.empty_cache()
    cfg["c5_ga"] = measure_ga(torch, J, dev)
    torch.cuda.empty_cache()
    return cfg


KSWEEP = (1, 2, 4, 8, 16, 20, 32, 64, 128)


def ksweep_arm(args, torch, J, dev):
    """The k sweep of the paper's S_{2,8} result (Section 3.1): all 8^8
    genotypes classified at each k, for the lattice of the bench (L = 16) and
    the paper's (L = 19).  With one seed the first k replicates of a run at k'
    > k are the run at k, so DET(k') is a subset of DET(k); the genotypes
    called DET at k but not at the largest k are non-deterministic genotypes
    misclassified at k.  Reports their share of DET(k) and the GPU time."""
    n, c, seed, count = 2, 8, 2, 8 ** 8
    out = torch.empty(count * 8, dtype=torch.uint8, device=dev)
    J.jatam_profile(1)
    lines = {}
    for L in (16, 19):
        rows = {}
        for k in KSWEEP:
            for _ in range(2):  # the first call of a shape pays for its set-up
                J.enumerate_space(n, c, L, k, seed, 0, count, out=out, sync=True)
            kms = J.last_kernel_ms()
            cls = J.results_view(out)["cls"]
            counts = np.bincount(cls.astype(np.int64), minlength=4)
            rows[k] = {"det": int(counts[0]), "nd_local": int(counts[1]), "nd_steric": int(counts[2]),
                       "unbounded": int(counts[3]), "growth_kernels_ms": round(kms, 3)}
        det_ref = rows[KSWEEP[-1]]["det"]
        for k in KSWEEP:
            d = rows[k]["det"]
            rows[k]["misclassified_share_of_det"] = round((d - det_ref) / d, 6) if d else 0.0
        lines[f"L{L}"] = rows
    line = {"metric": "k sweep of S_{2,8}: genotypes called DET at k that are not DET at k = 128",
            "value": lines["L19"][8]["misclassified_share_of_det"], "unit": "share of DET(k=8) at L=19",
            "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
            "config": {"workload": f"ksweep: all 8^8 genotypes of S_{{2,8}}, seed {seed}, k in {list(KSWEEP)}, "
                                   "L in {16, 19}", "sweep": lines}}
    print(json.dumps(line), flush=True)
    return 0


def run_oracle_sample(nthreads):
    from oracle import oracle as O
    n, c, L, k, seed, _, _, _ = WORKLOAD_SPEC()
    done = 0
    t0 = time.perf_counter()
    for first, cnt in cpu_sample_plan():
        O.enumerate_space(n, c, L, k, seed, first, cnt, nthreads=nthreads)
        done += cnt
    return done, time.perf_counter() - t0


def reference_arm(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    cores = getattr(args, "cpu_threads", 0) or os.cpu_count() or 1
    times, units = [], 0
    for _ in range(args.warmup):
        run_oracle_sample(cores)
    for _ in range(args.steps):
        u, dt = run_oracle_sample(cores)
        units = u
        times.append(dt)
    per_step = float(np.mean(times))
    value = units / per_step
    n, c, L, k, seed, first, count, _ = WORKLOAD_SPEC()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: S_{{{n},{c}}} n={n} c={c} L={L} k={k} seed={seed}",
                   "step": f"oracle on a stratified sample of {units} genotypes (64 x 65536)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{cpu_sample_text()} ({units} per step)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def network_profile_case(args, torch, J, dev):
    """Small cases of the network and pre-screen kernels for ncu: screened GA
    generations (population 8192, ratio 8, device-side best) or predictions."""
    from paper_2205_15311_gb300 import surrogate as S
    from paper_2205_15311_gb300 import workloads as W
    N, ratio = 8192, 8
    net = J.Surrogate(max_batch=max(N * ratio, args.profile_predict))
    net.set_params(S.initial_params(5))
    if args.profile_predict:
        n = args.profile_predict
        g = torch.from_numpy(W.random_genomes(n, 3, 8, seed=3).view(np.int64)).to(dev)
        logits = torch.empty((n, 8), dtype=torch.float32, device=dev)
        for i in range(args.warmup + args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            net.predict(g, logits)
            b.record()
            torch.cuda.synchronize()
            if i >= args.warmup:
                print(json.dumps({"profile_predict": n, "ms": round(a.elapsed_time(b), 4)}))
    else:
        G = args.profile_screen
        thr = J.poisson_thresholds(0.01)
        ga = J.make_ga(3, 8, 5, selection=J.TOURNAMENT, tournament=4, crossover=J.NO_CROSSOVER,
                       mutation_thresholds=thr)
        pop = torch.from_numpy(W.random_genomes(N, 3, 8, seed=5).view(np.int64)).to(dev)
        best = torch.zeros(G, dtype=torch.int32, device=dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        J.run_ga_screened(ga, pop, G, ratio, net, online_lr=1e-3, L=16, k=20, seed=5, best=best)
        b.record()
        torch.cuda.synchronize()
        print(json.dumps({"profile_screen_generations": G, "ms_per_generation": round(a.elapsed_time(b) / G, 4)}))
    net.close()
    return 0


def main():
    global WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="s28_full",
                    help="s28_full (the bench line), or s24_full / s28_paper / s38_sample / mixed / ga / ksweep "
                         "for measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-threads", type=int, default=0, help="threads of the oracle arm (default: all cores)")
    ap.add_argument("--lifo", action="store_true",
                    help="the movelist process (JATAM_LIFO) instead of the row-major frontier; a measurement")
    ap.add_argument("--orbits", action="store_true",
                    help="orbit mode (JATAM_ORBITS): one classification per orbit of the exact symmetries; "
                         "a measurement, not the bench line")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations (S_{2,4}, the 2^28 S_{3,8} sample, the 10^7 mixed "
                         "batch, the GA arms) measured after the bench line")
    ap.add_argument("--profile-genomes", type=int, default=0,
                    help="instead of the bench: ga_evaluate on this many uniform random genomes of the "
                         "workload's space (a representative small case for ncu); prints timings only")
    ap.add_argument("--profile-screen", type=int, default=0,
                    help="instead of the bench: this many screened GA generations (population 8192 of "
                         "S_{3,8}, screen ratio 8, an untrained network) -- the network and pre-screen "
                         "kernels for ncu; prints timings only")
    ap.add_argument("--profile-predict", type=int, default=0,
                    help="instead of the bench: network predictions of this many S_{3,8} genomes "
                         "(the warm-up count, then the step count); prints timings only")
    ap.add_argument("--count", type=int, default=0,
                    help="classify only the first COUNT genotypes (small profiling cases; not a bench line)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    WORKLOAD = args.workload
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import torch.distributed as dist

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_15311_gb300 import binding as J
    if args.profile_screen or args.profile_predict:
        return network_profile_case(args, torch, J, dev)
    if WORKLOAD == "mixed":
        return mixed_arm(args, torch, J, dev)
    if WORKLOAD == "ga":
        return ga_arm(args, torch, J, dev)
    if WORKLOAD == "ksweep":
        return ksweep_arm(args, torch, J, dev)

    n, c, L, k, seed0, first, count, sampled = WORKLOAD_SPEC()
    if args.profile_genomes:
        from paper_2205_15311_gb300 import workloads as W
        g = torch.from_numpy(W.random_genomes(args.profile_genomes, n, c, seed=7).view(np.int64)).to(dev)
        fit = torch.empty(args.profile_genomes, dtype=torch.int32, device=dev)
        J.jatam_profile(1)
        for i in range(args.warmup + args.steps):
            J.evaluate_genomes(g, fit, n=n, c=c, L=L, k=k, seed=seed0, sync=True)
            if i >= args.warmup:
                print(json.dumps({"profile_genomes": args.profile_genomes, "kernel_ms": J.last_kernel_ms()}))
        return 0
    if args.count:
        count = min(count, args.count)
    seed = seed0 + rank  # every rank: its own independent classification of the space
    hist_cap = 1 << 16
    stream = torch.cuda.Stream(device=dev)
    out = torch.empty(count * 8, dtype=torch.uint8, device=dev)
    hist = torch.empty(hist_cap * 32, dtype=torch.uint8, device=dev)
    hlen = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # larger than the 129 MB L2

    def step():
        J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out, hist=hist, hist_len=hlen,
                          hist_cap=hist_cap, stream=stream, orbits=args.orbits, lifo=args.lifo)

    J.jatam_profile(1)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    # one untimed counted pass: the work the growth kernel executes per step
    J.jatam_profile(3)
    with torch.cuda.stream(stream):
        step()
    stream.synchronize()
    work = J.work_counters()
    J.jatam_profile(1)

    # a sustained run of at least SOAK_S seconds of back-to-back steps just before the timed steps, inside
    # the clock record: the sampler sees the GPU under load even when the timed steps are short
    est = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    est[0].record(stream)
    with torch.cuda.stream(stream):
        step()
    est[1].record(stream)
    torch.cuda.synchronize()
    soak_steps = max(1, int(np.ceil(SOAK_S * 1e3 / max(est[0].elapsed_time(est[1]), 1e-3))))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kernel_ms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        soak = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        soak[0].record(stream)
        with torch.cuda.stream(stream):
            for _ in range(soak_steps):
                step()
        soak[1].record(stream)
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(i & 255)
                starts[i].record(stream)
                step()
                stops[i].record(stream)
            kernel_ms.append(J.last_kernel_ms())
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    soak_ms = soak[0].elapsed_time(soak[1])
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, stops)]
    ms = float(np.mean(step_ms))
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * count / (ms / 1e3)

    # end to end through the C ABI with host buffers: results and histogram land in pinned host memory;
    # the calls a user makes, without the kernel timing of the profiling mode
    J.jatam_profile(0)
    out_h = torch.empty(count * 8, dtype=torch.uint8, pin_memory=True)
    hist_h = np.zeros(hist_cap, J.HIST_DTYPE)
    hlen_h = np.zeros(1, np.uint32)
    if not args.no_e2e:
        J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out_h, hist=hist_h,
                          hist_len=hlen_h, hist_cap=hist_cap, stream=stream, orbits=args.orbits, lifo=args.lifo)
    e2e_times = []
    for i in range(0 if args.no_e2e else max(3, min(args.steps, 5))):
        flush.fill_(i & 255)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J.enumerate_space(n, c, L, k, seed, first, count, sampled=sampled, out=out_h, hist=hist_h,
                          hist_len=hlen_h, hist_cap=hist_cap, stream=stream, orbits=args.orbits, lifo=args.lifo)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e_times)) if e2e_times else float("nan")
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    nk = int(hlen_h[0]) if e2e_times else int(hlen.item())
    collisions = _collisions(J)

    line = None
    if rank == 0:
        res = J.results_view(out)
        peaks = measured_peaks()
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        props = torch.cuda.get_device_properties(dev)
        n_sms = props.multi_processor_count
        alu_peak = n_sms * 128 * sm_max * 1e6 / 1e12  # int32 lane-ops per second, T
        placements = None
        golden = os.path.join(ROOT, "tests", "golden",
                              {"s28_full": "c2_summary.json", "s24_full": "c1_summary.json"}.get(WORKLOAD, "-"))
        if os.path.exists(golden) and rank == 0 and not args.count and not args.orbits and not args.lifo:
            placements = json.load(open(golden))["placements"]
        roofline = None
        kms = float(np.mean(kernel_ms))
        ops = executed_ops(work, res["cls"], res["size"])
        achieved = ops / (kms / 1e3) / 1e12
        traffic = measured_traffic(os.path.join(ROOT, "paper_2205_15311_gb300", "csrc", "jatam_kernels.cu"))
        if WORKLOAD != "s28_full":
            traffic = None
        roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(alu_peak, 2),
                    "unit": "Tops/s", "frac": round(achieved / alu_peak, 4), "traffic": traffic,
                    "kernel": f"classify_kernel<{8 if L <= 8 else 16 if L <= 16 else 32}, {8 if n <= 2 else 16}, "
                              f"{1 if args.lifo else 0}>",
                    "kernel_ms": round(kms, 4),
                    "peak_source": f"{n_sms} SMs x 128 int32 lanes x {sm_max:.0f} MHz (MEASURED_PEAKS sm_max)",
                    "executed": work,
                    "lane_utilisation": round((work["placements"] + work["seeds"]) / max(work["lane_slots"], 1), 4),
                    "hbm_gbs": round(count * 8 / (kms / 1e3) / 1e9, 1),
                    "hbm_frac_of_measured": round(count * 8 / (kms / 1e3) / 1e9 / float(peaks.get("hbm_gbs", 6753.1)), 4)}
        pipes = measured_pipes(os.path.join(ROOT, "paper_2205_15311_gb300", "csrc", "jatam_kernels.cu"))
        if pipes is not None and n <= 2 and L <= 16 and not args.lifo:
            # context for the ALU fraction: how busy the kernel keeps the SM (ncu, same source)
            roofline["ncu_pipes"] = pipes
        if placements is not None:
            # the same rate counted in the work of the process as the paper states it
            # (all k replicates of every genotype, the oracle's placement count)
            mops = algorithmic_ops(res["cls"], res["decided_rep"], res["size"], k, placements)
            roofline["method_placements"] = placements
            roofline["method_ops_frac"] = round(mops / (kms / 1e3) / 1e12 / alu_peak, 4)
        cpu = None
        if not args.no_cpu_baseline and world == 1 and not args.orbits and not args.lifo:
            from oracle import oracle as O
            O.build()
            cores = getattr(args, "cpu_threads", 0) or os.cpu_count() or 1
            units, dt = run_oracle_sample(cores)
            cpu = {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{cpu_sample_text()} ({units} genotypes, {dt:.1f} s)"}
        configs = None
        if world == 1 and not args.no_configs and WORKLOAD == "s28_full" and not (args.count or args.orbits
                                                                                  or args.lifo):
            configs = measure_configs(torch, J, dev, steps=5, warmup=3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}{' (orbit mode)' if args.orbits else ''}"
                                   f"{' (movelist process)' if args.lifo else ''}: "
                                   f"{'sampled' if sampled else 'all'} {count} genotypes of "
                                   f"S_{{{n},{c}}}, n={n} c={c} L={L} k={k} seed={seed0}",
                       "global_batch": world * count, "parallelism": f"replicas x{world}",
                       "l2": "256 MB buffer written between timed steps; outputs 134 MB > L2",
                       "distinct_phenotypes": nk,
                       "shape_collisions": collisions,
                       "sustained": {"steps": soak_steps, "seconds": round(soak_ms / 1e3, 3),
                                     "ms_per_step": round(soak_ms / soak_steps, 4),
                                     "value": world * count / (soak_ms / soak_steps / 1e3),
                                     "note": "back-to-back steps just before the timed ones, no L2 flush; "
                                             "the clock record covers them and the timed steps"}},
            "configs": configs,
            "e2e": None if not e2e_times else {"value": world * count / e2e_s, "unit": UNIT,
                                               "h2d_bytes_per_step": 0,
                                               "d2h_bytes_per_step": count * 8 + nk * 32 + 8},
            "gpu_launches": 5 * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
