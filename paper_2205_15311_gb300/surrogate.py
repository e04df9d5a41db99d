"""Training the surrogate network on labels the classification produced.

Host orchestration only: the labels come from jatam_enumerate / ga_evaluate,
the genomes are embedded into the 36-bit S_{3,8} encoding and mapped to the 8
classes by the library's kernels, and every training step is
jatam_mlp_train_step.  torch supplies device buffers.

Training set (all classified by the library itself):
  * S_{2,4} in full (4^8 genotypes, L = 16, k = 10, seed 1), embedded;
  * a uniform sample of S_{2,8} (L = 16, k = 20, seed 2), embedded;
  * a uniform sample of S_{3,8} at the genetic algorithm's settings (L = 16,
    k = 20, its classification seed).
"""
from __future__ import annotations

import numpy as np

from . import binding as J
from . import workloads as W


def _classify_genomes(torch, genomes_dev, n, c, L, k, seed):
    N = int(genomes_dev.shape[0])
    out = torch.empty(N * 8, dtype=torch.uint8, device=genomes_dev.device)
    fit = torch.empty(N, dtype=torch.int32, device=genomes_dev.device)
    J.evaluate_genomes(genomes_dev, fit, n=n, c=c, L=L, k=k, seed=seed, out=out, sync=True)
    return out


def build_training_set(torch, device, *, s28_sample=1 << 21, s38_sample=1 << 21, L=16, k=20, seed38=7):
    """Genomes (36-bit, int64 view) and labels (uint8) on the device."""
    parts_g, parts_y = [], []

    def add(genomes_np, n, c, Lc, kc, sd):
        g = torch.from_numpy(np.ascontiguousarray(genomes_np, np.uint64).view(np.int64)).to(device)
        res = _classify_genomes(torch, g, n, c, Lc, kc, sd)
        y = torch.empty(g.shape[0], dtype=torch.uint8, device=device)
        J.labels_of(res, y)
        if n == 3 and c == 8:
            e = g
        else:
            e = torch.empty_like(g)
            J.embed(g, n, c, e)
        parts_g.append(e)
        parts_y.append(y)

    add(np.arange(1 << 16, dtype=np.uint64), 2, 4, 16, 10, 1)
    add(W.random_genomes(s28_sample, 2, 8, seed=12), 2, 8, 16, 20, 2)
    if s38_sample:
        add(W.random_genomes(s38_sample, 3, 8, seed=13), 3, 8, L, k, seed38)
    genomes = torch.cat(parts_g)
    labels = torch.cat(parts_y)
    torch.cuda.synchronize()
    return genomes, labels


def train(torch, net, genomes, labels, *, steps=3000, batch=4096, lr=2e-3, seed=0):
    """Adam on shuffled minibatches; returns the loss of each step."""
    n = int(genomes.shape[0])
    perm = torch.from_numpy(np.random.default_rng(seed).permutation(n)).to(genomes.device)
    g = genomes[perm].contiguous()
    y = labels[perm].contiguous()
    losses = []
    for s in range(steps):
        lo = (s * batch) % max(n - batch, 1)
        losses.append(net.train_step(g[lo: lo + batch], y[lo: lo + batch], lr=lr))
    return losses


def initial_params(seed=0):
    """He-scaled normal initialisation as a flat float32 vector."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.standard_normal((48, 256)) * np.sqrt(2.0 / 36), "b1": np.zeros(256),
         "W2": rng.standard_normal((256, 256)) * np.sqrt(2.0 / 256), "b2": np.zeros(256),
         "W3": rng.standard_normal((256, 8)) * np.sqrt(1.0 / 256), "b3": np.zeros(8)}
    return J.flatten_params(p)


def accuracy(torch, net, genomes, labels, batch=1 << 16):
    """Fraction of genomes whose most probable class is their class."""
    hit = 0
    n = int(genomes.shape[0])
    logits = torch.empty((batch, 8), dtype=torch.float32, device=genomes.device)
    for lo in range(0, n, batch):
        m = min(batch, n - lo)
        net.predict(genomes[lo: lo + m], logits[:m])
        hit += int((logits[:m].argmax(dim=1).to(torch.uint8) == labels[lo: lo + m]).sum().item())
    return hit / n
