"""Pins of the surrogate network's CPU oracle: its backward pass against
central finite differences (float64), its bfloat16 rounding against PyTorch's
conversion, closed-form losses, and the class buckets.  No GPU needed."""
import numpy as np
import pytest

from oracle import mlp as M


def _small_problem(seed=0, B=7):
    rng = np.random.default_rng(seed)
    params = M.init_params(seed)
    for k in params:
        params[k] = params[k] + 0.01 * rng.standard_normal(params[k].shape)
    g = rng.integers(0, 1 << 36, size=B, dtype=np.int64).astype(np.uint64)
    return params, M.genome_bits(g), rng.integers(0, 8, size=B)


def test_backward_matches_finite_differences():
    params, x, y = _small_problem()
    loss, grads, _ = M.forward_backward(params, x, y, bf16=False)
    rng = np.random.default_rng(1)
    eps = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = params[name].reshape(-1)
        for idx in rng.choice(flat.size, size=6, replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _, _ = M.forward_backward(params, x, y, bf16=False)
            flat[idx] = old - eps
            lm, _, _ = M.forward_backward(params, x, y, bf16=False)
            flat[idx] = old
            num = (lp - lm) / (2 * eps)
            ana = grads[name].reshape(-1)[idx]
            assert abs(num - ana) <= 1e-6 + 1e-4 * abs(num), (name, idx, num, ana)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.standard_normal(5000) * 10 ** rng.uniform(-6, 6, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 65504.0, 3.0e38]])
    want = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(v), want)


def test_zero_network_has_log8_loss_and_uniform_gradient():
    params = {k: np.zeros_like(v) for k, v in M.init_params(0).items()}
    x = M.genome_bits(np.arange(5, dtype=np.uint64))
    y = np.array([0, 1, 2, 7, 7])
    loss, grads, logits = M.forward_backward(params, x, y, bf16=False)
    assert abs(loss - np.log(8.0)) < 1e-12
    # with all logits 0, dL/db3 = mean over the batch of (1/8 - onehot)
    want = np.full(8, 1 / 8) - np.bincount(y, minlength=8) / 5
    assert np.allclose(grads["b3"], want)


def test_genome_bits_are_msb_first():
    x = M.genome_bits(np.array([1 << 35, 1, 0b101], dtype=np.uint64))
    assert x[0, 0] == 1 and x[0, 1:].sum() == 0
    assert x[1, 35] == 1 and x[1, :35].sum() == 0
    assert x[2, 33] == 1 and x[2, 35] == 1 and x[:, 36:].sum() == 0


def test_class_buckets():
    res = np.zeros(9, dtype=[("cls", "u1"), ("decided_rep", "u1"), ("size", "<u2"), ("shape_hash", "<u4")])
    res["cls"] = [3, 1, 2, 0, 0, 0, 0, 0, 0]
    res["size"] = [0, 0, 9, 1, 3, 4, 15, 16, 200]
    assert M.class_of(res).tolist() == [0, 1, 2, 3, 4, 5, 6, 7, 7]


def test_adam_step_matches_torch_optim_adam():
    """The oracle's Adam (Kingma & Ba 2015, bias-corrected moments, eps outside
    the square root) equals torch.optim.Adam in float64 over several steps."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    params = {k: v + 0.01 * rng.standard_normal(v.shape) for k, v in M.init_params(8).items()}
    tp = {k: torch.tensor(v.copy(), dtype=torch.float64, requires_grad=True) for k, v in params.items()}
    opt = torch.optim.Adam(list(tp.values()), lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    state = {}
    for step in range(5):
        grads = {k: rng.standard_normal(v.shape) * 10.0 ** rng.uniform(-9, 1, v.shape) for k, v in params.items()}
        grads["b3"][0] = 0.0  # a zero gradient leaves the parameter in place on the first step
        for k in tp:
            tp[k].grad = torch.tensor(grads[k], dtype=torch.float64)
        opt.step()
        M.adam_step(params, grads, state, lr=3e-3)
        for k in params:
            assert np.allclose(params[k], tp[k].detach().numpy(), rtol=1e-12, atol=1e-15), (step, k)
