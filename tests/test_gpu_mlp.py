"""The surrogate network's tensor-core kernels against its CPU oracle, element
by element.

Tolerance.  The GPU and the oracle round the same tensors to bfloat16
(weights, activations, output gradients) and differ in two ways only:
  (a) float32 (GPU) vs float64 (oracle) accumulation.  A sum of K products
      computed in float32, in any order, and rounded once more when stored,
      differs from the exact sum by at most (K + 1) u sum_i |a_i b_i| to first
      order, u = 2^-24; split-K partial sums add one more rounding per split,
      so the tight bound is 2 (K + 2) 2^-24 S, with S = sum_i |a_i b_i| the
      magnitude sum of the element's own dot product (oracle/mlp.py,
      magnitude_sums);
  (b) bfloat16 rounding-boundary flips: where the float32 and float64 values
      of an activation or output gradient straddle a rounding boundary, the
      two sides store values one bfloat16 ulp apart (2^-8 relative).  A flip
      of one operand changes its term by at most 2^-8 of the term, a flip of
      both by about 2^-7, and the terms' magnitudes add up to S, so the flips
      move an element by at most 2^-7 S in all.
Every element must be within tight + 2^-7 S, and at most 2 % of the elements
of a gradient (5 % of the logits, which read 256 rounded activations each)
may exceed the tight bound -- the explicit cap on flip-affected elements.
Measured on a GB300: the largest |got - want| / S of any element was 7e-4
(2^-7 = 7.8e-3), and at most 0.9 % of a gradient's elements (0.3 % of the
logits) exceeded the tight bound.  A mis-indexed row or column, a transposed
operand or a dropped term moves elements by an amount of the order of S
itself and fails the loose bound."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as M  # noqa: E402
from paper_2205_15311_gb300 import binding as J  # noqa: E402
from paper_2205_15311_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def assert_elementwise(got, want, S, K, name, cap_frac=0.02):
    """|got - want| <= tight + 2^-7 S everywhere, and <= tight = 2 (K + 2)
    2^-24 S except on at most max(8, cap_frac of the elements)."""
    got = np.asarray(got, np.float64)
    d = np.abs(got - want)
    tiny = 1e-37  # float32 denormal floor
    tight = 2.0 * (K + 2) * 2.0 ** -24 * S + tiny
    loose = tight + 2.0 ** -7 * S
    worst = int(np.argmax(d - loose))
    assert np.all(d <= loose), (name, "loose", np.unravel_index(worst, d.shape), got.reshape(-1)[worst],
                                want.reshape(-1)[worst], S.reshape(-1)[worst])
    over = int(np.count_nonzero(d > tight))
    assert over <= max(8, int(cap_frac * d.size)), (name, "tight", over, d.size)
    return over


@pytest.mark.parametrize("B", [64, 512, 1000, 8192, 40000])
def test_gradients_match_oracle(B):
    params = M.init_params(3)
    rng = np.random.default_rng(B)
    for k in ("b1", "b2", "b3"):
        params[k] = 0.1 * rng.standard_normal(params[k].shape)
    genomes = W.random_genomes(B, 3, 8, seed=B)
    labels = rng.integers(0, 8, size=B).astype(np.uint8)
    net = J.Surrogate(max_batch=max(B, 2048))
    flat = J.flatten_params(params)
    net.set_params(flat)
    grads = np.zeros(J.MLP_NPARAM, np.float32)
    loss = net.train_step(genomes, labels, lr=0.0, grads=grads)
    # the oracle sees exactly the float32 parameters the GPU holds
    p32 = J.unflatten_params(flat)
    want_loss, want, _ = M.forward_backward(p32, M.genome_bits(genomes), labels.astype(np.int64), bf16=True)
    assert abs(loss - want_loss) <= 1e-4 * max(1.0, abs(want_loss))
    got = J.unflatten_params(grads)
    S = M.magnitude_sums(p32, M.genome_bits(genomes), labels.astype(np.int64))
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        if k == "W1":
            assert np.all(got[k][36:] == 0)  # zero input features give zero weight gradients
        assert_elementwise(got[k], want[k], S[k], B, k)
    # device buffers give the same numbers
    dg = torch.from_numpy(genomes.view(np.int64)).cuda()
    dl = torch.from_numpy(labels).cuda()
    dgr = torch.zeros(J.MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss2 = net.train_step(dg, dl, lr=0.0, grads=dgr)
    assert loss2 == loss and np.array_equal(dgr.cpu().numpy(), grads)
    net.close()


def test_predict_matches_oracle_and_training_lowers_the_loss():
    params = M.init_params(5)
    net = J.Surrogate(max_batch=4096)
    net.set_params(J.flatten_params(params))
    genomes = W.random_genomes(3000, 3, 8, seed=9)
    logits = np.zeros((3000, 8), np.float32)
    net.predict(genomes, logits)
    p32 = J.unflatten_params(J.flatten_params(params))
    want = M.predict(p32, M.genome_bits(genomes))
    S = M.magnitude_sums(p32, M.genome_bits(genomes), np.zeros(3000, np.int64))
    assert_elementwise(logits, want, S["logits"], 256, "logits", cap_frac=0.05)
    # a learnable target: class = the genome's top 3 bits
    labels = (genomes >> np.uint64(33)).astype(np.uint8)
    first = net.train_step(genomes[:1024], labels[:1024], lr=3e-3)
    for _ in range(300):
        last = net.train_step(genomes[:1024], labels[:1024], lr=3e-3)
    assert last < 0.3 * first
    after = J.unflatten_params(net.get_params())
    assert not np.allclose(after["W1"], params["W1"])
    net.close()


def test_predict_at_screening_size_matches_oracle():
    """A prediction over more rows than the tensor-core product has CTAs (65,613:
    several 128-row tiles a CTA, a ragged last tile), where the logits come out
    of the second layer's epilogue without the layer being stored."""
    params = M.init_params(7)
    rng = np.random.default_rng(7)
    for k in ("b1", "b2", "b3"):
        params[k] = 0.1 * rng.standard_normal(params[k].shape)
    n = 65613
    net = J.Surrogate(max_batch=n)
    net.set_params(J.flatten_params(params))
    genomes = W.random_genomes(n, 3, 8, seed=21)
    dg = torch.from_numpy(genomes.view(np.int64)).cuda()
    logits = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    net.predict(dg, logits)
    got = logits.cpu().numpy()
    p32 = J.unflatten_params(J.flatten_params(params))
    want = M.predict(p32, M.genome_bits(genomes))
    S = M.magnitude_sums(p32, M.genome_bits(genomes), np.zeros(n, np.int64))
    assert_elementwise(got, want, S["logits"], 256, "logits", cap_frac=0.05)
    net.close()


@pytest.mark.parametrize("B", [200, 1000, 4096])
def test_tensor_core_products_match_mma_sync(B, monkeypatch):
    """The tcgen05 products (the 256-column ones: both hidden layers and the
    first layer's activation gradient) against the mma.sync kernel on the same
    bfloat16 operands: only float32 summation order and bfloat16 rounding of
    the stored activations differ."""
    params = J.flatten_params(M.init_params(11))
    genomes = W.random_genomes(B, 3, 8, seed=B + 1)
    labels = np.random.default_rng(B).integers(0, 8, size=B).astype(np.uint8)
    out = {}
    for mode in ("mma", "tc"):
        monkeypatch.setenv("JATAM_MLP_PRODUCTS", mode)
        net = J.Surrogate(max_batch=4096)
        net.set_params(params)
        logits = np.zeros((B, 8), np.float32)
        net.predict(genomes, logits)
        grads = np.zeros(J.MLP_NPARAM, np.float32)
        loss = net.train_step(genomes, labels, lr=0.0, grads=grads)
        out[mode] = (logits, grads, loss)
        net.close()
    assert _rel(out["tc"][0], out["mma"][0]) < 1e-2
    assert _rel(out["tc"][1], out["mma"][1]) < 1e-2
    assert abs(out["tc"][2] - out["mma"][2]) <= 1e-3 * abs(out["mma"][2])
    # and against the oracle
    p32 = J.unflatten_params(params)
    want_loss, want, _ = M.forward_backward(p32, M.genome_bits(genomes), labels.astype(np.int64), bf16=True)
    S = M.magnitude_sums(p32, M.genome_bits(genomes), labels.astype(np.int64))
    got = J.unflatten_params(out["tc"][1])
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert_elementwise(got[k], want[k], S[k], B, k)


def test_adam_update_matches_oracle():
    """Four training steps: after each, the float32 parameters the GPU holds
    equal the oracle's Adam (float64) applied to the gradients the GPU
    reported for that step, within float32 rounding of the update (a few
    2^-24 of |p| plus a few 2^-24 of lr per step)."""
    params = M.init_params(21)
    rng = np.random.default_rng(21)
    net = J.Surrogate(max_batch=1024)
    flat = J.flatten_params(params)
    net.set_params(flat)
    ref = J.unflatten_params(flat)
    state = {}
    lr = 2e-3
    for t in range(1, 5):
        genomes = W.random_genomes(1000, 3, 8, seed=100 + t)
        labels = rng.integers(0, 8, size=1000).astype(np.uint8)
        grads = np.zeros(J.MLP_NPARAM, np.float32)
        net.train_step(genomes, labels, lr=lr, grads=grads)
        M.adam_step(ref, J.unflatten_params(grads), state, lr=lr)
        got = J.unflatten_params(net.get_params())
        for k in ref:
            d = np.abs(got[k] - ref[k])
            assert np.all(d <= 8 * 2.0 ** -24 * (np.abs(ref[k]) + 4 * t * lr)), (t, k, float(d.max()))
        # the parameters moved by about lr per step where the gradient is not zero
        assert np.abs(got["W2"] - J.unflatten_params(flat)["W2"]).max() > 0.5 * lr
    net.close()


def test_labels_match_oracle_class_buckets():
    """jatam_mlp_labels on the device equals the oracle's class buckets, on
    hand-made results at every bucket boundary and on classified genomes."""
    res = np.zeros(14, J.RESULT_DTYPE)
    res["cls"] = [3, 1, 2, 2, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0]
    res["size"] = [0, 0, 5, 40, 1, 2, 3, 4, 7, 8, 15, 16, 17, 1000]
    genomes = W.random_genomes(50000, 3, 8, seed=77)
    fit = torch.zeros(50000, dtype=torch.int32, device="cuda")
    out = torch.empty(50000 * 8, dtype=torch.uint8, device="cuda")
    J.evaluate_genomes(torch.from_numpy(genomes.view(np.int64)).cuda(), fit, n=3, c=8, L=16, k=20, seed=5,
                       out=out, sync=True)
    classified = J.results_view(out)
    assert len(set(classified["cls"].tolist())) == 4  # every class occurs
    for r in (res, classified):
        dr = torch.from_numpy(np.ascontiguousarray(r).view(np.uint8)).cuda()
        lab = torch.zeros(r.shape[0], dtype=torch.uint8, device="cuda")
        J.labels_of(dr, lab)
        torch.cuda.synchronize()
        assert lab.cpu().numpy().astype(np.int64).tolist() == M.class_of(r).tolist()
