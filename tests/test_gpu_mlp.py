"""The surrogate network's tensor-core kernels against its CPU oracle.

Tolerance: the GPU and the oracle round the same tensors to bfloat16 (weights,
activations, output gradients) and differ in (a) float32 vs float64
accumulation, relative error below K * 2^-24 ~ 3e-5 for K <= 512, and (b)
bfloat16 rounding-boundary flips of an activation (one bfloat16 ulp, 2^-8
relative) when the float32 and float64 pre-activations straddle a rounding
boundary, which touch a handful of elements.  Per tensor the relative
Frobenius error is therefore a few 1e-3; the tests allow 1e-2 for gradients
and logits and 1e-4 for the loss."""
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


@pytest.mark.parametrize("B", [64, 512, 1000])
def test_gradients_match_oracle(B):
    params = M.init_params(3)
    rng = np.random.default_rng(B)
    for k in ("b1", "b2", "b3"):
        params[k] = 0.1 * rng.standard_normal(params[k].shape)
    genomes = W.random_genomes(B, 3, 8, seed=B)
    labels = rng.integers(0, 8, size=B).astype(np.uint8)
    net = J.Surrogate(max_batch=2048)
    flat = J.flatten_params(params)
    net.set_params(flat)
    grads = np.zeros(J.MLP_NPARAM, np.float32)
    loss = net.train_step(genomes, labels, lr=0.0, grads=grads)
    # the oracle sees exactly the float32 parameters the GPU holds
    p32 = J.unflatten_params(flat)
    want_loss, want, _ = M.forward_backward(p32, M.genome_bits(genomes), labels.astype(np.int64), bf16=True)
    assert abs(loss - want_loss) <= 1e-4 * max(1.0, abs(want_loss))
    got = J.unflatten_params(grads)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        if k == "W1":
            assert np.all(got[k][36:] == 0)  # zero input features give zero weight gradients
        assert _rel(got[k], want[k]) < 1e-2, k
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
    want = M.predict(J.unflatten_params(J.flatten_params(params)), M.genome_bits(genomes))
    assert _rel(logits, want) < 1e-2
    # a learnable target: class = the genome's top 3 bits
    labels = (genomes >> np.uint64(33)).astype(np.uint8)
    first = net.train_step(genomes[:1024], labels[:1024], lr=3e-3)
    for _ in range(300):
        last = net.train_step(genomes[:1024], labels[:1024], lr=3e-3)
    assert last < 0.3 * first
    after = J.unflatten_params(net.get_params())
    assert not np.allclose(after["W1"], params["W1"])
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
    want_loss, want, _ = M.forward_backward(J.unflatten_params(params), M.genome_bits(genomes),
                                            labels.astype(np.int64), bf16=True)
    got = J.unflatten_params(out["tc"][1])
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert _rel(got[k], want[k]) < 1e-2, k
