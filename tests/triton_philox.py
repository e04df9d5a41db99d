"""Philox4x32-10 from Triton's own implementation, run by its CPU interpreter:
a library routine written independently of the oracle, used by the pins of
everything the oracle draws."""
import os

import numpy as np
import pytest


def triton_philox(ctrs, key):
    """Philox4x32-10 words from Triton's own implementation (run by its CPU
    interpreter), a library routine written independently of the oracle."""
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    tl = pytest.importorskip("triton.language")
    torch = pytest.importorskip("torch")

    @triton.jit
    def kern(out_ptr, c_ptr, seed, NB: tl.constexpr):
        i = tl.arange(0, NB)
        c0 = tl.load(c_ptr + 4 * i + 0)
        c1 = tl.load(c_ptr + 4 * i + 1)
        c2 = tl.load(c_ptr + 4 * i + 2)
        c3 = tl.load(c_ptr + 4 * i + 3)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
        tl.store(out_ptr + 4 * i + 0, a)
        tl.store(out_ptr + 4 * i + 1, b)
        tl.store(out_ptr + 4 * i + 2, c)
        tl.store(out_ptr + 4 * i + 3, d)

    nb = len(ctrs)
    npad = 1 << max(0, (nb - 1).bit_length())  # tl.arange needs a power of two
    arr = np.zeros((npad, 4), np.uint32)
    arr[:nb] = np.array(ctrs, dtype=np.uint64).astype(np.uint32).reshape(nb, 4)
    cbuf = torch.tensor(arr.reshape(-1).view(np.int32))
    out = torch.zeros(4 * npad, dtype=torch.int32)
    seed = (int(key[1]) << 32) | int(key[0])
    kern[(1,)](out, cbuf, seed, NB=npad)
    return out.numpy().view(np.uint32).reshape(npad, 4)[:nb].tolist()
