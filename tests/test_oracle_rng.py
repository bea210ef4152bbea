"""Pin the oracle's Philox4x32-10 against an independent implementation.

Triton's language library ships a Philox4x32-10 (its random-number routines);
run through Triton's CPU interpreter it gives a third-party reference for the
same counter/key definition (Salmon et al. 2011).
"""
import os

import numpy as np
import pytest

import oracle as O


def triton_philox(ctrs, seed):
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    import torch
    import triton.language as tl

    @triton.jit
    def k(out_ptr, c_ptr, seed, N: tl.constexpr):
        offs = tl.arange(0, N)
        c0 = tl.load(c_ptr + offs * 4 + 0)
        c1 = tl.load(c_ptr + offs * 4 + 1)
        c2 = tl.load(c_ptr + offs * 4 + 2)
        c3 = tl.load(c_ptr + offs * 4 + 3)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + offs * 4 + 0, a)
        tl.store(out_ptr + offs * 4 + 1, b)
        tl.store(out_ptr + offs * 4 + 2, c)
        tl.store(out_ptr + offs * 4 + 3, d)

    n = len(ctrs)
    c = torch.from_numpy(np.asarray(ctrs, np.uint32).view(np.int32).copy())
    out = torch.zeros(n * 4, dtype=torch.int32)
    k[(1,)](out, c, seed, N=n)
    return out.numpy().view(np.uint32).reshape(n, 4)


def test_philox_matches_triton():
    rng = np.random.default_rng(7)
    ctrs = rng.integers(0, 2 ** 32, size=(16, 4), dtype=np.uint64).astype(np.uint32)
    ctrs[0] = 0
    ctrs[1] = 0xFFFFFFFF
    for seed in (0, 1, 0x123456789ABCDEF, 2 ** 64 - 1):
        ref = triton_philox(ctrs, seed if seed < 2 ** 63 else seed - 2 ** 64)
        key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
        got = np.stack([O.philox(c, key) for c in ctrs])
        assert np.array_equal(got, ref), seed


def test_philox_avalanche():
    # flipping one counter bit changes about half of the 128 output bits
    base = O.philox((1, 2, 3, 4), (5, 6))
    flips = []
    for w in range(4):
        for b in range(32):
            c = [1, 2, 3, 4]
            c[w] ^= 1 << b
            diff = np.bitwise_xor(O.philox(c, (5, 6)), base)
            flips.append(sum(bin(int(x)).count("1") for x in diff))
    assert 56 < np.mean(flips) < 72
