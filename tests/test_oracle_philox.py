"""Pins of the oracle's Philox4x32-10 against an independent implementation.

Triton ships its own Philox4x32-10 (``tl.philox_impl``, written from the same
SC'11 definition, with its own code).  Its CPU interpreter runs it here with
no GPU, so the oracle's block function is compared word for word with it on
counters and keys that exercise every word, carries in the key schedule and
the all-ones corner.  A transposed multiplier, a dropped key bump or swapped
output words would all fail.
"""
import os
import numpy as np
import pytest

import oracle


def _triton_philox(ctrs, keys):
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    tl = pytest.importorskip("triton.language")
    torch = pytest.importorskip("torch")

    @triton.jit
    def kern(out, cp, kp, n: tl.constexpr):
        i = tl.arange(0, n)
        c0 = tl.load(cp + 4 * i).to(tl.uint32)
        c1 = tl.load(cp + 4 * i + 1).to(tl.uint32)
        c2 = tl.load(cp + 4 * i + 2).to(tl.uint32)
        c3 = tl.load(cp + 4 * i + 3).to(tl.uint32)
        k0 = tl.load(kp + 2 * i).to(tl.uint32)
        k1 = tl.load(kp + 2 * i + 1).to(tl.uint32)
        a, b, c, d = tl.philox_impl(c0, c1, c2, c3, k0, k1, 10)
        tl.store(out + 4 * i, a.to(tl.int64))
        tl.store(out + 4 * i + 1, b.to(tl.int64))
        tl.store(out + 4 * i + 2, c.to(tl.int64))
        tl.store(out + 4 * i + 3, d.to(tl.int64))

    n = len(ctrs)
    ct = torch.tensor(np.asarray(ctrs, dtype=np.int64))
    kt = torch.tensor(np.asarray(keys, dtype=np.int64))
    out = torch.zeros((n, 4), dtype=torch.int64)
    kern[(1,)](out, ct, kt, n)
    return (out.numpy() & 0xFFFFFFFF).astype(np.uint64)


def test_philox_matches_independent_triton_implementation():
    rng = np.random.default_rng(12345)
    n = 64
    ctrs = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64)
    keys = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64)
    # corners: all zero, all ones, single bits in every word
    ctrs[0] = 0
    keys[0] = 0
    ctrs[1] = 0xFFFFFFFF
    keys[1] = 0xFFFFFFFF
    for w in range(4):
        ctrs[2 + w] = 0
        ctrs[2 + w, w] = 1
        keys[2 + w] = 0
    keys[6] = (1, 0)
    keys[7] = (0, 1)
    ref = _triton_philox(ctrs.astype(np.int64), keys.astype(np.int64))
    ours = np.array([oracle.philox4x32_10(c, k) for c, k in zip(ctrs, keys)], dtype=np.uint64)
    assert np.array_equal(ours, ref)


def test_philox_words_uniform_and_independent():
    """Chi-square of the top byte of each word over 2^14 counters, and no
    correlation between words of one block (a broken round mixes poorly)."""
    n = 1 << 14
    words = np.array([oracle.philox4x32_10((i, 7, 0, 3), (99, 0)) for i in range(n)], dtype=np.uint64)
    from scipy.stats import chi2
    for w in range(4):
        top = (words[:, w] >> np.uint64(24)).astype(np.int64)
        counts = np.bincount(top, minlength=256)
        stat = ((counts - n / 256) ** 2 / (n / 256)).sum()
        assert chi2.sf(stat, 255) > 1e-4
    u = words.astype(np.float64) / 2 ** 32
    c = np.corrcoef(u.T)
    assert np.all(np.abs(c[np.triu_indices(4, 1)]) < 5.0 / np.sqrt(n))
