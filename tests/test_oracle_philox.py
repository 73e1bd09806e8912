"""Pins of the oracle's Philox4x64-10 against numpy's independent implementation.

numpy.random.Philox is Philox4x64-10 (Salmon et al., SC'11); its
``random_raw`` increments the 256-bit counter and then encrypts it, so a
generator started at counter c-1 yields the block of counter c first.
"""
import numpy as np
import pytest


def _numpy_block(ctr, key):
    c = 0
    for i, w in enumerate(ctr):
        c |= int(w) << (64 * i)
    k = int(key[0]) | (int(key[1]) << 64)
    bg = np.random.Philox(counter=(c - 1) % (1 << 256), key=k)
    return bg.random_raw(4).astype(np.uint64)


def test_philox_matches_numpy_random_counters(orc):
    rng = np.random.default_rng(7)
    for _ in range(200):
        ctr = rng.integers(0, 2**64, size=4, dtype=np.uint64)
        key = rng.integers(0, 2**64, size=2, dtype=np.uint64)
        np.testing.assert_array_equal(orc.philox4x64(ctr, key), _numpy_block(ctr, key))


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([2**64 - 1] * 4, [2**64 - 1] * 2),
    ([5, 0, 2, 0], [20260301, 1]),
])
def test_philox_matches_numpy_special_counters(orc, ctr, key):
    np.testing.assert_array_equal(orc.philox4x64(ctr, key), _numpy_block(ctr, key))


def test_stream_layout(orc):
    """Step t of particle i uses 32-bit word (t-1)&7 of block (t-1)>>3 of the
    STEP purpose; the component draw uses word 0 of block 0 of SELECT."""
    seed, human, i = 123456789, 7, 42
    for t in (1, 2, 8, 9, 17, 150):
        q = t - 1
        out = orc.philox4x64([i, q >> 3, orc.PURPOSE_STEP, 0], [seed, human])
        word = (int(out[(q & 7) >> 1]) >> (32 * (q & 1))) & 0xFFFFFFFF
        assert orc.uniform_step(seed, human, i, t) == (word >> 8) / 2.0**24
    out = orc.philox4x64([i, 0, orc.PURPOSE_SELECT, 0], [seed, human])
    assert orc.uniform_select(seed, human, i) == ((int(out[0]) & 0xFFFFFFFF) >> 8) / 2.0**24


def test_uniform_statistics(orc):
    """Mean, chi-square over 64 bins and lag-1 correlation of 2^16 step uniforms."""
    u = np.array([orc.uniform_step(99, 3, i, t) for i in range(2048) for t in range(1, 33)])
    assert u.min() >= 0.0 and u.max() < 1.0
    n = u.size
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    hist = np.bincount((u * 64).astype(int), minlength=64)
    chi2 = ((hist - n / 64) ** 2 / (n / 64)).sum()
    assert chi2 < 120  # 63 dof: p < 1e-5 above ~120
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 5 / np.sqrt(n)
