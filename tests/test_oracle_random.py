"""Pins of the oracle's random stream: Philox4x32-10 and the bounded draw U(m).

The paper only fixes that random numbers depend on a frame/sample index and not
on a thread (Appendix D.2, indexed frames); the generator itself is Philox4x32-10
(Salmon et al., SC 2011) and the bounded draw is Lemire's multiply-and-reject.
"""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answer_vectors():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert list(O.philox4x32_10(ctr, key)) == out


def test_stream_layout_counter_and_word_order():
    # counter = (index lo, index hi, block, domain), key = (seed lo, seed hi);
    # each block gives two words, (out0 | out1<<32) then (out2 | out3<<32).
    seed, index, domain = 0x1234_5678_9abc_def0, (7 << 32) | 5, 1
    words = O.stream_words(seed, index, domain, 6)
    key = [seed & 0xffffffff, seed >> 32]
    for blk in range(3):
        o = [int(x) for x in O.philox4x32_10([index & 0xffffffff, index >> 32, blk, domain], key)]
        assert int(words[2 * blk]) == o[0] | (o[1] << 32)
        assert int(words[2 * blk + 1]) == o[2] | (o[3] << 32)


def test_uniform_power_of_two_is_top_bits():
    # For m = 2^k the multiply-and-reject draw never rejects and returns the top k bits.
    seed, idx = 99, 3
    for k in (1, 5, 17, 32, 63):
        ms = np.full(50, 1 << k, dtype=np.uint64)
        vals, used = O.stream_draws(seed, idx, 0, ms)
        words = O.stream_words(seed, idx, 0, 50)
        assert used == 50
        assert [int(v) for v in vals] == [int(w) >> (64 - k) for w in words]


def test_uniform_m1_consumes_one_word_each():
    vals, used = O.stream_draws(5, 0, 0, np.ones(40, dtype=np.uint64))
    assert used == 40 and not vals.any()


def test_uniform_small_ranges_exact_rule():
    # For every m <= 64: output = floor(x*m / 2^64) of the first accepted word,
    # where x is rejected iff (x*m mod 2^64) < (2^64 - m) mod m.
    for m in range(1, 65):
        ms = np.full(200, m, dtype=np.uint64)
        vals, used = O.stream_draws(11, m, 0, ms)
        words = [int(w) for w in O.stream_words(11, m, 0, used)]
        thresh = (2**64 - m) % m
        j = 0
        for v in vals:
            while (words[j] * m) % 2**64 < thresh:
                j += 1
            assert int(v) == (words[j] * m) >> 64
            assert 0 <= int(v) < m
            j += 1
        assert j == used


def test_uniform_rejects_and_stays_uniform_for_large_m():
    # m just above 2^63: about half of all words are rejected; outputs must still
    # be uniform over [0, m).  Chi-square over 8 equal-width bins.
    m = (1 << 63) + 12345
    n = 40000
    vals, used = O.stream_draws(3, 1, 0, np.full(n, m, dtype=np.uint64))
    assert 1.8 * n < used < 2.2 * n
    v = np.array([int(x) for x in vals], dtype=object)
    assert all(0 <= x < m for x in v)
    bins = np.bincount(np.array([(x * 8) // m for x in v], dtype=np.int64), minlength=8)
    exp = n / 8
    chi2 = float(((bins - exp) ** 2 / exp).sum())
    assert chi2 < 30.0  # 7 dof, p ~ 1e-4


@pytest.mark.parametrize("m", [3, 7, 1000, 4097])
def test_uniform_chi_square(m):
    n = 200 * m if m < 1000 else 100 * m
    n = min(n, 400000)
    vals, _ = O.stream_draws(17, m, 0, np.full(n, m, dtype=np.uint64))
    bins = np.bincount(vals.astype(np.int64), minlength=m)
    exp = n / m
    chi2 = float(((bins - exp) ** 2 / exp).sum())
    dof = m - 1
    # mean dof, sd sqrt(2 dof); 6 sd is far beyond any honest fluctuation
    assert chi2 < dof + 6 * np.sqrt(2 * dof)
