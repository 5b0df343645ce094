"""Pins of the oracle's enhancement-layer coder (static rANS over the
residual planes), against what information theory and the coder's
definition fix rather than against itself: lossless round trips at every
chunk / stream boundary, the code length of arithmetic coding (the words
written equal the ideal cost sum log2(M / f) of the symbols plus the
32-bit final state per stream, to within one 16-bit word per stream), the
exact cost in the degenerate cases (one symbol: zero bits; two equally
likely symbols: one bit each), and the table's defining properties."""
import math

import numpy as np
import pytest

from oracle import oracle as O

M = 1 << 14


def _hist(r3, n):
    return np.stack([np.bincount(r3[c * n:(c + 1) * n].astype(np.int64) + 255, minlength=511) for c in range(3)])


def _laplace(n, scale, seed):
    rng = np.random.default_rng(seed)
    return np.clip(np.round(rng.laplace(0, scale, size=3 * n)), -255, 255).astype(np.int16)


def _streams(n):
    """Non-empty streams of one plane of n symbols."""
    chunks = (n + 8191) // 8192
    return sum(1 for k in range(chunks) for l in range(32) if k * 8192 + l < n)


@pytest.mark.parametrize("n", [1, 31, 32, 33, 255, 8191, 8192, 8193, 20000])
def test_round_trip_is_lossless_at_every_boundary(n):
    r3 = _laplace(n, 7.0, seed=n)
    f3 = np.stack([O.rans_table(h) for h in _hist(r3, n)])
    w, cn = O.rans_encode(r3, f3)
    assert np.array_equal(O.rans_decode(w, cn, n, f3), r3)


@pytest.mark.parametrize("n,scale", [(20000, 3.0), (50000, 20.0), (9000, 100.0)])
def test_code_length_matches_the_ideal_cost(n, scale):
    r3 = _laplace(n, scale, seed=int(scale))
    f3 = np.stack([O.rans_table(h) for h in _hist(r3, n)])
    w, cn = O.rans_encode(r3, f3)
    cn = cn.reshape(3, -1)
    for c in range(3):
        ideal = sum(math.log2(M / f3[c][s + 255]) for s in r3[c * n:(c + 1) * n].tolist())
        streams = _streams(n)
        bits = 16 * int(cn[c].sum())
        # every stream ends with its 32-bit state; renormalisation wastes less
        # than one 16-bit word per stream
        assert ideal + 32 * streams - 16 * streams <= bits <= ideal + 32 * streams + 16 * streams


def test_single_symbol_costs_nothing():
    n = 10000
    r3 = np.full(3 * n, -4, np.int16)
    f3 = np.stack([O.rans_table(h) for h in _hist(r3, n)])
    assert (f3[:, 251] == M).all() and (f3.sum(1) == M).all()
    w, cn = O.rans_encode(r3, f3)
    assert (cn == 2).all()                       # only the final states
    # the state never leaves L = 2^16: every stream is the word pair (1, 0),
    # packed stream after stream from the start of its chunk's block
    blocks = w.reshape(-1, 32 * 258)
    assert (blocks[:, :64] == np.tile([1, 0], 32)).all() and (blocks[:, 64:] == 0).all()
    assert np.array_equal(O.rans_decode(w, cn, n, f3), r3)


def test_two_equally_likely_symbols_cost_one_bit_each():
    n = 8192
    # residuals -4 and 5, equally often in each plane: the table is exactly M / 2 each
    r3 = np.concatenate([np.tile([-4, 5], n // 2), np.tile([5, -4], n // 2),
                         np.repeat([-4, 5], n // 2)]).astype(np.int16)
    f3 = np.stack([O.rans_table(hh) for hh in _hist(r3, n)])
    assert (f3[:, 251] == M // 2).all() and (f3[:, 260] == M // 2).all()
    w, cn = O.rans_encode(r3, f3)
    # 256 symbols per stream at one bit each: 16 words, plus the 2-word state
    assert (cn == 18).all()
    assert np.array_equal(O.rans_decode(w, cn, n, f3), r3)


def test_table_properties():
    rng = np.random.default_rng(7)
    for trial in range(50):
        k = int(rng.integers(1, 511))
        counts = np.zeros(511, np.uint32)
        idx = rng.choice(511, size=k, replace=False)
        counts[idx] = rng.integers(1, 10 ** int(rng.integers(1, 7)), size=k)
        f = O.rans_table(counts)
        N = int(counts.sum())
        assert int(f.sum()) == M                          # total exactly M
        assert np.array_equal(f > 0, counts > 0)          # every occurring symbol codable, no other
        # each entry is within the correction of its exact share c M / N
        exact = counts.astype(np.float64) * M / N
        assert np.all(np.abs(f[counts > 0] - exact[counts > 0]) <= k + 1)
    assert not O.rans_table(np.zeros(511, np.uint32)).any()   # empty histogram: no table


def test_table_tie_rules_on_hand_worked_histograms():
    # shortfall: three symbols seen once each get floor(2^14 / 3) = 5461,
    # 16,383 in all; the missing unit goes to the most frequent symbol, the
    # smallest one on ties
    c = np.zeros(511, np.uint32)
    c[[10, 20, 30]] = 1
    f = O.rans_table(c)
    assert f[[10, 20, 30]].tolist() == [5462, 5461, 5461]
    # excess: two symbols seen 10^6 times and 299 seen once (N = 2,000,299)
    # get floor(10^6 2^14 / N) = 8190 twice and 1 each: 16,679, 295 too many;
    # units go one at a time from the largest entry, the smaller symbol on
    # ties, so symbol 5 gives 148 and symbol 6 gives 147
    c = np.zeros(511, np.uint32)
    c[5] = c[6] = 10 ** 6
    c[100:399] = 1
    f = O.rans_table(c)
    assert (f[5], f[6]) == (8190 - 148, 8190 - 147)
    assert (f[100:399] == 1).all() and int(f.sum()) == M


def test_zero_frequency_is_rejected():
    n = 100
    r3 = np.zeros(3 * n, np.int16)
    f3 = np.zeros((3, 511), np.uint32)
    f3[:, 256] = M                                     # the table does not cover residual 0
    with pytest.raises(ValueError):
        O.rans_encode(r3, f3)
