"""The GPU rANS encoder divides the 32-bit state by the symbol frequency f
(1 <= f <= 2^14) with a multiply: m = ceil(2^46 / f) in two 32-bit halves
(mh, ml), and floor(x / f) = floor((x mh + floor(x ml / 2^32)) / 2^14)
(division by invariant integers, Granlund and Montgomery 1994).  This
checks that identity on the host for every f, at the states where it is
tightest (just below and at each multiple of f near 2^32, and the smallest
states), and on random states."""
import numpy as np

M_BITS = 14


def _magic_quotient(x: np.ndarray, f: np.ndarray) -> np.ndarray:
    m = ((np.uint64(1) << np.uint64(46)) + f - np.uint64(1)) // f
    ml, mh = m & np.uint64(0xFFFFFFFF), m >> np.uint64(32)
    t = x * mh + ((x * ml) >> np.uint64(32))          # x mh < 2^46 and x ml < 2^64: exact in uint64
    return t >> np.uint64(M_BITS)


def test_every_frequency_at_its_tightest_states():
    f = np.arange(1, (1 << M_BITS) + 1, dtype=np.uint64)
    top = np.uint64((1 << 32) - 1)
    last = top - top % f                                # the largest multiple of f below 2^32
    cands = [top, last, last - np.uint64(1), last - f, last - f + np.uint64(1), f - np.uint64(1), f,
             np.full_like(f, 1 << 16), np.full_like(f, (1 << 16) - 1)]
    for x in cands:
        x = np.minimum(x, top)
        assert np.array_equal(_magic_quotient(x, f), x // f)


def test_random_states():
    rng = np.random.default_rng(46)
    for _ in range(20):
        f = rng.integers(1, (1 << M_BITS) + 1, size=200_000).astype(np.uint64)
        x = rng.integers(0, 1 << 32, size=200_000).astype(np.uint64)
        assert np.array_equal(_magic_quotient(x, f), x // f)
