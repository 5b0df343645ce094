"""The GPU builds each rANS frequency table in closed form, not by the
oracle's one-unit-at-a-time excess removal: every entry above a level T is
cut to T, where T is the smallest level whose cut removes at most the
excess D, and the remaining r = D - (units cut) units come one each from the
first r entries at T in symbol order.  This restates that construction in
numpy and checks it against the oracle's rule on many adversarial
histograms (ties, long tails of rare symbols, shortfalls and excesses); the
GPU kernel itself is compared with the oracle in tests/test_gpu_rans.py and
tests/test_gpu_dwt.py."""
import numpy as np

from oracle import oracle as O

M = 1 << 14


def closed_form(counts: np.ndarray) -> np.ndarray:
    c = counts.astype(np.int64)
    N = int(c.sum())
    f = np.zeros(511, np.int64)
    if N == 0:
        return f
    f[c > 0] = np.maximum(1, (c[c > 0] << 14) // N)
    diff = M - int(f.sum())
    if diff > 0:
        f[int(np.argmax(c))] += diff           # the first maximum: the smallest symbol on ties
    elif diff < 0:
        D = -diff
        cut = lambda T: int(np.maximum(f - T, 0).sum())
        lo, hi = max(1, int(f.max()) - D), int(f.max())
        while lo < hi:
            mid = (lo + hi) // 2
            if cut(mid) <= D:
                hi = mid
            else:
                lo = mid + 1
        T = lo
        r = D - cut(T)
        at = np.nonzero(f >= T)[0]
        f = np.minimum(f, T)
        f[at[:r]] = T - 1
    return f


def _histograms(rng, n):
    for _ in range(n):
        kind = rng.integers(0, 4)
        c = np.zeros(511, np.uint32)
        k = int(rng.integers(1, 512))
        idx = rng.choice(511, size=k, replace=False)
        if kind == 0:                              # a few heavy symbols, a long tail of ones
            c[idx] = 1
            heavy = idx[: int(rng.integers(1, 4))]
            c[heavy] = rng.integers(10 ** 5, 10 ** 7)
        elif kind == 1:                            # ties among the heaviest
            c[idx] = rng.integers(1, 50, size=k)
            c[idx[: int(rng.integers(2, 6))]] = int(rng.integers(1000, 10 ** 6))
        elif kind == 2:                            # Laplace-like
            v = np.clip(np.round(rng.laplace(0, rng.uniform(0.3, 40), size=int(rng.integers(1, 10 ** 6)))), -255, 255)
            c = np.bincount((v + 255).astype(np.int64), minlength=511).astype(np.uint32)
        else:                                      # uniform counts
            c[idx] = rng.integers(1, int(rng.integers(2, 10 ** 6)), size=k)
        yield c


def test_closed_form_equals_the_oracle_rule():
    rng = np.random.default_rng(2309)
    excess = shortfall = 0
    for c in _histograms(rng, 1500):
        want = O.rans_table(c).astype(np.int64)
        got = closed_form(c)
        assert np.array_equal(got, want)
        N = int(c.sum())
        base = np.where(c > 0, np.maximum(1, (c.astype(np.int64) << 14) // max(N, 1)), 0).sum()
        excess += base > M
        shortfall += base < M
    assert excess > 200 and shortfall > 200          # both corrections exercised
