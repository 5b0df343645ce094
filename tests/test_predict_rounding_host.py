"""The GPU evaluates Eq. (8)'s rounding without a branch: t is clamped to
[0, 255], v = round_down(t + 1/2) and floor(v) = round_down(v + 2^23) - 2^23
(a float32 add with directed rounding).  Restated here with exact float64
sums rounded down to float32, it must give the oracle's rule (0 for t <= 0,
255 for t >= 255, else half away from zero) at every half-integer and its
neighbouring float32 values, and on random values."""
import numpy as np


def _round_down_f32(x: np.ndarray) -> np.ndarray:
    # x: float64 values that are exact sums of two float32 values
    f = x.astype(np.float32)
    return np.where(f.astype(np.float64) > x, np.nextafter(f, np.float32(-np.inf)), f)


def _gpu_round(t: np.ndarray) -> np.ndarray:
    t = np.minimum(np.maximum(t, np.float32(0)), np.float32(255))
    v = _round_down_f32(t.astype(np.float64) + 0.5)
    w = _round_down_f32(v.astype(np.float64) + 8388608.0)
    return w.astype(np.float64).astype(np.int64) - 8388608


def _oracle_round(t: np.ndarray) -> np.ndarray:
    t = t.astype(np.float64)
    fl = np.floor(t)
    r = fl + (t - fl >= 0.5)
    return np.where(t <= 0, 0, np.where(t >= 255, 255, r)).astype(np.int64)


def test_branch_free_rounding_equals_half_away_from_zero():
    halves = np.arange(-2, 258, dtype=np.float32) + np.float32(0.5)
    near = [halves]
    for k in range(1, 5):
        near.append(np.nextafter(near[-1], np.float32(np.inf)))
    down = [halves]
    for k in range(1, 5):
        down.append(np.nextafter(down[-1], np.float32(-np.inf)))
    rng = np.random.default_rng(8)
    t = np.concatenate(near + down + [np.arange(-3, 259, dtype=np.float32),
                                      rng.uniform(-20, 300, 500_000).astype(np.float32),
                                      np.array([0.0, -0.0, 1e-45, 254.99998, 255.0, 3e38, -3e38], np.float32)])
    assert np.array_equal(_gpu_round(t), _oracle_round(t))
