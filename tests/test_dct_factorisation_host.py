"""The base kernel evaluates the 8x8 integer DCT with an even/odd
factorisation of each 8-point pass (the constants C1..C7 of csrc/base.cu),
the rounding term of each shift folded into the sums, and the +128 of the
decoded samples folded into the last one.  Restated here in int64 numpy,
it must give the oracle's plain matrix products with rounded shifts on
every block, including the extreme ones, and every intermediate must fit
the kernel's int32."""
import os
import re

import numpy as np

from oracle import oracle as O


def _c_block(fn, *arrays):
    args = [np.ascontiguousarray(a, dtype=np.int32).reshape(64) for a in arrays]
    out = np.empty(64, dtype=np.int32)
    getattr(O.lib(), fn)(*[O._p(a) for a in args], O._p(out))
    return out.reshape(8, 8).astype(np.int64)

BASE_CU = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2309_11072_gb300", "csrc",
                       "base.cu")


def _constants():
    text = open(BASE_CU).read()
    c = {k: int(v) for k, v in re.findall(r"\b(C[1-7])\s*=\s*(\d+)", text)}
    assert sorted(c) == ["C1", "C2", "C3", "C4", "C5", "C6", "C7"]
    return c


def _fdct8(x, r, C):
    # x: int64 [..., 8] along the transformed axis
    s07, d07 = x[..., 0] + x[..., 7], x[..., 0] - x[..., 7]
    s16, d16 = x[..., 1] + x[..., 6], x[..., 1] - x[..., 6]
    s25, d25 = x[..., 2] + x[..., 5], x[..., 2] - x[..., 5]
    s34, d34 = x[..., 3] + x[..., 4], x[..., 3] - x[..., 4]
    e0, e1, e2, e3 = s07 + s34, s16 + s25, s07 - s34, s16 - s25
    C1, C2, C3, C4, C5, C6, C7 = (C[f"C{i}"] for i in range(1, 8))
    F = [C4 * (e0 + e1) + r,
         C1 * d07 + r + C3 * d16 + C5 * d25 + C7 * d34,
         C2 * e2 + r + C6 * e3,
         C3 * d07 + r - C7 * d16 - C1 * d25 - C5 * d34,
         C4 * (e0 - e1) + r,
         C5 * d07 + r - C1 * d16 + C7 * d25 + C3 * d34,
         C6 * e2 + r - C2 * e3,
         C7 * d07 + r - C5 * d16 + C3 * d25 - C1 * d34]
    return np.stack(F, axis=-1)


def _idct8(F, r, C):
    C1, C2, C3, C4, C5, C6, C7 = (C[f"C{i}"] for i in range(1, 8))
    f = [F[..., i] for i in range(8)]
    a, b = C4 * (f[0] + f[4]) + r, C4 * (f[0] - f[4]) + r
    c, d = C2 * f[2] + C6 * f[6], C6 * f[2] - C2 * f[6]
    E0, E3, E1, E2 = a + c, a - c, b + d, b - d
    O0 = C1 * f[1] + C3 * f[3] + C5 * f[5] + C7 * f[7]
    O1 = C3 * f[1] - C7 * f[3] - C1 * f[5] - C5 * f[7]
    O2 = C5 * f[1] - C1 * f[3] + C7 * f[5] + C3 * f[7]
    O3 = C7 * f[1] - C5 * f[3] + C3 * f[5] - C1 * f[7]
    return np.stack([E0 + O0, E1 + O1, E2 + O2, E3 + O3, E3 - O3, E2 - O2, E1 - O1, E0 - O0], axis=-1)


def _blocks():
    rng = np.random.default_rng(88)
    yy, xx = np.mgrid[0:8, 0:8]
    out = [np.full((8, 8), -128), np.full((8, 8), 127), np.where((yy + xx) % 2 == 0, 127, -128),
           np.where(xx < 4, 127, -128), np.where(yy % 2 == 0, -128, 127)]
    out += list(rng.choice([-128, 127], size=(300, 8, 8)))
    out += list(rng.integers(-128, 128, size=(700, 8, 8)))
    return np.array(out, np.int64)


def test_factorised_forward_and_inverse_equal_the_matrix_products():
    C = _constants()
    X = _blocks()
    big = []
    # forward: rows (x), shift 9; then columns (y), shift 15
    A = _fdct8(X, 1 << 8, C)                       # [b, y, u]
    big.append(np.abs(A).max())
    T = A >> 9
    B = _fdct8(np.swapaxes(T, 1, 2), 1 << 14, C)   # [b, u, v]
    big.append(np.abs(B).max())
    F = np.swapaxes(B >> 15, 1, 2)                 # [b, v, u]
    for k in range(0, len(X), 7):
        assert np.array_equal(F[k], _c_block("oracle_fdct_block", X[k]))
    # inverse: columns (v -> y), shift 9; then rows (u -> x), shift 15, +128 folded
    Q = O.quant_table(50)
    Fq = np.array([_c_block("oracle_quant_dequant_block", F[k], Q) for k in range(len(F))], np.int64)
    for Fin in (F, Fq):
        G = _idct8(np.swapaxes(Fin, 1, 2), 1 << 8, C)      # [b, u, y]
        big.append(np.abs(G).max())
        G = np.swapaxes(G >> 9, 1, 2)                      # [b, y, u]
        Xr = _idct8(G, (1 << 14) + (128 << 15), C)         # [b, y, x]
        big.append(np.abs(Xr).max())
        S = np.clip(Xr >> 15, 0, 255)
        for k in range(0, len(X), 7):
            assert np.array_equal(S[k], np.clip(_c_block("oracle_idct_block", Fin[k]) + 128, 0, 255))
    assert max(big) < 2 ** 31                       # every sum fits the kernel's int32
