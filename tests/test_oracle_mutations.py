"""Strength of the oracle's pins: plausible mistakes are planted one at a
time in a scratch copy of the C oracle (never in the oracle itself), the
copy is compiled, and the pin tests of that part of the codec must fail
against it.  Each mistake is the kind a careful reading of the paper or a
standard could still make: a dropped or wrong term, a wrong sign, index or
shift, a wrong tie rule or offset, a transposed operand."""
import os
import subprocess
import sys
import tempfile

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text in slrme_oracle.c, replacement, occurrences replaced, pin test files)
MUTATIONS = [
    ("frexp exponent offset 129", "int E = ex + 128;", "int E = ex + 129;", 1, ["test_oracle_format.py"]),
    ("Eq. 3 without the half", "ldexp(M + 0.5, E - 128 - 8)", "ldexp(M + 0.0, E - 128 - 8)", 1,
     ["test_oracle_format.py"]),
    ("luma weight of R", "return 2126 * (2 * R + 1)", "return 2127 * (2 * R + 1)", 1, ["test_oracle_tmo.py"]),
    ("log-average offset 136", "65536 * (int64_t)(E - 137 + k)", "65536 * (int64_t)(E - 136 + k)", 1,
     ["test_oracle_tmo.py"]),
    ("key rounds below half", "stats[0] + 2048 * stats[1]", "stats[0] + 2047 * stats[1]", 1, ["test_oracle_tmo.py"]),
    ("operator denominator 2 + L", "float den = 1.0f + L;\n        float num = ldexpf(wr[r], d);\n        float H",
     "float den = 2.0f + L;\n        float num = ldexpf(wr[r], d);\n        float H", 1, ["test_oracle_tmo.py"]),
    ("white point from the smallest L", "if (L > best) best = L;", "if (best == 0.0f || L < best) best = L;", 1,
     ["test_oracle_tmo.py"]),
    ("white point factor dropped", "float f = 1.0f + q;", "float f = 1.0f + 0.0f * q;", 1, ["test_oracle_tmo.py"]),
    ("key split truncates toward zero", "int64_t Jj = floor_div(j, 16);", "int64_t Jj = j / 16;", 1,
     ["test_oracle_tmo.py"]),
    ("DCT DC basis scale", "double a = (u == 0) ? sqrt(1.0 / 8.0) : 0.5;", "double a = (u == 0) ? 0.5 : 0.5;", 1,
     ["test_oracle_base.py"]),
    ("right edge from column 0", "int xx = bx + x < w ? bx + x : w - 1;", "int xx = bx + x < w ? bx + x : 0;", 1,
     ["test_oracle_base.py"]),
    ("IJG scale rounding", "(k_luma_q50[i] * s + 50) / 100", "(k_luma_q50[i] * s + 49) / 100", 1,
     ["test_oracle_base.py"]),
    ("DCT shift truncates", "return (int32_t)((v + ((int64_t)1 << (s - 1))) >> s);", "return (int32_t)(v >> s);", 1,
     ["test_oracle_base.py"]),
    ("quantiser rounds half down", "int32_t lvl = (a + q / 2) / q;", "int32_t lvl = (a + (q - 1) / 2) / q;", 1,
     ["test_oracle_base.py"]),
    ("IDCT operand transposed", "acc += (int64_t)D[v * 8 + y] * F[v * 8 + u];",
     "acc += (int64_t)D[v * 8 + y] * F[u * 8 + v];", 1, ["test_oracle_base.py"]),
    ("filter weight index", "acc += wt[dy + 1] * wt[dx + 1] * S", "acc += wt[dx + 1] * wt[dx + 1] * S", 1,
     ["test_oracle_slrme.py"]),
    ("sum of x y takes x x", "s[3 + 4 * c] += x * y;", "s[3 + 4 * c] += x * x;", 1, ["test_oracle_slrme.py"]),
    ("D_xy sign", "__int128 dxy = (__int128)N * sxy - (__int128)sx * sy;",
     "__int128 dxy = (__int128)N * sxy + (__int128)sx * sy;", 1, ["test_oracle_slrme.py"]),
    ("intercept from the unquantised slope", "double t = (double)af * (double)sx;", "double t = ad * (double)sx;", 1,
     ["test_oracle_slrme.py"]),
    ("flat region intercept dropped", "*bc = (float)((double)sy / (double)N);", "*bc = 0.0f;", 1,
     ["test_oracle_slrme.py"]),
    ("unfiltered x scale 15", "= 16 * S[(int64_t)y * w + x]; continue;", "= 15 * S[(int64_t)y * w + x]; continue;", 1,
     ["test_oracle_slrme.py"]),
    ("int128 to double ties away from even", "(rem == half && (mant & 1))", "(rem == half)", 1,
     ["test_oracle_slrme.py"]),
    ("prediction ties round down", "if (t - tr >= 0.5f) r += 1;", "if (t - tr > 0.5f) r += 1;", 1,
     ["test_oracle_slrme.py"]),
    ("prediction fused multiply-add", "float t = a * (float)x;\n    t = t + b;", "float t = fmaf(a, (float)x, b);",
     1, ["test_oracle_slrme.py"]),
    ("residual sign", "int r = (int)m3[c * n_px + p] - (int)mstar3[c * n_px + p];",
     "int r = (int)mstar3[c * n_px + p] - (int)m3[c * n_px + p];", 1, ["test_oracle_slrme.py",
                                                                        "test_oracle_pipeline.py"]),
    ("rANS shortfall to the largest symbol on ties", "if (counts[s] > counts[best]) best = s;",
     "if (counts[s] >= counts[best]) best = s;", 1, ["test_oracle_rans.py"]),
    ("rANS excess from the largest symbol on ties", "if (freq[s] > 1 && (best < 0 || freq[s] > freq[best])) best = s;",
     "if (freq[s] > 1 && (best < 0 || freq[s] >= freq[best])) best = s;", 1, ["test_oracle_rans.py"]),
    ("rANS renormalises one bit early", "if ((x >> 18) >= fs) {", "if ((x >> 17) >= fs) {", 1,
     ["test_oracle_rans.py"]),
    ("rANS initial state L + 1", "uint32_t x = RANS_L;", "uint32_t x = RANS_L + 1;", 1, ["test_oracle_rans.py"]),
    ("wavelet right edge zero, both directions", ": x[(2 * i) * step];", ": 0;", 2, ["test_oracle_dwt.py"]),
    ("raw chunk from 255", "if (src[i] < -255 || src[i] > 255) raw = 1;",
     "if (src[i] < -255 || src[i] > 254) raw = 1;", 1, ["test_oracle_dwt.py", "test_oracle_rans.py"]),
    ("wavelet prediction rounds up", "hi[i] = (int32_t)(x[(2 * i + 1) * step] - floor_div2(left + right));",
     "hi[i] = (int32_t)(x[(2 * i + 1) * step] - floor_div2(left + right + 1));", 1, ["test_oracle_dwt.py"]),
    ("wavelet update bias 1, both directions", "floor_div4(dl + dr + 2)", "floor_div4(dl + dr + 1)", 2,
     ["test_oracle_dwt.py"]),
    ("luminance DC length of category 5", "{2, 3, 3, 3, 3, 3, 4, 5, 6, 7, 8, 9}", "{2, 3, 3, 3, 3, 4, 4, 5, 6, 7, 8, 9}",
     1, ["test_oracle_jpeg.py"]),
    ("EOB and 0x05 lengths swapped", "0x01, 0x02, 0x03, 0x00, 0x04, 0x11, 0x05,", "0x01, 0x02, 0x03, 0x05, 0x04, 0x11, 0x00,",
     1, ["test_oracle_jpeg.py"]),
    ("chrominance DC length of category 2", "{2, 2, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11}",
     "{2, 2, 3, 3, 4, 5, 6, 7, 8, 9, 10, 11}", 1, ["test_oracle_420.py"]),
    ("ZRL after 17 zeros", "while (run > 15) {", "while (run > 16) {", 1, ["test_oracle_jpeg.py"]),
    ("zigzag transposed", "int lv = L[u * 8 + v];", "int lv = L[v * 8 + u];", 1, ["test_oracle_jpeg.py"]),
    ("DC prediction dropped", "        pred = L[0];\n", "        pred = 0;\n", 1, ["test_oracle_jpeg.py"]),
    ("EOB dropped", "if (run > 0) bits +=", "if (run > 63) bits +=", 1, ["test_oracle_jpeg.py"]),
    ("Cb weight of B", "32768 * b + 32768) >> 16) + 128", "32767 * b + 32768) >> 16) + 128", 1,
     ["test_oracle_420.py"]),
    ("2x2 chroma average rounds down", "(uint8_t)((sum + 2) >> 2)", "(uint8_t)((sum + 1) >> 2)", 1,
     ["test_oracle_420.py"]),
    ("chroma upsampled from the wrong row", "k = (int64_t)(y / 2) * wc + x / 2;",
     "k = (int64_t)((y + 1) / 2 < hc ? (y + 1) / 2 : hc - 1) * wc + x / 2;", 1, ["test_oracle_420.py"]),
    ("inverse colour: Cr weight of G", "- 46802 * cr + 32768) >> 16", "- 46803 * cr + 32768) >> 16", 1,
     ["test_oracle_420.py"]),
]


def _mutant(src: str, old: str, new: str, count: int, where: str) -> str:
    assert src.count(old) == count, f"the planted text must occur {count} time(s)"
    path_c = os.path.join(where, "mutant.c")
    with open(path_c, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(where, "libmutant.so")
    subprocess.check_call(["gcc", *O.CFLAGS, "-o", so, path_c, "-lm"])
    return so


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new,count,files", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(name, old, new, count, files):
    with open(O._SRC) as f:
        src = f.read()
    with tempfile.TemporaryDirectory() as tmp:
        so = _mutant(src, old, new, count, tmp)
        env = dict(os.environ, SLRME_ORACLE_LIB=so)
        p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                            *[os.path.join(ROOT, "tests", f) for f in files]],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    # exit status 1: tests ran and at least one failed (not a crash or a collection error)
    assert p.returncode == 1, f"{name}: no pin failed\n{p.stdout[-1500:]}"


# The CNN oracle is Python: its mistakes are planted in a scratch copy of the
# module, loaded under its own name before the pin tests are collected.
CNN_MUTATIONS = [
    ("input exponent offset 136", "np.asarray(e, np.int64) - 137 - int(J)", "np.asarray(e, np.int64) - 136 - int(J)"),
    ("convolution window flipped", 'np.einsum("oc,chw->ohw", w[:, :, dy, dx], win)',
     'np.einsum("oc,chw->ohw", w[:, :, 2 - dy, 2 - dx], win)'),
    ("requantisation rounds down", "(acc * m + (1 << (shift - 1))) >> shift", "(acc * m) >> shift"),
    ("hidden clamp 128", "0, 127 if l < 3 else 255", "0, 128 if l < 3 else 255"),
    ("correction offset 127", "+ np.asarray(y3, np.int64) - 128", "+ np.asarray(y3, np.int64) - 127"),
    ("weight step over 128", "max(axis=1) / 127.0", "max(axis=1) / 128.0"),
    ("activation steps of 1/4", "q = z / SCALE_A", "q = z / (2 * SCALE_A)"),
    ("backward ignores the quantiser mask", "        g = g * mask\n", "        g = g\n"),
    ("L1 gradient not averaged", "np.sign(d) / d.size", "np.sign(d)"),
    ("Adam without bias correction", "mh = m / (1 - b1 ** step)", "mh = m"),
]

_LOAD_AND_TEST = """
import importlib.util, sys
import oracle
spec = importlib.util.spec_from_file_location("oracle.cnn_oracle", sys.argv[1])
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle.cnn_oracle"] = mod
spec.loader.exec_module(mod)
oracle.cnn_oracle = mod
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", sys.argv[2]]))
"""


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new", CNN_MUTATIONS, ids=[m[0] for m in CNN_MUTATIONS])
def test_planted_cnn_mistake_fails_a_pin(name, old, new):
    src_path = os.path.join(ROOT, "oracle", "cnn_oracle.py")
    with open(src_path) as f:
        src = f.read()
    assert src.count(old) == 1, "the planted text must occur once"
    with tempfile.TemporaryDirectory() as tmp:
        mut = os.path.join(tmp, "cnn_oracle.py")
        with open(mut, "w") as f:
            f.write(src.replace(old, new))
        p = subprocess.run([sys.executable, "-c", _LOAD_AND_TEST, mut, os.path.join(ROOT, "tests", "test_oracle_cnn.py")],
                           cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 1, f"{name}: no pin failed\n{p.stdout[-1500:]}"
