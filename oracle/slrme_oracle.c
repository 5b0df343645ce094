/*
 * CPU oracle for the dual-layer lossless Radiance (RGBE) coder with the
 * simple linear regressive mantissa estimator (SLRME), arXiv 2309.11072.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It is a plain, slow,
 * single-threaded statement of what the codec computes, written from the
 * paper (sections and equations cited per function) and from the readings
 * the paper leaves open (marked READING).  It shares no code, header, table
 * or constant generator with the CUDA library.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared
 * (float and double arithmetic is plain IEEE round-to-nearest, no FMA
 * contraction; >> on negative int is an arithmetic shift under gcc).
 *
 * Layouts: images are row-major, h rows by w columns.  Colour planes are
 * planar, plane c (R=0, G=1, B=2) at offset c*h*w.  A packed RGBE word is
 * R | G<<8 | B<<16 | E<<24.
 *
 * Parity status: every function here is pinned by a test against something
 * other than itself (closed forms, invariants, brute force, library
 * routines); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NBIN 256        /* one region per 8-bit exponent value E            */
#define NSUM 13         /* N_E, then (sum x, sum y, sum xy, sum xx) per channel */
#define NRES 511        /* residual values -255..255                         */

/* ----------------------------------------------------------------------
 * Sec. II-A, Eqs. (1)-(2): RGBE forward conversion.
 * READING: Eq. (1) with a ceiling gives M = 256 at exact powers of two,
 * which does not fit 8 bits; the Radiance convention (frexp exponent + 128,
 * so the largest mantissa is in [128, 255]) is used instead.  It agrees
 * with Eq. (1) everywhere else.  Returns -1 if an exponent leaves [1, 255].
 * ---------------------------------------------------------------------- */
int oracle_rgbe_from_float(const double* f, int64_t n_px, uint32_t* rgbe)
{
    for (int64_t p = 0; p < n_px; ++p) {
        double r = f[3 * p], g = f[3 * p + 1], b = f[3 * p + 2];
        double v = r > g ? r : g;
        v = v > b ? v : b;
        if (v < 1e-32) { rgbe[p] = 0; continue; }
        int ex;
        frexp(v, &ex);                     /* v = m * 2^ex, m in [0.5, 1) */
        int E = ex + 128;
        if (E < 1 || E > 255) return -1;
        /* Eq. (2): M = floor(256 f / 2^(E-128)) = floor(f * 2^(136-E)) */
        uint32_t M[3];
        const double c3[3] = {r, g, b};
        for (int c = 0; c < 3; ++c) M[c] = (uint32_t)floor(ldexp(c3[c], 136 - E));
        rgbe[p] = M[0] | (M[1] << 8) | (M[2] << 16) | ((uint32_t)E << 24);
    }
    return 0;
}

/* Sec. II-A, Eq. (3): f = (M + 0.5) / 256 * 2^(E-128); E = 0 is the zero pixel. */
void oracle_rgbe_to_float(const uint32_t* rgbe, int64_t n_px, double* f)
{
    for (int64_t p = 0; p < n_px; ++p) {
        uint32_t wd = rgbe[p];
        int E = (int)(wd >> 24);
        for (int c = 0; c < 3; ++c) {
            int M = (int)((wd >> (8 * c)) & 255u);
            f[3 * p + c] = (E == 0) ? 0.0 : ldexp(M + 0.5, E - 128 - 8);
        }
    }
}

/* Sec. III-A: the coder works on the mantissas M_R, M_G, M_B and the
 * exponent E directly; the split takes the bytes of each word apart. */
void oracle_rgbe_split(const uint32_t* rgbe, int64_t n_px, uint8_t* m3, uint8_t* e)
{
    for (int64_t p = 0; p < n_px; ++p) {
        uint32_t wd = rgbe[p];
        m3[p] = (uint8_t)(wd & 255u);
        m3[n_px + p] = (uint8_t)((wd >> 8) & 255u);
        m3[2 * n_px + p] = (uint8_t)((wd >> 16) & 255u);
        e[p] = (uint8_t)(wd >> 24);
    }
}

/* ======================================================================
 * Base layer, part 1: the tone-mapping operator (Sec. II-B, Fig. 2; the
 * experiments of Sec. IV use Reinhard et al.'s global operator).  The
 * paper gives no parameters; every constant below is a READING:
 *   key 0.18 over the log-average luminance, L_d = L / (1 + L), colour
 *   carried by the ratio f_c / Y, BT.709 luma weights, display gamma 2.2.
 * The pixel luminance is exact in integers: with f_c = (2M_c+1) 2^(E-137)
 * (Eq. 3), 10^4 * Y = Yq * 2^(E-137) where
 *   Yq = 2126 (2M_R+1) + 7152 (2M_G+1) + 722 (2M_B+1)   (10^4 <= Yq < 2^23).
 * ====================================================================== */

/* lut[i] = round(65536 * log2(2048 + i)), i = 0..2047 */
void oracle_log2_table(int32_t* lut)
{
    for (int i = 0; i < 2048; ++i) lut[i] = (int32_t)llround(65536.0 * log2((double)(2048 + i)));
}

/* t[k] = float32(((k - 0.5) / 255) ^ 2.2), k = 1..255; t[0] = 0 (unused).
 * The 8-bit display value of a linear value v is #{k in 1..255 : v >= t[k]},
 * i.e. round(255 v^(1/2.2)) with ties settled by the table. */
void oracle_gamma_thresholds(float* t)
{
    t[0] = 0.0f;
    for (int k = 1; k < 256; ++k) t[k] = (float)pow((k - 0.5) / 255.0, 2.2);
}

/* Key scale tables for the fractional sixteenth r = 0..15 of the log-average:
 * kr[r] = float32(0.18 * 2^(-r/16)),  wr[r] = float32(1800 * 2^(-r/16)). */
void oracle_key_tables(float* kr, float* wr)
{
    for (int r = 0; r < 16; ++r) {
        kr[r] = (float)(0.18 * pow(2.0, -r / 16.0));
        wr[r] = (float)(1800.0 * pow(2.0, -r / 16.0));
    }
}

static int64_t yq_of(uint32_t wd)
{
    int64_t R = wd & 255u, G = (wd >> 8) & 255u, B = (wd >> 16) & 255u;
    return 2126 * (2 * R + 1) + 7152 * (2 * G + 1) + 722 * (2 * B + 1);
}

static int bitlen64(int64_t v)
{
    int n = 0;
    while (v > 0) { ++n; v >>= 1; }
    return n;
}

/* Log-average statistic: stats[0] = sum over E > 0 of l(p), stats[1] = count,
 * where l = 65536 (E - 137 + k) + lut[m - 2048], k = bitlen(Yq) - 12,
 * m = Yq >> k, so l / 65536 ~ log2(10^4 Y). */
void oracle_lum_stats(const uint32_t* rgbe, int64_t n_px, int64_t* stats)
{
    int32_t lut[2048];
    oracle_log2_table(lut);
    int64_t s = 0, n = 0;
    for (int64_t p = 0; p < n_px; ++p) {
        int E = (int)(rgbe[p] >> 24);
        if (E == 0) continue;
        int64_t Yq = yq_of(rgbe[p]);
        int k = bitlen64(Yq) - 12;
        int64_t m = Yq >> k;
        s += 65536 * (int64_t)(E - 137 + k) + lut[m - 2048];
        n += 1;
    }
    stats[0] = s;
    stats[1] = n;
}

static int64_t floor_div(int64_t a, int64_t b)   /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

/* j = round-half-up(16 * mu), mu = stats[0] / (65536 stats[1]); j = 16 J + r.
 * An image with no non-zero pixel takes j = 0. */
void oracle_key(const int64_t* stats, int32_t* J, int32_t* r)
{
    int64_t j = 0;
    if (stats[1] > 0) j = floor_div(stats[0] + 2048 * stats[1], 4096 * stats[1]);
    int64_t Jj = floor_div(j, 16);
    *J = (int32_t)Jj;
    *r = (int32_t)(j - 16 * Jj);
}

/* Per pixel, float32 round-to-nearest, as the READING fixes it:
 *   d = clamp(E - 137 - J, -100, 100)
 *   L = (kr[r] * Yq) * 2^d                       (scaled luminance, exact scale)
 *   H = (wr[r] * 2^d) / (1 + L)                  (= L_d / Y, times 10^4)
 *   v_c = H * (2 M_c + 1)                        (= L_d * f_c / Y)
 *   SDR_c = #{k : v_c >= t[k]};   E = 0 gives SDR = 0. */
void oracle_tmo(const uint32_t* rgbe, int64_t n_px, int32_t J, int32_t r, uint8_t* sdr3)
{
    float t[256], kr[16], wr[16];
    oracle_gamma_thresholds(t);
    oracle_key_tables(kr, wr);
    for (int64_t p = 0; p < n_px; ++p) {
        uint32_t wd = rgbe[p];
        int E = (int)(wd >> 24);
        if (E == 0) { sdr3[p] = sdr3[n_px + p] = sdr3[2 * n_px + p] = 0; continue; }
        int d = E - 137 - J;
        if (d < -100) d = -100;
        if (d > 100) d = 100;
        float P = kr[r] * (float)yq_of(wd);
        float L = ldexpf(P, d);
        float den = 1.0f + L;
        float num = ldexpf(wr[r], d);
        float H = num / den;
        for (int c = 0; c < 3; ++c) {
            int M = (int)((wd >> (8 * c)) & 255u);
            float v = H * (float)(2 * M + 1);
            /* count thresholds <= v by bisection over the increasing table */
            int lo = 0, hi = 256;            /* invariant: t[1..lo] <= v < t[hi..255] */
            while (hi - lo > 1) {
                int mid = (lo + hi) / 2;
                if (v >= t[mid]) lo = mid; else hi = mid;
            }
            sdr3[(int64_t)c * n_px + p] = (uint8_t)lo;
        }
    }
}

/* Reinhard's operator with a white point (his Eq. 4, the variant of Eq. 3
 * that maps the luminance L_white to 1): L_d = L (1 + L / L_white^2) / (1 + L).
 * READING: L_white is the largest scaled luminance L of the image (L as
 * oracle_tmo computes it, over the pixels with E > 0; Reinhard's own
 * suggestion), and per pixel, in float32 round-to-nearest,
 *   H = ((num * (1 + L / (L_white * L_white))) / den)
 * with num, den and L as in oracle_tmo, each operation rounded once in
 * that order.  L_white = +inf gives oracle_tmo exactly. */
static float tmo_L(uint32_t wd, int32_t J, float kr)
{
    int E = (int)(wd >> 24);
    int d = E - 137 - J;
    if (d < -100) d = -100;
    if (d > 100) d = 100;
    return ldexpf(kr * (float)yq_of(wd), d);
}

float oracle_white_point(const uint32_t* rgbe, int64_t n_px, int32_t J, int32_t r)
{
    float t[256], kr[16], wr[16];
    (void)t;
    oracle_key_tables(kr, wr);
    float best = 0.0f;
    for (int64_t p = 0; p < n_px; ++p) {
        if ((rgbe[p] >> 24) == 0) continue;
        float L = tmo_L(rgbe[p], J, kr[r]);
        if (L > best) best = L;
    }
    return best;
}

void oracle_tmo_white(const uint32_t* rgbe, int64_t n_px, int32_t J, int32_t r, float l_white, uint8_t* sdr3)
{
    float t[256], kr[16], wr[16];
    oracle_gamma_thresholds(t);
    oracle_key_tables(kr, wr);
    float lw2 = l_white * l_white;
    for (int64_t p = 0; p < n_px; ++p) {
        uint32_t wd = rgbe[p];
        int E = (int)(wd >> 24);
        if (E == 0) { sdr3[p] = sdr3[n_px + p] = sdr3[2 * n_px + p] = 0; continue; }
        int d = E - 137 - J;
        if (d < -100) d = -100;
        if (d > 100) d = 100;
        float L = tmo_L(wd, J, kr[r]);
        float den = 1.0f + L;
        float num = ldexpf(wr[r], d);
        float q = L / lw2;
        float f = 1.0f + q;
        float nf = num * f;
        float H = nf / den;
        for (int c = 0; c < 3; ++c) {
            int M = (int)((wd >> (8 * c)) & 255u);
            float v = H * (float)(2 * M + 1);
            int lo = 0, hi = 256;            /* count thresholds <= v */
            while (hi - lo > 1) {
                int mid = (lo + hi) / 2;
                if (v >= t[mid]) lo = mid; else hi = mid;
            }
            sdr3[(int64_t)c * n_px + p] = (uint8_t)lo;
        }
    }
}

/* ======================================================================
 * Base layer, part 2: the lossy base coder round trip (Sec. IV uses JPEG
 * at quality Q).  Only the transform and quantiser change the decoded
 * SDRI S, so only they are computed (entropy coding does not change S).
 * READINGS: each colour plane is coded on its own, 4:4:4, with the ITU-T
 * T.81 Annex K.1 luminance table scaled by the IJG quality rule; the
 * last row/column is replicated up to a multiple of 8; the DCT is a
 * fixed-point matrix product with constants round(4096 * D) and a
 * round-half-up shift after each 1-D pass (9, 15 forward; 9, 15 inverse).
 * ====================================================================== */

static const int32_t k_luma_q50[64] = {
    16, 11, 10, 16, 24, 40, 51, 61,
    12, 12, 14, 19, 26, 58, 60, 55,
    14, 13, 16, 24, 40, 57, 69, 56,
    14, 17, 22, 29, 51, 87, 80, 62,
    18, 22, 37, 56, 68, 109, 103, 77,
    24, 35, 55, 64, 81, 104, 113, 92,
    49, 64, 78, 87, 103, 121, 120, 101,
    72, 92, 95, 98, 112, 100, 103, 99};

/* q[v*8+u]: quantiser step for vertical frequency v, horizontal u. */
void oracle_quant_table(int quality, int32_t* q)
{
    int s = quality < 50 ? 5000 / quality : 200 - 2 * quality;
    for (int i = 0; i < 64; ++i) {
        int v = (k_luma_q50[i] * s + 50) / 100;
        q[i] = v < 1 ? 1 : (v > 255 ? 255 : v);
    }
}

/* d[u*8+x] = round(4096 * alpha_u * cos((2x+1) u pi / 16)),
 * alpha_0 = sqrt(1/8), alpha_u = 1/2 (orthonormal DCT-II). */
void oracle_dct_matrix(int32_t* d)
{
    const double pi = 3.14159265358979323846;
    for (int u = 0; u < 8; ++u)
        for (int x = 0; x < 8; ++x) {
            double a = (u == 0) ? sqrt(1.0 / 8.0) : 0.5;
            d[u * 8 + x] = (int32_t)llround(4096.0 * a * cos((2 * x + 1) * u * pi / 16.0));
        }
}

static int32_t rshift_round(int64_t v, int s) { return (int32_t)((v + ((int64_t)1 << (s - 1))) >> s); }

/* Forward 2-D DCT of one block, X[y*8+x] in [-128, 127] -> F[v*8+u]:
 * along x first, T[y][u] = (sum_x D[u][x] X[y][x]) >> 9 (rounded), then
 * along y, F[v][u] = (sum_y D[v][y] T[y][u]) >> 15 (rounded).  The scale
 * 4096^2 = 2^(9+15) makes F the orthonormal DCT-II up to rounding. */
static const int32_t* dct_constants(void)
{
    static int32_t D[64];
    static int ready = 0;
    if (!ready) { oracle_dct_matrix(D); ready = 1; }
    return D;
}

void oracle_fdct_block(const int32_t* X, int32_t* F)
{
    const int32_t* D = dct_constants();
    int32_t T[64];
    for (int y = 0; y < 8; ++y)
        for (int u = 0; u < 8; ++u) {
            int64_t acc = 0;
            for (int x = 0; x < 8; ++x) acc += (int64_t)D[u * 8 + x] * X[y * 8 + x];
            T[y * 8 + u] = rshift_round(acc, 9);
        }
    for (int v = 0; v < 8; ++v)
        for (int u = 0; u < 8; ++u) {
            int64_t acc = 0;
            for (int y = 0; y < 8; ++y) acc += (int64_t)D[v * 8 + y] * T[y * 8 + u];
            F[v * 8 + u] = rshift_round(acc, 15);
        }
}

/* Quantise (level = sign(F) floor((|F| + floor(q/2)) / q), i.e. half away
 * from zero) and dequantise (level * q), coefficient by coefficient. */
void oracle_quant_dequant_block(const int32_t* F, const int32_t* Q, int32_t* Fq)
{
    for (int i = 0; i < 64; ++i) {
        int32_t q = Q[i];
        int32_t a = F[i] < 0 ? -F[i] : F[i];
        int32_t lvl = (a + q / 2) / q;
        Fq[i] = (F[i] < 0 ? -lvl : lvl) * q;
    }
}

/* Inverse 2-D DCT: along y first, G[y][u] = (sum_v D[v][y] F[v][u]) >> 9,
 * then along x, X[y][x] = (sum_u D[u][x] G[y][u]) >> 15 (both rounded). */
void oracle_idct_block(const int32_t* F, int32_t* X)
{
    const int32_t* D = dct_constants();
    int32_t G[64];
    for (int y = 0; y < 8; ++y)
        for (int u = 0; u < 8; ++u) {
            int64_t acc = 0;
            for (int v = 0; v < 8; ++v) acc += (int64_t)D[v * 8 + y] * F[v * 8 + u];
            G[y * 8 + u] = rshift_round(acc, 9);
        }
    for (int y = 0; y < 8; ++y)
        for (int x = 0; x < 8; ++x) {
            int64_t acc = 0;
            for (int u = 0; u < 8; ++u) acc += (int64_t)D[u * 8 + x] * G[y * 8 + u];
            X[y * 8 + x] = rshift_round(acc, 15);
        }
}

/* sdr3 (planar uint8) -> decoded SDRI s3 (planar uint8). Returns -1 on bad quality. */
int oracle_base_roundtrip(const uint8_t* sdr3, int h, int w, int quality, uint8_t* s3)
{
    if (quality < 1 || quality > 100) return -1;
    int32_t Q[64];
    oracle_quant_table(quality, Q);
    int64_t n_px = (int64_t)h * w;
    for (int c = 0; c < 3; ++c) {
        const uint8_t* in = sdr3 + c * n_px;
        uint8_t* out = s3 + c * n_px;
        for (int by = 0; by < h; by += 8)
            for (int bx = 0; bx < w; bx += 8) {
                int32_t X[64], F[64], Fq[64], Y[64];
                for (int y = 0; y < 8; ++y)
                    for (int x = 0; x < 8; ++x) {
                        int yy = by + y < h ? by + y : h - 1;
                        int xx = bx + x < w ? bx + x : w - 1;
                        X[y * 8 + x] = (int32_t)in[(int64_t)yy * w + xx] - 128;
                    }
                oracle_fdct_block(X, F);
                oracle_quant_dequant_block(F, Q, Fq);
                oracle_idct_block(Fq, Y);
                for (int y = 0; y < 8 && by + y < h; ++y)
                    for (int x = 0; x < 8 && bx + x < w; ++x) {
                        int32_t s = Y[y * 8 + x] + 128;
                        out[(int64_t)(by + y) * w + bx + x] = (uint8_t)(s < 0 ? 0 : (s > 255 ? 255 : s));
                    }
            }
    }
    return 0;
}

/* ======================================================================
 * Sec. III-B: SLRME.
 * ====================================================================== */

/* Gaussian-filter restoration S -> S* (Sec. III-B and its footnote).
 * READING: 3x3 binomial kernel [1 2 1]^T [1 2 1] with edge replication,
 * kept unrounded as an integer in 1/16 units: x = 16 S* in [0, 4080].
 * gf_on = 0 gives x = 16 S (no restoration). */
void oracle_gf(const uint8_t* s3, int h, int w, int gf_on, int32_t* x3)
{
    int64_t n_px = (int64_t)h * w;
    static const int wt[3] = {1, 2, 1};
    for (int c = 0; c < 3; ++c) {
        const uint8_t* S = s3 + c * n_px;
        int32_t* X = x3 + c * n_px;
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                if (!gf_on) { X[(int64_t)y * w + x] = 16 * S[(int64_t)y * w + x]; continue; }
                int32_t acc = 0;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int yy = y + dy, xx = x + dx;
                        yy = yy < 0 ? 0 : (yy >= h ? h - 1 : yy);
                        xx = xx < 0 ? 0 : (xx >= w ? w - 1 : xx);
                        acc += wt[dy + 1] * wt[dx + 1] * S[(int64_t)yy * w + xx];
                    }
                X[(int64_t)y * w + x] = acc;
            }
    }
}

/* Eqs. (9)-(10) need, for each region E (all q with that exponent) and each
 * channel c, the sums over q of 1, S*, M, S* M and S*^2.  Layout:
 * sums[E*13 + 0] = N_E, sums[E*13 + 1 + 4c + {0,1,2,3}] =
 * {sum x, sum y, sum x y, sum x x} with x = 16 S*_c, y = M_c.  Exact int64. */
void oracle_bin_sums(const int32_t* x3, const uint8_t* m3, const uint8_t* e, int64_t n_px, int64_t* sums)
{
    memset(sums, 0, sizeof(int64_t) * NBIN * NSUM);
    for (int64_t p = 0; p < n_px; ++p) {
        int64_t* s = sums + (int64_t)e[p] * NSUM;
        s[0] += 1;
        for (int c = 0; c < 3; ++c) {
            int64_t x = x3[c * n_px + p], y = m3[c * n_px + p];
            s[1 + 4 * c] += x;
            s[2 + 4 * c] += y;
            s[3 + 4 * c] += x * y;
            s[4 + 4 * c] += x * x;
        }
    }
}

/* Correctly rounded (nearest, ties to even) conversion of a signed 128-bit
 * integer to double, written out: keep the top 53 significant bits and
 * round on the rest. */
double oracle_i128_to_double(__int128 v)
{
    if (v == 0) return 0.0;
    int neg = v < 0;
    unsigned __int128 u = neg ? (unsigned __int128)0 - (unsigned __int128)v : (unsigned __int128)v;
    int nb = 0;
    for (unsigned __int128 t = u; t != 0; t >>= 1) ++nb;
    double r;
    if (nb <= 53) {
        r = (double)(uint64_t)u;
    } else {
        int sh = nb - 53;
        unsigned __int128 mant = u >> sh;
        unsigned __int128 rem = u - (mant << sh);
        unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (mant & 1))) mant += 1;   /* may reach 2^53: still exact */
        r = ldexp((double)(uint64_t)mant, sh);
    }
    return neg ? -r : r;
}

/* Entry point so tests can check the conversion: v = hi * 2^64 + lo. */
double oracle_i128_to_double_parts(int64_t hi, uint64_t lo)
{
    __int128 v = ((__int128)hi << 64) | (__int128)lo;
    return oracle_i128_to_double(v);
}

/* Eqs. (9)-(10) (the normal equations (6)-(7) of Sec. II-C restricted to
 * region E), quantised to the 32-bit values Sec. III-C transmits.
 *   D_xx = N sum x^2 - (sum x)^2,  D_xy = N sum xy - sum x sum y   (exact int128)
 *   a_E  = float32( double(D_xy) / double(D_xx) )
 *   b_E  = float32( (double(sum y) - double(a_E) * double(sum x)) / double(N) )
 * READINGS: per channel and per E (Eq. 8 is written per mantissa); x is
 * S* in 1/16 units, so a_E is per 1/16 step; b_E is computed from the
 * quantised a_E (the intercept that is optimal for the slope actually
 * sent); N_E = 0 leaves the region unused (a = b = 0, not sent); D_xx = 0
 * (all x equal) gives a = 0, b = float32(sum y / N). */
void oracle_solve(const int64_t* sums, float* a, float* b, int32_t* n_e, int32_t* n_used)
{
    int used = 0;
    for (int E = 0; E < NBIN; ++E) {
        const int64_t* s = sums + E * NSUM;
        int64_t N = s[0];
        n_e[E] = (int32_t)N;
        if (N > 0) ++used;
        for (int c = 0; c < 3; ++c) {
            float* ac = a + c * NBIN + E;
            float* bc = b + c * NBIN + E;
            if (N == 0) { *ac = 0.0f; *bc = 0.0f; continue; }
            int64_t sx = s[1 + 4 * c], sy = s[2 + 4 * c], sxy = s[3 + 4 * c], sxx = s[4 + 4 * c];
            __int128 dxx = (__int128)N * sxx - (__int128)sx * sx;
            __int128 dxy = (__int128)N * sxy - (__int128)sx * sy;
            if (dxx == 0) {
                *ac = 0.0f;
                *bc = (float)((double)sy / (double)N);
                continue;
            }
            double ad = oracle_i128_to_double(dxy) / oracle_i128_to_double(dxx);
            float af = (float)ad;
            double t = (double)af * (double)sx;
            double bd = ((double)sy - t) / (double)N;
            *ac = af;
            *bc = (float)bd;
        }
    }
    *n_used = used;
}

/* Eq. (8): M*(q) = round(a_E S*(q) + b_E) clipped to [0, 255].
 * READINGS: t = float32(float32(a x) + b) with x = 16 S* (no fused
 * multiply-add); round is half away from zero (MATLAB's round, the
 * paper's platform). */
static uint8_t predict1(float a, float b, int32_t x)
{
    float t = a * (float)x;
    t = t + b;
    if (!(t > 0.0f)) return 0;            /* t <= 0 (round of t <= 0 is <= 0) */
    if (t >= 255.0f) return 255;
    float tr = truncf(t);
    int r = (int)tr;
    if (t - tr >= 0.5f) r += 1;
    return (uint8_t)(r > 255 ? 255 : r);
}

void oracle_predict(const int32_t* x3, const uint8_t* e, int64_t n_px, const float* a, const float* b, uint8_t* mstar3)
{
    for (int c = 0; c < 3; ++c)
        for (int64_t p = 0; p < n_px; ++p) {
            int E = e[p];
            mstar3[c * n_px + p] = predict1(a[c * NBIN + E], b[c * NBIN + E], x3[c * n_px + p]);
        }
}

/* Sec. III-C: the enhancement layer carries R = M - M*; hist[c*511 + R + 255]
 * counts each value (the order-0 statistics used for the bit rate). */
void oracle_residual(const uint8_t* m3, const uint8_t* mstar3, int64_t n_px, int16_t* r3, uint32_t* hist)
{
    if (hist) memset(hist, 0, sizeof(uint32_t) * 3 * NRES);
    for (int c = 0; c < 3; ++c)
        for (int64_t p = 0; p < n_px; ++p) {
            int r = (int)m3[c * n_px + p] - (int)mstar3[c * n_px + p];
            r3[c * n_px + p] = (int16_t)r;
            if (hist) hist[c * NRES + r + 255] += 1;
        }
}

/* Decoder (Sec. I, III-C): M = R + M*(S, E, a, b), M* recomputed from the
 * decoded SDRI and the transmitted parameters without refitting; the word
 * is repacked with the transmitted exponent plane. */
void oracle_decode(const uint8_t* s3, const uint8_t* e, const int16_t* r3, int h, int w, int gf_on,
                   const float* a, const float* b, uint32_t* rgbe)
{
    int64_t n_px = (int64_t)h * w;
    int32_t* x3 = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)n_px);
    uint8_t* ms = (uint8_t*)malloc(3 * (size_t)n_px);
    oracle_gf(s3, h, w, gf_on, x3);
    oracle_predict(x3, e, n_px, a, b, ms);
    for (int64_t p = 0; p < n_px; ++p) {
        uint32_t wd = (uint32_t)e[p] << 24;
        for (int c = 0; c < 3; ++c) {
            int M = (int)r3[c * n_px + p] + (int)ms[c * n_px + p];
            wd |= ((uint32_t)M & 255u) << (8 * c);
        }
        rgbe[p] = wd;
    }
    free(x3);
    free(ms);
}

/* ===================================================================== enhancement-layer coder
 * The reversible coder of the residual planes (Sec. III-C sends R to a
 * lossless coder; the paper uses JPEG 2000 lossless, Sec. IV).  Here: a
 * static rANS coder with one frequency table per channel, written from the
 * published rANS construction (J. Duda, "Asymmetric numeral systems", 2013)
 * as specified for this library:
 *   symbols s = R + 255 in 0..510; table total M = 2^14;
 *   state x in [L, 2^32) with L = 2^16; 16-bit words in and out;
 *   encode s (f, c): if floor(x / 2^18) >= f, emit x mod 2^16, x = floor(x / 2^16);
 *                    then x = floor(x / f) M + (x mod f) + c;
 *   decode: slot = x mod M, s the symbol with c <= slot < c + f,
 *           x = f floor(x / M) + slot - c; if x < L, x = 2^16 x + next word.
 * A plane's symbols (raster order) are cut into chunks of 8192; stream l
 * (0..31) of chunk k codes symbols k 8192 + l + 32 j in increasing j.  Each
 * chunk owns a block of 32 x 258 words; its streams' words are packed from
 * the start of the block, stream after stream (stream l from the sum of the
 * word counts of streams 0..l-1), each in decoding order: the final encoder
 * state (high word, low word), then the renormalisation words.  counts[]
 * holds the words used per stream; the rest of the block is left as it was. */

#define RANS_BITS 14
#define RANS_M (1u << RANS_BITS)
#define RANS_L (1u << 16)
#define RANS_CHUNK 8192
#define RANS_LANES 32
#define RANS_CAP (RANS_CHUNK / RANS_LANES + 2)

/* Frequency table of one channel from its residual histogram: every symbol
 * that occurs gets max(1, floor(count M / N)); the shortfall to M goes to the
 * most frequent symbol (smallest on ties), an excess is taken one at a time
 * from the largest entry above 1 (smallest symbol on ties).  Returns the
 * number of symbols that occur (0: an empty histogram, all entries 0). */
int oracle_rans_table(const uint32_t* counts, uint32_t* freq)
{
    uint64_t N = 0;
    int used = 0;
    for (int s = 0; s < NRES; ++s) {
        N += counts[s];
        used += counts[s] != 0;
    }
    for (int s = 0; s < NRES; ++s) freq[s] = 0;
    if (N == 0) return 0;
    int64_t sum = 0;
    for (int s = 0; s < NRES; ++s)
        if (counts[s]) {
            uint64_t f = (uint64_t)counts[s] * RANS_M / N;
            freq[s] = (uint32_t)(f < 1 ? 1 : f);
            sum += freq[s];
        }
    int64_t diff = (int64_t)RANS_M - sum;
    if (diff > 0) {
        int best = 0;
        for (int s = 1; s < NRES; ++s)
            if (counts[s] > counts[best]) best = s;
        freq[best] += (uint32_t)diff;
    }
    while (diff < 0) {
        int best = -1;
        for (int s = 0; s < NRES; ++s)
            if (freq[s] > 1 && (best < 0 || freq[s] > freq[best])) best = s;
        freq[best] -= 1;
        diff += 1;
    }
    return used;
}

static void rans_cum(const uint32_t* freq, uint32_t* cum)
{
    uint32_t c = 0;
    for (int s = 0; s < NRES; ++s) {
        cum[s] = c;
        c += freq[s];
    }
}

/* Symbols of stream l of chunk k of a plane of n symbols. */
static int64_t rans_stream_len(int64_t n, int64_t k, int l)
{
    int64_t end = (k + 1) * RANS_CHUNK < n ? (k + 1) * RANS_CHUNK : n;
    int64_t first = k * RANS_CHUNK + l;
    return first < end ? (end - 1 - first) / RANS_LANES + 1 : 0;
}

/* Segments: the symbol array is a run of segments, each with its own table
 * (freq[g * 511 ...]) and cut into its own chunks; segment g's chunks follow
 * those of segments 0..g-1 in `words` and `counts`.  A chunk holding a value
 * outside -255..255 is stored raw: its block holds the chunk's values (the
 * int16 bit patterns, in order) and all 32 of its counts are RANS_RAW. */
#define RANS_RAW 0xFFFFFFFFu

static int64_t rans_chunks(int64_t len) { return (len + RANS_CHUNK - 1) / RANS_CHUNK; }

/* Returns 0, or -1 when a value inside -255..255 has a zero frequency. */
int oracle_rans_encode_segments(const int16_t* sym, int nseg, const int64_t* len, const uint32_t* freq,
                                uint16_t* words, uint32_t* counts)
{
    int64_t sym_at = 0, chunk_at = 0;
    for (int g = 0; g < nseg; ++g) {
        const uint32_t* f = freq + (int64_t)g * NRES;
        uint32_t cum[NRES];
        rans_cum(f, cum);
        int64_t chunks = rans_chunks(len[g]);
        for (int64_t k = 0; k < chunks; ++k) {
            const int16_t* src = sym + sym_at + k * RANS_CHUNK;
            int64_t m = len[g] - k * RANS_CHUNK < RANS_CHUNK ? len[g] - k * RANS_CHUNK : RANS_CHUNK;
            uint16_t* block = words + (chunk_at + k) * RANS_LANES * RANS_CAP;
            uint32_t* cnt = counts + (chunk_at + k) * RANS_LANES;
            int raw = 0;
            for (int64_t i = 0; i < m; ++i)
                if (src[i] < -255 || src[i] > 255) raw = 1;
            if (raw) {
                for (int64_t i = 0; i < m; ++i) block[i] = (uint16_t)src[i];
                for (int l = 0; l < RANS_LANES; ++l) cnt[l] = RANS_RAW;
                continue;
            }
            int64_t at = 0;   /* where the next stream starts in the block */
            for (int l = 0; l < RANS_LANES; ++l) {
                /* the words are produced last-first: build them at the end of
                 * a scratch region, then copy them to the block */
                uint16_t region[RANS_CAP];
                int64_t slen = rans_stream_len(m, 0, l);
                uint32_t x = RANS_L;
                int p = RANS_CAP;
                for (int64_t j = slen - 1; j >= 0; --j) {
                    int s = src[l + RANS_LANES * j] + 255;
                    uint32_t fs = f[s];
                    if (fs == 0) return -1;
                    if ((x >> 18) >= fs) {
                        region[--p] = (uint16_t)(x & 0xFFFFu);
                        x >>= 16;
                    }
                    x = (x / fs) * RANS_M + (x % fs) + cum[s];
                }
                region[--p] = (uint16_t)(x & 0xFFFFu);
                region[--p] = (uint16_t)(x >> 16);
                int used = RANS_CAP - p;
                memcpy(block + at, region + p, (size_t)used * sizeof(uint16_t));
                at += used;
                cnt[l] = (uint32_t)used;
            }
        }
        sym_at += len[g];
        chunk_at += chunks;
    }
    return 0;
}

/* Decodes what oracle_rans_encode_segments wrote. */
void oracle_rans_decode_segments(const uint16_t* words, const uint32_t* counts, int nseg, const int64_t* len,
                                 const uint32_t* freq, int16_t* sym)
{
    int64_t sym_at = 0, chunk_at = 0;
    for (int g = 0; g < nseg; ++g) {
        const uint32_t* f = freq + (int64_t)g * NRES;
        uint32_t cum[NRES];
        rans_cum(f, cum);
        int64_t chunks = rans_chunks(len[g]);
        for (int64_t k = 0; k < chunks; ++k) {
            int16_t* dst = sym + sym_at + k * RANS_CHUNK;
            int64_t m = len[g] - k * RANS_CHUNK < RANS_CHUNK ? len[g] - k * RANS_CHUNK : RANS_CHUNK;
            const uint16_t* block = words + (chunk_at + k) * RANS_LANES * RANS_CAP;
            const uint32_t* cnt = counts + (chunk_at + k) * RANS_LANES;
            if (cnt[0] == RANS_RAW) {
                for (int64_t i = 0; i < m; ++i) dst[i] = (int16_t)block[i];
                continue;
            }
            int64_t at = 0;
            for (int l = 0; l < RANS_LANES; ++l) {
                const uint16_t* stream = block + at;
                at += cnt[l];
                int64_t slen = rans_stream_len(m, 0, l);
                uint32_t x = ((uint32_t)stream[0] << 16) | stream[1];
                int p = 2;
                for (int64_t j = 0; j < slen; ++j) {
                    uint32_t slot = x & (RANS_M - 1);
                    int s = 0;
                    while (!(cum[s] <= slot && slot < cum[s] + f[s])) ++s;
                    x = f[s] * (x >> RANS_BITS) + slot - cum[s];
                    if (x < RANS_L) x = (x << 16) | stream[p++];
                    dst[l + RANS_LANES * j] = (int16_t)(s - 255);
                }
            }
        }
        sym_at += len[g];
        chunk_at += chunks;
    }
}

/* The three residual planes (int16 [3][n]) as three segments of n symbols
 * with the channels' tables freq3 ([3][511]).  words: [3][chunks] blocks of
 * 32 x 258 uint16, counts: [3][chunks][32]; chunks = ceil(n / 8192). */
int oracle_rans_encode(const int16_t* r3, int64_t n, const uint32_t* freq3, uint16_t* words, uint32_t* counts)
{
    const int64_t len[3] = {n, n, n};
    return oracle_rans_encode_segments(r3, 3, len, freq3, words, counts);
}

void oracle_rans_decode(const uint16_t* words, const uint32_t* counts, int64_t n, const uint32_t* freq3,
                        int16_t* r3)
{
    const int64_t len[3] = {n, n, n};
    oracle_rans_decode_segments(words, counts, 3, len, freq3, r3);
}

/* ------------------------------------------------------------------ reversible 5/3 wavelet
 * The enhancement layer of Sec. IV is coded by JPEG 2000's lossless mode,
 * whose transform is the reversible LeGall 5/3 wavelet: integer lifting with
 * whole-sample symmetric extension (x[-k] = x[k], x[n-1+k] = x[n-1-k]).
 * For n >= 2 samples, nH = floor(n / 2) high-pass and nL = ceil(n / 2)
 * low-pass values:
 *   d[i] = x[2i+1] - floor((x[2i] + x[2i+2]) / 2),        i < nH
 *   s[i] = x[2i]   + floor((d[i-1] + d[i] + 2) / 4),       i < nL
 * where the extension gives x[n] = x[n-2], d[-1] = d[0] and, for odd n,
 * d[nL-1] = d[nL-2].  A single sample is its own low-pass value.  The
 * inverse runs the two steps backwards.  One 2-D level transforms every row,
 * then every column of the row-transformed array; the next level transforms
 * the low-low band.  Each pass at most doubles the largest magnitude, so
 * three levels of residuals in -255..255 stay within +-16320 (int16).
 * Output order per plane (subband-major, each band row-major):
 *   LL_L, HL_L, LH_L, HH_L, HL_(L-1), LH_(L-1), HH_(L-1), ..., HL_1, LH_1, HH_1
 * with HL high-pass along rows (columns nL..n-1 of a row), LH along columns. */

#define DWT_MAX_LEVELS 3

static int64_t floor_div2(int64_t a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }
static int64_t floor_div4(int64_t a) { return a >= 0 ? a / 4 : -((-a + 3) / 4); }

/* one 1-D forward step over n samples read with stride `step`: low-pass
 * values to lo[0..nL), high-pass to hi[0..nH) */
static void dwt53_fwd_1d(const int32_t* x, int n, int step, int32_t* lo, int32_t* hi)
{
    if (n == 1) {
        lo[0] = x[0];
        return;
    }
    int nH = n / 2, nL = n - nH;
    for (int i = 0; i < nH; ++i) {
        int64_t left = x[(2 * i) * step];
        int64_t right = (2 * i + 2 <= n - 1) ? x[(2 * i + 2) * step] : x[(2 * i) * step];
        hi[i] = (int32_t)(x[(2 * i + 1) * step] - floor_div2(left + right));
    }
    for (int i = 0; i < nL; ++i) {
        int64_t dl = hi[i >= 1 ? i - 1 : 0];
        int64_t dr = hi[i < nH ? i : nH - 1];
        lo[i] = (int32_t)(x[(2 * i) * step] + floor_div4(dl + dr + 2));
    }
}

static void dwt53_inv_1d(const int32_t* lo, const int32_t* hi, int n, int32_t* x, int step)
{
    if (n == 1) {
        x[0] = lo[0];
        return;
    }
    int nH = n / 2, nL = n - nH;
    for (int i = 0; i < nL; ++i) {
        int64_t dl = hi[i >= 1 ? i - 1 : 0];
        int64_t dr = hi[i < nH ? i : nH - 1];
        x[(2 * i) * step] = (int32_t)(lo[i] - floor_div4(dl + dr + 2));
    }
    for (int i = 0; i < nH; ++i) {
        int64_t left = x[(2 * i) * step];
        int64_t right = (2 * i + 2 <= n - 1) ? x[(2 * i + 2) * step] : x[(2 * i) * step];
        x[(2 * i + 1) * step] = (int32_t)(hi[i] + floor_div2(left + right));
    }
}

/* Band sizes in output order: dims[2 b] = rows, dims[2 b + 1] = columns of
 * band b; returns the number of bands (1 + 3 levels). */
int oracle_dwt53_bands(int h, int w, int levels, int32_t* dims)
{
    int hs[DWT_MAX_LEVELS + 1], ws[DWT_MAX_LEVELS + 1];
    hs[0] = h;
    ws[0] = w;
    for (int l = 1; l <= levels; ++l) {
        hs[l] = (hs[l - 1] + 1) / 2;
        ws[l] = (ws[l - 1] + 1) / 2;
    }
    int b = 0;
    dims[2 * b] = hs[levels];
    dims[2 * b + 1] = ws[levels];
    ++b;
    for (int l = levels; l >= 1; --l) {
        int H = hs[l - 1], W = ws[l - 1];
        int HL = (H + 1) / 2, HH = H / 2, WL = (W + 1) / 2, WH = W / 2;
        dims[2 * b] = HL; dims[2 * b + 1] = WH; ++b;   /* HL: rows low, columns high */
        dims[2 * b] = HH; dims[2 * b + 1] = WL; ++b;   /* LH */
        dims[2 * b] = HH; dims[2 * b + 1] = WH; ++b;   /* HH */
    }
    return b;
}

/* Forward transform of one plane (h x w, row-major) into the subband-major
 * order above.  0 on success, -1 for levels outside 0..3. */
int oracle_dwt53_forward(const int16_t* r, int h, int w, int levels, int16_t* coef)
{
    if (levels < 0 || levels > DWT_MAX_LEVELS) return -1;
    int64_t n = (int64_t)h * w;
    if (n == 0) return 0;
    int32_t* cur = malloc(sizeof(int32_t) * n);     /* the band being split, H x W */
    int32_t* tmp = malloc(sizeof(int32_t) * n);
    int32_t* col = malloc(sizeof(int32_t) * (h > w ? h : w) * 2);
    for (int64_t i = 0; i < n; ++i) cur[i] = r[i];
    int32_t dims[2 * (1 + 3 * DWT_MAX_LEVELS)];
    int nb = oracle_dwt53_bands(h, w, levels, dims);
    /* band offsets in output order */
    int64_t off[1 + 3 * DWT_MAX_LEVELS];
    int64_t at = 0;
    for (int b = 0; b < nb; ++b) {
        off[b] = at;
        at += (int64_t)dims[2 * b] * dims[2 * b + 1];
    }
    int H = h, W = w;
    for (int l = 1; l <= levels; ++l) {
        int WL = (W + 1) / 2, WH = W / 2, HL = (H + 1) / 2, HH = H / 2;
        /* rows: tmp[y][0..WL) low, tmp[y][WL..W) high */
        for (int y = 0; y < H; ++y) dwt53_fwd_1d(cur + (int64_t)y * W, W, 1, tmp + (int64_t)y * W, tmp + (int64_t)y * W + WL);
        /* columns */
        int bHL = 1 + 3 * (levels - l), bLH = bHL + 1, bHH = bHL + 2;
        for (int x = 0; x < W; ++x) {
            int32_t* lo = col;
            int32_t* hi = col + H;
            dwt53_fwd_1d(tmp + x, H, W, lo, hi);
            for (int y = 0; y < HL; ++y) {
                if (x < WL) cur[(int64_t)y * WL + x] = lo[y];           /* next level's input, HL x WL */
                else coef[off[bHL] + (int64_t)y * WH + (x - WL)] = (int16_t)lo[y];
            }
            for (int y = 0; y < HH; ++y) {
                if (x < WL) coef[off[bLH] + (int64_t)y * WL + x] = (int16_t)hi[y];
                else coef[off[bHH] + (int64_t)y * WH + (x - WL)] = (int16_t)hi[y];
            }
        }
        H = HL;
        W = WL;
    }
    for (int64_t i = 0; i < (int64_t)H * W; ++i) coef[i] = (int16_t)cur[i];   /* LL_L (band 0 at offset 0) */
    free(cur);
    free(tmp);
    free(col);
    return 0;
}

/* Inverse of oracle_dwt53_forward. */
int oracle_dwt53_inverse(const int16_t* coef, int h, int w, int levels, int16_t* r)
{
    if (levels < 0 || levels > DWT_MAX_LEVELS) return -1;
    int64_t n = (int64_t)h * w;
    if (n == 0) return 0;
    int32_t dims[2 * (1 + 3 * DWT_MAX_LEVELS)];
    int nb = oracle_dwt53_bands(h, w, levels, dims);
    int64_t off[1 + 3 * DWT_MAX_LEVELS];
    int64_t at = 0;
    for (int b = 0; b < nb; ++b) {
        off[b] = at;
        at += (int64_t)dims[2 * b] * dims[2 * b + 1];
    }
    int hs[DWT_MAX_LEVELS + 1], ws[DWT_MAX_LEVELS + 1];
    hs[0] = h;
    ws[0] = w;
    for (int l = 1; l <= levels; ++l) {
        hs[l] = (hs[l - 1] + 1) / 2;
        ws[l] = (ws[l - 1] + 1) / 2;
    }
    int32_t* cur = malloc(sizeof(int32_t) * n);
    int32_t* tmp = malloc(sizeof(int32_t) * n);
    int32_t* col = malloc(sizeof(int32_t) * (h > w ? h : w) * 2);
    for (int64_t i = 0; i < (int64_t)hs[levels] * ws[levels]; ++i) cur[i] = coef[i];
    for (int l = levels; l >= 1; --l) {
        int H = hs[l - 1], W = ws[l - 1];
        int WL = (W + 1) / 2, WH = W / 2, HL = (H + 1) / 2, HH = H / 2;
        int bHL = 1 + 3 * (levels - l), bLH = bHL + 1, bHH = bHL + 2;
        /* columns back into tmp (H x W, row-transformed layout) */
        for (int x = 0; x < W; ++x) {
            int32_t* lo = col;
            int32_t* hi = col + H;
            for (int y = 0; y < HL; ++y)
                lo[y] = x < WL ? cur[(int64_t)y * WL + x] : coef[off[bHL] + (int64_t)y * WH + (x - WL)];
            for (int y = 0; y < HH; ++y)
                hi[y] = x < WL ? coef[off[bLH] + (int64_t)y * WL + x] : coef[off[bHH] + (int64_t)y * WH + (x - WL)];
            dwt53_inv_1d(lo, hi, H, tmp + x, W);
        }
        /* rows back into cur (H x W) */
        for (int y = 0; y < H; ++y) dwt53_inv_1d(tmp + (int64_t)y * W, tmp + (int64_t)y * W + WL, W, cur + (int64_t)y * W, 1);
    }
    for (int64_t i = 0; i < n; ++i) r[i] = (int16_t)cur[i];
    free(cur);
    free(tmp);
    free(col);
    return 0;
}

/* ------------------------------------------------------------------ base-layer entropy coding
 * Sec. IV codes the base layer with JPEG.  The base round trip above models
 * only what changes S; its quantised levels are also what a baseline JPEG
 * encoder entropy-codes (T.81 Annex F.1.2), so their coded size gives the
 * base layer's rate.  Each colour plane is its own single-component scan
 * (reading 4), blocks in raster order, with the typical luminance Huffman
 * tables of T.81 Annex K.3 (Tables K.3 and K.5):
 *   DC: diff = level_DC - level_DC of the previous block of the plane (0
 *       before the first); category SSSS = bit length of |diff|; cost =
 *       length of the DC code of SSSS + SSSS extra bits;
 *   AC: zigzag order k = 1..63; a run of r zeros before a nonzero level c
 *       costs, for every 16 zeros beyond 15, one ZRL code (symbol 0xF0), then
 *       the code of symbol (r mod 16) << 4 | SSSS(c) plus SSSS extra bits;
 *       zeros after the last nonzero level cost one EOB code (symbol 0x00).
 * The size is the sum of code lengths and extra bits: the entropy-coded
 * data before byte stuffing, padding and markers.
 * Levels layout: levels3[(c * bh + by) * bw + bx][64], bh = ceil(h / 8),
 * bw = ceil(w / 8); within a block, coefficient (v vertical, u horizontal
 * frequency) at u * 8 + v. */

/* Code lengths of Table K.3 (DC luminance), by category 0..11. */
static const int jpeg_dc_len[12] = {2, 3, 3, 3, 3, 3, 4, 5, 6, 7, 8, 9};

/* Table K.5 (AC luminance): the symbols with codes shorter than 16 bits, in
 * the table's order of increasing length, with their lengths; every other
 * symbol (r << 4 | s, s = 1..10) has a 16-bit code. */
static const uint8_t jpeg_ac_short_sym[37] = {
    0x01, 0x02, 0x03, 0x00, 0x04, 0x11, 0x05, 0x12, 0x21, 0x31, 0x41, 0x06, 0x13,
    0x51, 0x61, 0x07, 0x22, 0x71, 0x14, 0x32, 0x81, 0x91, 0xa1, 0x08, 0x23, 0x42,
    0xb1, 0xc1, 0x15, 0x52, 0xd1, 0xf0, 0x24, 0x33, 0x62, 0x72, 0x82};
static const uint8_t jpeg_ac_short_len[37] = {
    2, 2, 3, 4, 4, 4, 5, 5, 5, 6, 6, 7, 7, 7, 7, 8, 8, 8, 9, 9, 9, 9, 9,
    10, 10, 10, 10, 10, 11, 11, 11, 11, 12, 12, 12, 12, 15};

/* Code length of AC symbol `sym`, 0 for a symbol the table does not have. */
int oracle_jpeg_ac_len(int sym)
{
    for (int i = 0; i < 37; ++i)
        if (jpeg_ac_short_sym[i] == sym) return jpeg_ac_short_len[i];
    int s = sym & 15;
    return (s >= 1 && s <= 10) ? 16 : 0;
}

int oracle_jpeg_dc_len(int cat) { return cat >= 0 && cat <= 11 ? jpeg_dc_len[cat] : 0; }

/* Natural index (v * 8 + u) of zigzag position k (T.81 Figure A.6): the
 * anti-diagonals s = u + v in turn, v rising on odd s and falling on even s. */
void oracle_zigzag(int32_t* zz)
{
    int k = 0;
    for (int s = 0; s <= 14; ++s) {
        int vlo = s - 7 > 0 ? s - 7 : 0, vhi = s < 7 ? s : 7;
        if (s & 1)
            for (int v = vlo; v <= vhi; ++v) zz[k++] = v * 8 + (s - v);
        else
            for (int v = vhi; v >= vlo; --v) zz[k++] = v * 8 + (s - v);
    }
}

static int bitlen(int a) { int n = 0; while (a) { ++n; a >>= 1; } return n; }

/* The quantised levels of the base round trip (same blocks, transform and
 * quantiser as oracle_base_roundtrip).  Returns -1 for a bad quality. */
int oracle_base_levels(const uint8_t* sdr3, int h, int w, int quality, int16_t* levels3)
{
    if (quality < 1 || quality > 100) return -1;
    int32_t Q[64];
    oracle_quant_table(quality, Q);
    int64_t n_px = (int64_t)h * w;
    int bh = (h + 7) / 8, bw = (w + 7) / 8;
    for (int c = 0; c < 3; ++c) {
        const uint8_t* in = sdr3 + c * n_px;
        for (int by = 0; by < bh; ++by)
            for (int bx = 0; bx < bw; ++bx) {
                int32_t X[64], F[64], Fq[64];
                for (int y = 0; y < 8; ++y)
                    for (int x = 0; x < 8; ++x) {
                        int yy = 8 * by + y < h ? 8 * by + y : h - 1;
                        int xx = 8 * bx + x < w ? 8 * bx + x : w - 1;
                        X[y * 8 + x] = (int32_t)in[(int64_t)yy * w + xx] - 128;
                    }
                oracle_fdct_block(X, F);
                oracle_quant_dequant_block(F, Q, Fq);
                int16_t* L = levels3 + (((int64_t)c * bh + by) * bw + bx) * 64;
                for (int v = 0; v < 8; ++v)
                    for (int u = 0; u < 8; ++u) L[u * 8 + v] = (int16_t)(Fq[v * 8 + u] / Q[v * 8 + u]);
            }
    }
    return 0;
}

/* Table K.4 (DC chrominance) code lengths by category, and Table K.6 (AC
 * chrominance): its symbols with codes shorter than 16 bits, in the table's
 * order, with their lengths; the other 119 symbols have 16-bit codes. */
static const int jpeg_dc_len_c[12] = {2, 2, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11};
static const uint8_t jpeg_ac_short_sym_c[43] = {
    0x00, 0x01, 0x02, 0x03, 0x11, 0x04, 0x05, 0x21, 0x31, 0x06, 0x12, 0x41, 0x51, 0x07, 0x61,
    0x71, 0x13, 0x22, 0x32, 0x81, 0x08, 0x14, 0x42, 0x91, 0xa1, 0xb1, 0xc1, 0x09, 0x23, 0x33,
    0x52, 0xf0, 0x15, 0x62, 0x72, 0xd1, 0x0a, 0x16, 0x24, 0x34, 0xe1, 0x25, 0xf1};
static const uint8_t jpeg_ac_short_len_c[43] = {
    2, 2, 3, 4, 4, 5, 5, 5, 5, 6, 6, 6, 6, 7, 7, 7, 8, 8, 8, 8, 9, 9, 9, 9, 9, 9, 9, 10, 10, 10,
    10, 10, 11, 11, 11, 11, 12, 12, 12, 12, 14, 15, 15};

/* Code lengths of the chrominance tables (0 for a symbol or category they lack). */
int oracle_jpeg_ac_len_c(int sym)
{
    for (int i = 0; i < 43; ++i)
        if (jpeg_ac_short_sym_c[i] == sym) return jpeg_ac_short_len_c[i];
    int s = sym & 15;
    return (s >= 1 && s <= 10) ? 16 : 0;
}

int oracle_jpeg_dc_len_c(int cat) { return cat >= 0 && cat <= 11 ? jpeg_dc_len_c[cat] : 0; }

/* Coded bits of one plane's nb blocks (64 levels each, raster order, one
 * scan) with the luminance (chroma = 0) or chrominance tables.  Returns the
 * total, or -1 when a category exceeds the baseline tables. */
static int64_t jpeg_plane_bits(const int16_t* levels, int64_t nb, int chroma, uint32_t* block_bits)
{
    int32_t zz[64];
    oracle_zigzag(zz);
    int64_t total = 0;
    int pred = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const int16_t* L = levels + b * 64;
        uint32_t bits = 0;
        int diff = L[0] - pred;
        pred = L[0];
        int cat = bitlen(diff < 0 ? -diff : diff);
        if (cat > 11) return -1;
        bits += (uint32_t)((chroma ? jpeg_dc_len_c[cat] : jpeg_dc_len[cat]) + cat);
        int run = 0;
        for (int k = 1; k < 64; ++k) {
            int nat = zz[k];
            int v = nat / 8, u = nat % 8;
            int lv = L[u * 8 + v];
            if (lv == 0) {
                ++run;
                continue;
            }
            while (run > 15) {
                bits += (uint32_t)(chroma ? oracle_jpeg_ac_len_c(0xF0) : oracle_jpeg_ac_len(0xF0));
                run -= 16;
            }
            int sz = bitlen(lv < 0 ? -lv : lv);
            if (sz > 10) return -1;
            int sym = (run << 4) | sz;
            bits += (uint32_t)((chroma ? oracle_jpeg_ac_len_c(sym) : oracle_jpeg_ac_len(sym)) + sz);
            run = 0;
        }
        if (run > 0) bits += (uint32_t)(chroma ? oracle_jpeg_ac_len_c(0x00) : oracle_jpeg_ac_len(0x00));
        if (block_bits) block_bits[b] = bits;
        total += bits;
    }
    return total;
}

/* Entropy-coded bits of each plane (bits3[3]) and of each block
 * (block_bits[(c * bh + by) * bw + bx], may be NULL), three planes of the
 * 4:4:4 base layer with the luminance tables.  Returns -1 when a category
 * exceeds the baseline tables (DC 11, AC 10). */
int oracle_jpeg_bits(const int16_t* levels3, int h, int w, uint64_t* bits3, uint32_t* block_bits)
{
    int64_t nb = (int64_t)((h + 7) / 8) * ((w + 7) / 8);
    for (int c = 0; c < 3; ++c) {
        int64_t t = jpeg_plane_bits(levels3 + c * nb * 64, nb, 0, block_bits ? block_bits + c * nb : NULL);
        if (t < 0) return -1;
        bits3[c] = (uint64_t)t;
    }
    return 0;
}

/* Planes of any block counts, each with its table class (chroma[p]). */
int oracle_jpeg_bits_planes(const int16_t* levels, int np, const int64_t* nblocks, const int32_t* chroma,
                            uint64_t* bits, uint32_t* block_bits)
{
    int64_t at = 0;
    for (int p = 0; p < np; ++p) {
        int64_t t = jpeg_plane_bits(levels + at * 64, nblocks[p], chroma[p], block_bits ? block_bits + at : NULL);
        if (t < 0) return -1;
        bits[p] = (uint64_t)t;
        at += nblocks[p];
    }
    return 0;
}

/* ------------------------------------------------------------------ YCbCr 4:2:0 base layer
 * The base layer as a default JPEG encoder codes colour: the SDRI converted
 * to YCbCr (T.871, the JFIF equations), chroma averaged over 2x2 pixels,
 * each plane through the 8x8 round trip above (Y with the Annex K.1
 * luminance table, Cb and Cr with the Annex K.2 chrominance table, both
 * scaled by the IJG quality rule), chroma replicated back over its 2x2
 * pixels, and converted back to RGB.  READING (fixed point, all rounding
 * half up by adding half before an arithmetic right shift, then clamping
 * to 0..255): with weights round(65536 c) of the T.871 coefficients c,
 *   Y  = (19595 R + 38470 G + 7471 B + 32768) >> 16
 *   Cb = ((-11058 R - 21710 G + 32768 B + 32768) >> 16) + 128
 *   Cr = ((32768 R - 27439 G - 5329 B + 32768) >> 16) + 128
 * chroma sample (i, j) = (sum of pixels (2i..2i+1, 2j..2j+1), edges
 * replicated, + 2) >> 2, planes of ceil(h/2) x ceil(w/2); back:
 *   R = Y + ((91881 (Cr - 128) + 32768) >> 16)
 *   G = Y + ((-22554 (Cb - 128) - 46802 (Cr - 128) + 32768) >> 16)
 *   B = Y + ((116130 (Cb - 128) + 32768) >> 16). */
static const int32_t k_chroma_q50[64] = {
    17, 18, 24, 47, 99, 99, 99, 99,
    18, 21, 26, 66, 99, 99, 99, 99,
    24, 26, 56, 99, 99, 99, 99, 99,
    47, 66, 99, 99, 99, 99, 99, 99,
    99, 99, 99, 99, 99, 99, 99, 99,
    99, 99, 99, 99, 99, 99, 99, 99,
    99, 99, 99, 99, 99, 99, 99, 99,
    99, 99, 99, 99, 99, 99, 99, 99};

void oracle_quant_table_chroma(int quality, int32_t* q)
{
    int s = quality < 50 ? 5000 / quality : 200 - 2 * quality;
    for (int i = 0; i < 64; ++i) {
        int v = (k_chroma_q50[i] * s + 50) / 100;
        q[i] = v < 1 ? 1 : (v > 255 ? 255 : v);
    }
}

static int clamp255(int v) { return v < 0 ? 0 : (v > 255 ? 255 : v); }

void oracle_rgb_to_ycc(const uint8_t* rgb3, int64_t n, uint8_t* ycc3)
{
    for (int64_t i = 0; i < n; ++i) {
        int r = rgb3[i], g = rgb3[n + i], b = rgb3[2 * n + i];
        ycc3[i] = (uint8_t)clamp255((19595 * r + 38470 * g + 7471 * b + 32768) >> 16);
        ycc3[n + i] = (uint8_t)clamp255(((-11058 * r - 21710 * g + 32768 * b + 32768) >> 16) + 128);
        ycc3[2 * n + i] = (uint8_t)clamp255(((32768 * r - 27439 * g - 5329 * b + 32768) >> 16) + 128);
    }
}

/* T.871's inverse, R = Y + 1.402 (Cr - 128), G = Y - 0.344136 (Cb - 128) -
 * 0.714136 (Cr - 128), B = Y + 1.772 (Cb - 128), with the weights
 * round(65536 c), rounded half up and clamped, on full-resolution planes. */
void oracle_ycc_to_rgb(const uint8_t* ycc3, int64_t n, uint8_t* rgb3)
{
    for (int64_t i = 0; i < n; ++i) {
        int Y = ycc3[i], cb = ycc3[n + i] - 128, cr = ycc3[2 * n + i] - 128;
        rgb3[i] = (uint8_t)clamp255(Y + ((91881 * cr + 32768) >> 16));
        rgb3[n + i] = (uint8_t)clamp255(Y + ((-22554 * cb - 46802 * cr + 32768) >> 16));
        rgb3[2 * n + i] = (uint8_t)clamp255(Y + ((116130 * cb + 32768) >> 16));
    }
}

/* One plane (ph x pw) through the 8x8 round trip with steps Q; levels (may
 * be NULL) as in oracle_base_levels for one plane. */
static void plane_roundtrip(const uint8_t* in, int ph, int pw, const int32_t* Q, uint8_t* out, int16_t* levels)
{
    int bh = (ph + 7) / 8, bw = (pw + 7) / 8;
    for (int by = 0; by < bh; ++by)
        for (int bx = 0; bx < bw; ++bx) {
            int32_t X[64], F[64], Fq[64], Y[64];
            for (int y = 0; y < 8; ++y)
                for (int x = 0; x < 8; ++x) {
                    int yy = 8 * by + y < ph ? 8 * by + y : ph - 1;
                    int xx = 8 * bx + x < pw ? 8 * bx + x : pw - 1;
                    X[y * 8 + x] = (int32_t)in[(int64_t)yy * pw + xx] - 128;
                }
            oracle_fdct_block(X, F);
            oracle_quant_dequant_block(F, Q, Fq);
            if (levels) {
                int16_t* L = levels + ((int64_t)by * bw + bx) * 64;
                for (int v = 0; v < 8; ++v)
                    for (int u = 0; u < 8; ++u) L[u * 8 + v] = (int16_t)(Fq[v * 8 + u] / Q[v * 8 + u]);
            }
            oracle_idct_block(Fq, Y);
            for (int y = 0; y < 8 && 8 * by + y < ph; ++y)
                for (int x = 0; x < 8 && 8 * bx + x < pw; ++x)
                    out[(int64_t)(8 * by + y) * pw + 8 * bx + x] = (uint8_t)clamp255(Y[y * 8 + x] + 128);
        }
}

/* The 4:2:0 base layer of the SDRI sdr3 (RGB planes) at `quality`: s3
 * (RGB planes) and, if levels is not NULL, the levels of the Y blocks, then
 * the Cb blocks, then the Cr blocks (each plane's blocks in raster order).
 * Returns -1 for a bad quality. */
int oracle_base_roundtrip_420(const uint8_t* sdr3, int h, int w, int quality, uint8_t* s3, int16_t* levels)
{
    if (quality < 1 || quality > 100) return -1;
    int64_t n = (int64_t)h * w;
    if (n == 0) return 0;
    int hc = (h + 1) / 2, wc = (w + 1) / 2;
    int64_t nc = (int64_t)hc * wc;
    int32_t QY[64], QC[64];
    oracle_quant_table(quality, QY);
    oracle_quant_table_chroma(quality, QC);
    uint8_t* ycc = malloc(3 * n);
    uint8_t* cs = malloc(2 * nc);      /* subsampled Cb, Cr */
    uint8_t* yd = malloc(n);
    uint8_t* cd = malloc(2 * nc);
    oracle_rgb_to_ycc(sdr3, n, ycc);
    for (int c = 0; c < 2; ++c) {
        const uint8_t* P = ycc + (1 + c) * n;
        for (int i = 0; i < hc; ++i)
            for (int j = 0; j < wc; ++j) {
                int y0 = 2 * i, y1 = 2 * i + 1 < h ? 2 * i + 1 : h - 1;
                int x0 = 2 * j, x1 = 2 * j + 1 < w ? 2 * j + 1 : w - 1;
                int sum = P[(int64_t)y0 * w + x0] + P[(int64_t)y0 * w + x1] + P[(int64_t)y1 * w + x0] +
                          P[(int64_t)y1 * w + x1];
                cs[c * nc + (int64_t)i * wc + j] = (uint8_t)((sum + 2) >> 2);
            }
    }
    int64_t nbY = (int64_t)((h + 7) / 8) * ((w + 7) / 8), nbC = (int64_t)((hc + 7) / 8) * ((wc + 7) / 8);
    plane_roundtrip(ycc, h, w, QY, yd, levels);
    for (int c = 0; c < 2; ++c)
        plane_roundtrip(cs + c * nc, hc, wc, QC, cd + c * nc, levels ? levels + (nbY + c * nbC) * 64 : NULL);
    /* chroma replicated over its 2x2 pixels, then back to RGB */
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            int64_t i = (int64_t)y * w + x, k = (int64_t)(y / 2) * wc + x / 2;
            ycc[i] = yd[i];
            ycc[n + i] = cd[k];
            ycc[2 * n + i] = cd[nc + k];
        }
    oracle_ycc_to_rgb(ycc, n, s3);
    free(ycc);
    free(cs);
    free(yd);
    free(cd);
    return 0;
}
