// Base layer round trip: tone-mapping operator + fixed-point 8x8 DCT,
// quantise, dequantise, inverse DCT (Sec. II-B, Fig. 2; Sec. IV's JPEG
// base layer at quality Q).
//
// Work unit: one warp owns a band of 8 rows x 32 columns = four 8x8 blocks
// per colour plane.  Lane l handles block (l >> 3) and row (l & 7):
//   phase 1  (lane = row):     load 8 pixels of M_R, M_G, M_B, E; tone map;
//                              forward 1-D DCT along x; T' -> shared
//   phase 2  (lane = column):  forward 1-D DCT along y, quantise/dequantise,
//                              inverse 1-D DCT along y; G -> shared
//   phase 3  (lane = row):     inverse 1-D DCT along x, +128, clamp, store S
// Only __syncwarp is needed between phases.  A block's tile is 8 lines of 8
// words, blocks 72 words apart: phase 1 writes its row transposed (word
// 8u + r for coefficient u of row r) and phase 2 writes its column
// transposed (word 8y + u), so each phase reads its own line as two 16-byte
// loads, and every scattered 4-byte store of a warp hits 32 distinct banks
// (lanes differ in 8 * block + line index).
//
// Exactness: every product and sum is an exact int32 (worst cases: 2^21
// after pass 1, 2^25.1 before the second shift, 2^24 and 2^28.2 in the
// inverse), so the even/odd factorisation below yields the same integers as
// the plain matrix products with the same rounding shifts; the rounding
// term of each shift (and the +128 of the last one) is added before the
// shift as part of the sums, which changes no integer.
#include "slrme_internal.cuh"

#define SLRME_TABLE static __device__ const
#include "tables.inc"
#undef SLRME_TABLE

namespace slrme {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kTileWords = 3 * 4 * 72;    // per warp: 3 planes x 4 blocks x 72 words (64 used)
// CTAs per SM of the round-trip kernel: three give it up to 85 registers a
// thread (measured faster at 7680x4320 than four CTAs at 64 registers)
constexpr int kBaseCtas = 3;

// Fixed-point DCT constants round(4096 * alpha_u * cos((2x+1) u pi / 16)).
constexpr int C4 = 1448;   // alpha_0 * 4096 and cos(pi/4) / 2 * 4096
constexpr int C1 = 2009, C2 = 1892, C3 = 1703, C5 = 1138, C6 = 784, C7 = 400;

// Forward 8-point transform along one line: out[u] = sum_x D[u][x] in[x] + r
// (r, the rounding term of the shift that follows, enters each output's
// first multiply-add).
__device__ __forceinline__ void fdct8(const int (&x)[8], int (&F)[8], int r) {
    const int s07 = x[0] + x[7], d07 = x[0] - x[7];
    const int s16 = x[1] + x[6], d16 = x[1] - x[6];
    const int s25 = x[2] + x[5], d25 = x[2] - x[5];
    const int s34 = x[3] + x[4], d34 = x[3] - x[4];
    const int e0 = s07 + s34, e1 = s16 + s25, e2 = s07 - s34, e3 = s16 - s25;
    F[0] = C4 * (e0 + e1) + r;
    F[4] = C4 * (e0 - e1) + r;
    F[2] = C2 * e2 + r + C6 * e3;
    F[6] = C6 * e2 + r - C2 * e3;
    F[1] = C1 * d07 + r + C3 * d16 + C5 * d25 + C7 * d34;
    F[3] = C3 * d07 + r - C7 * d16 - C1 * d25 - C5 * d34;
    F[5] = C5 * d07 + r - C1 * d16 + C7 * d25 + C3 * d34;
    F[7] = C7 * d07 + r - C5 * d16 + C3 * d25 - C1 * d34;
}

// Inverse 8-point transform along one line: out[x] = sum_u D[u][x] in[u] + r.
__device__ __forceinline__ void idct8(const int (&F)[8], int (&x)[8], int r) {
    const int a = C4 * (F[0] + F[4]) + r, b = C4 * (F[0] - F[4]) + r;
    const int c = C2 * F[2] + C6 * F[6], d = C6 * F[2] - C2 * F[6];
    const int E0 = a + c, E3 = a - c, E1 = b + d, E2 = b - d;
    const int O0 = C1 * F[1] + C3 * F[3] + C5 * F[5] + C7 * F[7];
    const int O1 = C3 * F[1] - C7 * F[3] - C1 * F[5] - C5 * F[7];
    const int O2 = C5 * F[1] - C1 * F[3] + C7 * F[5] + C3 * F[7];
    const int O3 = C7 * F[1] - C5 * F[3] + C3 * F[5] - C1 * F[7];
    x[0] = E0 + O0; x[7] = E0 - O0;
    x[1] = E1 + O1; x[6] = E1 - O1;
    x[2] = E2 + O2; x[5] = E2 - O2;
    x[3] = E3 + O3; x[4] = E3 - O3;
}

// 8-bit display value: #{k in 1..255 : v >= gamma[k]} for the increasing
// threshold table (v >= 0, not NaN).  The float bits of v, clamped to the
// bucket below 2^-20 and the one at 1.0 by a min and a max, pick a bucket by
// their high half (exponent and top 7 mantissa bits; positive floats order
// like their bits); a bucket holds at most one threshold, and its word makes
// (bits + word) >> 16 equal the count below the bucket plus one exactly when
// the low 16 bits reach that threshold's (the word holds (count - high half)
// * 2^16 + 2^16 - t, mod 2^32).  One lookup, one addition, one shift; no
// branch.
__device__ __forceinline__ int gamma_code(float v, const uint32_t* code) {
    const int bits = min(max(__float_as_int(v), 0x357F0000), 0x3F800000);
    const uint32_t e = code[(bits >> 16) - 0x357F];
    return (int)(((uint32_t)bits + e) >> 16);
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// float(v) for 0 <= v < 2^23, exactly (the 2^23 bias).
__device__ __forceinline__ float small_int_to_float(int v) {
    return __fsub_rn(__int_as_float(0x4B000000 | v), 8388608.0f);
}

// Row y of a plane of row pitch p: columns x0 .. x0 + 7, the last row and
// column replicated past the edges.
__device__ __forceinline__ void load8(const uint8_t* __restrict__ plane, int h, int w, int y, int x0, bool fast,
                                      uint8_t (&out)[8], int p) {
    y = y < h ? y : h - 1;
    if (fast && x0 + 8 <= w) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(plane + (int64_t)y * p + x0));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            out[i] = (uint8_t)byte_of(v.x, i);
            out[4 + i] = (uint8_t)byte_of(v.y, i);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int x = x0 + i;
            x = x < w ? x : w - 1;
            out[i] = __ldg(plane + (int64_t)y * p + x);
        }
    }
}

__device__ __forceinline__ uint2 pack8(const uint8_t (&b)[8]) {
    return make_uint2((uint32_t)b[0] | ((uint32_t)b[1] << 8) | ((uint32_t)b[2] << 16) | ((uint32_t)b[3] << 24),
                      (uint32_t)b[4] | ((uint32_t)b[5] << 8) | ((uint32_t)b[6] << 16) | ((uint32_t)b[7] << 24));
}

__device__ __forceinline__ void store8(uint8_t* __restrict__ plane, int h, int w, int y, int x0, bool fast,
                                       const uint32_t lo, const uint32_t hi, int p) {
    if (y >= h) return;
    if (fast && x0 + 8 <= w) {
        *reinterpret_cast<uint2*>(plane + (int64_t)y * p + x0) = make_uint2(lo, hi);
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (x0 + i < w) plane[(int64_t)y * p + x0 + i] = (uint8_t)byte_of(i < 4 ? lo : hi, i & 3);
    }
}

// The bucket words of the display code into shared memory; ends with a
// block barrier.
constexpr int kGammaWords = 2562;
__device__ __forceinline__ void load_gamma(uint32_t* code) {
    for (int i = threadIdx.x; i < kGammaWords; i += blockDim.x) code[i] = kGammaCode[i];
    __syncthreads();
}

// The scaled luminance L of one pixel (the operator's input).
__device__ __forceinline__ float tmo_L(int mr, int mg, int mb, int E, int J, float kr, float* p2d_out) {
    const int yq = 2126 * (2 * mr + 1) + 7152 * (2 * mg + 1) + 722 * (2 * mb + 1);
    int d = E - 137 - J;
    d = d < -100 ? -100 : (d > 100 ? 100 : d);
    const float p2d = __int_as_float((127 + d) << 23);      // 2^d, a normal float
    *p2d_out = p2d;
    return __fmul_rn(__fmul_rn(kr, small_int_to_float(yq)), p2d);
}

// The tone-mapping operator of one pixel (Sec. II-B with Sec. IV's
// Reinhard operator): the three display codes of mantissas (mr, mg, mb) and
// exponent E, computed for every pixel without a branch.  Where E = 0 the
// numerator is 0, so H = 0 / (1 + L) = 0 (1 + L is finite and at least 1),
// every v is 0 and every code 0.
// kWhite: the operator with a white point (Reinhard's Eq. 4), lw2 = L_white^2:
// the numerator is multiplied by 1 + L / lw2 before the division.
template <bool kWhite = false>
__device__ __forceinline__ void tmo_pixel(int mr, int mg, int mb, int E, int J, float kr, float wr,
                                          const uint32_t* gcode, int& r, int& g, int& b, float lw2 = 0.0f) {
    float p2d;
    const float L = tmo_L(mr, mg, mb, E, J, kr, &p2d);
    const float den = __fadd_rn(1.0f, L);
    float num = E == 0 ? 0.0f : __fmul_rn(wr, p2d);
    if (kWhite) num = __fmul_rn(num, __fadd_rn(1.0f, __fdiv_rn(L, lw2)));
    const float H = __fdiv_rn(num, den);
    r = gamma_code(__fmul_rn(H, small_int_to_float(2 * mr + 1)), gcode);
    g = gamma_code(__fmul_rn(H, small_int_to_float(2 * mg + 1)), gcode);
    b = gamma_code(__fmul_rn(H, small_int_to_float(2 * mb + 1)), gcode);
}

// The same operator from the biased words 0x4B000000 | m of the three
// mantissas (one byte permute each from the packed planes): Y from the
// biased words with the bias folded into the constant (exact mod 2^32; Y is
// small), and float(2 m + 1) = 2 (2^23 + m) + 1 - 2^24 by one exact FMA.
__device__ __forceinline__ void tmo_pixel_biased(uint32_t br, uint32_t bg, uint32_t bb, int E, int J, float kr,
                                                 float wr, const uint32_t* gcode, int& r, int& g, int& b) {
    const uint32_t yq = 4252u * br + 14304u * bg + 1444u * bb + (10000u - 20000u * 0x4B000000u);
    // 2^d with d = clamp(E - 137 - J, -100, 100) (its exponent field 127 + d);
    // 0 where E = 0 (the min with E * 256 > 227 acts only there), which makes
    // L = 0 and the numerator 0, so H = 0 as the operator gives for E = 0
    const int field = __vimin3_s32(max(E - 10 - J, 27), 227, E << 8);
    const float p2d = __int_as_float(field << 23);
    const float L = __fmul_rn(__fmul_rn(kr, small_int_to_float((int)yq)), p2d);
    const float den = __fadd_rn(1.0f, L);
    const float num = __fmul_rn(wr, p2d);
    const float H = __fdiv_rn(num, den);
    constexpr float kOdd = 1.0f - 16777216.0f;
    r = gamma_code(__fmul_rn(H, __fmaf_rn(__uint_as_float(br), 2.0f, kOdd)), gcode);
    g = gamma_code(__fmul_rn(H, __fmaf_rn(__uint_as_float(bg), 2.0f, kOdd)), gcode);
    b = gamma_code(__fmul_rn(H, __fmaf_rn(__uint_as_float(bb), 2.0f, kOdd)), gcode);
}

// Key and quantiser state of one image, as a lane needs it.
struct BaseKey {
    int J;
    float kr, wr;
    int qcol[8];        // quantiser column `sub` of the block: q[v][sub], v = 0..7
    uint32_t qmcol[8];
};

__device__ __forceinline__ void base_key(const int64_t* __restrict__ stats, const QuantTable& QT, int sub,
                                         BaseKey& K) {
    int r;
    key_from_stats(stats, &K.J, &r);
    K.kr = __uint_as_float(kKrBits[r]);
    K.wr = __uint_as_float(kWrBits[r]);
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        K.qcol[v] = QT.q[v * 8 + sub];
        K.qmcol[v] = QT.qm[v * 8 + sub];
    }
}

// One band task of one image (all 32 lanes): rows y0 .. y0+7, columns xb .. xb+31.
// kLevels: also store the quantised levels to lv3, block (by, bx) of plane
// c at ((c * bh + by) * bw + bx) * 64, coefficient (v, u) at u * 8 + v, so a
// lane's column of a block is one 16-byte store (a separate instantiation,
// so the plain round trip compiles without it).
template <bool kLevels = false, bool kWhite = false>
__device__ __forceinline__ void base_band(const uint8_t* __restrict__ m3, const uint8_t* __restrict__ e, int h, int w,
                                          bool fast, int y0, int xb, int lane, const BaseKey& K,
                                          const uint32_t* gcode, int* T, uint8_t* __restrict__ s3,
                                          uint8_t* __restrict__ sdr3, const uint2* pre, int16_t* __restrict__ lv3,
                                          float lw2 = 0.0f, int p = 0) {
    // planes of h rows of pitch p (p = 0: p = w)
    p = p ? p : w;
    const int blk = lane >> 3, sub = lane & 7;   // block in the band, row (phases 1, 3) or column (phase 2)
    const int64_t n = (int64_t)h * p;
    const int J = K.J;
    const float kr = K.kr, wr = K.wr;
    const int x0 = xb + 8 * blk;                 // first column of this lane's block
    const int y = y0 + sub;                      // this lane's row in phases 1 and 3
    // ---------------- phase 1: tone map and forward DCT along x
    {
        uint2 wr8, wg8, wb8, we8;   // the lane's 8 pixels of each plane, packed
        if (pre) {
            // the band's bytes, copied to shared memory while the previous band was processed
            wr8 = pre[0];
            wg8 = pre[32];
            wb8 = pre[64];
            we8 = pre[96];
        } else {
            // rows past the bottom and columns past the right edge replicate the last row/column
            uint8_t mr[8], mg[8], mb[8], ee[8];
            load8(m3, h, w, y, x0, fast, mr, p);
            load8(m3 + n, h, w, y, x0, fast, mg, p);
            load8(m3 + 2 * n, h, w, y, x0, fast, mb, p);
            load8(e, h, w, y, x0, fast, ee, p);
            wr8 = pack8(mr);
            wg8 = pack8(mg);
            wb8 = pack8(mb);
            we8 = pack8(ee);
        }
        int sdr[3][8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t sel = 0x7540u | (uint32_t)(i & 3);   // byte i & 3 under the 0x4B000000 bias
            const uint32_t br = __byte_perm(i < 4 ? wr8.x : wr8.y, 0x4B000000u, sel);
            const uint32_t bg = __byte_perm(i < 4 ? wg8.x : wg8.y, 0x4B000000u, sel);
            const uint32_t bb = __byte_perm(i < 4 ? wb8.x : wb8.y, 0x4B000000u, sel);
            const int E = (int)byte_of(i < 4 ? we8.x : we8.y, i & 3);
            if (kWhite)
                tmo_pixel<true>((int)(br & 255u), (int)(bg & 255u), (int)(bb & 255u), E, J, kr, wr, gcode, sdr[0][i],
                                sdr[1][i], sdr[2][i], lw2);
            else
                tmo_pixel_biased(br, bg, bb, E, J, kr, wr, gcode, sdr[0][i], sdr[1][i], sdr[2][i]);
        }
        if (sdr3 && x0 < w) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const uint32_t lo = sdr[c][0] | (sdr[c][1] << 8) | (sdr[c][2] << 16) | (sdr[c][3] << 24);
                const uint32_t hi = sdr[c][4] | (sdr[c][5] << 8) | (sdr[c][6] << 16) | (sdr[c][7] << 24);
                store8(sdr3 + c * n, h, w, y, x0, fast, lo, hi, p);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // the transform of (sdr - 128): only F[0] sees the level shift
            // (every other output's coefficients sum to zero), by -1024 C4
            int F[8];
            fdct8(sdr[c], F, 1 << 8);
            F[0] -= 1024 * C4;
            int* tile = T + (c * 4 + blk) * 72 + sub;   // coefficient u of row sub at word 8u + sub
#pragma unroll
            for (int u = 0; u < 8; ++u) tile[8 * u] = F[u] >> 9;
        }
    }
    __syncwarp();

    // ---------------- phase 2: along y: forward DCT, quantiser, inverse DCT
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        int* tile = T + (c * 4 + blk) * 72;
        const int4 c0 = *reinterpret_cast<const int4*>(tile + 8 * sub);       // column sub, rows 0-3
        const int4 c1 = *reinterpret_cast<const int4*>(tile + 8 * sub + 4);   // rows 4-7
        const int Tc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
        int F[8], G[8];
        fdct8(Tc, F, 1 << 14);
        int L[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int f = F[v] >> 15;
            const uint32_t a = (uint32_t)(f < 0 ? -f : f);
            const int lvl = (int)__umulhi((a + (uint32_t)(K.qcol[v] >> 1)) << 8, K.qmcol[v]);
            L[v] = f < 0 ? -lvl : lvl;
            F[v] = L[v] * K.qcol[v];
        }
        if (kLevels && x0 < w) {
            const int bh = (h + 7) >> 3, bw = (w + 7) >> 3;
            const int64_t blk_idx = ((int64_t)c * bh + (y0 >> 3)) * bw + (x0 >> 3);
            int4 pk;
            pk.x = (int)(((uint32_t)L[0] & 0xffffu) | ((uint32_t)L[1] << 16));
            pk.y = (int)(((uint32_t)L[2] & 0xffffu) | ((uint32_t)L[3] << 16));
            pk.z = (int)(((uint32_t)L[4] & 0xffffu) | ((uint32_t)L[5] << 16));
            pk.w = (int)(((uint32_t)L[6] & 0xffffu) | ((uint32_t)L[7] << 16));
            *reinterpret_cast<int4*>(lv3 + blk_idx * 64 + sub * 8) = pk;
        }
        idct8(F, G, 1 << 8);
        __syncwarp();   // every lane has read its column before the rows are written
#pragma unroll
        for (int yy = 0; yy < 8; ++yy) tile[8 * yy + sub] = G[yy] >> 9;   // row yy, column sub
    }
    __syncwarp();

    // ---------------- phase 3: inverse DCT along x, store S
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int* tile = T + (c * 4 + blk) * 72 + 8 * sub;   // row sub
        const int4 g0 = *reinterpret_cast<const int4*>(tile);
        const int4 g1 = *reinterpret_cast<const int4*>(tile + 4);
        const int G[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
        int X[8];
        idct8(G, X, (1 << 14) + (128 << 15));
        uint32_t q[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) q[i] = (uint32_t)__vimin_s32_relu(X[i] >> 15, 255);
        const uint32_t lo = __byte_perm(__byte_perm(q[0], q[1], 0x0040), __byte_perm(q[2], q[3], 0x0040), 0x5410);
        const uint32_t hi = __byte_perm(__byte_perm(q[4], q[5], 0x0040), __byte_perm(q[6], q[7], 0x0040), 0x5410);
        if (x0 < w) store8(s3 + c * n, h, w, y, x0, fast, lo, hi, p);
    }
    __syncwarp();
}

// Copies this lane's bytes of band t (M_R, M_G, M_B, E: 8 each) into its
// prefetch slot and commits the copies as one group (an empty group when
// the band is not whole -- the right edge of a ragged image -- or the image
// has no 8-byte rows); false when nothing was copied.
__device__ __forceinline__ bool prefetch_band(const uint8_t* __restrict__ m3, const uint8_t* __restrict__ e, int h,
                                              int w, bool fast, int cols, int64_t t, int lane, uint2* slot,
                                              int p = 0) {
    // planes of h rows of pitch p (p = 0: p = w)
    p = p ? p : w;
    bool ok = false;
    if (fast) {
        const int y0 = (int)(t / cols) * 8, xb = (int)(t % cols) * 32;
        if (xb + 32 <= w) {
            const int y = min(y0 + (lane & 7), h - 1), x0 = xb + 8 * (lane >> 3);
            const int64_t n = (int64_t)h * p, off = (int64_t)y * p + x0;
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(slot);
            cp_async8(dst, m3 + off);
            cp_async8(dst + 256, m3 + n + off);
            cp_async8(dst + 512, m3 + 2 * n + off);
            cp_async8(dst + 768, e + off);
            ok = true;
        }
    }
    cp_async_commit();
    return ok;
}

template <bool kLevels, bool kWhite = false>
__global__ void __launch_bounds__(kThreads, kBaseCtas) k_base(const uint8_t* __restrict__ m3, const uint8_t* __restrict__ e,
                                                      int h, int w, const int64_t* __restrict__ lum_stats,
                                                      uint8_t* __restrict__ s3, uint8_t* __restrict__ sdr3,
                                                      int16_t* __restrict__ lv3, int fast_io, const QuantTable QT,
                                                      const float* __restrict__ l_white = nullptr) {
    __shared__ uint32_t gcode[kGammaWords];
    __shared__ __align__(16) int tile[kWarps][kTileWords];
    __shared__ __align__(16) uint2 pre[kWarps][2][4][32];   // [warp][slot][plane][lane]
    load_gamma(gcode);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BaseKey K;
    base_key(lum_stats, QT, lane & 7, K);
    float lw2 = 0.0f;
    if (kWhite) {
        const float lw = __ldg(l_white);
        lw2 = __fmul_rn(lw, lw);
    }
    const int cols = (w + 31) >> 5;
    const int64_t tasks = (int64_t)((h + 7) >> 3) * cols;
    const int64_t step = (int64_t)gridDim.x * kWarps;
    const bool fast = fast_io != 0;
    int64_t t = (int64_t)blockIdx.x * kWarps + warp;
    int slot = 0;
    bool have = t < tasks && prefetch_band(m3, e, h, w, fast, cols, t, lane, &pre[warp][0][0][lane]);
    while (t < tasks) {
        // the next band's copies go out before this band is processed
        const int64_t tn = t + step;
        const bool next = tn < tasks && prefetch_band(m3, e, h, w, fast, cols, tn, lane, &pre[warp][slot ^ 1][0][lane]);
        if (!next) cp_async_commit();   // keep one group per band, so "all but the newest" is this band's
        cp_async_wait_prev();
        base_band<kLevels, kWhite>(m3, e, h, w, fast, (int)(t / cols) * 8, (int)(t % cols) * 32, lane, K, gcode,
                                   tile[warp], s3, sdr3, have ? &pre[warp][slot][0][lane] : nullptr, lv3, lw2);
        t = tn;
        slot ^= 1;
        have = next;
    }
}

// Batch: CTA tasks of 8 band tasks of one image, contiguous ranges per CTA;
// a warp takes band (k - first task of the image) * 8 + warp of CTA task k.
// As in k_base, each warp copies its next band's bytes into shared memory
// (cp.async) while it processes the current one, across image changes too.
struct BatchBand {
    int img;            // -1: none
    int64_t t;          // band of the image, or past its last band
};

// Band of CTA task k for this warp; `img` tracks the image of the tasks
// seen last (they come in increasing order), so a lookup is one compare in
// the common case.
__device__ __forceinline__ BatchBand batch_band(const BatchDev& B, int64_t k, int warp, int& img) {
    if (img < 0) img = batch_image_of(B.base_prefix, B.n, k);
    while (B.base_prefix[img + 1] <= k) ++img;
    return BatchBand{img, (k - B.base_prefix[img]) * kWarps + warp};
}

__device__ __forceinline__ bool batch_fast(const BatchImage& im, const uint8_t* m3b, const uint8_t* eb,
                                           const uint8_t* s3b) {
    // pitched rows: 8-byte loads and stores are aligned wherever 8 columns lie inside the image
    return (im.pitch % 8 == 0) && ((uintptr_t)(m3b + 3 * im.px) % 8 == 0) && ((uintptr_t)(eb + im.px) % 8 == 0) &&
           ((uintptr_t)(s3b + 3 * im.px) % 8 == 0);
}

__device__ __forceinline__ bool batch_prefetch(const BatchDev& B, const BatchBand& b, const uint8_t* m3b,
                                               const uint8_t* eb, const uint8_t* s3b, int lane, uint2* slot) {
    const BatchImage im = B.img[b.img];
    const int cols = (im.w + 31) >> 5;
    const int64_t bands = (int64_t)((im.h + 7) >> 3) * cols;
    if ((int64_t)im.h * im.w == 0 || b.t >= bands) {
        cp_async_commit();
        return false;
    }
    return prefetch_band(m3b + 3 * im.px, eb + im.px, im.h, im.w, batch_fast(im, m3b, eb, s3b), cols, b.t, lane, slot,
                         im.pitch);
}

__global__ void __launch_bounds__(kThreads, 3) k_base_batch(const BatchDev B, int64_t cta_tasks,
                                                            const uint8_t* __restrict__ m3b,
                                                            const uint8_t* __restrict__ eb, uint8_t* __restrict__ s3b) {
    __shared__ uint32_t gcode[kGammaWords];
    __shared__ __align__(16) int tile[kWarps][kTileWords];
    __shared__ __align__(16) uint2 pre[kWarps][2][4][32];   // [warp][slot][plane][lane]
    load_gamma(gcode);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t per = (cta_tasks + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = (int64_t)blockIdx.x * per, k1 = min(k0 + per, cta_tasks);
    if (k0 >= k1) return;
    int cur = -1, slot = 0, track = -1;
    BaseKey K;
    BatchBand b = batch_band(B, k0, warp, track);
    bool have = batch_prefetch(B, b, m3b, eb, s3b, lane, &pre[warp][0][0][lane]);
    for (int64_t k = k0; k < k1; ++k) {
        // the next task's band goes out before this one is processed
        BatchBand nb{-1, 0};
        bool next = false;
        if (k + 1 < k1) {
            nb = batch_band(B, k + 1, warp, track);
            next = batch_prefetch(B, nb, m3b, eb, s3b, lane, &pre[warp][slot ^ 1][0][lane]);
        } else {
            cp_async_commit();   // one group per band, so "all but the newest" is this band's
        }
        cp_async_wait_prev();
        if (b.img != cur) {
            base_key(B.lum_stats + 2 * b.img, B.quant[b.img], lane & 7, K);
            cur = b.img;
        }
        const BatchImage im = B.img[b.img];
        const int cols = (im.w + 31) >> 5;
        const int64_t bands = (int64_t)((im.h + 7) >> 3) * cols;
        if ((int64_t)im.h * im.w > 0 && b.t < bands)
            base_band(m3b + 3 * im.px, eb + im.px, im.h, im.w, batch_fast(im, m3b, eb, s3b), (int)(b.t / cols) * 8,
                      (int)(b.t % cols) * 32, lane, K, gcode, tile[warp], s3b + 3 * im.px, nullptr,
                      have ? &pre[warp][slot][0][lane] : nullptr, nullptr, 0.0f, im.pitch);
        b = nb;
        have = next;
        slot ^= 1;
    }
}

}  // namespace

// ---------------------------------------------------------------- YCbCr 4:2:0 base layer
// The base layer with a default JPEG encoder's colour handling: the tone-
// mapped SDRI in YCbCr (T.871's equations in 16-bit fixed point, rounded
// half up, clamped), chroma averaged over 2x2 pixels (edges replicated,
// rounded half up), each plane through the 8x8 round trip (Y with the K.1
// table, Cb and Cr with K.2), chroma replicated back over its 2x2 pixels and
// converted to RGB:
//   Y  = (19595 R + 38470 G + 7471 B + 32768) >> 16
//   Cb = ((-11058 R - 21710 G + 32768 B + 32768) >> 16) + 128
//   Cr = ((32768 R - 27439 G - 5329 B + 32768) >> 16) + 128
//   R = Y + ((91881 (Cr - 128) + 32768) >> 16)
//   G = Y + ((-22554 (Cb - 128) - 46802 (Cr - 128) + 32768) >> 16)
//   B = Y + ((116130 (Cb - 128) + 32768) >> 16)
__device__ __forceinline__ int clamp255(int v) {
    return min(max(v, 0), 255);
}

// One thread per 2x2 cell: tone mapping, the colour transform, Y of the
// cell's pixels and the cell's chroma averages.
__global__ void __launch_bounds__(256) k_ycc420_fwd(const uint8_t* __restrict__ m3, const uint8_t* __restrict__ e,
                                                    int h, int w, const int64_t* __restrict__ lum_stats,
                                                    uint8_t* __restrict__ yp, uint8_t* __restrict__ cbp,
                                                    uint8_t* __restrict__ crp) {
    __shared__ uint32_t gcode[kGammaWords];
    load_gamma(gcode);
    int J, r;
    key_from_stats(lum_stats, &J, &r);
    const float kr = __uint_as_float(kKrBits[r]), wr = __uint_as_float(kWrBits[r]);
    const int hc = (h + 1) >> 1, wc = (w + 1) >> 1;
    const int cj = blockIdx.x * 32 + threadIdx.x, ci = blockIdx.y * 8 + threadIdx.y;
    if (ci >= hc || cj >= wc) return;
    const int64_t n = (int64_t)h * w;
    int sum_cb = 0, sum_cr = 0;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int y = min(2 * ci + dy, h - 1), x = min(2 * cj + dx, w - 1);
            const int64_t i = (int64_t)y * w + x;
            int R, G, B;
            tmo_pixel(__ldg(m3 + i), __ldg(m3 + n + i), __ldg(m3 + 2 * n + i), __ldg(e + i), J, kr, wr, gcode, R,
                      G, B);
            const int Y = clamp255((19595 * R + 38470 * G + 7471 * B + 32768) >> 16);
            sum_cb += clamp255(((-11058 * R - 21710 * G + 32768 * B + 32768) >> 16) + 128);
            sum_cr += clamp255(((32768 * R - 27439 * G - 5329 * B + 32768) >> 16) + 128);
            if (2 * ci + dy < h && 2 * cj + dx < w) yp[i] = (uint8_t)Y;
        }
    cbp[(int64_t)ci * wc + cj] = (uint8_t)((sum_cb + 2) >> 2);
    crp[(int64_t)ci * wc + cj] = (uint8_t)((sum_cr + 2) >> 2);
}

// The 8x8 round trip of single planes, in place: plane p (h[p] x w[p]) with
// the luminance steps for p = 0 and the chrominance steps otherwise; one warp
// per band of 8 rows x 32 columns as in base_band, without the tone mapping.
// levels (may be null): plane p's blocks from block lv_off[p], 64 levels
// each, coefficient (v, u) at u * 8 + v.
struct Planes420 {
    uint8_t* p[3];
    int h[3], w[3];
    int64_t lv_off[3];
};

__global__ void __launch_bounds__(kThreads) k_plane_rt(const Planes420 P, const QuantTable QY, const QuantTable QC,
                                                       int16_t* __restrict__ levels) {
    __shared__ __align__(16) int tiles[kWarps][4 * 72];
    const int pl = blockIdx.y;
    const QuantTable& Q = pl == 0 ? QY : QC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int blk = lane >> 3, sub = lane & 7;
    int qcol[8];
    uint32_t qmcol[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        qcol[v] = Q.q[v * 8 + sub];
        qmcol[v] = Q.qm[v * 8 + sub];
    }
    uint8_t* plane = P.p[pl];
    const int h = P.h[pl], w = P.w[pl];
    const int cols = (w + 31) >> 5, bw = (w + 7) >> 3;
    const int64_t tasks = (int64_t)((h + 7) >> 3) * cols;
    int* T = tiles[warp];
    for (int64_t t = (int64_t)blockIdx.x * kWarps + warp; t < tasks; t += (int64_t)gridDim.x * kWarps) {
        const int y0 = (int)(t / cols) * 8, xb = (int)(t % cols) * 32;
        const int x0 = xb + 8 * blk, y = y0 + sub;
        {
            uint8_t px[8];
            load8(plane, h, w, y, x0, false, px, w);   // rows and columns past the edge replicate it
            int X[8], F[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) X[i] = px[i];
            fdct8(X, F, 1 << 8);
            F[0] -= 1024 * C4;   // the level shift by -128 (only F[0] sees it)
            int* tile = T + blk * 72 + sub;
#pragma unroll
            for (int u = 0; u < 8; ++u) tile[8 * u] = F[u] >> 9;
        }
        __syncwarp();
        {
            int* tile = T + blk * 72;
            const int4 c0 = *reinterpret_cast<const int4*>(tile + 8 * sub);
            const int4 c1 = *reinterpret_cast<const int4*>(tile + 8 * sub + 4);
            const int Tc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
            int F[8], G[8], L[8];
            fdct8(Tc, F, 1 << 14);
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const int f = F[v] >> 15;
                const uint32_t a = (uint32_t)(f < 0 ? -f : f);
                const int lvl = (int)__umulhi((a + (uint32_t)(qcol[v] >> 1)) << 8, qmcol[v]);
                L[v] = f < 0 ? -lvl : lvl;
                F[v] = L[v] * qcol[v];
            }
            if (levels && x0 < w) {
                const int64_t b = P.lv_off[pl] + (int64_t)(y0 >> 3) * bw + (x0 >> 3);
                int4 pk;
                pk.x = (int)(((uint32_t)L[0] & 0xffffu) | ((uint32_t)L[1] << 16));
                pk.y = (int)(((uint32_t)L[2] & 0xffffu) | ((uint32_t)L[3] << 16));
                pk.z = (int)(((uint32_t)L[4] & 0xffffu) | ((uint32_t)L[5] << 16));
                pk.w = (int)(((uint32_t)L[6] & 0xffffu) | ((uint32_t)L[7] << 16));
                *reinterpret_cast<int4*>(levels + b * 64 + sub * 8) = pk;
            }
            idct8(F, G, 1 << 8);
            __syncwarp();
#pragma unroll
            for (int yy = 0; yy < 8; ++yy) tile[8 * yy + sub] = G[yy] >> 9;
        }
        __syncwarp();
        {
            const int* tile = T + blk * 72 + 8 * sub;
            const int4 g0 = *reinterpret_cast<const int4*>(tile);
            const int4 g1 = *reinterpret_cast<const int4*>(tile + 4);
            const int G[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
            int X[8];
            idct8(G, X, (1 << 14) + (128 << 15));
            uint32_t q[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) q[i] = (uint32_t)clamp255(X[i] >> 15);
            const uint32_t lo = q[0] | (q[1] << 8) | (q[2] << 16) | (q[3] << 24);
            const uint32_t hi = q[4] | (q[5] << 8) | (q[6] << 16) | (q[7] << 24);
            if (x0 < w) store8(plane, h, w, y, x0, false, lo, hi, w);
        }
        __syncwarp();
    }
}

// Chroma back over its 2x2 pixels and the inverse colour transform.
__global__ void __launch_bounds__(256) k_ycc420_inv(const uint8_t* __restrict__ yp, const uint8_t* __restrict__ cbp,
                                                    const uint8_t* __restrict__ crp, int h, int w,
                                                    uint8_t* __restrict__ s3) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= w || y >= h) return;
    const int wc = (w + 1) >> 1;
    const int64_t n = (int64_t)h * w, i = (int64_t)y * w + x, k = (int64_t)(y >> 1) * wc + (x >> 1);
    const int Y = __ldg(yp + i), cb = (int)__ldg(cbp + k) - 128, cr = (int)__ldg(crp + k) - 128;
    s3[i] = (uint8_t)clamp255(Y + ((91881 * cr + 32768) >> 16));
    s3[n + i] = (uint8_t)clamp255(Y + ((-22554 * cb - 46802 * cr + 32768) >> 16));
    s3[2 * n + i] = (uint8_t)clamp255(Y + ((116130 * cb + 32768) >> 16));
}

int launch_base_420(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats, const QuantTable& qy,
                    const QuantTable& qc, uint8_t* s_dec3, int16_t* levels, uint8_t* ws, cudaStream_t s) {
    const int hc = (h + 1) / 2, wc = (w + 1) / 2;
    const int64_t n = (int64_t)h * w, nc = (int64_t)hc * wc;
    uint8_t* yp = ws;
    uint8_t* cbp = ws + n;
    uint8_t* crp = cbp + nc;
    k_ycc420_fwd<<<dim3((unsigned)((wc + 31) / 32), (unsigned)((hc + 7) / 8)), dim3(32, 8), 0, s>>>(
        m3, e, h, w, lum_stats, yp, cbp, crp);
    Planes420 P;
    P.p[0] = yp;
    P.p[1] = cbp;
    P.p[2] = crp;
    P.h[0] = h;
    P.w[0] = w;
    P.h[1] = P.h[2] = hc;
    P.w[1] = P.w[2] = wc;
    const int64_t nbY = (int64_t)((h + 7) / 8) * ((w + 7) / 8), nbC = (int64_t)((hc + 7) / 8) * ((wc + 7) / 8);
    P.lv_off[0] = 0;
    P.lv_off[1] = nbY;
    P.lv_off[2] = nbY + nbC;
    const int64_t tasks = (int64_t)((h + 7) / 8) * ((w + 31) / 32);
    int64_t gx = (tasks + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)geometry().sms * 4;
    gx = gx < 1 ? 1 : (gx > cap ? cap : gx);
    k_plane_rt<<<dim3((unsigned)gx, 3), kThreads, 0, s>>>(P, qy, qc, levels);
    k_ycc420_inv<<<dim3((unsigned)((w + 31) / 32), (unsigned)((h + 7) / 8)), dim3(32, 8), 0, s>>>(yp, cbp, crp, h, w,
                                                                                                  s_dec3);
    return cuda_status("sdri_base_roundtrip_420 launch");
}

// The white point: the largest scaled luminance L over the pixels with
// E > 0, as the float bits (positive floats order like their bits), one
// atomic per warp.
__global__ void __launch_bounds__(256) k_white_point(const uint8_t* __restrict__ m3, const uint8_t* __restrict__ e,
                                                     int64_t n, const int64_t* __restrict__ lum_stats,
                                                     unsigned int* __restrict__ out) {
    int J, r;
    key_from_stats(lum_stats, &J, &r);
    const float kr = __uint_as_float(kKrBits[r]);
    unsigned int best = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int E = __ldg(e + i);
        float p2d;
        const float L = tmo_L(__ldg(m3 + i), __ldg(m3 + n + i), __ldg(m3 + 2 * n + i), E, J, kr, &p2d);
        if (E != 0) best = max(best, __float_as_uint(L));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}

int launch_white_point(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats, float* l_white,
                       cudaStream_t s) {
    if (cudaMemsetAsync(l_white, 0, sizeof(float), s) != cudaSuccess) return cuda_status("sdri_white_point clear");
    const int64_t n = (int64_t)h * w;
    if (n == 0) return SLRME_OK;
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)geometry().sms * 8;
    blocks = blocks > cap ? cap : blocks;
    k_white_point<<<(unsigned)blocks, 256, 0, s>>>(m3, e, n, lum_stats, reinterpret_cast<unsigned int*>(l_white));
    return cuda_status("sdri_white_point launch");
}

int launch_base_white(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats,
                      const float* l_white, const QuantTable& qt, uint8_t* s_dec3, uint8_t* sdr3, cudaStream_t s) {
    const int64_t n = (int64_t)h * w;
    const bool fast = (w % 8 == 0) && ((uintptr_t)m3 % 8 == 0) && ((uintptr_t)e % 8 == 0) &&
                      ((uintptr_t)s_dec3 % 8 == 0) && (!sdr3 || (uintptr_t)sdr3 % 8 == 0) && (n % 8 == 0);
    const int64_t tasks = (int64_t)((h + 7) / 8) * ((w + 31) / 32);
    int64_t blocks = (tasks + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)geometry().sms * kBaseCtas;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_base<false, true><<<(unsigned)blocks, kThreads, 0, s>>>(m3, e, h, w, lum_stats, s_dec3, sdr3, nullptr,
                                                              fast ? 1 : 0, qt, l_white);
    return cuda_status("sdri_base_roundtrip_white launch");
}

int launch_base(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats, const QuantTable& qt,
                uint8_t* s_dec3, uint8_t* sdr3, int16_t* levels3, cudaStream_t s) {
    const Geometry g = geometry();
    const int64_t n = (int64_t)h * w;
    const bool fast = (w % 8 == 0) && ((uintptr_t)m3 % 8 == 0) && ((uintptr_t)e % 8 == 0) &&
                      ((uintptr_t)s_dec3 % 8 == 0) && (!sdr3 || (uintptr_t)sdr3 % 8 == 0) && (n % 8 == 0);
    const int64_t tasks = (int64_t)((h + 7) / 8) * ((w + 31) / 32);
    int64_t blocks = (tasks + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)g.sms * kBaseCtas;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (levels3)
        k_base<true><<<(unsigned)blocks, kThreads, 0, s>>>(m3, e, h, w, lum_stats, s_dec3, sdr3, levels3,
                                                           fast ? 1 : 0, qt);
    else
        k_base<false><<<(unsigned)blocks, kThreads, 0, s>>>(m3, e, h, w, lum_stats, s_dec3, sdr3, nullptr,
                                                            fast ? 1 : 0, qt);
    return cuda_status("sdri_base_roundtrip launch");
}

}  // namespace slrme

namespace slrme {

int launch_base_batch(const BatchDev& B, int64_t cta_tasks, int ctas_per_sm, const uint8_t* m3, const uint8_t* e,
                      uint8_t* s3, cudaStream_t s) {
    if (cta_tasks == 0) return SLRME_OK;
    const int64_t cap = (int64_t)geometry().sms * (ctas_per_sm < 3 ? ctas_per_sm : 3);
    const int64_t g = cta_tasks < cap ? cta_tasks : cap;
    k_base_batch<<<(unsigned)(g < 1 ? 1 : g), kThreads, 0, s>>>(B, cta_tasks, m3, e, s3);
    return cuda_status("batch base launch");
}

}  // namespace slrme
