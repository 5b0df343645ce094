// Learned mantissa estimator: integer CNN inference on the tensor cores.
//
// Network (4 -> 16 -> 16 -> 16 -> 3, 3x3, zero padding, int8 weights and
// activations, int32 accumulation, per-channel requantisation) as declared
// in include/slrme.h.  One CTA computes a 15 x 56 output tile: the input tile
// with a 4-pixel halo (23 x 64) is staged in shared memory and the four
// layers run back to back, each as an implicit GEMM on the tensor cores
// (mma.sync.m16n8k16, f16 operands carrying the int8 values exactly, f32
// accumulators holding integers below 2^24 exactly: M = 16 pixels, N = 8
// output channels, K = 16 input channels per 3x3 tap).  On this GPU the
// int8 form of the same MMA (m16n8k32.s8) runs at a quarter of the f16
// rate, and tcgen05 has no int8 kind for sm_103a.
//
// Shared activations: 32 bytes per pixel (16 f16 channels; the two 16-byte
// halves swapped on every other group of 4 pixels, so ldmatrix rows and
// epilogue stores hit distinct banks), every layer's buffer with the same
// row pitch P = 64 pixels.  A layer's outputs are computed over the
// flattened index o = r P + x of its output rows, 16 at a time: the A rows
// of tap (dy, dx) are then the 16 consecutive input pixels from
// o + dy P + dx.  Columns x at or past the layer's output width are
// computed and stored but never read by a valid output of the next layer.
//
// Operand encoding: a hidden activation a in 0..127 is stored as the f16
// value 128 + a (bits 0x5800 + 8 a: no conversion instruction) and an
// input value v in -128..127 as 384 + v (bits 0x5C00 + 4 (v + 128)); zero
// padding is the encoded zero.  Each accumulator starts at -offset * (sum
// of the output channel's weights), so it ends at sum w a exactly
// (|sum w a| < 2^22, every partial sum below 2^24).
//
// Requantisation a' = clamp(floor((acc m + 2^(s-1)) / 2^s), 0, hi) with
// acc = b + sum w a: the float sum is turned into the integer
// 0x4B400000 + sum w a by adding 1.5 * 2^23 (exact below 2^22), and the
// per-channel constant (b - 0x4B400000) m + 2^(s-1) makes the product and
// all additions one 32 x 32 -> 64-bit multiply-add.  When m <= 2^(s+7) for
// every channel of the layer (|acc| < 2^24 then keeps the quotient inside
// int32) the low word of the 64-bit shift is the quotient and one
// min/max-with-zero instruction clamps it; otherwise the clamp reads the
// whole 64-bit quotient.
#include "slrme_internal.cuh"

namespace slrme {
namespace {

constexpr int TH = 15, TW = 56;                 // output tile
constexpr int P = TW + 8;                       // row pitch of every activation buffer (pixels)
constexpr int H0 = TH + 8;                      // rows of the input tile (halo 4)
constexpr int kThreadsC = 256, kWarpsC = 8;
constexpr int kBufAPx = H0 * P + 2;             // the input and layer-2 activations (+2: flattened overreach)
constexpr int kBufBPx = (H0 - 2) * P + 2;       // layer-1 and layer-3 activations
constexpr int GH = TH + 2, GW = TW + 2;         // S with a one-pixel halo, edges replicated (the filter's input)
constexpr int kNetBytes = 16 * 4 * 9 + 2 * 16 * 16 * 9 + 3 * 16 * 9;   // int8 weights of the four layers
constexpr size_t kOffB = (size_t)kBufAPx * 32;
constexpr size_t kOffHist = kOffB + (size_t)kBufBPx * 32;
constexpr size_t kOffCst = (kOffHist + 3 * kNres * 4 + 15) / 16 * 16;   // int64 [4][16]
constexpr size_t kOffMul = kOffCst + 4 * 16 * 8;              // int32 [4][16]
constexpr size_t kOffCor = kOffMul + 4 * 16 * 4;              // float [4][16]
constexpr size_t kOffNarrow = kOffCor + 4 * 16 * 4;           // int32 [4]
// B fragments (f16 pairs) of every layer, tap and n-tile, in lane order
constexpr int kFragWords = 2 * 32 * 9 * (2 + 2 + 2 + 1);
constexpr size_t kOffFrag = kOffNarrow + 16;
constexpr int kSmemBytes = (int)(kOffFrag + 4 * kFragWords);
__host__ __device__ constexpr int frag_base(int layer) { return 32 * 9 * 2 * layer; }   // in uint2 units
// after layer 3 the input buffer is free: the last layer's outputs and the
// staged S of the refinement live there
constexpr size_t kOffMh = 0;
constexpr size_t kOffSg = kOffMh + 3 * TH * TW;
static_assert(kOffSg + 3 * GH * GW <= (size_t)kBufAPx * 32, "refinement staging fits the input buffer");
static_assert(kNetBytes <= kBufAPx * 32, "the raw weights are staged in the input buffer");
static_assert(kOffB % 16 == 0 && kOffCst % 8 == 0, "cnn shared layout");
static_assert(2 * (kSmemBytes + 1024) <= 228 * 1024, "two CNN CTAs per SM");

enum Mode { kInfer = 0, kEncode = 1, kDecode = 2 };

__device__ __forceinline__ uint32_t swz(int pix, int chunk) {   // byte offset of (pixel, 16-byte chunk)
    return (uint32_t)(pix * 32 + ((chunk ^ ((pix >> 2) & 1)) << 4));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&a)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// f16 bits of an int8 weight (exact): sign, and |w| <= 127 as an f16 integer.
__device__ __forceinline__ uint32_t w_f16(int v) {
    const uint32_t a = (uint32_t)(v < 0 ? -v : v);
    // |w| = 2^e (1 + f): the f16 word for 1 <= |w| < 128, 0 for w = 0
    const int e = 31 - __clz((int)(a | 1u));
    const uint32_t bits = a ? (((uint32_t)(e + 15) << 10) | ((a << (10 - e)) & 0x3FFu)) : 0u;
    return bits | (v < 0 ? 0x8000u : 0u);
}

// Encoded operands (see above).
__device__ __forceinline__ uint32_t enc_in_pair(int v0, int v1) {   // inputs -128..127
    return (0x5C00u + 4u * (uint32_t)(v0 + 128)) | ((0x5C00u + 4u * (uint32_t)(v1 + 128)) << 16);
}
constexpr uint32_t kInZeroPair = 0x5E005E00u;    // two encoded input zeros (384)

struct LayerRef {
    int shift, hi;
};

// One layer over the tile: input rows HIN (pitch P) -> output rows HOUT =
// HIN - 2.  `halo` is the output's halo around the 15 x 56 tile; outputs
// outside the image are the encoded zero (the next layer's zero padding).
// The last layer writes its clamped values to `mh` (uint8 [3][TH][TW]).
template <int HIN, int NT, bool LAST>
__device__ __forceinline__ void conv_layer(uint32_t in_s, char* out_b, uint8_t* mh, const LayerRef& L, int layer,
                                           const uint2* frag, const long long* cst_s, const int* mul_s,
                                           const float* cor_s, const int* narrow_s, int halo, int oy, int ox, int h,
                                           int w) {
    constexpr int HOUT = HIN - 2;
    const int wout = P - 2 * (4 - halo);            // output width of this layer: 62, 60, 58, 56
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane & 3, g = lane >> 2;
    // B fragments of the nine taps (k = input channel, n = output channel), prepared per CTA
    uint32_t bf[9][NT][2];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const uint2 v = frag[frag_base(layer) + (t * NT + nt) * 32 + lane];
            bf[t][nt][0] = v.x;
            bf[t][nt][1] = v.y;
        }
    int mult[NT][2];
    long long cst[NT][2];
    float cor[NT][2];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int co = layer * 16 + nt * 8 + 2 * q + j;
            mult[nt][j] = mul_s[co];
            cst[nt][j] = cst_s[co];
            cor[nt][j] = cor_s[co];
        }
    const bool narrow = narrow_s[layer] != 0;
    const int s = L.shift;
    // this lane's A row (pixel) and 16-byte half
    const int ar = lane & 15, ah = lane >> 4;
    for (int c = warp; c < HOUT * (P / 16); c += kWarpsC) {
        const int o0 = 16 * c;
        float acc[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            acc[nt][0] = acc[nt][2] = cor[nt][0];
            acc[nt][1] = acc[nt][3] = cor[nt][1];
        }
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int pix = o0 + ar + (t / 3) * P + t % 3;
            uint32_t a[4];
            ldsm_x4(in_s + swz(pix, ah), a);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) mma16816(acc[nt], a, bf[t][nt][0], bf[t][nt][1]);
        }
        // epilogue: pixels o0 + g and o0 + g + 8, channels 2q, 2q + 1 of each n-tile
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            const int o = o0 + g + 8 * hf;
            const int r = o / P, x = o % P;
            const int gy = oy - halo + r, gx = ox - halo + x;
            const bool inside = x < wout && gy >= 0 && gy < h && gx >= 0 && gx < w;
            int y[NT][2];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int bits = __float_as_int(__fadd_rn(acc[nt][2 * hf + j], 12582912.0f));
                    const long long pv = (long long)bits * mult[nt][j] + cst[nt][j];
                    int z;
                    if (narrow) {
                        z = __vimin_s32_relu((int)(pv >> s), L.hi);
                    } else {
                        const long long zz = pv >> s;
                        z = zz < 0 ? 0 : (zz > L.hi ? L.hi : (int)zz);
                    }
                    y[nt][j] = inside ? z : 0;
                }
            if (LAST) {
                if (x < TW) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int co = 2 * q + j;
                        if (co < 3) mh[(co * TH + r) * TW + x] = (uint8_t)y[0][j];
                    }
                }
            } else {
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
                    *reinterpret_cast<uint32_t*>(out_b + swz(o, nt) + 4 * q) =
                        __byte_perm((uint32_t)y[nt][0], (uint32_t)y[nt][1], 0x5410) * 8u + 0x58005800u;
            }
        }
    }
}

struct CnnArgs {
    const uint8_t* s3;
    const uint8_t* e;
    const uint8_t* m3;     // encode: mantissas
    const int16_t* r3;     // decode: residuals
    uint8_t* mhat3;        // infer: predictions
    int16_t* r3_out;       // encode: residuals
    uint32_t* hist;        // encode: histograms (may be null)
    uint32_t* rgbe_out;    // decode: words
    const slrme_cnn_net* net;
    const slrme_params* params;   // encode / decode: the regression being refined
    int h, w, J, mode, gf_on;
};

// x = 16 S* (3x3 binomial, edge replicated) or 16 S at tile pixel (r, c) of
// one plane of the staged S (rows and columns with a one-pixel halo).
__device__ __forceinline__ int gf_tile(const uint8_t* Sg, int r, int c, bool gf) {
    const uint8_t* p = Sg + (r + 1) * GW + (c + 1);
    if (!gf) return 16 * (int)p[0];
    const int a = p[-GW - 1] + 2 * p[-GW] + p[-GW + 1];
    const int b = p[-1] + 2 * p[0] + p[1];
    const int d = p[GW - 1] + 2 * p[GW] + p[GW + 1];
    return a + 2 * b + d;
}

__global__ void __launch_bounds__(kThreadsC, 2) k_cnn(const CnnArgs A) {
    extern __shared__ __align__(128) char smem[];
    char* bufA = smem;
    char* bufB = smem + kOffB;
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + kOffHist);
    long long* cst_s = reinterpret_cast<long long*>(smem + kOffCst);
    int* mul_s = reinterpret_cast<int*>(smem + kOffMul);
    float* cor_s = reinterpret_cast<float*>(smem + kOffCor);
    int* narrow_s = reinterpret_cast<int*>(smem + kOffNarrow);
    uint2* frag = reinterpret_cast<uint2*>(smem + kOffFrag);
    int8_t* wsm = reinterpret_cast<int8_t*>(smem);   // the raw weights, staged in the input buffer at the start
    uint8_t* mh = reinterpret_cast<uint8_t*>(smem + kOffMh);
    uint8_t* Sg = reinterpret_cast<uint8_t*>(smem + kOffSg);     // [3][GH][GW]
    const uint32_t sA = (uint32_t)__cvta_generic_to_shared(bufA), sB = (uint32_t)__cvta_generic_to_shared(bufB);
    const int h = A.h, w = A.w;
    const int64_t n = (int64_t)h * w;
    const bool want_hist = A.mode == kEncode && A.hist;
    const bool gf = A.gf_on != 0;
    const float* pa = &A.params->a[0][0];   // regression slopes [3][256] (encode / decode)
    const float* pb = &A.params->b[0][0];   // intercepts

    const slrme_cnn_net* N = A.net;
    const LayerRef L1{N->shift[0], 127}, L2{N->shift[1], 127}, L3{N->shift[2], 127}, L4{N->shift[3], 255};
    // the network's B fragments, and per layer and output channel the
    // multiplier, the 64-bit constant and the accumulator's start value
    {
        const int8_t* src = &N->w1[0][0][0];   // w1..w4 are contiguous in the struct
        for (int i = threadIdx.x; i < kNetBytes; i += kThreadsC) wsm[i] = src[i];
        if (want_hist)
            for (int i = threadIdx.x; i < 3 * kNres; i += kThreadsC) hist[i] = 0u;
        __syncthreads();
        // fragment word (layer, tap t, n-tile nt, lane, j): f16 pair of w[n][c0][t], w[n][c0 + 1][t]
        // with n = 8 nt + lane / 4, c0 = 2 (lane % 4) + 8 j
        for (int i = threadIdx.x; i < kFragWords; i += kThreadsC) {
            int l = 0, k = i;
            while (l < 3 && k >= 2 * 32 * 9 * 2) {
                k -= 2 * 32 * 9 * 2;
                ++l;
            }
            const int NTl = l == 3 ? 1 : 2;
            const int j = k & 1, ln = (k >> 1) & 31, tn = k >> 6, t = tn / NTl, nt = tn % NTl;
            const int nco = l == 3 ? 3 : 16, nci = l == 0 ? 4 : 16;
            const int woff = l == 0 ? 0 : 16 * 4 * 9 + (l - 1) * 16 * 16 * 9;
            const int nn = nt * 8 + (ln >> 2), c0 = 2 * (ln & 3) + 8 * j;
            const int v0 = (nn < nco && c0 < nci) ? (int)wsm[woff + (nn * nci + c0) * 9 + t] : 0;
            const int v1 = (nn < nco && c0 + 1 < nci) ? (int)wsm[woff + (nn * nci + c0 + 1) * 9 + t] : 0;
            reinterpret_cast<uint32_t*>(frag)[i] = w_f16(v0) | (w_f16(v1) << 16);
        }
        if (threadIdx.x < 64) {
            const int l = threadIdx.x >> 4, co = threadIdx.x & 15;
            const int nco = l == 3 ? 3 : 16, nci = l == 0 ? 4 : 16, offset = l == 0 ? 384 : 128;
            const int woff = l == 0 ? 0 : 16 * 4 * 9 + (l - 1) * 16 * 16 * 9;
            const int32_t* bl = l == 0 ? N->b1 : (l == 1 ? N->b2 : (l == 2 ? N->b3 : N->b4));
            const int32_t* ml = l == 0 ? N->m1 : (l == 1 ? N->m2 : (l == 2 ? N->m3 : N->m4));
            const int sh = N->shift[l];
            const int m = co < nco ? ml[co] : 0, b = co < nco ? bl[co] : 0;
            int sw = 0;
            if (co < nco)
                for (int i = 0; i < nci * 9; ++i) sw += wsm[woff + co * nci * 9 + i];
            mul_s[threadIdx.x] = m;
            cst_s[threadIdx.x] = ((long long)b - 0x4B400000ll) * m + (1ll << (sh - 1));
            cor_s[threadIdx.x] = (float)(-offset * sw);
            const bool ok = (long long)m <= (1ll << (sh + 7));
            const unsigned all = __ballot_sync(0xffffffffu, ok);
            if ((threadIdx.x & 15) == 0) narrow_s[l] = ((all >> (threadIdx.x & 16)) & 0xFFFFu) == 0xFFFFu;
        }
        // (the first tile's barrier orders these writes before their use)
    }

    const int tiles_x = (w + TW - 1) / TW, tiles_y = (h + TH - 1) / TH;
    const int64_t tiles = (int64_t)tiles_x * tiles_y;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int oy = (int)(tile / tiles_x) * TH, ox = (int)(tile % tiles_x) * TW;
        __syncthreads();   // the previous tile's readers are done with the buffers
        // input tile: encoded (S - 128, key-relative exponent, 0 ...) per pixel; encoded zero outside the
        // image.  Every load of the thread's pixels is issued before the first is used.
        {
            constexpr int kIt = (H0 * P + kThreadsC - 1) / kThreadsC;
            int sv[kIt][4];
            bool in[kIt];
#pragma unroll
            for (int it = 0; it < kIt; ++it) {
                const int p = threadIdx.x + it * kThreadsC;
                const int gy = oy - 4 + p / P, gx = ox - 4 + p % P;
                in[it] = p < H0 * P && gy >= 0 && gy < h && gx >= 0 && gx < w;
                const int64_t o = in[it] ? (int64_t)gy * w + gx : 0;
                sv[it][0] = in[it] ? (int)A.s3[o] : 0;
                sv[it][1] = in[it] ? (int)A.s3[n + o] : 0;
                sv[it][2] = in[it] ? (int)A.s3[2 * n + o] : 0;
                sv[it][3] = in[it] ? (int)A.e[o] : 0;
            }
#pragma unroll
            for (int it = 0; it < kIt; ++it) {
                const int p = threadIdx.x + it * kThreadsC;
                if (p >= H0 * P) break;
                uint32_t v0 = kInZeroPair, v1 = kInZeroPair;
                if (in[it]) {
                    int d = sv[it][3] - 137 - A.J;
                    d = d < -128 ? -128 : (d > 127 ? 127 : d);
                    v0 = enc_in_pair(sv[it][0] - 128, sv[it][1] - 128);
                    v1 = enc_in_pair(sv[it][2] - 128, d);
                }
                *reinterpret_cast<uint4*>(bufA + swz(p, 0)) = make_uint4(v0, v1, 0u, 0u);
                *reinterpret_cast<uint4*>(bufA + swz(p, 1)) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        __syncthreads();
        conv_layer<H0, 2, false>(sA, bufB, nullptr, L1, 0, frag, cst_s, mul_s, cor_s, narrow_s, 3, oy, ox, h, w);
        __syncthreads();
        conv_layer<H0 - 2, 2, false>(sB, bufA, nullptr, L2, 1, frag, cst_s, mul_s, cor_s, narrow_s, 2, oy, ox, h,
                                     w);
        __syncthreads();
        conv_layer<H0 - 4, 2, false>(sA, bufB, nullptr, L3, 2, frag, cst_s, mul_s, cor_s, narrow_s, 1, oy, ox, h,
                                     w);
        __syncthreads();
        // S around the tile for the restoration filter (edges replicated), into the free input buffer
        if (A.mode != kInfer) {
            constexpr int kIt = (GH * GW + kThreadsC - 1) / kThreadsC;
            uint8_t sv[kIt][3];
#pragma unroll
            for (int it = 0; it < kIt; ++it) {
                const int p = min(threadIdx.x + it * kThreadsC, GH * GW - 1);
                const int gy = min(max(oy - 1 + p / GW, 0), h - 1), gx = min(max(ox - 1 + p % GW, 0), w - 1);
                const int64_t o = (int64_t)gy * w + gx;
#pragma unroll
                for (int c = 0; c < 3; ++c) sv[it][c] = A.s3[c * n + o];
            }
#pragma unroll
            for (int it = 0; it < kIt; ++it) {
                const int p = threadIdx.x + it * kThreadsC;
                if (p < GH * GW) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) Sg[c * GH * GW + p] = sv[it][c];
                }
            }
        }
        conv_layer<H0 - 6, 1, true>(sB, nullptr, mh, L4, 3, frag, cst_s, mul_s, cor_s, narrow_s, 0, oy, ox, h, w);
        __syncthreads();
        // outputs of the tile: a thread's pixels p = threadIdx.x + k * kThreadsC; the exponents and
        // the mantissas (encoder) or residuals (decoder) of all of them are loaded first
        {
            constexpr int kIt = (TH * TW + kThreadsC - 1) / kThreadsC;
            int Ev[kIt], in3[kIt][3];
            int64_t ov[kIt];
            bool ok[kIt];
#pragma unroll
            for (int k = 0; k < kIt; ++k) {
                const int p = threadIdx.x + k * kThreadsC;
                const int gy = oy + p / TW, gx = ox + p % TW;
                ok[k] = p < TH * TW && gy < h && gx < w;
                ov[k] = ok[k] ? (int64_t)gy * w + gx : 0;
                const int64_t o = ov[k];
                Ev[k] = ok[k] && A.mode != kInfer ? (int)A.e[o] : 0;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch)
                    in3[k][ch] = !ok[k] || A.mode == kInfer ? 0
                                 : (A.mode == kEncode ? (int)A.m3[ch * n + o] : (int)A.r3[ch * n + o]);
            }
#pragma unroll
            for (int k = 0; k < kIt; ++k) {
                if (!ok[k]) continue;
                const int p = threadIdx.x + k * kThreadsC;
                const int r = p / TW, c = p % TW;
                const int64_t o = ov[k];
                const int y3[3] = {mh[p], mh[TH * TW + p], mh[2 * TH * TW + p]};
                if (A.mode == kInfer) {
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) A.mhat3[ch * n + o] = (uint8_t)y3[ch];
                    continue;
                }
                // refined estimate: M^ = clamp(M* + y - 128, 0, 255), M* from Eq. (8)
                const int E = Ev[k];
                int mhat[3];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const int ms = predict(__ldg(pa + ch * kNbin + E), __ldg(pb + ch * kNbin + E),
                                           gf_tile(Sg + ch * GH * GW, r, c, gf));
                    const int v = ms + y3[ch] - 128;
                    mhat[ch] = v < 0 ? 0 : (v > 255 ? 255 : v);
                }
                if (A.mode == kEncode) {
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        const int rr = in3[k][ch] - mhat[ch];
                        A.r3_out[ch * n + o] = (int16_t)rr;
                        if (want_hist) atomicAdd(&hist[ch * kNres + rr + 255], 1u);
                    }
                } else {
                    uint32_t wd = (uint32_t)E << 24;
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) wd |= ((uint32_t)(in3[k][ch] + mhat[ch]) & 255u) << (8 * ch);
                    A.rgbe_out[o] = wd;
                }
            }
        }
    }
    if (want_hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * kNres; i += kThreadsC)
            if (hist[i]) atomicAdd(A.hist + i, hist[i]);
    }
}

int launch_cnn(const CnnArgs& A, cudaStream_t s) {
    // the kernel needs more than 48 KB of dynamic shared memory: opt in once per device
    static bool attr_set[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cuda_status("cnn device");
    if (!attr_set[dev]) {
        if (cudaFuncSetAttribute(k_cnn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess)
            return cuda_status("cnn smem attribute");
        attr_set[dev] = true;
    }
    const int64_t tiles = (int64_t)((A.w + TW - 1) / TW) * ((A.h + TH - 1) / TH);
    const int64_t cap = (int64_t)geometry().sms * 2;
    const int64_t g = tiles < cap ? tiles : cap;
    k_cnn<<<(unsigned)(g < 1 ? 1 : g), kThreadsC, kSmemBytes, s>>>(A);
    return cuda_status("cnn launch");
}

bool net_ok(const slrme_cnn_net* net) { return net && (uintptr_t)net % 4 == 0; }

}  // namespace
}  // namespace slrme

using namespace slrme;

extern "C" {

int cnn_infer(const uint8_t* s_dec3, const uint8_t* e, int h, int w, int32_t J, const slrme_cnn_net* net,
              uint8_t* mhat3, slrme_stream_t stream) {
    if (h < 0 || w < 0 || (int64_t)h * w >= ((int64_t)1 << 31) || !net_ok(net)) {
        set_error("cnn_infer: bad size or network pointer");
        return SLRME_EINVAL;
    }
    if ((int64_t)h * w == 0) return SLRME_OK;
    if (!s_dec3 || !e || !mhat3) {
        set_error("cnn_infer: null pointer");
        return SLRME_EINVAL;
    }
    CnnArgs A{s_dec3, e, nullptr, nullptr, mhat3, nullptr, nullptr, nullptr, net, nullptr, h, w, J, kInfer, 0};
    return launch_cnn(A, (cudaStream_t)stream);
}

int cnn_residual_encode(const uint8_t* s_dec3, const uint8_t* m3, const uint8_t* e, int h, int w, int32_t J,
                        const slrme_cnn_net* net, const slrme_params* params, int gf_on, int16_t* r3, uint32_t* hist,
                        slrme_stream_t stream) {
    if (h < 0 || w < 0 || (int64_t)h * w >= ((int64_t)1 << 31) || !net_ok(net) || (uintptr_t)r3 % 2 ||
        (uintptr_t)hist % 4 || !params || (uintptr_t)params % 4 || (gf_on != 0 && gf_on != 1)) {
        set_error("cnn_residual_encode: bad size, alignment or network pointer");
        return SLRME_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (hist && cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 3 * kNres, s) != cudaSuccess)
        return cuda_status("cnn_residual_encode memset");
    if ((int64_t)h * w == 0) return SLRME_OK;
    if (!s_dec3 || !m3 || !e || !r3) {
        set_error("cnn_residual_encode: null pointer");
        return SLRME_EINVAL;
    }
    CnnArgs A{s_dec3, e, m3, nullptr, nullptr, r3, hist, nullptr, net, params, h, w, J, kEncode, gf_on};
    return launch_cnn(A, s);
}

int cnn_residual_decode(const uint8_t* s_dec3, const uint8_t* e, const int16_t* r3, int h, int w, int32_t J,
                        const slrme_cnn_net* net, const slrme_params* params, int gf_on, uint32_t* rgbe_out,
                        slrme_stream_t stream) {
    if (h < 0 || w < 0 || (int64_t)h * w >= ((int64_t)1 << 31) || !net_ok(net) || (uintptr_t)r3 % 2 ||
        (uintptr_t)rgbe_out % 4 || !params || (uintptr_t)params % 4 || (gf_on != 0 && gf_on != 1)) {
        set_error("cnn_residual_decode: bad size, alignment or network pointer");
        return SLRME_EINVAL;
    }
    if ((int64_t)h * w == 0) return SLRME_OK;
    if (!s_dec3 || !e || !r3 || !rgbe_out) {
        set_error("cnn_residual_decode: null pointer");
        return SLRME_EINVAL;
    }
    CnnArgs A{s_dec3, e, nullptr, r3, nullptr, nullptr, nullptr, rgbe_out, net, params, h, w, J, kDecode, gf_on};
    return launch_cnn(A, (cudaStream_t)stream);
}

}  // extern "C"
