// Learned mantissa estimator: integer CNN inference on the tensor cores.
//
// Network (4 -> 16 -> 16 -> 16 -> 3, 3x3, zero padding, int8 weights and
// activations, int32 accumulation, per-channel requantisation) as declared
// in include/slrme.h.  One CTA computes a 16 x 32 output tile: the input tile
// with a 4-pixel halo is staged in shared memory and the four layers run
// back to back, each as an implicit GEMM (M = 16 pixels of a row, N = 8
// output channels, K = 16 input channels per 3x3 tap) with ldmatrix and
// mma.sync.m16n8k16.  int8 values are carried exactly in f16; products and
// sums are integers below 2^24 (at most 144 * 127 * 127), so the f32
// accumulator holds them exactly and the integer requantisation follows.
//
// Shared activations: 32 bytes per pixel (16 f16 channels), the two 16-byte
// halves swapped on every other group of 4 pixels so that both ldmatrix rows
// and epilogue stores hit distinct banks.
#include <cuda_fp16.h>

#include "slrme_internal.cuh"

namespace slrme {
namespace {

constexpr int TH = 16, TW = 32;                 // output tile
constexpr int H0 = TH + 8, W0 = TW + 8;         // input tile (halo 4)
constexpr int H1 = TH + 6, W1 = TW + 6;
constexpr int H2 = TH + 4, W2 = TW + 4;
constexpr int H3 = TH + 2, W3 = TW + 2;
constexpr int kThreadsC = 256, kWarpsC = 8;
constexpr int kBufAPx = H0 * W0;                // holds the input and layer-2 activations
constexpr int kBufBPx = H1 * W1;                // holds layer-1 and layer-3 activations
constexpr int kSmemBytes = (kBufAPx + kBufBPx) * 32 + 3 * TH * TW + 3 * kNres * 4 + 2 * 3 * kNbin * 4;

enum Mode { kInfer = 0, kEncode = 1, kDecode = 2 };

__device__ __forceinline__ uint32_t swz(int pix, int chunk) {   // byte offset of (pixel, 16-byte chunk)
    return (uint32_t)(pix * 32 + ((chunk ^ ((pix >> 2) & 1)) << 4));
}

__device__ __forceinline__ uint32_t pack_h2(int lo, int hi) {
    const __half2 h = __halves2half2(__int2half_rn(lo), __int2half_rn(hi));
    return *reinterpret_cast<const uint32_t*>(&h);
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

struct LayerRef {
    const int8_t* w;     // [co][ci][9]
    const int32_t* b;    // [co]
    const int32_t* m;    // [co]
    int ci, co, shift, hi;
};

// One layer over the tile: input buffer HIN x WIN -> output HOUT x WOUT
// (HOUT = HIN - 2).  `halo` is the output's halo around the 16 x 32 tile;
// outputs outside the image are zero (the next layer's zero padding).  The
// last layer writes its clamped values to `mh` (uint8 [3][TH][TW]).
template <int HIN, int WIN, int NT, bool LAST>
__device__ __forceinline__ void conv_layer(uint32_t in_s, char* out_b, uint8_t* mh, const LayerRef& L, int halo,
                                           int oy, int ox, int h, int w) {
    constexpr int HOUT = HIN - 2, WOUT = WIN - 2;
    constexpr int G = (WOUT + 15) / 16;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane & 3, r4 = lane >> 2;
    // B fragments of all 9 taps: k = input channel, n = output channel
    uint32_t bf[9][NT][2];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int n = nt * 8 + r4;
            int v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int ci = 2 * q + (j & 1) + 8 * (j >> 1);
                v[j] = (n < L.co && ci < L.ci) ? (int)__ldg(L.w + (n * L.ci + ci) * 9 + t) : 0;
            }
            bf[t][nt][0] = pack_h2(v[0], v[1]);
            bf[t][nt][1] = pack_h2(v[2], v[3]);
        }
    int bias[NT][2], mult[NT][2];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int co = nt * 8 + 2 * q + j;
            bias[nt][j] = co < L.co ? __ldg(L.b + co) : 0;
            mult[nt][j] = co < L.co ? __ldg(L.m + co) : 0;
        }
    const long long rnd = 1ll << (L.shift - 1);
    for (int it = warp; it < HOUT * G; it += kWarpsC) {
        const int r = it / G;
        const int x0 = min((it % G) * 16, WOUT - 16);
        float acc[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int pix = (r + t / 3) * WIN + x0 + t % 3 + (lane & 15);
            uint32_t a[4];
            ldsm_x4(in_s + swz(pix, lane >> 4), a);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) mma16816(acc[nt], a, bf[t][nt][0], bf[t][nt][1]);
        }
        // epilogue: rows r4 and r4 + 8 of the group, channels 2q, 2q + 1 of each n-tile
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int xo = x0 + r4 + 8 * half;
            const int gy = oy - halo + r, gx = ox - halo + xo;
            const bool inside = gy >= 0 && gy < h && gx >= 0 && gx < w;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                int y[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const long long v = (long long)(__float2int_rn(acc[nt][2 * half + j]) + bias[nt][j]);
                    long long z = (v * mult[nt][j] + rnd) >> L.shift;
                    z = z < 0 ? 0 : (z > L.hi ? L.hi : z);
                    y[j] = inside ? (int)z : 0;
                }
                if (LAST) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int co = nt * 8 + 2 * q + j;
                        if (co < 3) mh[(co * TH + r) * TW + xo] = (uint8_t)y[j];
                    }
                } else {
                    const int pix = r * WOUT + xo;
                    *reinterpret_cast<uint32_t*>(out_b + swz(pix, nt) + 4 * q) = pack_h2(y[0], y[1]);
                }
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

// x = 16 S* (3x3 binomial, edge replicated) or 16 S at one pixel of one plane.
__device__ __forceinline__ int gf_at(const uint8_t* __restrict__ S, int h, int w, int y, int x, bool gf) {
    if (!gf) return 16 * (int)S[(int64_t)y * w + x];
    int acc = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const int yy = min(max(y + dy, 0), h - 1);
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int xx = min(max(x + dx, 0), w - 1);
            acc += (2 - (dy != 0)) * (2 - (dx != 0)) * (int)S[(int64_t)yy * w + xx];
        }
    }
    return acc;
}

__global__ void __launch_bounds__(kThreadsC, 2) k_cnn(const CnnArgs A) {
    extern __shared__ __align__(128) char smem[];
    char* bufA = smem;
    char* bufB = smem + kBufAPx * 32;
    uint8_t* mh = reinterpret_cast<uint8_t*>(bufB + kBufBPx * 32);
    uint32_t* hist = reinterpret_cast<uint32_t*>(mh + 3 * TH * TW);
    float* pa = reinterpret_cast<float*>(hist + 3 * kNres);      // regression slopes [3][256]
    float* pb = pa + 3 * kNbin;                                   // intercepts [3][256]
    const uint32_t sA = (uint32_t)__cvta_generic_to_shared(bufA), sB = (uint32_t)__cvta_generic_to_shared(bufB);
    const int h = A.h, w = A.w;
    const int64_t n = (int64_t)h * w;
    const bool want_hist = A.mode == kEncode && A.hist;
    if (want_hist)
        for (int i = threadIdx.x; i < 3 * kNres; i += kThreadsC) hist[i] = 0u;
    if (A.mode != kInfer)
        for (int i = threadIdx.x; i < 3 * kNbin; i += kThreadsC) {
            pa[i] = (&A.params->a[0][0])[i];
            pb[i] = (&A.params->b[0][0])[i];
        }

    const slrme_cnn_net* N = A.net;
    const LayerRef L1{&N->w1[0][0][0], N->b1, N->m1, 4, 16, N->shift[0], 127};
    const LayerRef L2{&N->w2[0][0][0], N->b2, N->m2, 16, 16, N->shift[1], 127};
    const LayerRef L3{&N->w3[0][0][0], N->b3, N->m3, 16, 16, N->shift[2], 127};
    const LayerRef L4{&N->w4[0][0][0], N->b4, N->m4, 16, 3, N->shift[3], 255};

    const int tiles_x = (w + TW - 1) / TW, tiles_y = (h + TH - 1) / TH;
    const int64_t tiles = (int64_t)tiles_x * tiles_y;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int oy = (int)(tile / tiles_x) * TH, ox = (int)(tile % tiles_x) * TW;
        __syncthreads();   // the previous tile's readers are done with the buffers
        // input tile: S - 128 and the key-relative exponent; zero outside the image
        for (int p = threadIdx.x; p < kBufAPx; p += kThreadsC) {
            const int gy = oy - 4 + p / W0, gx = ox - 4 + p % W0;
            uint4 lo = make_uint4(0u, 0u, 0u, 0u);
            if (gy >= 0 && gy < h && gx >= 0 && gx < w) {
                const int64_t o = (int64_t)gy * w + gx;
                int d = (int)A.e[o] - 137 - A.J;
                d = d < -128 ? -128 : (d > 127 ? 127 : d);
                lo.x = pack_h2((int)A.s3[o] - 128, (int)A.s3[n + o] - 128);
                lo.y = pack_h2((int)A.s3[2 * n + o] - 128, d);
            }
            *reinterpret_cast<uint4*>(bufA + swz(p, 0)) = lo;
            *reinterpret_cast<uint4*>(bufA + swz(p, 1)) = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        conv_layer<H0, W0, 2, false>(sA, bufB, nullptr, L1, 3, oy, ox, h, w);
        __syncthreads();
        conv_layer<H1, W1, 2, false>(sB, bufA, nullptr, L2, 2, oy, ox, h, w);
        __syncthreads();
        conv_layer<H2, W2, 2, false>(sA, bufB, nullptr, L3, 1, oy, ox, h, w);
        __syncthreads();
        conv_layer<H3, W3, 1, true>(sB, nullptr, mh, L4, 0, oy, ox, h, w);
        __syncthreads();
        // outputs of the tile, one pixel per thread per step
        for (int p = threadIdx.x; p < TH * TW; p += kThreadsC) {
            const int gy = oy + p / TW, gx = ox + p % TW;
            if (gy >= h || gx >= w) continue;
            const int64_t o = (int64_t)gy * w + gx;
            int y3[3] = {mh[p], mh[TH * TW + p], mh[2 * TH * TW + p]};
            if (A.mode == kInfer) {
#pragma unroll
                for (int c = 0; c < 3; ++c) A.mhat3[c * n + o] = (uint8_t)y3[c];
                continue;
            }
            // refined estimate: M^ = clamp(M* + y - 128, 0, 255), M* from Eq. (8)
            const int E = A.e[o];
            int mhat[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int ms = predict(pa[c * kNbin + E], pb[c * kNbin + E], gf_at(A.s3 + c * n, h, w, gy, gx,
                                                                                    A.gf_on != 0));
                const int v = ms + y3[c] - 128;
                mhat[c] = v < 0 ? 0 : (v > 255 ? 255 : v);
            }
            if (A.mode == kEncode) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int r = (int)A.m3[c * n + o] - mhat[c];
                    A.r3_out[c * n + o] = (int16_t)r;
                    if (want_hist) atomicAdd(&hist[c * kNres + r + 255], 1u);
                }
            } else {
                uint32_t wd = (uint32_t)E << 24;
#pragma unroll
                for (int c = 0; c < 3; ++c) wd |= ((uint32_t)((int)A.r3[c * n + o] + mhat[c]) & 255u) << (8 * c);
                A.rgbe_out[o] = wd;
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
