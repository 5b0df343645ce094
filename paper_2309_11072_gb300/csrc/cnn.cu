// Learned mantissa estimator: integer CNN inference on the tensor cores.
//
// Network (4 -> 16 -> 16 -> 16 -> 3, 3x3, zero padding, int8 weights and
// activations, int32 accumulation, per-channel requantisation) as declared
// in include/slrme.h.  One CTA computes a 32 x 56 output tile: the input tile
// with a 4-pixel halo (40 x 64) is staged in shared memory and the four
// layers run back to back, each as an implicit GEMM on the int8 tensor path
// (mma.sync.m16n8k32.s32.s8.s8.s32: M = 16 pixels, N = 8 output channels,
// K = 32 = two 3x3 taps of 16 input channels, int32 accumulators).
//
// Shared activations: 16 bytes per pixel (16 int8 channels), every layer's
// buffer with the same row pitch P = 64 pixels.  A layer's outputs are
// computed over the flattened index o = r P + x of its output rows, 16 at a
// time: the A rows of tap (dy, dx) are then the 16 consecutive input pixels
// from o + dy P + dx, one ldmatrix row (16 bytes) each, so an ldmatrix.x4
// loads two taps at once (lanes 0-15 one tap, 16-31 the other).  Columns x
// at or past the layer's output width are computed and stored but never
// read by a valid output of the next layer.
//
// Requantisation a' = clamp(floor((acc m + 2^(s-1)) / 2^s), 0, hi): the MMA
// gives sum w a; (b m + 2^(s-1)) is a per-channel 64-bit constant, so the
// product and both additions are one 32 x 32 -> 64-bit multiply-add.  When
// m <= 2^(s+7) for every channel of the layer (|acc| < 2^24 then keeps the
// quotient inside int32), the low word of the 64-bit shift is the quotient
// and one min/max-with-zero instruction clamps it; otherwise the clamp
// reads the whole 64-bit quotient.
#include "slrme_internal.cuh"

namespace slrme {
namespace {

constexpr int TH = 32, TW = 56;                 // output tile
constexpr int P = TW + 8;                       // row pitch of every activation buffer (pixels)
constexpr int H0 = TH + 8;                      // rows of the input tile (halo 4)
constexpr int kThreadsC = 256, kWarpsC = 8;
constexpr int kBufAPx = H0 * P + 2;             // the input and layer-2 activations (+2: flattened overreach)
constexpr int kBufBPx = (H0 - 2) * P + 2;       // layer-1 and layer-3 activations
constexpr int GH = TH + 2, GW = TW + 2;         // S with a one-pixel halo, edges replicated (the filter's input)
constexpr size_t kOffB = (size_t)kBufAPx * 16;
constexpr size_t kOffMh = kOffB + (size_t)kBufBPx * 16;
constexpr size_t kOffHist = kOffMh + 3 * TH * TW;
constexpr size_t kOffPa = kOffHist + 3 * kNres * 4;
constexpr size_t kOffSg = kOffPa + 2 * 3 * kNbin * 4;
constexpr int kSmemBytes = (int)(kOffSg + 3 * GH * GW);
static_assert(kOffB % 16 == 0 && kOffPa % 4 == 0, "cnn shared layout");
static_assert(2 * (kSmemBytes + 1024) <= 228 * 1024, "two CNN CTAs per SM");

enum Mode { kInfer = 0, kEncode = 1, kDecode = 2 };

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&a)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}

// D += A B, A 16 x 32 int8 (row), B 32 x 8 int8 (column), D 16 x 8 int32.
__device__ __forceinline__ void mma_s8(int (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack4_s8(int a, int b, int c, int d) {
    return ((uint32_t)a & 255u) | (((uint32_t)b & 255u) << 8) | (((uint32_t)c & 255u) << 16) | ((uint32_t)d << 24);
}

struct LayerRef {
    const int8_t* w;     // [co][ci][9]
    const int32_t* b;    // [co]
    const int32_t* m;    // [co]
    int ci, co, shift, hi;
};

// One layer over the tile: input rows HIN (pitch P) -> output rows HOUT =
// HIN - 2.  `halo` is the output's halo around the 32 x 56 tile; outputs
// outside the image are zero (the next layer's zero padding).  The last
// layer writes its clamped values to `mh` (uint8 [3][TH][TW]).
template <int HIN, int NT, bool LAST>
__device__ __forceinline__ void conv_layer(uint32_t in_s, char* out_b, uint8_t* mh, const LayerRef& L, int halo,
                                           int oy, int ox, int h, int w) {
    constexpr int HOUT = HIN - 2;
    const int wout = P - 2 * (4 - halo);            // output width of this layer: 62, 60, 58, 56
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane & 3, g = lane >> 2;
    // B fragments of the five tap pairs (taps 2p, 2p + 1; tap 9 is zero):
    // k = 16 * (tap - 2p) + input channel, n = output channel
    uint32_t bf[5][NT][2];
#pragma unroll
    for (int pr = 0; pr < 5; ++pr)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int n = nt * 8 + g;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int t = 2 * pr + half;
                int v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int ci = 4 * q + i;
                    v[i] = (t < 9 && n < L.co && ci < L.ci) ? (int)__ldg(L.w + (n * L.ci + ci) * 9 + t) : 0;
                }
                bf[pr][nt][half] = pack4_s8(v[0], v[1], v[2], v[3]);
            }
        }
    // per output channel (2q + j of n-tile nt): m and b m + 2^(s-1)
    const int s = L.shift;
    int mult[NT][2];
    long long cst[NT][2];
    bool narrow = true;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int co = nt * 8 + 2 * q + j;
            const int m = co < L.co ? __ldg(L.m + co) : 0;
            const int b = co < L.co ? __ldg(L.b + co) : 0;
            mult[nt][j] = m;
            cst[nt][j] = (long long)b * m + (1ll << (s - 1));
            narrow = narrow && (long long)m <= (1ll << (s + 7));
        }
    narrow = __all_sync(0xffffffffu, narrow);
    // this lane's A row offsets (pixels) for the five tap pairs
    int off[5];
#pragma unroll
    for (int pr = 0; pr < 5; ++pr) {
        const int t = min(2 * pr + (lane >> 4), 8);
        off[pr] = (lane & 15) + (t / 3) * P + t % 3;
    }
    for (int c = warp; c < HOUT * (P / 16); c += kWarpsC) {
        const int o0 = 16 * c;
        int acc[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0;
#pragma unroll
        for (int pr = 0; pr < 5; ++pr) {
            uint32_t a[4];
            ldsm_x4(in_s + 16u * (uint32_t)(o0 + off[pr]), a);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) mma_s8(acc[nt], a, bf[pr][nt][0], bf[pr][nt][1]);
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
                    const long long pv = (long long)acc[nt][2 * hf + j] * mult[nt][j] + cst[nt][j];
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
                if (x < TW && r < TH) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int co = 2 * q + j;
                        if (co < 3) mh[(co * TH + r) * TW + x] = (uint8_t)y[0][j];
                    }
                }
            } else {
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
                    *reinterpret_cast<uint16_t*>(out_b + 16 * o + 8 * nt + 2 * q) =
                        (uint16_t)((y[nt][0] & 255) | (y[nt][1] << 8));
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
    uint8_t* mh = reinterpret_cast<uint8_t*>(smem + kOffMh);
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + kOffHist);
    float* pa = reinterpret_cast<float*>(smem + kOffPa);         // regression slopes [3][256]
    float* pb = pa + 3 * kNbin;                                   // intercepts [3][256]
    uint8_t* Sg = reinterpret_cast<uint8_t*>(smem + kOffSg);     // [3][GH][GW]
    const uint32_t sA = (uint32_t)__cvta_generic_to_shared(bufA), sB = (uint32_t)__cvta_generic_to_shared(bufB);
    const int h = A.h, w = A.w;
    const int64_t n = (int64_t)h * w;
    const bool want_hist = A.mode == kEncode && A.hist;
    const bool gf = A.gf_on != 0;
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
        // input tile: (S - 128, key-relative exponent, 0 ...) per pixel; zero outside the image
        for (int p = threadIdx.x; p < H0 * P; p += kThreadsC) {
            const int gy = oy - 4 + p / P, gx = ox - 4 + p % P;
            uint32_t v = 0u;
            if (gy >= 0 && gy < h && gx >= 0 && gx < w) {
                const int64_t o = (int64_t)gy * w + gx;
                int d = (int)A.e[o] - 137 - A.J;
                d = d < -128 ? -128 : (d > 127 ? 127 : d);
                v = pack4_s8((int)A.s3[o] - 128, (int)A.s3[n + o] - 128, (int)A.s3[2 * n + o] - 128, d);
            }
            *reinterpret_cast<uint4*>(bufA + 16 * p) = make_uint4(v, 0u, 0u, 0u);
        }
        // S around the tile for the restoration filter (edges replicated)
        if (A.mode != kInfer)
            for (int p = threadIdx.x; p < GH * GW; p += kThreadsC) {
                const int gy = min(max(oy - 1 + p / GW, 0), h - 1), gx = min(max(ox - 1 + p % GW, 0), w - 1);
                const int64_t o = (int64_t)gy * w + gx;
#pragma unroll
                for (int c = 0; c < 3; ++c) Sg[c * GH * GW + p] = A.s3[c * n + o];
            }
        __syncthreads();
        conv_layer<H0, 2, false>(sA, bufB, nullptr, L1, 3, oy, ox, h, w);
        __syncthreads();
        conv_layer<H0 - 2, 2, false>(sB, bufA, nullptr, L2, 2, oy, ox, h, w);
        __syncthreads();
        conv_layer<H0 - 4, 2, false>(sA, bufB, nullptr, L3, 1, oy, ox, h, w);
        __syncthreads();
        conv_layer<H0 - 6, 1, true>(sB, nullptr, mh, L4, 0, oy, ox, h, w);
        __syncthreads();
        // outputs of the tile, one pixel per thread per step
        for (int p = threadIdx.x; p < TH * TW; p += kThreadsC) {
            const int r = p / TW, c = p % TW;
            const int gy = oy + r, gx = ox + c;
            if (gy >= h || gx >= w) continue;
            const int64_t o = (int64_t)gy * w + gx;
            int y3[3] = {mh[p], mh[TH * TW + p], mh[2 * TH * TW + p]};
            if (A.mode == kInfer) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) A.mhat3[ch * n + o] = (uint8_t)y3[ch];
                continue;
            }
            // refined estimate: M^ = clamp(M* + y - 128, 0, 255), M* from Eq. (8)
            const int E = A.e[o];
            int mhat[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const int ms = predict(pa[ch * kNbin + E], pb[ch * kNbin + E], gf_tile(Sg + ch * GH * GW, r, c, gf));
                const int v = ms + y3[ch] - 128;
                mhat[ch] = v < 0 ? 0 : (v > 255 ? 255 : v);
            }
            if (A.mode == kEncode) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const int rr = (int)A.m3[ch * n + o] - mhat[ch];
                    A.r3_out[ch * n + o] = (int16_t)rr;
                    if (want_hist) atomicAdd(&hist[ch * kNres + rr + 255], 1u);
                }
            } else {
                uint32_t wd = (uint32_t)E << 24;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) wd |= ((uint32_t)((int)A.r3[ch * n + o] + mhat[ch]) & 255u) << (8 * ch);
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
