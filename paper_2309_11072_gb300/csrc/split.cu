// RGBE split (Sec. II-A, Sec. III-A) fused with the log-average luminance
// statistic of the tone-mapping operator.
//
// HBM-bound: 4 bytes read and 4 bytes written per pixel.  The vector path
// reads 16 bytes (4 words) per thread per step with non-allocating loads and
// writes one 32-bit word to each of the four planes; the byte transposition
// is 6 byte-permutes per 4 pixels.  The statistic of the vector path is
// 65536 (sum (E + k) - 137 n) + sum LUT16[m] over the nonzero pixels, the
// same integer as the per-pixel sum of l(p): Yq comes from two 16x8-bit dot
// products, the three partial sums are 32-bit per loop step and folded into
// int64 after it.  It is reduced per thread, then per warp and block, with
// one 64-bit atomic per block.
#include "slrme_internal.cuh"

#define SLRME_TABLE static __device__ const
#include "tables.inc"
#undef SLRME_TABLE

namespace slrme {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// l(p) of one word (0 for E = 0), from the table in shared memory.
__device__ __forceinline__ int32_t log_lum(uint32_t wd, const int32_t* lut) {
    const int E = (int)(wd >> 24);
    if (E == 0) return 0;
    const int yq = 2126 * (2 * (int)(wd & 255u) + 1) + 7152 * (2 * (int)((wd >> 8) & 255u) + 1) +
                   722 * (2 * (int)((wd >> 16) & 255u) + 1);
    const int k = (32 - __clz(yq)) - 12;        // bitlen(Yq) - 12, in [2, 11]
    const int m = yq >> k;                       // 2048 .. 4095
    return 65536 * (E - 137 + k) + lut[m - 2048];
}

// The statistic's parts for the four words of v: sl += LUT16[m], se += E + k
// and cn += 1 for each word with E > 0 (se also adds E = 0, which is 0).
// Yq = 4252 R + 14304 G + 1444 B + 10000 = 2126 (2R+1) + 7152 (2G+1) +
// 722 (2B+1); lut[m - 2048] is LUT16[m].
__device__ __forceinline__ void lum4(const uint4& v, const int32_t* lut, uint32_t& sl, uint32_t& se,
                                     uint32_t& cn) {
    const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t wd = w4[q];
        const uint32_t yq = __dp2a_hi(1444u, wd, __dp2a_lo(4252u | (14304u << 16), wd, 10000u));
        const uint32_t k = 20u - __clz(yq);   // bitlen(Yq) - 12, in [2, 11]
        const int32_t t = lut[(yq >> k) - 2048u];
        const bool nz = wd > 0xFFFFFFu;
        sl += nz ? (uint32_t)t : 0u;
        se += (wd >> 24) + (nz ? k : 0u);
        cn += nz ? 1u : 0u;
    }
}

__device__ __forceinline__ void block_reduce_add(int64_t s, int64_t c, int64_t* stats) {
    __shared__ int64_t red[2][kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = s;
        red[1][wid] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t ts = 0, tc = 0;
        for (int i = 0; i < kThreads / 32; ++i) {
            ts += red[0][i];
            tc += red[1][i];
        }
        if (tc != 0 || ts != 0) {
            atomicAdd(reinterpret_cast<unsigned long long*>(stats), (unsigned long long)ts);
            atomicAdd(reinterpret_cast<unsigned long long*>(stats + 1), (unsigned long long)tc);
        }
    }
    __syncthreads();   // `red` may be reused by the next call
}

// Vector path: n % 4 == 0, rgbe 16-byte aligned, planes 4-byte aligned.
__global__ void __launch_bounds__(kThreads) k_split_vec(const uint4* __restrict__ rgbe4, int64_t nv,
                                                        uint32_t* __restrict__ mR, uint32_t* __restrict__ mG,
                                                        uint32_t* __restrict__ mB, uint32_t* __restrict__ eP,
                                                        int64_t* __restrict__ stats) {
    __shared__ int32_t lut[2048];
    for (int i = threadIdx.x; i < 2048; i += kThreads) lut[i] = kLog2Lut[i];
    __syncthreads();

    int64_t sl64 = 0, se64 = 0, c = 0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    constexpr int U = 8;   // independent 16-byte loads in flight per thread
    // 32-bit parts per step: at most 32 words, each below 2^20 (LUT) and 267 (E + k)
    for (; i + (U - 1) * stride < nv; i += U * stride) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = ld_stream(rgbe4 + i + u * stride);
        uint32_t sl = 0, se = 0, cn = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t lo01 = __byte_perm(v[u].x, v[u].y, 0x5140), hi01 = __byte_perm(v[u].x, v[u].y, 0x7362);
            const uint32_t lo23 = __byte_perm(v[u].z, v[u].w, 0x5140), hi23 = __byte_perm(v[u].z, v[u].w, 0x7362);
            const int64_t j = i + u * stride;
            mR[j] = __byte_perm(lo01, lo23, 0x5410);
            mG[j] = __byte_perm(lo01, lo23, 0x7632);
            mB[j] = __byte_perm(hi01, hi23, 0x5410);
            eP[j] = __byte_perm(hi01, hi23, 0x7632);
            lum4(v[u], lut, sl, se, cn);
        }
        sl64 += sl;
        se64 += se;
        c += cn;
    }
    for (; i < nv; i += stride) {
        const uint4 v = ld_stream(rgbe4 + i);
        const uint32_t lo01 = __byte_perm(v.x, v.y, 0x5140), hi01 = __byte_perm(v.x, v.y, 0x7362);
        const uint32_t lo23 = __byte_perm(v.z, v.w, 0x5140), hi23 = __byte_perm(v.z, v.w, 0x7362);
        mR[i] = __byte_perm(lo01, lo23, 0x5410);
        mG[i] = __byte_perm(lo01, lo23, 0x7632);
        mB[i] = __byte_perm(hi01, hi23, 0x5410);
        eP[i] = __byte_perm(hi01, hi23, 0x7632);
        uint32_t sl = 0, se = 0, cn = 0;
        lum4(v, lut, sl, se, cn);
        sl64 += sl;
        se64 += se;
        c += cn;
    }
    block_reduce_add(65536 * (se64 - 137 * c) + sl64, c, stats);
}

// Scalar path: any size and alignment, one word per thread per step.
__global__ void __launch_bounds__(kThreads) k_split_scalar(const uint32_t* __restrict__ rgbe, int64_t n,
                                                           uint8_t* __restrict__ m3, uint8_t* __restrict__ e,
                                                           int64_t* __restrict__ stats) {
    __shared__ int32_t lut[2048];
    for (int i = threadIdx.x; i < 2048; i += kThreads) lut[i] = kLog2Lut[i];
    __syncthreads();
    int64_t s = 0, c = 0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
        const uint32_t wd = __ldg(rgbe + i);
        m3[i] = (uint8_t)(wd & 255u);
        m3[n + i] = (uint8_t)((wd >> 8) & 255u);
        m3[2 * n + i] = (uint8_t)((wd >> 16) & 255u);
        e[i] = (uint8_t)(wd >> 24);
        s += log_lum(wd, lut);
        c += (wd >> 24) != 0;
    }
    block_reduce_add(s, c, stats);
}


// Batch: one task per chunk of 4096 words of one image's pitched plane (the
// padding words are zero: no pixel, nothing added to the statistic); a CTA
// works through a contiguous range of chunks and adds each chunk's statistic
// to its image.
__global__ void __launch_bounds__(kThreads) k_split_batch(const BatchDev B, int64_t chunks,
                                                          const uint32_t* __restrict__ rgbeb,
                                                          uint8_t* __restrict__ m3b, uint8_t* __restrict__ eb) {
    __shared__ int32_t lut[2048];
    for (int i = threadIdx.x; i < 2048; i += kThreads) lut[i] = kLog2Lut[i];
    __syncthreads();
    const int64_t per = (chunks + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = (int64_t)blockIdx.x * per, k1 = min(k0 + per, chunks);
    // the statistic of the current image, added to its pair at each change
    // of image (the block's chunks are consecutive, so a block changes image
    // at most a few times)
    int cur = -1;
    int64_t s = 0, c = 0;
    int i = k0 < k1 ? batch_image_of(B.split_prefix, B.n, k0) : 0;
    for (int64_t k = k0; k < k1; ++k) {
        while (B.split_prefix[i + 1] <= k) ++i;   // chunks come in increasing order
        if (i != cur) {
            if (cur >= 0) block_reduce_add(s, c, B.lum_stats + 2 * cur);
            s = c = 0;
            cur = i;
        }
        const BatchImage im = B.img[i];
        const int64_t n = (int64_t)im.h * im.pitch;
        const int64_t w0 = (k - B.split_prefix[i]) * kSplitChunk, w1 = min(w0 + kSplitChunk, n);
        const uint32_t* rgbe = rgbeb + im.px;
        uint8_t* m3 = m3b + 3 * im.px;
        uint8_t* e = eb + im.px;
        const bool vec = (n % 4 == 0) && ((uintptr_t)rgbe % 16 == 0) && ((uintptr_t)m3 % 4 == 0) &&
                         ((uintptr_t)e % 4 == 0);
        if (vec) {
            // a chunk gives a thread kPer 16-byte units, all loaded before the first is used;
            // 32-bit parts per chunk
            constexpr int kPer = kSplitChunk / 4 / kThreads;
            static_assert(kSplitChunk / kThreads * (1 << 20) < (1ll << 32), "32-bit statistic parts");
            uint32_t sl = 0, se = 0, cn = 0;
            const uint4* r4 = reinterpret_cast<const uint4*>(rgbe);
            uint32_t* mR = reinterpret_cast<uint32_t*>(m3);
            uint32_t* mG = reinterpret_cast<uint32_t*>(m3 + n);
            uint32_t* mB = reinterpret_cast<uint32_t*>(m3 + 2 * n);
            uint32_t* eP = reinterpret_cast<uint32_t*>(e);
            uint4 v[kPer];
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const int64_t j = w0 / 4 + threadIdx.x + u * kThreads;
                v[u] = j < w1 / 4 ? ld_stream(r4 + j) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const int64_t j = w0 / 4 + threadIdx.x + u * kThreads;
                if (j < w1 / 4) {
                    const uint32_t lo01 = __byte_perm(v[u].x, v[u].y, 0x5140), hi01 = __byte_perm(v[u].x, v[u].y, 0x7362);
                    const uint32_t lo23 = __byte_perm(v[u].z, v[u].w, 0x5140), hi23 = __byte_perm(v[u].z, v[u].w, 0x7362);
                    mR[j] = __byte_perm(lo01, lo23, 0x5410);
                    mG[j] = __byte_perm(lo01, lo23, 0x7632);
                    mB[j] = __byte_perm(hi01, hi23, 0x5410);
                    eP[j] = __byte_perm(hi01, hi23, 0x7632);
                    lum4(v[u], lut, sl, se, cn);
                }
            }
            s += 65536 * ((int64_t)se - 137 * (int64_t)cn) + sl;
            c += cn;
        } else {
            for (int64_t j = w0 + threadIdx.x; j < w1; j += kThreads) {
                const uint32_t wd = __ldg(rgbe + j);
                m3[j] = (uint8_t)(wd & 255u);
                m3[n + j] = (uint8_t)((wd >> 8) & 255u);
                m3[2 * n + j] = (uint8_t)((wd >> 16) & 255u);
                e[j] = (uint8_t)(wd >> 24);
                s += log_lum(wd, lut);
                c += (wd >> 24) != 0;
            }
        }
    }
    if (cur >= 0) block_reduce_add(s, c, B.lum_stats + 2 * cur);
}

}  // namespace

int launch_split(const uint32_t* rgbe, int64_t n, uint8_t* m3, uint8_t* e, int64_t* lum_stats, cudaStream_t s) {
    const Geometry g = geometry();
    const bool vec = (n % 4 == 0) && ((uintptr_t)rgbe % 16 == 0) && ((uintptr_t)m3 % 4 == 0) &&
                     ((uintptr_t)e % 4 == 0);
    const int64_t units = vec ? n / 4 : n;
    int64_t blocks = (units + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)g.sms * 4;   // 4 resident blocks of 256 threads per SM
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (vec) {
        const int64_t nv = n / 4;
        k_split_vec<<<(unsigned)blocks, kThreads, 0, s>>>(
            reinterpret_cast<const uint4*>(rgbe), nv, reinterpret_cast<uint32_t*>(m3),
            reinterpret_cast<uint32_t*>(m3 + n), reinterpret_cast<uint32_t*>(m3 + 2 * n),
            reinterpret_cast<uint32_t*>(e), lum_stats);
    } else {
        k_split_scalar<<<(unsigned)blocks, kThreads, 0, s>>>(rgbe, n, m3, e, lum_stats);
    }
    return cuda_status("rgbe_split launch");
}

}  // namespace slrme

namespace slrme {

int launch_split_batch(const BatchDev& B, int64_t chunks, int ctas_per_sm, const uint32_t* rgbe, uint8_t* m3,
                       uint8_t* e, cudaStream_t s) {
    if (cudaMemsetAsync(B.lum_stats, 0, sizeof(int64_t) * 2 * (size_t)B.n, s) != cudaSuccess)
        return cuda_status("batch split memset");
    if (chunks == 0) return SLRME_OK;
    const int64_t cap = (int64_t)geometry().sms * ctas_per_sm;
    const int64_t g = chunks < cap ? chunks : cap;
    k_split_batch<<<(unsigned)(g < 1 ? 1 : g), kThreads, 0, s>>>(B, chunks, rgbe, m3, e);
    return cuda_status("batch split launch");
}

}  // namespace slrme
