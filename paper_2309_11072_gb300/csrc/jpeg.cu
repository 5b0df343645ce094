// Base-layer entropy coding: the size of the JPEG baseline Huffman coding
// (T.81 Annex F.1.2) of the base layer's quantised levels, with the typical
// luminance tables of T.81 Annex K.3 (Tables K.3 and K.5).  Sec. IV codes the
// base layer with JPEG; each colour plane is a single-component scan of its
// 8x8 blocks in raster order.
//   DC: diff = level_DC - level_DC of the plane's previous block (0 before the
//       first); category SSSS = bit length of |diff|; cost = DC code length of
//       SSSS + SSSS extra bits.
//   AC: zigzag positions 1..63; before a nonzero level c preceded by r zeros,
//       one ZRL code (symbol 0xF0) per 16 zeros while r > 15, then the code of
//       symbol (r << 4) | SSSS(c) and SSSS extra bits; zeros after the last
//       nonzero level cost one EOB code (symbol 0x00).
// The result is the entropy-coded data's size in bits, before byte stuffing,
// padding and markers.  One thread per block: its 64 levels (one 128-byte
// block, coefficient (v, u) at u * 8 + v) in registers, walked in zigzag
// order with compile-time positions, the previous block's DC read beside
// them, code lengths from shared copies of the generated tables; per-plane
// sums by warp reduction and one 64-bit atomic per warp.
#include <stdint.h>

#include <algorithm>
#include <utility>

#include "slrme_internal.cuh"

namespace slrme {
namespace {

#define SLRME_TABLE static __device__ const
#include "jpeg_tables.inc"
#undef SLRME_TABLE

// Natural index v * 8 + u of zigzag position k (T.81 Figure A.6): the
// anti-diagonals s = u + v in turn, v rising on odd s, falling on even s.
__host__ __device__ constexpr int zz_nat(int k) {
    int i = 0;
    for (int sd = 0; sd <= 14; ++sd) {
        const int vlo = sd > 7 ? sd - 7 : 0, vhi = sd < 7 ? sd : 7;
        for (int t = 0; t <= vhi - vlo; ++t) {
            const int v = (sd & 1) ? vlo + t : vhi - t;
            if (i == k) return v * 8 + (sd - v);
            ++i;
        }
    }
    return -1;
}
static_assert(zz_nat(0) == 0 && zz_nat(1) == 1 && zz_nat(2) == 8 && zz_nat(3) == 16 && zz_nat(63) == 63,
              "zigzag order of T.81 Figure A.6");

__device__ __forceinline__ int bitlen(int a) {
    return 32 - __clz(a);
}

constexpr int kStatusJpeg = 4;   // bit 2 of the status word: a level beyond the baseline categories

// AC position K (a compile-time index into the block's registers).
// Planes to size: plane p has nblocks[p] blocks from block first[p] of the
// levels array, coded with the chrominance tables when chroma[p].
constexpr int kMaxPlanes = 4;
struct JpegPlanes {
    int n;
    int64_t first[kMaxPlanes], nblocks[kMaxPlanes];
    int chroma[kMaxPlanes];
};

template <int K>
__device__ __forceinline__ void ac_step(const int16_t (&lv)[64], const uint8_t* aclen, int& run, uint32_t& bits,
                                        bool& bad) {
    constexpr int nat = zz_nat(K);
    constexpr int at = (nat & 7) * 8 + (nat >> 3);   // column-major position of (v, u)
    const int v = lv[at];
    if (v == 0) {
        ++run;
    } else {
        bits += (uint32_t)(run >> 4) * aclen[0xF0];   // one ZRL per 16 zeros of a longer run
        const int sz = bitlen(v < 0 ? -v : v);
        bad |= sz > 10;
        bits += aclen[(((run & 15) << 4) | sz) & 255] + sz;
        run = 0;
    }
}

template <int... K>
__device__ __forceinline__ void ac_steps(std::integer_sequence<int, K...>, const int16_t (&lv)[64],
                                         const uint8_t* aclen, int& run, uint32_t& bits, bool& bad) {
    (ac_step<K + 1>(lv, aclen, run, bits, bad), ...);
}

__global__ void __launch_bounds__(256) k_jpeg_bits(const int16_t* __restrict__ lv, const JpegPlanes P,
                                                   unsigned long long* __restrict__ bits3,
                                                   uint32_t* __restrict__ block_bits, int* status) {
    __shared__ uint8_t aclen[256];
    __shared__ uint8_t dclen[16];
    const int c = blockIdx.y;
    const bool chroma = P.chroma[c] != 0;
    aclen[threadIdx.x] = chroma ? kJpegAcLenC[threadIdx.x] : kJpegAcLen[threadIdx.x];
    if (threadIdx.x < 16) dclen[threadIdx.x] = chroma ? kJpegDcLenC[threadIdx.x] : kJpegDcLen[threadIdx.x];
    __syncthreads();
    const int64_t blocks_per_plane = P.nblocks[c];
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t bits = 0;
    bool bad = false;
    if (b < blocks_per_plane) {
        const int16_t* L = lv + (P.first[c] + b) * 64;
        int16_t lv[64];
        const int4* L4 = reinterpret_cast<const int4*>(L);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int4 q = __ldg(L4 + i);
            const int w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                lv[8 * i + 2 * j] = (int16_t)(w4[j] & 0xffff);
                lv[8 * i + 2 * j + 1] = (int16_t)(w4[j] >> 16);
            }
        }
        const int pred = b > 0 ? (int)__ldg(L - 64) : 0;   // the previous block in raster order, same plane
        const int diff = (int)lv[0] - pred;
        const int cat = bitlen(diff < 0 ? -diff : diff);
        bad |= cat > 11;
        bits += dclen[cat & 15] + cat;
        int run = 0;
        ac_steps(std::make_integer_sequence<int, 63>{}, lv, aclen, run, bits, bad);
        if (run > 0) bits += aclen[0x00];
        if (block_bits) block_bits[P.first[c] + b] = bits;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusJpeg);
    unsigned long long sum = bits;
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(bits3 + c, sum);
}

}  // namespace
}  // namespace slrme

namespace slrme {
namespace {

int launch_jpeg(const int16_t* levels, const JpegPlanes& P, unsigned long long* bits, uint32_t* block_bits,
                cudaStream_t s, const char* who) {
    int64_t most = 0;
    for (int p = 0; p < P.n; ++p) most = std::max(most, P.nblocks[p]);
    if (most > 0 && (!levels || ((uintptr_t)levels & 15u))) {
        set_error("%s: levels must be non-null and 16-byte aligned", who);
        return SLRME_EINVAL;
    }
    int* status = nullptr;
    int rc = status_word_address(&status);
    if (rc) return rc;
    if (cudaMemsetAsync(bits, 0, P.n * sizeof(unsigned long long), s) != cudaSuccess) return cuda_status(who);
    if (most == 0) return SLRME_OK;
    const dim3 grid((unsigned)((most + 255) / 256), (unsigned)P.n);
    k_jpeg_bits<<<grid, 256, 0, s>>>(levels, P, bits, block_bits, status);
    return cuda_status(who);
}

}  // namespace
}  // namespace slrme

extern "C" int jpeg_huffman_bits(const int16_t* levels3, int h, int w, unsigned long long* bits3, uint32_t* block_bits,
                                 slrme_stream_t stream) {
    using namespace slrme;
    if (h < 0 || w < 0 || (int64_t)h * w >= (int64_t(1) << 31) || !bits3 || ((uintptr_t)bits3 & 7u) ||
        (block_bits && ((uintptr_t)block_bits & 3u))) {
        set_error("jpeg_huffman_bits: need 0 <= h, w, h*w < 2^31, an 8-byte aligned bits3 and 4-byte aligned block_bits");
        return SLRME_EINVAL;
    }
    const int64_t blocks = (int64_t)((h + 7) / 8) * ((w + 7) / 8);
    JpegPlanes P;
    P.n = 3;
    for (int p = 0; p < kMaxPlanes; ++p) {
        P.first[p] = p * blocks;
        P.nblocks[p] = p < 3 ? blocks : 0;
        P.chroma[p] = 0;
    }
    return launch_jpeg(levels3, P, bits3, block_bits, (cudaStream_t)stream, "jpeg_huffman_bits");
}

extern "C" int jpeg_huffman_bits_planes(const int16_t* levels, int nplanes, const int64_t* nblocks,
                                        const int32_t* chroma, unsigned long long* bits, uint32_t* block_bits,
                                        slrme_stream_t stream) {
    using namespace slrme;
    if (nplanes < 1 || nplanes > kMaxPlanes || !nblocks || !chroma || !bits || ((uintptr_t)bits & 7u) ||
        (block_bits && ((uintptr_t)block_bits & 3u))) {
        set_error("jpeg_huffman_bits_planes: need 1 <= nplanes <= %d, nblocks and chroma, an 8-byte aligned bits and "
                  "4-byte aligned block_bits", kMaxPlanes);
        return SLRME_EINVAL;
    }
    JpegPlanes P;
    P.n = nplanes;
    int64_t at = 0;
    for (int p = 0; p < kMaxPlanes; ++p) {
        const bool in = p < nplanes;
        if (in && (nblocks[p] < 0 || nblocks[p] >= (int64_t(1) << 31) / 64 + 1 || (chroma[p] != 0 && chroma[p] != 1))) {
            set_error("jpeg_huffman_bits_planes: plane %d: bad block count or table class", p);
            return SLRME_EINVAL;
        }
        P.first[p] = at;
        P.nblocks[p] = in ? nblocks[p] : 0;
        P.chroma[p] = in ? chroma[p] : 0;
        at += P.nblocks[p];
    }
    return launch_jpeg(levels, P, bits, block_bits, (cudaStream_t)stream, "jpeg_huffman_bits_planes");
}
