// Enhancement-layer entropy coder: interleaved rANS over the residual planes.
//
// The paper codes the residuals R = M - M* of the enhancement layer with a
// reversible (lossless) coder, JPEG 2000's lossless mode in its experiments
// (Sec. II-A, Sec. IV); the residual is losslessly recoverable from the
// bitstream.  This file implements that layer's entropy coder as range
// asymmetric numeral systems (rANS, Duda 2013) with a static table per
// colour channel, laid out for the GPU: every 8192 symbols of a plane form
// a chunk, coded as 32 interleaved streams (stream l takes symbols
// l, l + 32, l + 64, ...), one warp per chunk and one lane per stream.
//
// Coder definition (M = 2^14, L = 2^16, 16-bit words):
//   symbol s = R + 255 with frequency f_s and cumulative frequency c_s;
//   encode (symbols of a stream in reverse order), state x in [L, 2^32):
//     if floor(x / 2^18) >= f_s: emit x mod 2^16, x = floor(x / 2^16);
//     x = floor(x / f_s) M + (x mod f_s) + c_s;
//   then emit the final state's low word, then its high word;
//   decode: slot = x mod M, s the symbol with c_s <= slot < c_s + f_s,
//     x = f_s floor(x / M) + slot - c_s; if x < L: x = 2^16 x + next word.
// Stream l of chunk k of plane c owns the region of 258 words at word
// ((c chunks + k) 32 + l) 258; its words fill the end of the region in
// decoding order (high word, low word, then renormalisation words), the
// words before them are zero, and counts[(c chunks + k) 32 + l] is the
// number of words used.
#include <stdint.h>

#include <algorithm>

#include "slrme_internal.cuh"

namespace slrme {
namespace {

constexpr int kRansBits = 14;
constexpr uint32_t kRansM = 1u << kRansBits;
constexpr uint32_t kRansL = 1u << 16;
constexpr int kChunk = SLRME_RANS_CHUNK;
constexpr int kLanes = SLRME_RANS_LANES;
constexpr int kCap = SLRME_RANS_CAP;
constexpr int kStatusRans = 2;   // bit 1 of the status word: rANS input outside its table or a corrupt stream
static_assert(kCap == kChunk / kLanes + 2, "a stream of 256 symbols emits at most one word per symbol plus the state");
static_assert((kLanes * kCap * 2) % 16 == 0, "chunk blocks must stay 16-byte aligned");

constexpr unsigned kFull = 0xffffffffu;

// Symbols of stream l of chunk k of a plane of n symbols.
__device__ __forceinline__ int stream_len(int64_t n, int64_t k, int l) {
    const int64_t first = k * kChunk + l;
    const int64_t end = min(n, (k + 1) * kChunk);
    return first < end ? (int)((end - 1 - first) / kLanes) + 1 : 0;
}

// ---------------------------------------------------------------- tables
// Normalisation of one channel's residual histogram to a table of total M:
//   f_s = max(1, floor(n_s M / N)) for every symbol that occurs (n_s > 0);
//   a shortfall D = M - sum f goes to the most frequent symbol (smallest s on
//   ties); an excess D = sum f - M is removed one unit at a time from the
//   largest entry above 1 (smallest s on ties).
// The one-at-a-time removal equals, in closed form: with
//   E(T) = sum_s max(0, f_s - T) and T the smallest level with E(T) <= D,
// every entry is cut to min(f_s, T) and the r = D - E(T) smallest symbols
// among those with f_s >= T lose one more unit (r is below their number).
// Each level the removal passes through has all entries above it already cut
// to it, and at the level T itself it walks the tied entries in symbol order.
// Since sum f <= M + 511 over at most 511 symbols, T > 32, so no entry
// reaches 0.  One warp per channel; lane t holds symbols t + 32 i.
__global__ void __launch_bounds__(32) k_rans_tables(const uint32_t* __restrict__ hist3, uint32_t* __restrict__ freq3) {
    constexpr int kPer = 16;   // 16 x 32 = 512 >= 511 symbols
    const int c = blockIdx.x, lane = threadIdx.x;
    const uint32_t* h = hist3 + c * kNres;
    uint32_t cnt[kPer], f[kPer];
    unsigned long long N = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int s = lane + 32 * i;
        cnt[i] = s < kNres ? h[s] : 0u;
        N += cnt[i];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) N += __shfl_xor_sync(kFull, N, o);
    uint32_t* out = freq3 + c * kNres;
    if (N == 0) {
#pragma unroll
        for (int i = 0; i < kPer; ++i)
            if (lane + 32 * i < kNres) out[lane + 32 * i] = 0u;
        return;
    }
    long long sum = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        uint32_t v = 0;
        if (cnt[i]) {
            const unsigned long long q = (unsigned long long)cnt[i] * kRansM / N;
            v = q < 1 ? 1u : (uint32_t)q;
        }
        f[i] = v;
        sum += v;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    const long long diff = (long long)kRansM - sum;
    if (diff > 0) {
        // most frequent symbol, smallest index on ties: key = (count, -s)
        uint32_t bc = 0;
        int bs = 1 << 30;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int s = lane + 32 * i;
            if (s < kNres && (cnt[i] > bc || (cnt[i] == bc && s < bs))) {
                bc = cnt[i];
                bs = s;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const uint32_t oc = __shfl_xor_sync(kFull, bc, o);
            const int os = __shfl_xor_sync(kFull, bs, o);
            if (oc > bc || (oc == bc && os < bs)) {
                bc = oc;
                bs = os;
            }
        }
#pragma unroll
        for (int i = 0; i < kPer; ++i)
            if (lane + 32 * i == bs) f[i] += (uint32_t)diff;
    } else if (diff < 0) {
        const long long D = -diff;
        uint32_t fmax = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) fmax = max(fmax, f[i]);
#pragma unroll
        for (int o = 16; o; o >>= 1) fmax = max(fmax, __shfl_xor_sync(kFull, fmax, o));
        // smallest T in [1, fmax] with E(T) <= D (E(fmax) = 0)
        uint32_t lo = 1, hi = fmax;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            long long e = 0;
#pragma unroll
            for (int i = 0; i < kPer; ++i) e += f[i] > mid ? (long long)(f[i] - mid) : 0;
#pragma unroll
            for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(kFull, e, o);
            if (e <= D) hi = mid;
            else lo = mid + 1;
        }
        const uint32_t T = lo;
        long long e = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) e += f[i] > T ? (long long)(f[i] - T) : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(kFull, e, o);
        const long long r = D - e;
        // rank of each entry with f >= T in symbol order s = lane + 32 i
        long long before = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const bool cand = f[i] >= T;
            const unsigned m = __ballot_sync(kFull, cand);
            const long long rank = before + __popc(m & ((1u << lane) - 1u));
            if (cand) f[i] = (rank < r) ? T - 1 : T;
            before += __popc(m);
        }
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i)
        if (lane + 32 * i < kNres) out[lane + 32 * i] = f[i];
}

// Exclusive prefix sums of one channel's table (512 entries, entry 511 = 0)
// by warp 0 of the block; cum[512] = the total.  Each lane scans 16
// consecutive entries.  *bad = 1 unless every entry is at most M and they
// sum to M (entries capped at M cannot wrap the 32-bit sums).
__device__ __forceinline__ void table_scan(const uint32_t* __restrict__ freq, uint32_t* fr, uint32_t* cum, int* bad) {
    const int lane = threadIdx.x & 31;
    uint32_t v[16], local = 0;
    bool big = false;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int s = lane * 16 + i;
        v[i] = s < kNres ? freq[s] : 0u;
        big |= v[i] > kRansM;
        v[i] = min(v[i], kRansM);
        local += v[i];
    }
    big = __any_sync(kFull, big);
    uint32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    uint32_t run = incl - local;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        fr[lane * 16 + i] = v[i];
        cum[lane * 16 + i] = run;
        run += v[i];
    }
    if (lane == 31) {
        cum[512] = incl;
        *bad = big || incl != kRansM;
    }
}

// ---------------------------------------------------------------- encoder
// Per-symbol entry: the divisor f with its reciprocal m = ceil(2^46 / f)
// split into 32-bit halves, and the cumulative frequency.  For x < 2^32 and
// 1 <= f <= 2^14 (so x f < 2^46), floor(x / f) = floor(x m / 2^46) exactly
// (division by invariant integers using multiplication, Granlund and
// Montgomery 1994): x m / 2^46 = x / f + x e / 2^46 with 0 <= e < 1, and the
// added term is below 1 / f, the gap between x / f and the next integer.
struct EncSym {
    uint32_t ml, mh, f, cum;
};

constexpr int kEncWarps = 8;

struct EncSmem {
    EncSym sym[512];
    uint32_t fr[512];
    uint32_t cum[513];
    int bad_table;
    __align__(16) uint16_t stage[kEncWarps][kLanes * kCap];
};

__device__ __forceinline__ uint32_t div_by_magic(uint32_t x, uint32_t ml, uint32_t mh) {
    // floor(x (mh 2^32 + ml) / 2^46): the low 32 bits of x ml never carry
    // into bit 46 once shifted out, so only its high half is needed.
    const unsigned long long t = (unsigned long long)x * mh + __umulhi(x, ml);
    return (uint32_t)(t >> 14);
}

__global__ void __launch_bounds__(kEncWarps * 32, 1)
    k_rans_encode(const int16_t* __restrict__ r3, int64_t n, int64_t chunks, const uint32_t* __restrict__ freq3,
                  uint16_t* __restrict__ words, uint32_t* __restrict__ counts, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    EncSmem& S = *reinterpret_cast<EncSmem*>(smem_raw);
    const int c = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) table_scan(freq3 + c * kNres, S.fr, S.cum, &S.bad_table);
    __syncthreads();
    for (int s = threadIdx.x; s < 512; s += blockDim.x) {
        const uint32_t f = S.fr[s];
        EncSym e;
        e.f = f;
        e.cum = S.cum[s];
        if (f) {
            const unsigned long long m = ((1ull << 46) + f - 1) / f;
            e.ml = (uint32_t)m;
            e.mh = (uint32_t)(m >> 32);
        } else {
            e.ml = e.mh = 0u;
        }
        S.sym[s] = e;
    }
    __syncthreads();
    const bool bad_table = S.bad_table != 0;
    if (bad_table && threadIdx.x == 0) atomicOr(status, kStatusRans);

    uint16_t* stage = S.stage[warp];
    uint4* stage4 = reinterpret_cast<uint4*>(stage);
    constexpr int kVec = kLanes * kCap * 2 / 16;   // uint4 per chunk block
    for (int64_t k = (int64_t)blockIdx.x * kEncWarps + warp; k < chunks; k += (int64_t)gridDim.x * kEncWarps) {
        const int64_t blk = (int64_t)c * chunks + k;
        if (bad_table) {
            counts[blk * kLanes + lane] = 0u;
            continue;
        }
        for (int i = lane; i < kVec; i += 32) stage4[i] = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        const int len = stream_len(n, k, lane);
        const int J = __shfl_sync(kFull, len, 0);   // lane 0 has the longest stream
        const int16_t* src = r3 + (int64_t)c * n + k * kChunk + lane;
        uint16_t* st = stage + lane * kCap;
        uint32_t x = kRansL;
        int p = kCap;
        bool ok = true;
        // symbols are loaded one block of 8 ahead of the state chain
        constexpr int kB = 8;
        int16_t cur[kB], nxt[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int j = J - 1 - u;
            cur[u] = (j >= 0 && j < len) ? src[(int64_t)kLanes * j] : (int16_t)0;
        }
        for (int j0 = J; j0 > 0; j0 -= kB) {
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int j = j0 - kB - 1 - u;
                nxt[u] = (j >= 0 && j < len) ? src[(int64_t)kLanes * j] : (int16_t)0;
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int j = j0 - 1 - u;
                if (j >= 0 && j < len && ok) {
                    const uint32_t s = (uint32_t)((int)cur[u] + 255);
                    if (s >= (uint32_t)kNres) {
                        ok = false;
                    } else {
                        const EncSym e = S.sym[s];
                        if (e.f == 0u) {
                            ok = false;
                        } else {
                            if ((x >> 18) >= e.f) {
                                st[--p] = (uint16_t)(x & 0xffffu);
                                x >>= 16;
                            }
                            const uint32_t q = div_by_magic(x, e.ml, e.mh);
                            x += q * (kRansM - e.f) + e.cum;
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) cur[u] = nxt[u];
        }
        if (ok) {
            st[--p] = (uint16_t)(x & 0xffffu);
            st[--p] = (uint16_t)(x >> 16);
        } else {
            atomicOr(status, kStatusRans);
        }
        counts[blk * kLanes + lane] = ok ? (uint32_t)(kCap - p) : 0u;
        __syncwarp();
        uint4* dst = reinterpret_cast<uint4*>(words + blk * (int64_t)(kLanes * kCap));
        for (int i = lane; i < kVec; i += 32) dst[i] = stage4[i];
        __syncwarp();
    }
}

// ---------------------------------------------------------------- decoder
// Slot tables: fb[slot] = f_s << 16 | (slot - c_s) (f_s <= 2^14, slot - c_s
// < f_s), sym[slot] = s, for the symbol s whose range holds the slot.  The
// state update reads fb only; the symbol is fetched beside it.
constexpr int kDecWarps = 8;

struct DecSmem {
    uint32_t fb[kRansM];
    uint16_t sym[kRansM];
    uint32_t fr[512];
    uint32_t cum[513];
    int bad_table;
};

__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__global__ void __launch_bounds__(kDecWarps * 32, 1)
    k_rans_decode(const uint16_t* __restrict__ words, const uint32_t* __restrict__ counts, int64_t n, int64_t chunks,
                  const uint32_t* __restrict__ freq3, int16_t* __restrict__ r3, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DecSmem& S = *reinterpret_cast<DecSmem*>(smem_raw);
    const int c = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) table_scan(freq3 + c * kNres, S.fr, S.cum, &S.bad_table);
    __syncthreads();
    if (S.bad_table) {
        if (threadIdx.x == 0) atomicOr(status, kStatusRans);
        return;
    }
    // Each thread fills a run of consecutive slots: the symbol of its first
    // slot is the largest s with cum[s] <= slot (that symbol has f > 0, as
    // cum[s + 1] > slot), then it walks forward.
    constexpr int kRun = kRansM / (kDecWarps * 32);
    static_assert(kRansM % (kDecWarps * 32) == 0, "slot runs must tile the table");
    {
        const uint32_t first = threadIdx.x * kRun;
        int lo = 0, hi = kNres - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (S.cum[mid] <= first) lo = mid;
            else hi = mid - 1;
        }
        int s = lo;
        for (uint32_t slot = first; slot < first + kRun; ++slot) {
            while (slot >= S.cum[s + 1]) ++s;
            S.fb[slot] = (S.fr[s] << 16) | (slot - S.cum[s]);
            S.sym[slot] = (uint16_t)s;
        }
    }
    __syncthreads();

    for (int64_t k = (int64_t)blockIdx.x * kDecWarps + warp; k < chunks; k += (int64_t)gridDim.x * kDecWarps) {
        const int64_t blk = (int64_t)c * chunks + k;
        const int len = stream_len(n, k, lane);
        const uint32_t cnt = counts[blk * kLanes + lane];
        const uint16_t* reg = words + (blk * kLanes + lane) * (int64_t)kCap;
        int16_t* dst = r3 + (int64_t)c * n + k * kChunk + lane;
        bool ok = cnt >= 2u && cnt <= (uint32_t)kCap;
        int p = kCap - (ok ? (int)cnt : 2);
        uint32_t x = kRansL;
        if (ok) {
            for (int q = (p & ~63); q < kCap; q += 64) prefetch_l1(reg + q);
            x = ((uint32_t)__ldg(reg + p) << 16) | __ldg(reg + p + 1);
            p += 2;
        }
        for (int j = 0; j < len; ++j) {
            int16_t v = 0;
            if (ok) {
                const uint32_t slot = x & (kRansM - 1u);
                const uint32_t e = S.fb[slot];
                v = (int16_t)((int)S.sym[slot] - 255);
                x = (e >> 16) * (x >> kRansBits) + (e & 0xffffu);
                if (x < kRansL) {
                    if (p < kCap) x = (x << 16) | __ldg(reg + p++);
                    else ok = false;
                }
            }
            dst[(int64_t)kLanes * j] = v;
        }
        // the decoder ends in the encoder's initial state with every word read
        if (!ok || p != kCap || x != kRansL) atomicOr(status, kStatusRans);
    }
}

int grid_x(int64_t chunks, int warps) {
    const int64_t need = (chunks + warps - 1) / warps;
    const int64_t cap = std::max(1, geometry().sms / 3);
    return (int)std::min<int64_t>(need, cap);
}

int set_smem(const void* fn, size_t bytes, const char* what) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return cuda_status(what);
    return SLRME_OK;
}

bool aligned(const void* p, size_t a) {
    return ((uintptr_t)p % a) == 0;
}

int check_n(const char* who, int64_t n) {
    if (n < 0 || n >= (int64_t(1) << 31)) {
        set_error("%s: n must be in 0..2^31-1 (n=%lld)", who, (long long)n);
        return SLRME_EINVAL;
    }
    return SLRME_OK;
}

}  // namespace
}  // namespace slrme

extern "C" int64_t rans_words_capacity(int64_t n) {
    if (n < 0) return 0;
    const int64_t chunks = (n + SLRME_RANS_CHUNK - 1) / SLRME_RANS_CHUNK;
    return 3 * chunks * SLRME_RANS_LANES * SLRME_RANS_CAP;
}

extern "C" int64_t rans_counts_capacity(int64_t n) {
    if (n < 0) return 0;
    const int64_t chunks = (n + SLRME_RANS_CHUNK - 1) / SLRME_RANS_CHUNK;
    return 3 * chunks * SLRME_RANS_LANES;
}

extern "C" int rans_tables(const uint32_t* hist3, uint32_t* freq3, slrme_stream_t stream) {
    using namespace slrme;
    if (!hist3 || !freq3 || !aligned(hist3, 4) || !aligned(freq3, 4)) {
        set_error("rans_tables: hist3 and freq3 must be non-null and 4-byte aligned");
        return SLRME_EINVAL;
    }
    k_rans_tables<<<3, 32, 0, (cudaStream_t)stream>>>(hist3, freq3);
    return cuda_status("rans_tables launch");
}

extern "C" int rans_encode(const int16_t* r3, int64_t n, const uint32_t* freq3, uint16_t* words, uint32_t* counts,
                           slrme_stream_t stream) {
    using namespace slrme;
    int rc = check_n("rans_encode", n);
    if (rc) return rc;
    if (n == 0) return SLRME_OK;
    if (!r3 || !freq3 || !words || !counts || !aligned(r3, 2) || !aligned(freq3, 4) || !aligned(words, 16) ||
        !aligned(counts, 4)) {
        set_error("rans_encode: null or misaligned pointer (r3 2, freq3 4, words 16, counts 4 bytes)");
        return SLRME_EINVAL;
    }
    int* status = nullptr;
    if ((rc = status_word_address(&status))) return rc;
    const size_t smem = sizeof(EncSmem);
    if ((rc = set_smem((const void*)k_rans_encode, smem, "rans_encode smem"))) return rc;
    const int64_t chunks = (n + kChunk - 1) / kChunk;
    const dim3 grid(grid_x(chunks, kEncWarps), 3);
    k_rans_encode<<<grid, kEncWarps * 32, smem, (cudaStream_t)stream>>>(r3, n, chunks, freq3, words, counts, status);
    return cuda_status("rans_encode launch");
}

extern "C" int rans_decode(const uint16_t* words, const uint32_t* counts, int64_t n, const uint32_t* freq3,
                           int16_t* r3, slrme_stream_t stream) {
    using namespace slrme;
    int rc = check_n("rans_decode", n);
    if (rc) return rc;
    if (n == 0) return SLRME_OK;
    if (!r3 || !freq3 || !words || !counts || !aligned(r3, 2) || !aligned(freq3, 4) || !aligned(words, 2) ||
        !aligned(counts, 4)) {
        set_error("rans_decode: null or misaligned pointer (words 2, counts 4, freq3 4, r3 2 bytes)");
        return SLRME_EINVAL;
    }
    int* status = nullptr;
    if ((rc = status_word_address(&status))) return rc;
    const size_t smem = sizeof(DecSmem);
    if ((rc = set_smem((const void*)k_rans_decode, smem, "rans_decode smem"))) return rc;
    const int64_t chunks = (n + kChunk - 1) / kChunk;
    const dim3 grid(grid_x(chunks, kDecWarps), 3);
    k_rans_decode<<<grid, kDecWarps * 32, smem, (cudaStream_t)stream>>>(words, counts, n, chunks, freq3, r3, status);
    return cuda_status("rans_decode launch");
}
