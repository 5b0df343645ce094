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
// Chunk k of plane c owns the block of 32 x 258 words at word
// (c chunks + k) 32 258; its streams' words are packed from the start of the
// block, stream l from the sum of the word counts of streams 0..l-1, each in
// decoding order (high word, low word, then renormalisation words), and
// counts[(c chunks + k) 32 + l] is the number of words of stream l.  The
// rest of a block is not written.
#include <stdint.h>

#include <algorithm>

#include "slrme_internal.cuh"
#include "tma.cuh"

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

// A run of segments, each with its own table and its own chunks.
constexpr int kMaxSeg = SLRME_RANS_MAX_SEGMENTS;
struct SegPlan {
    int n;
    int64_t sym_off[kMaxSeg];     // first symbol of each segment
    int64_t len[kMaxSeg];         // symbols of each segment
    int64_t chunk_off[kMaxSeg];   // first chunk (block, 32 counts) of each segment
};

// Warp-wide: does the chunk hold a value outside -255..255 (a raw chunk)?
__device__ __forceinline__ bool chunk_out_of_range(const int16_t* src, int64_t m, int lane) {
    bool oor = false;
    for (int64_t i = lane; i < m; i += 32) {
        const int v = src[i];
        oor |= v < -255 || v > 255;
    }
    return __any_sync(kFull, oor);
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
// reaches 0.  One CTA of 512 threads per table, thread s holding symbol s: every sum,
// maximum and rank is a block reduction (warp shuffles, then one warp over
// the 16 warp results).
constexpr int kTabThreads = 512;

template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v = op(v, __shfl_xor_sync(kFull, v, o));
    __syncthreads();   // the previous reduction's readers are done with red
    if (lane == 0) red[warp] = v;
    __syncthreads();
    v = red[lane & 15];
#pragma unroll
    for (int o = 8; o; o >>= 1) v = op(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__global__ void __launch_bounds__(kTabThreads) k_rans_tables(const uint32_t* __restrict__ hist3,
                                                             uint32_t* __restrict__ freq3) {
    __shared__ unsigned long long red64[16];
    __shared__ int red32[16];
    const int c = blockIdx.x, s = threadIdx.x, lane = s & 31, warp = s >> 5;
    auto add64 = [](unsigned long long a, unsigned long long b) { return a + b; };
    auto max64 = [](unsigned long long a, unsigned long long b) { return a > b ? a : b; };
    auto add32 = [](int a, int b) { return a + b; };
    auto max32 = [](int a, int b) { return a > b ? a : b; };
    const uint32_t cnt = s < kNres ? hist3[c * kNres + s] : 0u;
    uint32_t* out = freq3 + c * kNres;
    const unsigned long long N = block_reduce<unsigned long long>(cnt, add64, red64);
    if (N == 0) {
        if (s < kNres) out[s] = 0u;
        return;
    }
    // floor(n_s M / N) from a double estimate (relative error below 2^-51, so
    // at most one off, and only next to an integer) and one exact correction;
    // q N < 2^56 since q <= 2^14 and N < 2^41.
    int f = 0;
    if (cnt) {
        const unsigned long long a = (unsigned long long)cnt << kRansBits;
        unsigned long long q = (unsigned long long)((double)a * (1.0 / (double)N));
        if (q * N > a) --q;
        else if ((q + 1) * N <= a) ++q;
        f = q < 1 ? 1 : (int)q;
    }
    const int diff = (int)kRansM - block_reduce<int>(f, add32, red32);
    if (diff > 0) {
        // most frequent symbol, smallest index on ties: key (count, 65535 - s)
        const unsigned long long key = cnt ? ((unsigned long long)cnt << 16) | (unsigned)(0xffff - s) : 0ull;
        const unsigned long long best = block_reduce<unsigned long long>(key, max64, red64);
        if (s == 0xffff - (int)(best & 0xffffu)) f += diff;
    } else if (diff < 0) {
        const int D = -diff;   // at most 511
        const int fmax = block_reduce<int>(f, max32, red32);
        // smallest T with E(T) <= D: E(fmax) = 0, and E(fmax - D - 1) > D
        // because the largest entry alone contributes D + 1 there
        int lo = fmax > D ? fmax - D : 1, hi = fmax;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (block_reduce<int>(f > mid ? f - mid : 0, add32, red32) <= D) hi = mid;
            else lo = mid + 1;
        }
        const int T = lo;
        const int r = D - block_reduce<int>(f > T ? f - T : 0, add32, red32);
        // rank of each entry with f >= T in symbol order
        const bool cand = f >= T;
        const unsigned m = __ballot_sync(kFull, cand);
        __syncthreads();
        if (lane == 0) red32[warp] = __popc(m);
        __syncthreads();
        int before = 0;
        for (int w8 = 0; w8 < warp; ++w8) before += red32[w8];
        const int rank = before + __popc(m & ((1u << lane) - 1u));
        if (cand) f = (rank < r) ? T - 1 : T;
    }
    if (s < kNres) out[s] = (uint32_t)f;
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

// One encoder step for residual value v, without branches: the low word of
// x is stored at the next free position every step, and the position moves
// only when the word is emitted (a word stored without moving is overwritten
// by the next emitted word or by the final state, so it never survives).
// Each step emits at most one word, so the positions stay in 1..257.  A value
// outside -255..255 reads entry 511, whose frequency is 0 like that of any
// symbol the table leaves out; fmin records it (the stream is then
// reported).
__device__ __forceinline__ void enc_step(uint32_t& x, int& p, uint32_t& fmin, uint16_t* st, const EncSym* tab,
                                         int16_t v) {
    const uint32_t s = min((uint32_t)((int)v + 255), (uint32_t)kNres);
    const EncSym e = tab[s];
    fmin = min(fmin, e.f);
    const bool emit = (x >> 18) >= e.f;
    st[p - 1] = (uint16_t)(x & 0xffffu);
    p -= emit ? 1 : 0;
    x = emit ? (x >> 16) : x;
    const uint32_t q = div_by_magic(x, e.ml, e.mh);
    x += q * (kRansM - e.f) + e.cum;
}

__global__ void __launch_bounds__(kEncWarps * 32, 1)
    k_rans_encode(const int16_t* __restrict__ sym, SegPlan P, const uint32_t* __restrict__ freq,
                  uint16_t* __restrict__ words, uint32_t* __restrict__ counts, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    EncSmem& S = *reinterpret_cast<EncSmem*>(smem_raw);
    const int g = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t seg_len = P.len[g];
    const int64_t chunks = (seg_len + kChunk - 1) / kChunk;
    if ((int64_t)blockIdx.x * kEncWarps >= chunks) return;   // no chunk of this segment for this CTA
    if (warp == 0) table_scan(freq + (int64_t)g * kNres, S.fr, S.cum, &S.bad_table);
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

    uint16_t* stage = S.stage[warp];
    for (int64_t k = (int64_t)blockIdx.x * kEncWarps + warp; k < chunks; k += (int64_t)gridDim.x * kEncWarps) {
        const int64_t blk = P.chunk_off[g] + k;
        const int16_t* src0 = sym + P.sym_off[g] + k * kChunk;
        const int64_t m = min((int64_t)kChunk, seg_len - k * kChunk);   // symbols of this chunk
        if (bad_table) {
            // without a table only a raw chunk can be stored
            if (chunk_out_of_range(src0, m, lane)) {
                uint16_t* dst = words + blk * (int64_t)(kLanes * kCap);
                for (int64_t i = lane; i < m; i += 32) dst[i] = (uint16_t)src0[i];
                counts[blk * kLanes + lane] = SLRME_RANS_RAW;
            } else {
                if (lane == 0) atomicOr(status, kStatusRans);
                counts[blk * kLanes + lane] = 0u;
            }
            continue;
        }
        // The lanes' streams differ in length by at most one symbol (lane 0's
        // is the longest): the top step is taken by the lanes that have it,
        // every step below it by all lanes, without per-step conditions.
        const int len = stream_len(m, 0, lane);
        const int J = __shfl_sync(kFull, len, 0);
        const int16_t* src = src0 + lane;
        uint16_t* st = stage + lane * kCap;
        uint32_t x = kRansL, fmin = kRansM;
        int p = kCap;
        if (m == kChunk) {
            // a full chunk: 256 steps per lane in blocks of 32, the symbols of
            // the next block loaded while the current block runs
            constexpr int kF = 32;
            constexpr int kPerLane = kChunk / kLanes;
            int16_t cur[kF];
#pragma unroll
            for (int u = 0; u < kF; ++u) cur[u] = src[(int64_t)kLanes * (kPerLane - 1 - u)];
#pragma unroll 1
            for (int b = 0; b < kPerLane / kF; ++b) {
                const int jtop = kPerLane - 1 - kF * b;
                int16_t nxt[kF];
                const int16_t* sp = src + (int64_t)kLanes * (jtop - kF);
#pragma unroll
                for (int u = 0; u < kF; ++u) nxt[u] = b + 1 < kPerLane / kF ? sp[-kLanes * u] : (int16_t)0;
#pragma unroll
                for (int u = 0; u < kF; ++u) enc_step(x, p, fmin, st, S.sym, cur[u]);
#pragma unroll
                for (int u = 0; u < kF; ++u) cur[u] = nxt[u];
            }
        } else {
            // the plane's last, partial chunk
            if (J > 0 && len == J) enc_step(x, p, fmin, st, S.sym, src[(int64_t)kLanes * (J - 1)]);
            int j = J - 2;
            // symbols are loaded one block of 8 steps ahead of the state chain
            constexpr int kB = 8;
            if (j >= kB - 1) {
                int16_t cur[kB];
                const int16_t* sp = src + (int64_t)kLanes * j;
#pragma unroll
                for (int u = 0; u < kB; ++u) cur[u] = sp[-kLanes * u];
                for (; j >= kB - 1; j -= kB) {
                    int16_t nxt[kB];
                    const bool more = j - kB >= kB - 1;
                    sp = src + (int64_t)kLanes * (j - kB);
#pragma unroll
                    for (int u = 0; u < kB; ++u) nxt[u] = more ? sp[-kLanes * u] : (int16_t)0;
#pragma unroll
                    for (int u = 0; u < kB; ++u) enc_step(x, p, fmin, st, S.sym, cur[u]);
#pragma unroll
                    for (int u = 0; u < kB; ++u) cur[u] = nxt[u];
                }
            }
            for (; j >= 0; --j) enc_step(x, p, fmin, st, S.sym, src[(int64_t)kLanes * j]);
        }
        // at most one word per symbol and two for the state: p stays >= 0
        st[--p] = (uint16_t)(x & 0xffffu);
        st[--p] = (uint16_t)(x >> 16);
        if (__any_sync(kFull, fmin == 0u) && chunk_out_of_range(src0, m, lane)) {
            // a value outside the alphabet: the chunk is stored raw
            uint16_t* dst = words + blk * (int64_t)(kLanes * kCap);
            for (int64_t i = lane; i < m; i += 32) dst[i] = (uint16_t)src0[i];
            counts[blk * kLanes + lane] = SLRME_RANS_RAW;
            __syncwarp();
            continue;
        }
        const bool ok = fmin != 0u;
        if (!ok) atomicOr(status, kStatusRans);
        const int used = kCap - p;
        counts[blk * kLanes + lane] = ok ? (uint32_t)used : 0u;
        // the streams go to the block packed, stream after stream: the warp
        // copies one stream at a time (coalesced stores), stream r from the
        // sum of the word counts of streams 0..r-1
        int incl = used;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        const int off = incl - used;
        __syncwarp();
        // Each stream takes a fixed nine rounds of 32 words (258 at most),
        // predicated, so the loads of several rounds and streams are in
        // flight together.
        uint16_t* dst = words + blk * (int64_t)(kLanes * kCap);
        constexpr int kRounds = (kCap + 31) / 32;
#pragma unroll 2
        for (int r = 0; r < kLanes; ++r) {
            const int cr = __shfl_sync(kFull, used, r), orr = __shfl_sync(kFull, off, r);
            const uint16_t* from = stage + r * kCap + (kCap - cr);
            uint16_t v[kRounds];
#pragma unroll
            for (int i = 0; i < kRounds; ++i) v[i] = (32 * i + lane < cr) ? from[32 * i + lane] : (uint16_t)0;
#pragma unroll
            for (int i = 0; i < kRounds; ++i)
                if (32 * i + lane < cr) dst[orr + 32 * i + lane] = v[i];
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- decoder
// Slot tables: fb[slot] = f_s << 16 | (slot - c_s) (f_s <= 2^14, slot - c_s
// < f_s), sym[slot] = s, for the symbol s whose range holds the slot.  The
// state update reads fb only; the symbol is fetched beside it.  Each warp
// stages its chunk's 32 stream regions (16,512 bytes, contiguous) in shared
// memory with one bulk copy, so the word reads of the state chain are
// shared-memory loads; the staging buffers share their space with the scan
// arrays, which are dead once the slot tables are built.
constexpr int kDecWarps = 8;
constexpr uint32_t kBlockBytes = kLanes * kCap * 2;

struct DecSmem {
    uint32_t fb[kRansM];
    uint16_t sym[kRansM];
    unsigned long long bar[kDecWarps];
    int bad_table;
    __align__(16) union {
        struct {
            uint32_t fr[512];
            uint32_t cum[513];
        } t;
        uint16_t stage[kDecWarps][kLanes * kCap];
    } u;
};
static_assert(sizeof(DecSmem) <= 232448, "decoder shared memory exceeds the 227 KB a CTA may use");

// One decoder step: the symbol of the state's slot, the state update, one
// word taken when the state falls below L (reads are clamped to the staging
// buffer: a corrupt stream runs past its words only in p, which is checked
// at the end).
__device__ __forceinline__ void dec_step(uint32_t& x, int& p, const uint32_t* fb, const uint16_t* sym,
                                         const uint16_t* st, int16_t* out) {
    // the next word is read every step (its address does not depend on x)
    // and taken only when the state falls below L
    const uint32_t w = st[min(p, kLanes * kCap - 1)];
    const uint32_t slot = x & (kRansM - 1u);
    const uint32_t e = fb[slot];
    const int s = sym[slot];
    x = (e >> 16) * (x >> kRansBits) + (e & 0xffffu);
    const bool take = x < kRansL;
    x = take ? ((x << 16) | w) : x;
    p += take ? 1 : 0;
    *out = (int16_t)(s - 255);
}

__global__ void __launch_bounds__(kDecWarps * 32, 1)
    k_rans_decode(const uint16_t* __restrict__ words, const uint32_t* __restrict__ counts, SegPlan P,
                  const uint32_t* __restrict__ freq, int16_t* __restrict__ sym, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DecSmem& S = *reinterpret_cast<DecSmem*>(smem_raw);
    const int g = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t seg_len = P.len[g];
    const int64_t chunks = (seg_len + kChunk - 1) / kChunk;
    if ((int64_t)blockIdx.x * kDecWarps >= chunks) return;   // no chunk of this segment for this CTA
    if (warp == 0) table_scan(freq + (int64_t)g * kNres, S.u.t.fr, S.u.t.cum, &S.bad_table);
    if (lane == 0) mbar_init(smem_addr(&S.bar[warp]), 1);
    __syncthreads();
    const bool bad_table = S.bad_table != 0;
    if (!bad_table) {
    // The symbol of each slot: every symbol with f > 0 marks the first slot
    // of its range (cum[s]) in sym[], and a running maximum over the slots
    // carries each mark to the end of its range (the marks grow with the
    // slot).  Warp w takes slots w*2048 .. w*2048+2047, 32 consecutive slots
    // per step (conflict-free), starting from the symbol of the slot before
    // its range (the largest s with cum[s] at or below it; that s has f > 0).
    constexpr int kRange = kRansM / kDecWarps;
    static_assert(kRansM % (kDecWarps * 32) == 0, "slot ranges must tile the table");
    {
        const uint32_t* cum = S.u.t.cum;
        const uint32_t* fr = S.u.t.fr;
        uint32_t* sym32 = reinterpret_cast<uint32_t*>(S.sym);
        for (int i = threadIdx.x; i < kRansM / 2; i += blockDim.x) sym32[i] = 0u;
        __syncthreads();
        for (int t = threadIdx.x; t < kNres; t += blockDim.x)
            if (fr[t]) S.sym[cum[t]] = (uint16_t)t;
        __syncthreads();
        uint32_t carry = 0;
        if (warp > 0) {
            const uint32_t before = warp * kRange - 1;
            int lo = 0, hi = kNres - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (cum[mid] <= before) lo = mid;
                else hi = mid - 1;
            }
            carry = lo;
        }
        // eight rows of 32 slots at a time: their scans are independent, the
        // carry into each row is the maximum of the carry and the rows before it
        constexpr int kG = 8;
        for (int row = 0; row < kRange / 32; row += kG) {
            uint32_t v[kG];
#pragma unroll
            for (int u = 0; u < kG; ++u) v[u] = S.sym[warp * kRange + (row + u) * 32 + lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                for (int u = 0; u < kG; ++u) v[u] = max(v[u], __shfl_up_sync(kFull, v[u], o));
            }
            uint32_t top[kG];
#pragma unroll
            for (int u = 0; u < kG; ++u) top[u] = __shfl_sync(kFull, v[u], 31);
#pragma unroll
            for (int u = 0; u < kG; ++u) {
                const uint32_t sv = max(v[u], carry);
                carry = max(carry, top[u]);
                const uint32_t slot = warp * kRange + (row + u) * 32 + lane;
                S.fb[slot] = (fr[sv] << 16) | (slot - cum[sv]);
                S.sym[slot] = (uint16_t)sv;
            }
        }
    }
    }
    __syncthreads();   // the scan arrays are dead from here: the staging buffers reuse them

    const uint32_t bar = smem_addr(&S.bar[warp]);
    const uint32_t stage_addr = smem_addr(S.u.stage[warp]);
    uint32_t phase = 0;
    for (int64_t k = (int64_t)blockIdx.x * kDecWarps + warp; k < chunks; k += (int64_t)gridDim.x * kDecWarps) {
        const int64_t blk = P.chunk_off[g] + k;
        const int64_t m = min((int64_t)kChunk, seg_len - k * kChunk);
        int16_t* out0 = sym + P.sym_off[g] + k * kChunk;
        const uint32_t cnt = counts[blk * kLanes + lane];
        const bool raw = cnt == SLRME_RANS_RAW;
        if (__any_sync(kFull, raw)) {
            // a raw chunk (all 32 counts say so) holds its values verbatim
            const uint16_t* block = words + blk * (int64_t)(kLanes * kCap);
            for (int64_t i = lane; i < m; i += 32) out0[i] = (int16_t)block[i];
            if (!__all_sync(kFull, raw) && lane == 0) atomicOr(status, kStatusRans);
            continue;
        }
        if (bad_table) {
            if (lane == 0) atomicOr(status, kStatusRans);
            continue;
        }
        // stream offsets in the packed block; a count outside 2..258 (or a
        // sum beyond the block) is reported, and the whole block is copied
        const bool cnt_ok = cnt >= 2u && cnt <= (uint32_t)kCap;
        uint32_t incl = cnt_ok ? cnt : 2u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        const bool ok = __all_sync(kFull, cnt_ok);
        const uint32_t off = incl - (cnt_ok ? cnt : 2u);
        const uint32_t bytes = ok ? ((total * 2u + 15u) & ~15u) : kBlockBytes;
        if (lane == 0) {
            fence_async_shared();   // earlier generic accesses of the buffer before the copy overwrites it
            mbar_arrive_expect_tx(bar, bytes);
            tma_load_1d(stage_addr, words + blk * (int64_t)(kLanes * kCap), bytes, bar);
        }
        const int len = stream_len(m, 0, lane);
        int16_t* dst = out0 + lane;
        if (!mbar_wait(bar, phase, status)) {
            // the copy did not land within the bound: wait once more (bounded)
            // so that no copy is left in flight, then stop
            mbar_wait(bar, phase, status);
            return;
        }
        phase ^= 1u;
        // every read is clamped to the buffer (a corrupt count or stream only
        // decodes garbage, reported below)
        const uint16_t* sw = S.u.stage[warp];
        const uint32_t base = min(off, (uint32_t)(kLanes * kCap - 2));
        uint32_t x = ((uint32_t)sw[base] << 16) | sw[base + 1];
        int p = (int)base + 2;
        // steps 0 .. J-2 for every lane, step J-1 for the lanes that have it
        const int J = __shfl_sync(kFull, len, 0);
        int j = 0;
        for (; j + 4 <= J - 1; j += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) dec_step(x, p, S.fb, S.sym, sw, dst + (int64_t)kLanes * (j + u));
        }
        for (; j < J - 1; ++j) dec_step(x, p, S.fb, S.sym, sw, dst + (int64_t)kLanes * j);
        if (J > 0 && len == J) dec_step(x, p, S.fb, S.sym, sw, dst + (int64_t)kLanes * (J - 1));
        // the decoder ends in the encoder's initial state with every word read
        if (!ok || total > (uint32_t)(kLanes * kCap) || p != (int)(off + cnt) || x != kRansL)
            atomicOr(status, kStatusRans);
        __syncwarp();   // every lane is done with the buffer before the next copy
    }
}

// Raises the kernel's dynamic shared-memory limit once per device.
int set_smem(const void* fn, size_t bytes, bool* done, const char* what) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cuda_status(what);
    if (!done[dev]) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
            return cuda_status(what);
        done[dev] = true;
    }
    return SLRME_OK;
}

bool g_enc_attr[64], g_dec_attr[64];

// CTAs per segment: enough for every warp of the largest segment to take a
// chunk, at most a third of the SMs (then the CTAs loop over their chunks).
int grid_x(const SegPlan& P, int warps) {
    int64_t need = 1;
    for (int g = 0; g < P.n; ++g) need = std::max(need, ((P.len[g] + kChunk - 1) / kChunk + warps - 1) / warps);
    const int64_t cap = std::max(1, geometry().sms / 3);
    return (int)std::min<int64_t>(need, cap);
}

// Validates a run of segments and lays out its symbols and chunks.
int seg_plan(const char* who, int nseg, const int64_t* len, SegPlan* P, int64_t* total_chunks) {
    if (nseg < 1 || nseg > kMaxSeg || !len) {
        set_error("%s: need 1 <= nseg <= %d and the segment lengths", who, kMaxSeg);
        return SLRME_EINVAL;
    }
    P->n = nseg;
    int64_t at = 0, chunk = 0;
    for (int g = 0; g < nseg; ++g) {
        if (len[g] < 0) {
            set_error("%s: segment %d has a negative length", who, g);
            return SLRME_EINVAL;
        }
        P->sym_off[g] = at;
        P->len[g] = len[g];
        P->chunk_off[g] = chunk;
        at += len[g];
        chunk += (len[g] + kChunk - 1) / kChunk;
        if (at >= (int64_t(1) << 31)) {
            set_error("%s: the segments hold 2^31 symbols or more", who);
            return SLRME_EINVAL;
        }
    }
    for (int g = nseg; g < kMaxSeg; ++g) P->sym_off[g] = P->len[g] = P->chunk_off[g] = 0;
    *total_chunks = chunk;
    return SLRME_OK;
}

int encode_plan(const int16_t* sym, const SegPlan& P, int64_t chunks, const uint32_t* freq, uint16_t* words,
                uint32_t* counts, cudaStream_t s, const char* who) {
    if (chunks == 0) return SLRME_OK;
    if (!sym || !freq || !words || !counts || ((uintptr_t)sym & 1u) || ((uintptr_t)freq & 3u) ||
        ((uintptr_t)words & 15u) || ((uintptr_t)counts & 3u)) {
        set_error("%s: null or misaligned pointer (symbols 2, tables 4, words 16, counts 4 bytes)", who);
        return SLRME_EINVAL;
    }
    int* status = nullptr;
    int rc = status_word_address(&status);
    if (rc) return rc;
    const size_t smem = sizeof(EncSmem);
    if ((rc = set_smem((const void*)k_rans_encode, smem, g_enc_attr, "rans encoder shared memory"))) return rc;
    const dim3 grid(grid_x(P, kEncWarps), P.n);
    k_rans_encode<<<grid, kEncWarps * 32, smem, s>>>(sym, P, freq, words, counts, status);
    return cuda_status(who);
}

int decode_plan(const uint16_t* words, const uint32_t* counts, const SegPlan& P, int64_t chunks,
                const uint32_t* freq, int16_t* sym, cudaStream_t s, const char* who) {
    if (chunks == 0) return SLRME_OK;
    if (!sym || !freq || !words || !counts || ((uintptr_t)sym & 1u) || ((uintptr_t)freq & 3u) ||
        ((uintptr_t)words & 15u) || ((uintptr_t)counts & 3u)) {
        set_error("%s: null or misaligned pointer (words 16, counts 4, tables 4, symbols 2 bytes)", who);
        return SLRME_EINVAL;
    }
    int* status = nullptr;
    int rc = status_word_address(&status);
    if (rc) return rc;
    const size_t smem = sizeof(DecSmem);
    if ((rc = set_smem((const void*)k_rans_decode, smem, g_dec_attr, "rans decoder shared memory"))) return rc;
    const dim3 grid(grid_x(P, kDecWarps), P.n);
    k_rans_decode<<<grid, kDecWarps * 32, smem, s>>>(words, counts, P, freq, sym, status);
    return cuda_status(who);
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

extern "C" int64_t rans_segments_words_capacity(int nseg, const int64_t* len) {
    using namespace slrme;
    SegPlan P;
    int64_t chunks = 0;
    if (seg_plan("rans_segments_words_capacity", nseg, len, &P, &chunks)) return 0;
    return chunks * kLanes * kCap;
}

extern "C" int64_t rans_segments_counts_capacity(int nseg, const int64_t* len) {
    using namespace slrme;
    SegPlan P;
    int64_t chunks = 0;
    if (seg_plan("rans_segments_counts_capacity", nseg, len, &P, &chunks)) return 0;
    return chunks * kLanes;
}

extern "C" int rans_tables_n(const uint32_t* hist, int ntables, uint32_t* freq, slrme_stream_t stream) {
    using namespace slrme;
    if (!hist || !freq || !aligned(hist, 4) || !aligned(freq, 4) || ntables < 1 || ntables > 65535) {
        set_error("rans_tables_n: need 4-byte aligned hist and freq and 1 <= ntables <= 65535");
        return SLRME_EINVAL;
    }
    k_rans_tables<<<ntables, kTabThreads, 0, (cudaStream_t)stream>>>(hist, freq);
    return cuda_status("rans_tables_n launch");
}

extern "C" int rans_tables(const uint32_t* hist3, uint32_t* freq3, slrme_stream_t stream) {
    using namespace slrme;
    if (!hist3 || !freq3 || !aligned(hist3, 4) || !aligned(freq3, 4)) {
        set_error("rans_tables: hist3 and freq3 must be non-null and 4-byte aligned");
        return SLRME_EINVAL;
    }
    k_rans_tables<<<3, kTabThreads, 0, (cudaStream_t)stream>>>(hist3, freq3);
    return cuda_status("rans_tables launch");
}

extern "C" int rans_encode_segments(const int16_t* sym, int nseg, const int64_t* len, const uint32_t* freq,
                                    uint16_t* words, uint32_t* counts, slrme_stream_t stream) {
    using namespace slrme;
    SegPlan P;
    int64_t chunks = 0;
    int rc = seg_plan("rans_encode_segments", nseg, len, &P, &chunks);
    if (rc) return rc;
    return encode_plan(sym, P, chunks, freq, words, counts, (cudaStream_t)stream, "rans_encode_segments");
}

extern "C" int rans_decode_segments(const uint16_t* words, const uint32_t* counts, int nseg, const int64_t* len,
                                    const uint32_t* freq, int16_t* sym, slrme_stream_t stream) {
    using namespace slrme;
    SegPlan P;
    int64_t chunks = 0;
    int rc = seg_plan("rans_decode_segments", nseg, len, &P, &chunks);
    if (rc) return rc;
    return decode_plan(words, counts, P, chunks, freq, sym, (cudaStream_t)stream, "rans_decode_segments");
}

extern "C" int rans_encode(const int16_t* r3, int64_t n, const uint32_t* freq3, uint16_t* words, uint32_t* counts,
                           slrme_stream_t stream) {
    using namespace slrme;
    int rc = check_n("rans_encode", n);
    if (rc) return rc;
    const int64_t len[3] = {n, n, n};
    SegPlan P;
    int64_t chunks = 0;
    if ((rc = seg_plan("rans_encode", 3, len, &P, &chunks))) return rc;
    return encode_plan(r3, P, chunks, freq3, words, counts, (cudaStream_t)stream, "rans_encode");
}

extern "C" int rans_decode(const uint16_t* words, const uint32_t* counts, int64_t n, const uint32_t* freq3,
                           int16_t* r3, slrme_stream_t stream) {
    using namespace slrme;
    int rc = check_n("rans_decode", n);
    if (rc) return rc;
    const int64_t len[3] = {n, n, n};
    SegPlan P;
    int64_t chunks = 0;
    if ((rc = seg_plan("rans_decode", 3, len, &P, &chunks))) return rc;
    return decode_plan(words, counts, P, chunks, freq3, r3, (cudaStream_t)stream, "rans_decode");
}
