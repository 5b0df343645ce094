// SLRME (Sec. III-B, Eqs. 8-10) and the enhancement layer (Sec. III-C):
//   k_fit        Gaussian restoration of S + exponent-binned exact sums
//   k_solve      per (channel, region) slope/intercept from the sums
//   k_residual   restoration + Eq. (8) prediction + R = M - M* + histograms
//   k_decode     restoration + Eq. (8) prediction + M = R + M* + repack
//
// Shared structure: a warp owns a strip 256 columns wide (8 per lane) and
// 4, 8 or 16 rows tall and slides a 3-row window of S down it, so every row
// of S is loaded once per strip.  The neighbours a lane needs left and right
// of its 8 pixels come from the adjacent lanes by shuffle (strip edges load
// them).  The 3x3 binomial filter runs on 16-bit pairs: two pixels per
// 32-bit add (values stay <= 4080).
#include <initializer_list>
#include <mutex>

#include "slrme_internal.cuh"
#include "tma.cuh"

namespace slrme {

// Device status word of the TMA-staged kernels (0 = fine); read and cleared
// by slrme_device_status().
__device__ int g_slrme_status;


namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kMaxStripRows = 16;   // strip height is chosen per launch: 4, 8 or 16 rows
constexpr int kStripCols = 256;
// Per-lane run accumulators are 32-bit: a run holds at most 8 * kMaxStripRows
// pixels, and 8 * kMaxStripRows * 4080^2 must stay below 2^32.
static_assert(8ull * kMaxStripRows * 4080ull * 4080ull < (1ull << 32), "run accumulators would overflow");

struct Row10 {
    uint32_t lo, hi;   // bytes at x0 .. x0+7
    uint32_t l, r;     // bytes at x0-1 and x0+8 (edge replicated)
};

// One row of a plane for the 8 pixels of this lane plus its two neighbours.
// Must be called by all 32 lanes together (it shuffles).
__device__ __forceinline__ Row10 fetch_row(const uint8_t* __restrict__ plane, int h, int w, int y, int xs,
                                           bool fast, int lane) {
    y = y < 0 ? 0 : (y >= h ? h - 1 : y);
    const uint8_t* row = plane + (int64_t)y * w;
    const int x0 = xs + 8 * lane;
    Row10 R;
    if (fast && x0 + 8 <= w) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(row + x0));
        R.lo = v.x;
        R.hi = v.y;
    } else {
        uint32_t b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int x = x0 + i;
            x = x < w ? x : w - 1;
            b[i] = __ldg(row + x);
        }
        R.lo = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
        R.hi = b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24);
    }
    const uint32_t from_left = __shfl_up_sync(0xffffffffu, R.hi >> 24, 1);
    const uint32_t from_right = __shfl_down_sync(0xffffffffu, R.lo & 255u, 1);
    if (lane == 0) {
        const int xl = x0 > 0 ? x0 - 1 : 0;
        R.l = __ldg(row + (xl < w ? xl : w - 1));
    } else {
        R.l = from_left;
    }
    if (lane == 31) {
        const int xr = x0 + 8 < w ? x0 + 8 : w - 1;
        R.r = __ldg(row + xr);
    } else {
        R.r = from_right;
    }
    return R;
}

// 16-bit pairs (pixel 2k in the low half, 2k+1 in the high half) of the 8 bytes.
__device__ __forceinline__ void unpack_pairs(const Row10& a, uint32_t (&p)[4]) {
    p[0] = __byte_perm(a.lo, 0, 0x4140);
    p[1] = __byte_perm(a.lo, 0, 0x4342);
    p[2] = __byte_perm(a.hi, 0, 0x4140);
    p[3] = __byte_perm(a.hi, 0, 0x4342);
}

// x = 16 S* (3x3 binomial, gf_on = 1) or x = 16 S (gf_on = 0), as 16-bit pairs.
__device__ __forceinline__ void gf_pairs(const Row10& a, const Row10& b, const Row10& c, bool gf_on,
                                         uint32_t (&X)[4]) {
    uint32_t pb[4];
    unpack_pairs(b, pb);
    if (!gf_on) {
#pragma unroll
        for (int k = 0; k < 4; ++k) X[k] = pb[k] << 4;
        return;
    }
    uint32_t pa[4], pc[4], V[4];
    unpack_pairs(a, pa);
    unpack_pairs(c, pc);
#pragma unroll
    for (int k = 0; k < 4; ++k) V[k] = pa[k] + 2u * pb[k] + pc[k];
    const uint32_t Vl = a.l + 2u * b.l + c.l, Vr = a.r + 2u * b.r + c.r;
    const uint32_t L0 = __byte_perm(Vl, V[0], 0x5410);     // (V[-1], V[0])
    const uint32_t L1 = __byte_perm(V[0], V[1], 0x5432);   // (V[1], V[2])
    const uint32_t L2 = __byte_perm(V[1], V[2], 0x5432);   // (V[3], V[4])
    const uint32_t L3 = __byte_perm(V[2], V[3], 0x5432);   // (V[5], V[6])
    const uint32_t R3 = __byte_perm(V[3], Vr, 0x5432);     // (V[7], V[8])
    X[0] = L0 + 2u * V[0] + L1;
    X[1] = L1 + 2u * V[1] + L2;
    X[2] = L2 + 2u * V[2] + L3;
    X[3] = L3 + 2u * V[3] + R3;
}

// Sliding 3-row window of the three S planes down one strip.  With the
// filter on, rows y-1, y, y+1 are held and one new row is fetched per step;
// with it off only row y is needed.  All 32 lanes must call together.
struct GfWindow {
    const uint8_t* s3;
    int64_t n;
    int h, w, xs, lane;
    bool fast, gf;
    Row10 prv[3], cur[3];

    __device__ __forceinline__ void start(int y0) {
        if (!gf) return;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            prv[c] = fetch_row(s3 + c * n, h, w, y0 - 1, xs, fast, lane);
            cur[c] = fetch_row(s3 + c * n, h, w, y0, xs, fast, lane);
        }
    }

    // x values of row y (which must follow the previous call's row) as 16-bit pairs.
    __device__ __forceinline__ void row(int y, uint32_t (&X)[3][4]) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (gf) {
                const Row10 nxt = fetch_row(s3 + c * n, h, w, y + 1, xs, fast, lane);
                gf_pairs(prv[c], cur[c], nxt, true, X[c]);
                prv[c] = cur[c];
                cur[c] = nxt;
            } else {
                const Row10 r = fetch_row(s3 + c * n, h, w, y, xs, fast, lane);
                gf_pairs(r, r, r, false, X[c]);
            }
        }
    }
};

__device__ __forceinline__ int half_of(const uint32_t (&X)[4], int i) {
    return (int)((X[i >> 1] >> (16 * (i & 1))) & 0xFFFFu);
}

__device__ __forceinline__ void load_bytes8(const uint8_t* __restrict__ plane, int w, int y, int x0, bool fast,
                                            uint32_t& lo, uint32_t& hi) {
    const uint8_t* row = plane + (int64_t)y * w;
    if (fast && x0 + 8 <= w) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(row + x0));
        lo = v.x;
        hi = v.y;
    } else {
        uint32_t b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) b[i] = (x0 + i < w) ? (uint32_t)__ldg(row + x0 + i) : 0u;
        lo = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
        hi = b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24);
    }
}

// ====================================================================== fit

struct RunAcc {
    int E;            // region of the run, -1 = empty
    uint32_t n;
    uint32_t sx[3], sy[3], sxy[3], sxx[3];
};

__device__ __forceinline__ void run_reset(RunAcc& a, int E) {
    a.E = E;
    a.n = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) a.sx[c] = a.sy[c] = a.sxy[c] = a.sxx[c] = 0;
}

// Bins in shared memory, [E][13] twice: a sum is hi * 2^12 + lo, and every
// addend v goes in as v mod 2^12 (to lo) and v / 2^12 (to hi) with
// fire-and-forget shared-memory reductions, so no thread waits for an atomic.
// Exact while a block adds at most kMaxBlockPixels pixels between flushes to
// global memory: each addition covers at least one pixel, so lo stays below
// 2^20 (2^12 - 1) < 2^32, and hi below 2^20 * 4080^2 / 2^12 < 2^32.
constexpr int64_t kMaxBlockPixels = (int64_t)1 << 20;
static_assert((unsigned long long)kMaxBlockPixels * 4080ull * 4080ull / 4096ull < (1ull << 32), "hi words overflow");

struct SmemBins {
    uint32_t lo[kNbin * kNsum];
    uint32_t hi[kNbin * kNsum];
};

__device__ __forceinline__ void red_add(uint32_t addr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Adds the 13 sums of region E (values below 2^44) to the bins at shared
// address `bins`.
__device__ __forceinline__ void bins_add(uint32_t bins, int E, const unsigned long long (&v)[kNsum]) {
    const uint32_t lo = bins + 4u * (uint32_t)(E * kNsum), hi = lo + 4u * kNbin * kNsum;
#pragma unroll
    for (int j = 0; j < kNsum; ++j) {
        red_add(lo + 4u * j, (uint32_t)v[j] & 0xFFFu);
        red_add(hi + 4u * j, (uint32_t)(v[j] >> 12));
    }
}

__device__ __forceinline__ void bins_add32(uint32_t bins, int E, const uint32_t (&v)[kNsum]) {
    const uint32_t lo = bins + 4u * (uint32_t)(E * kNsum), hi = lo + 4u * kNbin * kNsum;
#pragma unroll
    for (int j = 0; j < kNsum; ++j) {
        red_add(lo + 4u * j, v[j] & 0xFFFu);
        red_add(hi + 4u * j, v[j] >> 12);
    }
}

__device__ __forceinline__ void run_values(const RunAcc& a, unsigned long long (&v)[kNsum]) {
    v[0] = a.n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[1 + 4 * c] = a.sx[c];
        v[2 + 4 * c] = a.sy[c];
        v[3 + 4 * c] = a.sxy[c];
        v[4 + 4 * c] = a.sxx[c];
    }
}

// Flush of one lane's run (divergent call sites).
__device__ __forceinline__ void run_flush(const RunAcc& a, SmemBins& B) {
    if (a.E < 0 || a.n == 0) return;
    unsigned long long v[kNsum];
    run_values(a, v);
    bins_add(smem_addr(&B), a.E, v);
}

// Flush of all lanes' runs at a warp-uniform point: when every non-empty run
// is in the same region the warp reduces them first and one lane adds.  A
// lane's run holds at most 8 * kMaxStripRows = 128 pixels, so warp totals of
// N, sum x, sum y and sum xy stay below 2^32 (4096 * 4080 * 255 < 2^32) and
// use the 32-bit warp reduction; sum xx needs 64 bits.
static_assert(32ull * 8 * kMaxStripRows * 4080ull * 255ull < (1ull << 32), "warp sums of x y exceed 32 bits");

__device__ __forceinline__ void warp_flush(const RunAcc& a, SmemBins& B, int lane) {
    const bool live = a.E >= 0 && a.n != 0;
    const unsigned liveMask = __ballot_sync(0xffffffffu, live);
    if (!liveMask) return;
    const int E0 = __shfl_sync(0xffffffffu, a.E, __ffs(liveMask) - 1);
    if (__all_sync(0xffffffffu, !live || a.E == E0)) {
        unsigned long long v[kNsum];
        v[0] = __reduce_add_sync(0xffffffffu, live ? a.n : 0u);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[1 + 4 * c] = __reduce_add_sync(0xffffffffu, live ? a.sx[c] : 0u);
            v[2 + 4 * c] = __reduce_add_sync(0xffffffffu, live ? a.sy[c] : 0u);
            v[3 + 4 * c] = __reduce_add_sync(0xffffffffu, live ? a.sxy[c] : 0u);
            unsigned long long q = live ? a.sxx[c] : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
            v[4 + 4 * c] = q;
        }
        if (lane == 0) bins_add(smem_addr(&B), E0, v);
    } else {
        run_flush(a, B);
    }
}

// Sums of one channel of an 8-pixel segment over the pixels whose byte of
// `klo/khi` is 0xFF; k16 is the mask expanded to the 16-bit x pairs.
__device__ __forceinline__ void chan_sums(const uint32_t (&X)[4], uint32_t ml, uint32_t mh, uint32_t klo,
                                          uint32_t khi, const uint32_t (&k16)[4], RunAcc& a, int c) {
    uint32_t x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = X[k] & k16[k];
    const uint32_t yl = ml & klo, yh = mh & khi;
    const uint32_t ps = x[0] + x[1] + x[2] + x[3];
    a.sx[c] = (ps & 0xFFFFu) + (ps >> 16);
    a.sy[c] = __dp4a(yl, 0x01010101u, __dp4a(yh, 0x01010101u, 0u));
    uint32_t q = __dp2a_lo(x[0], yl, 0u);
    q = __dp2a_hi(x[1], yl, q);
    q = __dp2a_lo(x[2], yh, q);
    a.sxy[c] = __dp2a_hi(x[3], yh, q);
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t lo16 = x[k] & 0xFFFFu, hi16 = x[k] >> 16;
        r += lo16 * lo16 + hi16 * hi16;
    }
    a.sxx[c] = r;
}

__device__ __forceinline__ void mask16(uint32_t klo, uint32_t khi, uint32_t (&k16)[4]) {
    k16[0] = __byte_perm(klo, 0, 0x1100);
    k16[1] = __byte_perm(klo, 0, 0x3322);
    k16[2] = __byte_perm(khi, 0, 0x1100);
    k16[3] = __byte_perm(khi, 0, 0x3322);
}

// Sums of one 8-pixel segment, restricted to the pixels whose byte of `klo/khi`
// is 0xFF (all ones for all pixels).
__device__ __forceinline__ void seg_sums(const uint32_t (&X)[3][4], const uint32_t (&mlo)[3], const uint32_t (&mhi)[3],
                                         uint32_t klo, uint32_t khi, RunAcc& a) {
    uint32_t k16[4];
    mask16(klo, khi, k16);
    a.n = (uint32_t)(__popc(klo) + __popc(khi)) >> 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) chan_sums(X[c], mlo[c], mhi[c], klo, khi, k16, a, c);
}

__device__ __forceinline__ void run_merge(RunAcc& a, const RunAcc& b) {
    a.n += b.n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a.sx[c] += b.sx[c];
        a.sy[c] += b.sy[c];
        a.sxy[c] += b.sxy[c];
        a.sxx[c] += b.sxx[c];
    }
}

__device__ __forceinline__ void run_minus(RunAcc& a, const RunAcc& b) {   // a -= b
    a.n -= b.n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a.sx[c] -= b.sx[c];
        a.sy[c] -= b.sy[c];
        a.sxy[c] -= b.sxy[c];
        a.sxx[c] -= b.sxx[c];
    }
}

// Largest byte of a pair of words.
__device__ __forceinline__ uint32_t max_byte(uint32_t lo, uint32_t hi) {
    uint32_t m = __vmaxu4(lo, hi);
    m = __vmaxu4(m, m >> 16);
    m = __vmaxu4(m, m >> 8);
    return m & 255u;
}

// Add a segment's sums for region E to the run of E's parity, flushing the
// run first when it holds another region of that parity.
__device__ __forceinline__ void run_feed(RunAcc& run, int E, const RunAcc& part, SmemBins& bins) {
    if (part.n == 0) return;
    if (E != run.E) {
        run_flush(run, bins);
        run_reset(run, E);
    }
    run_merge(run, part);
}

// Segments with three or more exponents (or ragged ones) are queued per warp
// and drained 32 at a time, one per lane, so the rare per-pixel work does not
// make every lane of the warp wait on it.  An entry is 21 words: the exponent
// bytes, the mantissa bytes of the three planes, the x pairs and the count;
// the odd stride keeps the lanes' accesses on distinct banks.
constexpr int kQueueStride = 21;

// Adds one queued entry to the bins: a flushed run (tag 256 + E; words 0-12
// hold N and the channel sums in bin order) or a segment (tag = pixel
// count), whose pixels are summed in order and added once per stretch of
// equal exponents.
template <bool kUnroll>
__device__ __forceinline__ void drain_entry(const uint32_t* q, uint32_t B) {
    const uint32_t tag = q[20];
    uint32_t acc[kNsum];
    if (tag >= 256u) {
#pragma unroll
        for (int j = 0; j < kNsum; ++j) acc[j] = q[j];
        bins_add32(B, (int)(tag - 256u), acc);
        return;
    }
    uint32_t elo = q[0], ehi = q[1];
    uint32_t mlo[3] = {q[2], q[3], q[4]}, mhi[3] = {q[5], q[6], q[7]};
    uint32_t X[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) X[c][k] = q[8 + 4 * c + k];
    const int cnt = (int)tag;
    int Ecur = (int)(elo & 255u);
#pragma unroll
    for (int j = 0; j < kNsum; ++j) acc[j] = 0u;
    if constexpr (kUnroll) {
        // fully unrolled: every byte and pair is picked with a constant index
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i < cnt) {
                const int E = (int)byte_of(i < 4 ? elo : ehi, i & 3);
                if (E != Ecur) {
                    bins_add32(B, Ecur, acc);
#pragma unroll
                    for (int j = 0; j < kNsum; ++j) acc[j] = 0u;
                    Ecur = E;
                }
                acc[0] += 1u;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const uint32_t x = (X[c][i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
                    const uint32_t yv = byte_of(i < 4 ? mlo[c] : mhi[c], i & 3);
                    acc[1 + 4 * c] += x;
                    acc[2 + 4 * c] += yv;
                    acc[3 + 4 * c] += x * yv;
                    acc[4 + 4 * c] += x * x;
                }
            }
        }
    } else {
        // compact loop (fewer registers): shift the next pixel into place
#pragma unroll 1
        for (int i = 0; i < cnt; ++i) {
            const int E = (int)(elo & 255u);
            elo = __funnelshift_r(elo, ehi, 8);
            ehi >>= 8;
            if (E != Ecur) {
                bins_add32(B, Ecur, acc);
#pragma unroll
                for (int j = 0; j < kNsum; ++j) acc[j] = 0u;
                Ecur = E;
            }
            acc[0] += 1u;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const uint32_t x = X[c][0] & 0xFFFFu, yv = mlo[c] & 255u;
                acc[1 + 4 * c] += x;
                acc[2 + 4 * c] += yv;
                acc[3 + 4 * c] += x * yv;
                acc[4 + 4 * c] += x * x;
                mlo[c] = __funnelshift_r(mlo[c], mhi[c], 8);
                mhi[c] >>= 8;
                X[c][0] = __funnelshift_r(X[c][0], X[c][1], 16);
                X[c][1] = __funnelshift_r(X[c][1], X[c][2], 16);
                X[c][2] = __funnelshift_r(X[c][2], X[c][3], 16);
                X[c][3] >>= 16;
            }
        }
    }
    bins_add32(B, Ecur, acc);
}

// Per-warp state of the fit: one run per exponent parity (adjacent regions
// of a smooth exponent field differ by one, so a boundary through a lane's
// column feeds the two runs without flushing either) and the queue of
// segments that need per-pixel work.
struct FitWarp {
    RunAcc even, odd;
    uint32_t* Q;
    int queued;   // entries in the queue (warp-uniform)
};

// Drains the warp's queue, one entry per lane (kUnroll: the faster drain
// that needs more registers).
template <bool kUnroll = false>
__device__ __forceinline__ void fit_drain(FitWarp& st, SmemBins& bins, int lane) {
    if (lane < st.queued) drain_entry<kUnroll>(st.Q + lane * kQueueStride, smem_addr(&bins));
    __syncwarp();
    st.queued = 0;
}

// Queues the run of every lane with `want` set (a run that must leave its
// accumulator in the middle of a strip); the warp drains them together later
// instead of waiting on one lane's atomics.
template <bool kUnroll = false>
__device__ __forceinline__ void enqueue_run(FitWarp& st, bool want, const RunAcc& r, SmemBins& bins, int lane) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return;
    if (st.queued + __popc(m) > 32) fit_drain<kUnroll>(st, bins, lane);
    if (want) {
        uint32_t* q = st.Q + (st.queued + __popc(m & ((1u << lane) - 1u))) * kQueueStride;
        q[0] = r.n;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            q[1 + 4 * c] = r.sx[c];
            q[2 + 4 * c] = r.sy[c];
            q[3 + 4 * c] = r.sxy[c];
            q[4 + 4 * c] = r.sxx[c];
        }
        q[20] = 256u + (uint32_t)r.E;
    }
    __syncwarp();
    st.queued += __popc(m);
}

// One strip of one image (all 32 lanes): rows y0 .. y0 + rows - 1, columns xs .. xs + 255.
__device__ __forceinline__ void fit_strip(const uint8_t* __restrict__ s3, const uint8_t* __restrict__ m3,
                                          const uint8_t* __restrict__ e, int h, int w, bool gf, bool fast, int y0,
                                          int rows, int xs, int lane, FitWarp& st, SmemBins& bins) {
    const int64_t n = (int64_t)h * w;
    const int x0 = xs + 8 * lane;
    const int y1 = min(y0 + rows, h);
    GfWindow win{s3, n, h, w, xs, lane, fast, gf};
    win.start(y0);
    for (int y = y0; y < y1; ++y) {
        uint32_t X[3][4];
        win.row(y, X);
        uint32_t mlo[3] = {0u, 0u, 0u}, mhi[3] = {0u, 0u, 0u}, elo = 0u, ehi = 0u;
        bool slow = false;
        if (x0 < w) {
#pragma unroll
            for (int c = 0; c < 3; ++c) load_bytes8(m3 + c * n, w, y, x0, fast, mlo[c], mhi[c]);
            load_bytes8(e, w, y, x0, fast, elo, ehi);
            // byte masks of the odd-exponent pixels and the two exponents
            const uint32_t olo = (elo & 0x01010101u) * 0xFFu, ohi = (ehi & 0x01010101u) * 0xFFu;
            const uint32_t Eo = max_byte(elo & olo, ehi & ohi);
            const uint32_t Ee = max_byte(elo & ~olo, ehi & ~ohi);
            const bool two = x0 + 8 <= w && ((elo ^ (Eo * 0x01010101u)) & olo) == 0 &&
                             ((ehi ^ (Eo * 0x01010101u)) & ohi) == 0 &&
                             ((elo ^ (Ee * 0x01010101u)) & ~olo) == 0 &&
                             ((ehi ^ (Ee * 0x01010101u)) & ~ohi) == 0;
            if (two) {
                // at most one even and one odd exponent in the segment
                RunAcc pe, po;
                seg_sums(X, mlo, mhi, 0xFFFFFFFFu, 0xFFFFFFFFu, pe);
                if ((olo | ohi) == 0u) {
                    run_reset(po, -1);
                } else if ((olo & ohi) == 0xFFFFFFFFu) {
                    po = pe;
                    run_reset(pe, -1);
                } else {
                    seg_sums(X, mlo, mhi, olo, ohi, po);
                    run_minus(pe, po);
                }
                run_feed(st.even, (int)Ee, pe, bins);
                run_feed(st.odd, (int)Eo, po, bins);
            } else {
                slow = true;
            }
        }
        // queue the segments with three or more exponents and the ragged ones
        const unsigned want = __ballot_sync(0xffffffffu, slow);
        if (want) {
            if (st.queued + __popc(want) > 32) fit_drain(st, bins, lane);
            if (slow) {
                uint32_t* q = st.Q + (st.queued + __popc(want & ((1u << lane) - 1u))) * kQueueStride;
                q[0] = elo;
                q[1] = ehi;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    q[2 + c] = mlo[c];
                    q[5 + c] = mhi[c];
#pragma unroll
                    for (int k = 0; k < 4; ++k) q[8 + 4 * c + k] = X[c][k];
                }
                q[20] = (uint32_t)min(8, w - x0);
            }
            __syncwarp();
            st.queued += __popc(want);
        }
    }
    // Every run ends with its strip, so the 32-bit run accumulators cannot
    // overflow; lanes hold their runs by parity, so equal regions flush in
    // the same warp-wide step.
    warp_flush(st.even, bins, lane);
    warp_flush(st.odd, bins, lane);
    run_reset(st.even, -1);
    run_reset(st.odd, -1);
}

__device__ __forceinline__ void bins_clear(SmemBins& bins) {
    for (int i = threadIdx.x; i < kNbin * kNsum; i += blockDim.x) bins.lo[i] = bins.hi[i] = 0u;
}

// Adds the block's bins to global int64 sums (and clears them when asked).
__device__ __forceinline__ void bins_to_global(SmemBins& bins, unsigned long long* __restrict__ g, bool clear) {
    for (int i = threadIdx.x; i < kNbin * kNsum; i += blockDim.x) {
        const unsigned long long v = ((unsigned long long)bins.hi[i] << 12) + bins.lo[i];
        if (v) {
            atomicAdd(g + i, v);
            if (clear) bins.lo[i] = bins.hi[i] = 0u;
        }
    }
}

__global__ void __launch_bounds__(kThreads, 2) k_fit(const uint8_t* __restrict__ s3, const uint8_t* __restrict__ m3,
                                                     const uint8_t* __restrict__ e, int h, int w, int gf_on,
                                                     int fast_io, int strip_rows,
                                                     unsigned long long* __restrict__ gbins) {
    __shared__ SmemBins bins;
    __shared__ uint32_t queue[kWarps][32 * kQueueStride];
    bins_clear(bins);
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cols = (w + kStripCols - 1) / kStripCols;
    const int64_t tasks = (int64_t)((h + strip_rows - 1) / strip_rows) * cols;
    FitWarp st;
    run_reset(st.even, -1);
    run_reset(st.odd, -1);
    st.Q = queue[warp];
    st.queued = 0;
    for (int64_t t = (int64_t)blockIdx.x * kWarps + warp; t < tasks; t += (int64_t)gridDim.x * kWarps)
        fit_strip(s3, m3, e, h, w, gf_on != 0, fast_io != 0, (int)(t / cols) * strip_rows, strip_rows,
                  (int)(t % cols) * kStripCols, lane, st, bins);
    fit_drain(st, bins, lane);
    __syncthreads();
    bins_to_global(bins, gbins, false);
}

// Vector loads need 8-byte aligned rows of every plane.
__device__ __forceinline__ bool planes_fast(int w, const void* a, const void* b, const void* c) {
    return (w % 8 == 0) && ((uintptr_t)a % 8 == 0) && ((uintptr_t)b % 8 == 0) && ((uintptr_t)c % 8 == 0);
}

// Batch: each CTA task is 8 strips of one image; a CTA works through a
// contiguous range of tasks, so its bins change image rarely.
__global__ void __launch_bounds__(kThreads, 2) k_fit_batch(const BatchDev B, int64_t cta_tasks,
                                                           const uint8_t* __restrict__ s3b,
                                                           const uint8_t* __restrict__ m3b,
                                                           const uint8_t* __restrict__ eb) {
    __shared__ SmemBins bins;
    __shared__ uint32_t queue[kWarps][32 * kQueueStride];
    bins_clear(bins);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    FitWarp st;
    run_reset(st.even, -1);
    run_reset(st.odd, -1);
    st.Q = queue[warp];
    st.queued = 0;
    const int64_t per = (cta_tasks + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = (int64_t)blockIdx.x * per, k1 = min(k0 + per, cta_tasks);
    int cur = -1;
    for (int64_t k = k0; k < k1; ++k) {
        const int i = batch_image_of(B.strip_prefix, B.n, k);
        if (i != cur) {
            if (cur >= 0) {
                fit_drain(st, bins, lane);
                __syncthreads();
                bins_to_global(bins, B.sums + (int64_t)cur * kNbin * kNsum, true);
                __syncthreads();
            }
            cur = i;
        }
        const BatchImage im = B.img[i];
        const int64_t n = (int64_t)im.h * im.w;
        const uint8_t* s3 = s3b + 3 * im.px;
        const uint8_t* m3 = m3b + 3 * im.px;
        const uint8_t* e = eb + im.px;
        const int cols = (im.w + kStripCols - 1) / kStripCols;
        const int64_t strips = (int64_t)((im.h + B.strip_rows - 1) / B.strip_rows) * cols;
        const int64_t t = (k - B.strip_prefix[i]) * kWarps + warp;
        if (n > 0 && t < strips)
            fit_strip(s3, m3, e, im.h, im.w, im.gf_on != 0, planes_fast(im.w, s3, m3, e),
                      (int)(t / cols) * B.strip_rows, B.strip_rows, (int)(t % cols) * kStripCols, lane, st, bins);
    }
    fit_drain(st, bins, lane);
    __syncthreads();
    if (cur >= 0) bins_to_global(bins, B.sums + (int64_t)cur * kNbin * kNsum, false);
}

// ====================================================================== solve

// Correctly rounded (nearest, ties to even) signed 128-bit integer -> double.
__device__ __forceinline__ double i128_to_f64(__int128 v) {
    if (v == 0) return 0.0;
    const bool neg = v < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)0 - (unsigned __int128)v : (unsigned __int128)v;
    const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
    const int nb = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
    double r;
    if (nb <= 53) {
        r = __ull2double_rn(lo);
    } else {
        const int sh = nb - 53;
        uint64_t mant = (uint64_t)(u >> sh);
        const unsigned __int128 rem = u - ((unsigned __int128)mant << sh);
        const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (mant & 1ull))) mant += 1;   // 2^53 is still exact
        r = __dmul_rn(__ull2double_rn(mant), __longlong_as_double((long long)(1023 + sh) << 52));
    }
    return neg ? -r : r;
}

// Slope and intercept of one (channel c, region E) of an image from its sums.
// FP64 work: a one-block solve would be bound by one SM's FP64 units, so the
// 768 solves of an image are spread over 24 warps (blocks of 32 threads).
__device__ __forceinline__ void solve_one(const int64_t* __restrict__ sums, slrme_params* __restrict__ P, int c,
                                          int E) {
    const int64_t* s = sums + E * kNsum;
    const int64_t N = s[0];
    float a = 0.0f, b = 0.0f;
    if (N > 0) {
        const int64_t sx = s[1 + 4 * c], sy = s[2 + 4 * c], sxy = s[3 + 4 * c], sxx = s[4 + 4 * c];
        const __int128 dxx = (__int128)N * sxx - (__int128)sx * sx;
        const __int128 dxy = (__int128)N * sxy - (__int128)sx * sy;
        if (dxx == 0) {
            b = __double2float_rn(__ddiv_rn(__ll2double_rn(sy), __ll2double_rn(N)));
        } else {
            a = __double2float_rn(__ddiv_rn(i128_to_f64(dxy), i128_to_f64(dxx)));
            const double t = __dmul_rn((double)a, __ll2double_rn(sx));
            b = __double2float_rn(__ddiv_rn(__dsub_rn(__ll2double_rn(sy), t), __ll2double_rn(N)));
        }
    }
    P->a[c][E] = a;
    P->b[c][E] = b;
    if (c == 0) P->n[E] = (int32_t)N;
}

// Block b (32 threads) of an image solves channel b / 8, regions 32 (b % 8) ..
// + 31; block 0 also counts the used regions.
__device__ __forceinline__ void solve_block(const int64_t* __restrict__ sums, slrme_params* __restrict__ P, int b) {
    const int lane = threadIdx.x;
    solve_one(sums, P, b >> 3, ((b & 7) << 5) + lane);
    if (b == 0) {
        int used = 0;
#pragma unroll
        for (int k = 0; k < kNbin / 32; ++k) used += __popc(__ballot_sync(0xffffffffu, sums[(32 * k + lane) * kNsum] > 0));
        if (lane == 0) {
            P->n_used = used;
            P->reserved[0] = P->reserved[1] = P->reserved[2] = 0;
        }
    }
}

constexpr int kSolveBlocks = 3 * kNbin / 32;

__global__ void __launch_bounds__(32) k_solve(const int64_t* __restrict__ sums, slrme_params* __restrict__ P) {
    solve_block(sums, P, blockIdx.x);
}

// grid (kSolveBlocks, images)
__global__ void __launch_bounds__(32) k_solve_batch(const unsigned long long* __restrict__ sums,
                                                     slrme_params* __restrict__ P) {
    solve_block(reinterpret_cast<const int64_t*>(sums) + (int64_t)blockIdx.y * kNbin * kNsum, P + blockIdx.y,
                blockIdx.x);
}

// ====================================================================== residual

__device__ __forceinline__ void load_params(const slrme_params* __restrict__ P, float* sa, float* sb) {
    for (int i = threadIdx.x; i < 3 * kNbin; i += blockDim.x) {
        sa[i] = (&P->a[0][0])[i];
        sb[i] = (&P->b[0][0])[i];
    }
}

// The parameters as (a, b) pairs, [c][E], so one 8-byte load gets both.
__device__ __forceinline__ void load_params_ab(const slrme_params* __restrict__ P, float2* ab) {
    for (int i = threadIdx.x; i < 3 * kNbin; i += blockDim.x) ab[i] = make_float2((&P->a[0][0])[i], (&P->b[0][0])[i]);
}

// One strip: R = M - M* for rows y0 .. y0 + rows - 1, columns xs .. xs + 255;
// `hist` (shared, may be null) counts the residual values.
__device__ __forceinline__ void residual_strip(const uint8_t* __restrict__ s3, const uint8_t* __restrict__ m3,
                                               const uint8_t* __restrict__ e, int h, int w, bool gf, bool fast,
                                               bool vec_r, int y0, int rows, int xs, int lane, const float* sa,
                                               const float* sb, int16_t* __restrict__ r3, uint32_t* hist) {
    const int64_t n = (int64_t)h * w;
    const int x0 = xs + 8 * lane;
    const int y1 = min(y0 + rows, h);
    GfWindow win{s3, n, h, w, xs, lane, fast, gf};
    win.start(y0);
    for (int y = y0; y < y1; ++y) {
        uint32_t X[3][4];
        win.row(y, X);
        if (x0 >= w) continue;
        uint32_t elo, ehi;
        load_bytes8(e, w, y, x0, fast, elo, ehi);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            uint32_t mlo, mhi;
            load_bytes8(m3 + c * n, w, y, x0, fast, mlo, mhi);
            int r[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int E = (int)byte_of(i < 4 ? elo : ehi, i & 3);
                const int M = (int)byte_of(i < 4 ? mlo : mhi, i & 3);
                r[i] = M - predict(sa[c * kNbin + E], sb[c * kNbin + E], half_of(X[c], i));
            }
            int16_t* row = r3 + c * n + (int64_t)y * w + x0;
            if (vec_r && x0 + 8 <= w) {
                uint4 v;
                v.x = (uint32_t)(r[0] & 0xFFFF) | ((uint32_t)r[1] << 16);
                v.y = (uint32_t)(r[2] & 0xFFFF) | ((uint32_t)r[3] << 16);
                v.z = (uint32_t)(r[4] & 0xFFFF) | ((uint32_t)r[5] << 16);
                v.w = (uint32_t)(r[6] & 0xFFFF) | ((uint32_t)r[7] << 16);
                *reinterpret_cast<uint4*>(row) = v;
                if (hist) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) atomicAdd(&hist[c * kNres + r[i] + 255], 1u);
                }
            } else {
                const int cnt = min(8, w - x0);
                for (int i = 0; i < cnt; ++i) {
                    row[i] = (int16_t)r[i];
                    if (hist) atomicAdd(&hist[c * kNres + r[i] + 255], 1u);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_residual(const uint8_t* __restrict__ s3, const uint8_t* __restrict__ m3,
                                                       const uint8_t* __restrict__ e, int h, int w, int gf_on,
                                                       int fast_io, int strip_rows, const slrme_params* __restrict__ P,
                                                       int16_t* __restrict__ r3, uint32_t* __restrict__ ghist) {
    __shared__ float sa[3 * kNbin], sb[3 * kNbin];
    __shared__ uint32_t hist[3 * kNres];
    load_params(P, sa, sb);
    if (ghist)
        for (int i = threadIdx.x; i < 3 * kNres; i += kThreads) hist[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cols = (w + kStripCols - 1) / kStripCols;
    const int64_t tasks = (int64_t)((h + strip_rows - 1) / strip_rows) * cols;
    const bool vec_r = fast_io != 0 && ((uintptr_t)r3 % 16 == 0);
    for (int64_t t = (int64_t)blockIdx.x * kWarps + warp; t < tasks; t += (int64_t)gridDim.x * kWarps)
        residual_strip(s3, m3, e, h, w, gf_on != 0, fast_io != 0, vec_r, (int)(t / cols) * strip_rows, strip_rows,
                       (int)(t % cols) * kStripCols, lane, sa, sb, r3, ghist ? hist : nullptr);
    if (ghist) {
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * kNres; i += kThreads)
            if (hist[i]) atomicAdd(ghist + i, hist[i]);
    }
}

// Batch: CTA tasks of 8 strips of one image; parameters and histogram of the
// current image stay in shared memory until the CTA moves to the next image.
__global__ void __launch_bounds__(kThreads) k_residual_batch(const BatchDev B, int64_t cta_tasks,
                                                             const uint8_t* __restrict__ s3b,
                                                             const uint8_t* __restrict__ m3b,
                                                             const uint8_t* __restrict__ eb,
                                                             const slrme_params* __restrict__ P,
                                                             int16_t* __restrict__ r3b, uint32_t* __restrict__ ghist) {
    __shared__ float sa[3 * kNbin], sb[3 * kNbin];
    __shared__ uint32_t hist[3 * kNres];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t per = (cta_tasks + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = (int64_t)blockIdx.x * per, k1 = min(k0 + per, cta_tasks);
    int cur = -1;
    for (int64_t k = k0; k < k1; ++k) {
        const int i = batch_image_of(B.strip_prefix, B.n, k);
        if (i != cur) {
            __syncthreads();
            if (cur >= 0 && ghist)
                for (int j = threadIdx.x; j < 3 * kNres; j += kThreads)
                    if (hist[j]) atomicAdd(ghist + (int64_t)cur * 3 * kNres + j, hist[j]);
            load_params(P + i, sa, sb);
            for (int j = threadIdx.x; j < 3 * kNres; j += kThreads) hist[j] = 0u;
            __syncthreads();
            cur = i;
        }
        const BatchImage im = B.img[i];
        const uint8_t* s3 = s3b + 3 * im.px;
        const uint8_t* m3 = m3b + 3 * im.px;
        const uint8_t* e = eb + im.px;
        int16_t* r3 = r3b + 3 * im.px;
        const int cols = (im.w + kStripCols - 1) / kStripCols;
        const int64_t strips = (int64_t)((im.h + B.strip_rows - 1) / B.strip_rows) * cols;
        const int64_t t = (k - B.strip_prefix[i]) * kWarps + warp;
        const bool fast = planes_fast(im.w, s3, m3, e);
        if ((int64_t)im.h * im.w > 0 && t < strips)
            residual_strip(s3, m3, e, im.h, im.w, im.gf_on != 0, fast, fast && ((uintptr_t)r3 % 16 == 0),
                           (int)(t / cols) * B.strip_rows, B.strip_rows, (int)(t % cols) * kStripCols, lane, sa, sb,
                           r3, ghist ? hist : nullptr);
    }
    __syncthreads();
    if (cur >= 0 && ghist)
        for (int j = threadIdx.x; j < 3 * kNres; j += kThreads)
            if (hist[j]) atomicAdd(ghist + (int64_t)cur * 3 * kNres + j, hist[j]);
}

// ====================================================================== decode

// One strip: M = R + M*, repacked with E into RGBE words.
__device__ __forceinline__ void decode_strip(const uint8_t* __restrict__ s3, const uint8_t* __restrict__ e,
                                             const int16_t* __restrict__ r3, int h, int w, bool gf, bool fast,
                                             bool vec, int y0, int rows, int xs, int lane, const float* sa,
                                             const float* sb, uint32_t* __restrict__ out) {
    const int64_t n = (int64_t)h * w;
    const int x0 = xs + 8 * lane;
    const int y1 = min(y0 + rows, h);
    GfWindow win{s3, n, h, w, xs, lane, fast, gf};
    win.start(y0);
    for (int y = y0; y < y1; ++y) {
        uint32_t X[3][4];
        win.row(y, X);
        if (x0 >= w) continue;
        uint32_t elo, ehi;
        load_bytes8(e, w, y, x0, fast, elo, ehi);
        uint32_t word[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) word[i] = byte_of(i < 4 ? elo : ehi, i & 3) << 24;
        const bool v8 = vec && x0 + 8 <= w;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int16_t* row = r3 + c * n + (int64_t)y * w + x0;
            int r[8];
            if (v8) {
                const uint4 v = __ldg(reinterpret_cast<const uint4*>(row));
                const uint32_t q[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    r[2 * k] = (int)(int16_t)(q[k] & 0xFFFFu);
                    r[2 * k + 1] = (int)(int16_t)(q[k] >> 16);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) r[i] = (x0 + i < w) ? (int)__ldg(row + i) : 0;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int E = (int)(word[i] >> 24);
                const int M = r[i] + predict(sa[c * kNbin + E], sb[c * kNbin + E], half_of(X[c], i));
                word[i] |= ((uint32_t)M & 255u) << (8 * c);
            }
        }
        uint32_t* orow = out + (int64_t)y * w + x0;
        if (v8) {
            reinterpret_cast<uint4*>(orow)[0] = make_uint4(word[0], word[1], word[2], word[3]);
            reinterpret_cast<uint4*>(orow)[1] = make_uint4(word[4], word[5], word[6], word[7]);
        } else {
            const int cnt = min(8, w - x0);
            for (int i = 0; i < cnt; ++i) orow[i] = word[i];
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_decode(const uint8_t* __restrict__ s3, const uint8_t* __restrict__ e,
                                                     const int16_t* __restrict__ r3, int h, int w, int gf_on,
                                                     int fast_io, int strip_rows, const slrme_params* __restrict__ P,
                                                     uint32_t* __restrict__ out) {
    __shared__ float sa[3 * kNbin], sb[3 * kNbin];
    load_params(P, sa, sb);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cols = (w + kStripCols - 1) / kStripCols;
    const int64_t tasks = (int64_t)((h + strip_rows - 1) / strip_rows) * cols;
    const bool vec = fast_io != 0 && ((uintptr_t)r3 % 16 == 0) && ((uintptr_t)out % 16 == 0);
    for (int64_t t = (int64_t)blockIdx.x * kWarps + warp; t < tasks; t += (int64_t)gridDim.x * kWarps)
        decode_strip(s3, e, r3, h, w, gf_on != 0, fast_io != 0, vec, (int)(t / cols) * strip_rows, strip_rows,
                     (int)(t % cols) * kStripCols, lane, sa, sb, out);
}

__global__ void __launch_bounds__(kThreads) k_decode_batch(const BatchDev B, int64_t cta_tasks,
                                                           const uint8_t* __restrict__ s3b,
                                                           const uint8_t* __restrict__ eb,
                                                           const int16_t* __restrict__ r3b,
                                                           const slrme_params* __restrict__ P,
                                                           uint32_t* __restrict__ outb) {
    __shared__ float sa[3 * kNbin], sb[3 * kNbin];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t per = (cta_tasks + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = (int64_t)blockIdx.x * per, k1 = min(k0 + per, cta_tasks);
    int cur = -1;
    for (int64_t k = k0; k < k1; ++k) {
        const int i = batch_image_of(B.strip_prefix, B.n, k);
        if (i != cur) {
            __syncthreads();
            load_params(P + i, sa, sb);
            __syncthreads();
            cur = i;
        }
        const BatchImage im = B.img[i];
        const uint8_t* s3 = s3b + 3 * im.px;
        const uint8_t* e = eb + im.px;
        const int16_t* r3 = r3b + 3 * im.px;
        uint32_t* out = outb + im.px;
        const int cols = (im.w + kStripCols - 1) / kStripCols;
        const int64_t strips = (int64_t)((im.h + B.strip_rows - 1) / B.strip_rows) * cols;
        const int64_t t = (k - B.strip_prefix[i]) * kWarps + warp;
        const bool fast = (im.w % 8 == 0) && ((uintptr_t)s3 % 8 == 0) && ((uintptr_t)e % 8 == 0);
        const bool vec = fast && ((uintptr_t)r3 % 16 == 0) && ((uintptr_t)out % 16 == 0);
        if ((int64_t)im.h * im.w > 0 && t < strips)
            decode_strip(s3, e, r3, im.h, im.w, im.gf_on != 0, fast, vec, (int)(t / cols) * B.strip_rows,
                         B.strip_rows, (int)(t % cols) * kStripCols, lane, sa, sb, out);
    }
}

// ====================================================================== TMA-staged row pipelines
//
// For images whose rows are 16-byte aligned (w % 16 == 0, 16-byte aligned
// planes).  The rows of all 256-column strips are taken in column-major
// order (strip, row) and cut into one contiguous range per warp, so every
// warp does the same number of rows to within one; a range becomes tasks of
// at most kMaxStripRows rows of one strip.  Each warp streams its rows
// through two rings of shared-memory slots filled by 1-D bulk copies
// (cp.async.bulk) that complete on the slot's mbarrier: S rows of the three
// planes with 16 halo columns (row j of a task needs S rows j - 1, j, j + 1,
// clamped to the image) and, up to two rows ahead, the row's other planes
// (M and E for the fit and the residual, R and E for the decoder).  No
// CTA-wide barrier is involved; data in flight costs shared memory, not
// registers.  Every wait is bounded (see tma.cuh).

constexpr int kSW = 288;          // S row segment: 16 halo + 256 + 16 halo bytes
constexpr int kRowWarps = 8;      // warps per CTA (independent pipelines)
constexpr int kSSlots = 5;        // S rows
constexpr int kAuxSlots = 3;      // M / E (or R / E) rows

enum class TmaMode { kResidual = 0, kDecode = 1, kFit = 2 };

struct SRow {
    uint8_t S[3][kSW];
};

template <TmaMode MODE>
struct AuxSlot {                  // fit and residual: M and E
    uint8_t M[3][kStripCols];
    uint8_t E[kStripCols];
};

template <>
struct AuxSlot<TmaMode::kDecode> {
    int16_t R[3][kStripCols];
    uint8_t E[kStripCols];
};

struct TmaImage {
    const uint8_t* s3;
    const uint8_t* m3;
    const uint8_t* e;
    const int16_t* r3_in;
    int16_t* r3_out;
    uint32_t* out;
    int h, w;
    bool gf;
};

// A warp's rows r .. end - 1 in (strip, row) order and its current task.
struct RowRange {
    int r, end, h;
    int y0, rows, xs;
    // Takes the next task; false when the range is done.
    __device__ __forceinline__ bool next() {
        if (r >= end) return false;
        const int c = r / h;
        y0 = r - c * h;
        rows = min(min(end - r, h - y0), kMaxStripRows);
        xs = c * kStripCols;
        r += rows;
        return true;
    }
};

// The warp's range of rows: warp gw of `warps` gets rows
// [gw total / warps, (gw + 1) total / warps).
__device__ __forceinline__ RowRange warp_rows(int64_t total_rows, int h, int per_block) {
    const int64_t warps = (int64_t)gridDim.x * per_block;
    const int64_t gw = (int64_t)blockIdx.x * per_block + (threadIdx.x >> 5);
    return RowRange{(int)(gw * total_rows / warps), (int)((gw + 1) * total_rows / warps), h, 0, 0, 0};
}

// One lane's S row segment from a slot: 8 bytes plus the neighbours at the
// precomputed offsets (which point at the lane's own edge byte where the
// image ends, replicating it).
__device__ __forceinline__ Row10 seg_row(const uint8_t* row, int own, int offl, int offr) {
    Row10 R;
    const uint2 v = *reinterpret_cast<const uint2*>(row + own);
    R.lo = v.x;
    R.hi = v.y;
    R.l = row[offl];
    R.r = row[offr];
    return R;
}

// Copies S row ys, columns xs - 16 .. xs + 271 (clipped to the image), of the
// three planes (lanes 0-2).
__device__ __forceinline__ void issue_s(const TmaImage& im, int64_t n, int ys, int xs, SRow& sl, uint32_t bar,
                                        int lane) {
    const int padl = xs >= 16 ? 16 : 0;
    const int bytes = min(xs + kStripCols + 16, im.w) - (xs - padl);
    fence_async_shared();
    if (lane == 0) mbar_arrive_expect_tx(bar, 3u * (uint32_t)bytes);
    __syncwarp();
    if (lane < 3)
        tma_load_1d(smem_addr(&sl.S[lane][16 - padl]), im.s3 + lane * n + (int64_t)ys * im.w + xs - padl,
                    (uint32_t)bytes, bar);
}

// Copies the other planes of row y, columns xs .. xs + 255 (lanes 0-3).
template <TmaMode MODE>
__device__ __forceinline__ void issue_aux(const TmaImage& im, int64_t n, int y, int xs, AuxSlot<MODE>& sl,
                                          uint32_t bar, int lane) {
    const int bytes = min(kStripCols, im.w - xs);
    constexpr int kRb = MODE == TmaMode::kDecode ? 2 : 1;   // bytes per element of planes 0-2
    fence_async_shared();
    if (lane == 0) mbar_arrive_expect_tx(bar, (3u * kRb + 1u) * (uint32_t)bytes);
    __syncwarp();
    const int64_t off = (int64_t)y * im.w + xs;
    if (lane < 3) {
        if constexpr (MODE == TmaMode::kDecode)
            tma_load_1d(smem_addr(&sl.R[lane][0]), im.r3_in + lane * n + off, 2u * (uint32_t)bytes, bar);
        else
            tma_load_1d(smem_addr(&sl.M[lane][0]), im.m3 + lane * n + off, (uint32_t)bytes, bar);
    } else if (lane == 3) {
        tma_load_1d(smem_addr(&sl.E[0]), im.e + off, (uint32_t)bytes, bar);
    }
}

// The two producers and the consumer's bookkeeping of one warp's rings.
template <TmaMode MODE>
struct RowPipe {
    SRow* ring;
    AuxSlot<MODE>* aux;
    unsigned long long* bars;    // kSSlots S barriers, then kAuxSlots aux barriers
    // S producer: task and item (0 .. rows + 1) issued next
    RowRange P;
    bool p_valid;
    int pk, p_slot, issued, released;
    // aux producer: the warp's rows one by one
    RowRange A;
    bool a_valid;
    int aj, a_slot, a_issued;
    // consumer: S slot of the task's first item, expected phase parities, the
    // warp's row count q and the aux slot of row q
    int c_slot, q, mc;
    uint32_t par, mpar;

    __device__ __forceinline__ void init(const RowRange& R) {
        P = R;
        p_valid = P.next();
        pk = p_slot = issued = released = 0;
        A = R;
        a_valid = A.next();
        aj = a_slot = a_issued = 0;
        c_slot = q = mc = 0;
        par = mpar = 0u;
    }
    __device__ __forceinline__ uint32_t sbar(int s) const { return smem_addr(&bars[s]); }
    __device__ __forceinline__ uint32_t abar(int s) const { return smem_addr(&bars[kSSlots + s]); }

    // keep kSSlots S items in flight or unreleased
    __device__ __forceinline__ void refill_s(const TmaImage& im, int64_t n, int lane) {
        while (p_valid && issued < released + kSSlots) {
            issue_s(im, n, min(max(P.y0 - 1 + pk, 0), im.h - 1), P.xs, ring[p_slot], sbar(p_slot), lane);
            ++issued;
            p_slot = p_slot + 1 == kSSlots ? 0 : p_slot + 1;
            if (++pk == P.rows + 2) {
                pk = 0;
                p_valid = P.next();
            }
        }
    }
    // keep rows q_done .. q_done + kAuxSlots - 1 in flight or ready
    __device__ __forceinline__ void refill_aux(const TmaImage& im, int64_t n, int q_done, int lane) {
        while (a_valid && a_issued < q_done + kAuxSlots) {
            issue_aux<MODE>(im, n, A.y0 + aj, A.xs, aux[a_slot], abar(a_slot), lane);
            ++a_issued;
            a_slot = a_slot + 1 == kAuxSlots ? 0 : a_slot + 1;
            if (++aj == A.rows) {
                aj = 0;
                a_valid = A.next();
            }
        }
    }
    // after a wait gave up: a bounded wait for every unreleased copy (each
    // has a slot of its own)
    __device__ __forceinline__ void drain_in_flight() {
        int s = p_slot;
        for (int g = issued - 1; g >= released; --g) {
            s = s == 0 ? kSSlots - 1 : s - 1;
            mbar_wait(sbar(s), (par >> s) & 1u, &g_slrme_status, 1 << 10);
        }
        s = a_slot;
        for (int g = a_issued - 1; g >= q; --g) {
            s = s == 0 ? kAuxSlots - 1 : s - 1;
            mbar_wait(abar(s), (mpar >> s) & 1u, &g_slrme_status, 1 << 10);
        }
    }
};

template <TmaMode MODE>
constexpr size_t rows_smem_bytes(int warps) {
    return (sizeof(SRow) * kSSlots + sizeof(AuxSlot<MODE>) * kAuxSlots + 8 * (kSSlots + kAuxSlots)) * warps;
}

// k_rows_tma<kResidual>: R = M - M* and histograms; k_rows_tma<kDecode>:
// M = R + M*, repacked with E.
template <TmaMode MODE>
__global__ void __launch_bounds__(kRowWarps * 32, 2) k_rows_tma(const TmaImage im, const slrme_params* __restrict__ P,
                                                                uint32_t* __restrict__ ghist, int64_t total_rows,
                                                                int max_spins) {
    extern __shared__ __align__(128) char dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RowPipe<MODE> pp;
    pp.ring = reinterpret_cast<SRow*>(dyn) + warp * kSSlots;
    char* tail = dyn + sizeof(SRow) * kSSlots * kRowWarps;
    pp.aux = reinterpret_cast<AuxSlot<MODE>*>(tail) + warp * kAuxSlots;
    tail += sizeof(AuxSlot<MODE>) * kAuxSlots * kRowWarps;
    pp.bars = reinterpret_cast<unsigned long long*>(tail) + warp * (kSSlots + kAuxSlots);
    tail += 8 * (kSSlots + kAuxSlots) * kRowWarps;
    float2* ab = reinterpret_cast<float2*>(tail);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ab + 3 * kNbin);

    load_params_ab(P, ab);
    if (MODE == TmaMode::kResidual && ghist)
        for (int i = threadIdx.x; i < 3 * kNres; i += blockDim.x) hist[i] = 0u;
    if (lane == 0) {
        for (int k = 0; k < kSSlots + kAuxSlots; ++k) mbar_init(smem_addr(&pp.bars[k]), 1);
        fence_async_shared();
    }
    __syncthreads();

    const int h = im.h, w = im.w;
    const int64_t n = (int64_t)h * w;
    const RowRange R0 = warp_rows(total_rows, h, kRowWarps);
    pp.init(R0);
    RowRange C = R0;
    bool c_valid = C.next();
    bool ok = true;
    pp.refill_aux(im, n, 0, lane);
    pp.refill_s(im, n, lane);

    while (c_valid && ok) {
        const int x0 = C.xs + 8 * lane;
        const int own = 16 + 8 * lane;
        const int offl = x0 == 0 ? own : own - 1;
        const int offr = x0 + 8 >= w ? own + 7 : own + 8;
        int a = pp.c_slot, b = a + 1 == kSSlots ? 0 : a + 1;
        ok = mbar_wait(pp.sbar(a), (pp.par >> a) & 1u, &g_slrme_status, max_spins) &&
             mbar_wait(pp.sbar(b), (pp.par >> b) & 1u, &g_slrme_status, max_spins);
        for (int j = 0; j < C.rows && ok; ++j, ++pp.q) {
            const int c2 = b + 1 == kSSlots ? 0 : b + 1;
            ok = mbar_wait(pp.sbar(c2), (pp.par >> c2) & 1u, &g_slrme_status, max_spins) &&
                 mbar_wait(pp.abar(pp.mc), (pp.mpar >> pp.mc) & 1u, &g_slrme_status, max_spins);
            if (!ok) break;
            const AuxSlot<MODE>& as = pp.aux[pp.mc];
            const int y = C.y0 + j;
            if (x0 < w) {
                const uint2 ev = *reinterpret_cast<const uint2*>(&as.E[8 * lane]);
                if constexpr (MODE == TmaMode::kResidual) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        uint32_t X[4];
                        gf_pairs(seg_row(pp.ring[a].S[c], own, offl, offr), seg_row(pp.ring[b].S[c], own, offl, offr),
                                 seg_row(pp.ring[c2].S[c], own, offl, offr), im.gf, X);
                        const uint2 mv = *reinterpret_cast<const uint2*>(&as.M[c][8 * lane]);
                        int rr[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int E = (int)byte_of(i < 4 ? ev.x : ev.y, i & 3);
                            const int M = (int)byte_of(i < 4 ? mv.x : mv.y, i & 3);
                            const float2 p = ab[c * kNbin + E];
                            rr[i] = M - predict(p.x, p.y, half_of(X, i));
                        }
                        uint4 v;
                        v.x = (uint32_t)(rr[0] & 0xFFFF) | ((uint32_t)rr[1] << 16);
                        v.y = (uint32_t)(rr[2] & 0xFFFF) | ((uint32_t)rr[3] << 16);
                        v.z = (uint32_t)(rr[4] & 0xFFFF) | ((uint32_t)rr[5] << 16);
                        v.w = (uint32_t)(rr[6] & 0xFFFF) | ((uint32_t)rr[7] << 16);
                        *reinterpret_cast<uint4*>(im.r3_out + c * n + (int64_t)y * w + x0) = v;
                        if (ghist) {
#pragma unroll
                            for (int i = 0; i < 8; ++i) atomicAdd(&hist[c * kNres + rr[i] + 255], 1u);
                        }
                    }
                } else {
                    uint32_t word[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) word[i] = byte_of(i < 4 ? ev.x : ev.y, i & 3) << 24;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        uint32_t X[4];
                        gf_pairs(seg_row(pp.ring[a].S[c], own, offl, offr), seg_row(pp.ring[b].S[c], own, offl, offr),
                                 seg_row(pp.ring[c2].S[c], own, offl, offr), im.gf, X);
                        const uint4 v = *reinterpret_cast<const uint4*>(&as.R[c][8 * lane]);
                        const uint32_t q4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int rv = (int)(int16_t)((q4[i >> 1] >> (16 * (i & 1))) & 0xFFFFu);
                            const int E = (int)(word[i] >> 24);
                            const float2 p = ab[c * kNbin + E];
                            const int M = rv + predict(p.x, p.y, half_of(X, i));
                            word[i] |= ((uint32_t)M & 255u) << (8 * c);
                        }
                    }
                    uint4* o4 = reinterpret_cast<uint4*>(im.out + (int64_t)y * w + x0);
                    o4[0] = make_uint4(word[0], word[1], word[2], word[3]);
                    o4[1] = make_uint4(word[4], word[5], word[6], word[7]);
                }
            }
            // S item j (slot a) and the aux row q are done: release and refill
            pp.par ^= 1u << a;
            ++pp.released;
            a = b;
            b = c2;
            pp.mpar ^= 1u << pp.mc;
            pp.mc = pp.mc + 1 == kAuxSlots ? 0 : pp.mc + 1;
            __syncwarp();
            pp.refill_aux(im, n, pp.q + 1, lane);
            pp.refill_s(im, n, lane);
        }
        if (!ok) break;
        // the last two S items of the task
        pp.par ^= (1u << a) | (1u << b);
        pp.released += 2;
        pp.c_slot = b + 1 == kSSlots ? 0 : b + 1;
        __syncwarp();
        pp.refill_s(im, n, lane);
        c_valid = C.next();
    }
    if (!ok) pp.drain_in_flight();
    if (MODE == TmaMode::kResidual && ghist) {
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * kNres; i += blockDim.x)
            if (hist[i]) atomicAdd(ghist + i, hist[i]);
    }
}

bool tma_eligible(int w, std::initializer_list<const void*> ptrs) {
    if (w % 16 != 0) return false;
    for (const void* p : ptrs)
        if ((uintptr_t)p % 16 != 0) return false;
    return true;
}

template <TmaMode MODE>
int launch_rows_tma(const TmaImage& im, const slrme_params* P, uint32_t* hist, cudaStream_t s) {
    static bool attr_set[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cuda_status("row pipeline device");
    constexpr size_t smem = rows_smem_bytes<MODE>(kRowWarps) + sizeof(float) * 6 * kNbin + sizeof(uint32_t) * 3 * kNres;
    if (!attr_set[dev]) {
        if (cudaFuncSetAttribute(k_rows_tma<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return cuda_status("row pipeline smem attribute");
        attr_set[dev] = true;
    }
    // every warp gets at least 4 rows; at most 2 CTAs of 8 warps per SM
    const int64_t total_rows = (int64_t)((im.w + kStripCols - 1) / kStripCols) * im.h;
    int64_t warps = (total_rows + 3) / 4;
    const int64_t cap = (int64_t)geometry().sms * 2 * kRowWarps;
    if (warps > cap) warps = cap;
    const int64_t g = (warps + kRowWarps - 1) / kRowWarps;
    k_rows_tma<MODE><<<(unsigned)(g < 1 ? 1 : g), kRowWarps * 32, smem, s>>>(im, P, hist, total_rows, kMaxSpins);
    return cuda_status(MODE == TmaMode::kResidual ? "residual_encode launch" : "residual_decode launch");
}

// ====================================================================== TMA-staged fit
//
// k_fit_tma: the fit on the row pipelines above (M / E as the other planes).
// Per lane one run per exponent parity is fed with the SIMD byte-mask sums of
// its 8-pixel segments; a run that has to leave its accumulator inside a
// strip goes to the warp's queue, with the segments that hold more exponents,
// and the warp drains the queue 32 entries at a time.

constexpr size_t kFitSmem = rows_smem_bytes<TmaMode::kFit>(kRowWarps) + sizeof(SmemBins) +
                            sizeof(uint32_t) * kRowWarps * 32 * kQueueStride;

__global__ void __launch_bounds__(kRowWarps * 32, 2) k_fit_tma(const TmaImage im, int64_t total_rows,
                                                                unsigned long long* __restrict__ gbins, int max_spins) {
    extern __shared__ __align__(128) char dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RowPipe<TmaMode::kFit> pp;
    pp.ring = reinterpret_cast<SRow*>(dyn) + warp * kSSlots;
    char* tail = dyn + sizeof(SRow) * kSSlots * kRowWarps;
    pp.aux = reinterpret_cast<AuxSlot<TmaMode::kFit>*>(tail) + warp * kAuxSlots;
    tail += sizeof(AuxSlot<TmaMode::kFit>) * kAuxSlots * kRowWarps;
    pp.bars = reinterpret_cast<unsigned long long*>(tail) + warp * (kSSlots + kAuxSlots);
    tail += 8 * (kSSlots + kAuxSlots) * kRowWarps;
    SmemBins& bins = *reinterpret_cast<SmemBins*>(tail);
    uint32_t* queue = reinterpret_cast<uint32_t*>(tail + sizeof(SmemBins));

    bins_clear(bins);
    if (lane == 0) {
        for (int k = 0; k < kSSlots + kAuxSlots; ++k) mbar_init(smem_addr(&pp.bars[k]), 1);
        fence_async_shared();
    }
    __syncthreads();

    const int h = im.h, w = im.w;
    const int64_t n = (int64_t)h * w;
    const RowRange R0 = warp_rows(total_rows, h, kRowWarps);
    pp.init(R0);

    FitWarp st;
    run_reset(st.even, -1);
    run_reset(st.odd, -1);
    st.Q = queue + warp * 32 * kQueueStride;
    st.queued = 0;

    RowRange C = R0;
    bool c_valid = C.next();
    bool ok = true;
    pp.refill_aux(im, n, 0, lane);
    pp.refill_s(im, n, lane);

    while (c_valid && ok) {
        const int x0 = C.xs + 8 * lane;
        const int own = 16 + 8 * lane;
        const int offl = x0 == 0 ? own : own - 1;
        const int offr = x0 + 8 >= w ? own + 7 : own + 8;
        const bool inside = x0 < w;
        int a = pp.c_slot, b = a + 1 == kSSlots ? 0 : a + 1;
        ok = mbar_wait(pp.sbar(a), (pp.par >> a) & 1u, &g_slrme_status, max_spins) &&
             mbar_wait(pp.sbar(b), (pp.par >> b) & 1u, &g_slrme_status, max_spins);
        for (int j = 0; j < C.rows && ok; ++j, ++pp.q) {
            const int c2 = b + 1 == kSSlots ? 0 : b + 1;
            ok = mbar_wait(pp.sbar(c2), (pp.par >> c2) & 1u, &g_slrme_status, max_spins) &&
                 mbar_wait(pp.abar(pp.mc), (pp.mpar >> pp.mc) & 1u, &g_slrme_status, max_spins);
            if (!ok) break;
            const AuxSlot<TmaMode::kFit>& ms = pp.aux[pp.mc];
            const uint2 ev = *reinterpret_cast<const uint2*>(&ms.E[8 * lane]);
            const uint32_t elo = ev.x, ehi = ev.y;
            // byte masks of the odd-exponent pixels and the two exponents
            const uint32_t olo = (elo & 0x01010101u) * 0xFFu, ohi = (ehi & 0x01010101u) * 0xFFu;
            const uint32_t Eo = max_byte(elo & olo, ehi & ohi);
            const uint32_t Ee = max_byte(elo & ~olo, ehi & ~ohi);
            const bool two = ((elo ^ (Eo * 0x01010101u)) & olo) == 0 && ((ehi ^ (Eo * 0x01010101u)) & ohi) == 0 &&
                             ((elo ^ (Ee * 0x01010101u)) & ~olo) == 0 &&
                             ((ehi ^ (Ee * 0x01010101u)) & ~ohi) == 0;
            // at most one even and one odd exponent: the odd pixels join the
            // odd run, the rest the even run; other segments go to the queue
            const bool slow = inside && !two;
            const bool take = inside && two;
            const uint32_t po_n = take ? (uint32_t)(__popc(olo) + __popc(ohi)) >> 3 : 0u;
            const uint32_t pe_n = take ? 8u - po_n : 0u;
            // a run whose region changes leaves its accumulator first
            enqueue_run<true>(st, pe_n != 0u && (int)Ee != st.even.E && st.even.n != 0u, st.even, bins, lane);
            enqueue_run<true>(st, po_n != 0u && (int)Eo != st.odd.E && st.odd.n != 0u, st.odd, bins, lane);
            if (pe_n != 0u && (int)Ee != st.even.E) run_reset(st.even, (int)Ee);
            if (po_n != 0u && (int)Eo != st.odd.E) run_reset(st.odd, (int)Eo);
            const unsigned want = __ballot_sync(0xffffffffu, slow);
            uint32_t* qe = nullptr;
            if (want) {
                if (st.queued + __popc(want) > 32) fit_drain<true>(st, bins, lane);
                qe = st.Q + (st.queued + __popc(want & ((1u << lane) - 1u))) * kQueueStride;
            }
            // channel by channel: x = 16 S* pairs, the sums of the odd pixels
            // (by mask) and of all pixels, added straight to the two runs
            uint32_t k16[4];
            mask16(olo, ohi, k16);
            const uint32_t ones[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
            RunAcc po, pa;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                uint32_t X[4];
                gf_pairs(seg_row(pp.ring[a].S[c], own, offl, offr), seg_row(pp.ring[b].S[c], own, offl, offr),
                         seg_row(pp.ring[c2].S[c], own, offl, offr), im.gf, X);
                const uint2 mv = *reinterpret_cast<const uint2*>(&ms.M[c][8 * lane]);
                chan_sums(X, mv.x, mv.y, olo, ohi, k16, po, c);
                chan_sums(X, mv.x, mv.y, 0xFFFFFFFFu, 0xFFFFFFFFu, ones, pa, c);
                if (take) {
                    st.odd.sx[c] += po.sx[c];
                    st.odd.sy[c] += po.sy[c];
                    st.odd.sxy[c] += po.sxy[c];
                    st.odd.sxx[c] += po.sxx[c];
                    st.even.sx[c] += pa.sx[c] - po.sx[c];
                    st.even.sy[c] += pa.sy[c] - po.sy[c];
                    st.even.sxy[c] += pa.sxy[c] - po.sxy[c];
                    st.even.sxx[c] += pa.sxx[c] - po.sxx[c];
                }
                if (slow) {
                    qe[2 + c] = mv.x;
                    qe[5 + c] = mv.y;
#pragma unroll
                    for (int k = 0; k < 4; ++k) qe[8 + 4 * c + k] = X[k];
                }
            }
            st.odd.n += po_n;
            st.even.n += pe_n;
            if (want) {
                if (slow) {
                    qe[0] = elo;
                    qe[1] = ehi;
                    qe[20] = 8u;
                }
                __syncwarp();
                st.queued += __popc(want);
            }
            // S item j (slot a) and the M / E of row q are done: release and refill
            pp.par ^= 1u << a;
            ++pp.released;
            a = b;
            b = c2;
            pp.mpar ^= 1u << pp.mc;
            pp.mc = pp.mc + 1 == kAuxSlots ? 0 : pp.mc + 1;
            __syncwarp();
            pp.refill_aux(im, n, pp.q + 1, lane);
            pp.refill_s(im, n, lane);
        }
        if (!ok) break;
        // the last two S items of the task; every run ends with its task
        // (bounded: a run holds at most 8 * kMaxStripRows pixels)
        pp.par ^= (1u << a) | (1u << b);
        pp.released += 2;
        pp.c_slot = b + 1 == kSSlots ? 0 : b + 1;
        warp_flush(st.even, bins, lane);
        warp_flush(st.odd, bins, lane);
        run_reset(st.even, -1);
        run_reset(st.odd, -1);
        __syncwarp();
        pp.refill_s(im, n, lane);
        c_valid = C.next();
    }
    if (!ok) pp.drain_in_flight();   // a copy did not arrive in time: stop
    else fit_drain<true>(st, bins, lane);
    __syncthreads();
    bins_to_global(bins, gbins, false);
}

int launch_fit_tma(const uint8_t* s3, const uint8_t* m3, const uint8_t* e, int h, int w, int gf_on,
                   unsigned long long* bins, cudaStream_t s) {
    static bool attr_set[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cuda_status("fit device");
    if (!attr_set[dev]) {
        if (cudaFuncSetAttribute(k_fit_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFitSmem) !=
            cudaSuccess)
            return cuda_status("fit smem attribute");
        attr_set[dev] = true;
    }
    // every warp gets at least 4 rows; at most 2 CTAs of 8 warps per SM,
    // unless a block would then add more than kMaxBlockPixels pixels (a warp
    // gets at most ceil(total_rows / warps) rows of at most 256 pixels)
    const int64_t total_rows = (int64_t)((w + kStripCols - 1) / kStripCols) * h;
    int64_t warps = (total_rows + 3) / 4;
    const int64_t cap = (int64_t)geometry().sms * 2 * kRowWarps;
    if (warps > cap) warps = cap;
    const int64_t rows_max = kMaxBlockPixels / ((int64_t)kRowWarps * kStripCols);
    if (warps < (total_rows + rows_max - 1) / rows_max) warps = (total_rows + rows_max - 1) / rows_max;
    const int64_t g = (warps + kRowWarps - 1) / kRowWarps;
    const TmaImage im{s3, m3, e, nullptr, nullptr, nullptr, h, w, gf_on != 0};
    k_fit_tma<<<(unsigned)(g < 1 ? 1 : g), kRowWarps * 32, kFitSmem, s>>>(im, total_rows, bins, kMaxSpins);
    return cuda_status("slr_fit launch");
}

int strip_ctas(int64_t cta_tasks, int per_sm) {
    const int64_t cap = (int64_t)geometry().sms * per_sm;
    int64_t g = cta_tasks < cap ? cta_tasks : cap;
    return (int)(g < 1 ? 1 : g);
}

struct StripLaunch {
    int rows;     // strip height
    int blocks;   // CTAs
};

// Strip height: the tallest of 16, 8, 4 rows that still gives about 32 warps
// of work per SM (short strips re-read two halo rows of S per strip).
StripLaunch strip_launch(int h, int w, int per_sm) {
    const int sms = geometry().sms;
    const int64_t cols = (w + kStripCols - 1) / kStripCols;
    int rows = kMaxStripRows;
    while (rows > 4 && (int64_t)((h + rows - 1) / rows) * cols < (int64_t)sms * 32) rows >>= 1;
    const int64_t tasks = (int64_t)((h + rows - 1) / rows) * cols;
    int64_t blocks = (tasks + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)sms * per_sm;
    if (blocks > cap) blocks = cap;
    return StripLaunch{rows, (int)(blocks < 1 ? 1 : blocks)};
}

// Blocks for the grid-stride strip fit: each block may add at most
// kMaxBlockPixels pixels to its bins, and a warp of a grid of `blocks` gets at
// most ceil(tasks / (kWarps blocks)) strips of rows x 256 pixels.
int64_t fit_strips_per_warp(int rows) { return kMaxBlockPixels / ((int64_t)kWarps * rows * kStripCols); }

int fit_strip_blocks(const StripLaunch& L, int h, int w) {
    const int64_t cols = (w + kStripCols - 1) / kStripCols;
    const int64_t tasks = (int64_t)((h + L.rows - 1) / L.rows) * cols;
    const int64_t per = kWarps * fit_strips_per_warp(L.rows);
    const int64_t need = (tasks + per - 1) / per;
    return (int)(need > L.blocks ? need : L.blocks);
}

}  // namespace

int launch_fit(const uint8_t* s3, const uint8_t* m3, const uint8_t* e, int h, int w, int gf_on, int64_t* bin_sums,
               slrme_params* params, cudaStream_t s) {
    if (cudaMemsetAsync(bin_sums, 0, sizeof(int64_t) * kNbin * kNsum, s) != cudaSuccess)
        return cuda_status("slr_fit memset");
    const int64_t n = (int64_t)h * w;
    if (n > 0) {
        const bool fast = (w % 8 == 0) && ((uintptr_t)s3 % 8 == 0) && ((uintptr_t)m3 % 8 == 0) &&
                          ((uintptr_t)e % 8 == 0);
        int st;
        if (tma_eligible(w, {s3, m3, e})) {
            st = launch_fit_tma(s3, m3, e, h, w, gf_on, reinterpret_cast<unsigned long long*>(bin_sums), s);
        } else {
            const StripLaunch L = strip_launch(h, w, 2);
            k_fit<<<fit_strip_blocks(L, h, w), kThreads, 0, s>>>(s3, m3, e, h, w, gf_on, fast ? 1 : 0, L.rows,
                                                                 reinterpret_cast<unsigned long long*>(bin_sums));
            st = cuda_status("slr_fit launch");
        }
        if (st != SLRME_OK) return st;
    }
    k_solve<<<kSolveBlocks, 32, 0, s>>>(bin_sums, params);
    return cuda_status("slr_fit solve launch");
}

int launch_residual_encode(const uint8_t* s3, const uint8_t* m3, const uint8_t* e, int h, int w, int gf_on,
                           const slrme_params* params, int16_t* r3, uint32_t* hist, cudaStream_t s) {
    const bool fast = (w % 8 == 0) && ((uintptr_t)s3 % 8 == 0) && ((uintptr_t)m3 % 8 == 0) &&
                      ((uintptr_t)e % 8 == 0);
    if (tma_eligible(w, {s3, m3, e, r3})) {
        const TmaImage im{s3, m3, e, nullptr, r3, nullptr, h, w, gf_on != 0};
        return launch_rows_tma<TmaMode::kResidual>(im, params, hist, s);
    }
    const StripLaunch L = strip_launch(h, w, 2);
    k_residual<<<L.blocks, kThreads, 0, s>>>(s3, m3, e, h, w, gf_on, fast ? 1 : 0, L.rows, params, r3, hist);
    return cuda_status("residual_encode launch");
}

int launch_residual_decode(const uint8_t* s3, const uint8_t* e, const int16_t* r3, int h, int w, int gf_on,
                           const slrme_params* params, uint32_t* rgbe_out, cudaStream_t s) {
    const bool fast = (w % 8 == 0) && ((uintptr_t)s3 % 8 == 0) && ((uintptr_t)e % 8 == 0);
    if (tma_eligible(w, {s3, e, r3, rgbe_out})) {
        const TmaImage im{s3, nullptr, e, r3, nullptr, rgbe_out, h, w, gf_on != 0};
        return launch_rows_tma<TmaMode::kDecode>(im, params, nullptr, s);
    }
    const StripLaunch L = strip_launch(h, w, 2);
    k_decode<<<L.blocks, kThreads, 0, s>>>(s3, e, r3, h, w, gf_on, fast ? 1 : 0, L.rows, params, rgbe_out);
    return cuda_status("residual_decode launch");
}


// ---------------------------------------------------------------- batch launchers

int launch_fit_batch(const BatchDev& B, int64_t cta_tasks, int ctas_per_sm, const uint8_t* s3, const uint8_t* m3,
                     const uint8_t* e, slrme_params* params, cudaStream_t s) {
    if (cudaMemsetAsync(B.sums, 0, sizeof(unsigned long long) * kNbin * kNsum * (size_t)B.n, s) != cudaSuccess)
        return cuda_status("batch fit memset");
    if (cta_tasks > 0) {
        // each block adds at most kMaxBlockPixels pixels (a CTA task is kWarps strips)
        const int64_t per = fit_strips_per_warp(B.strip_rows);
        int64_t blocks = strip_ctas(cta_tasks, ctas_per_sm < 2 ? ctas_per_sm : 2);
        if (blocks < (cta_tasks + per - 1) / per) blocks = (cta_tasks + per - 1) / per;
        k_fit_batch<<<(unsigned)blocks, kThreads, 0, s>>>(B, cta_tasks, s3, m3, e);
        const int st = cuda_status("batch fit launch");
        if (st != SLRME_OK) return st;
    }
    k_solve_batch<<<dim3(kSolveBlocks, B.n), 32, 0, s>>>(B.sums, params);
    return cuda_status("batch solve launch");
}

int launch_residual_batch(const BatchDev& B, int64_t cta_tasks, int ctas_per_sm, const uint8_t* s3,
                          const uint8_t* m3, const uint8_t* e, const slrme_params* params, int16_t* r3,
                          uint32_t* hist, cudaStream_t s) {
    if (hist && cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 3 * kNres * (size_t)B.n, s) != cudaSuccess)
        return cuda_status("batch residual memset");
    if (cta_tasks == 0) return SLRME_OK;
    k_residual_batch<<<strip_ctas(cta_tasks, ctas_per_sm), kThreads, 0, s>>>(B, cta_tasks, s3, m3, e, params, r3,
                                                                             hist);
    return cuda_status("batch residual launch");
}

int launch_decode_batch(const BatchDev& B, int64_t cta_tasks, int ctas_per_sm, const uint8_t* s3, const uint8_t* e,
                        const int16_t* r3, const slrme_params* params, uint32_t* out, cudaStream_t s) {
    if (cta_tasks == 0) return SLRME_OK;
    k_decode_batch<<<strip_ctas(cta_tasks, ctas_per_sm), kThreads, 0, s>>>(B, cta_tasks, s3, e, r3, params, out);
    return cuda_status("batch decode launch");
}

}  // namespace slrme

// ====================================================================== slr_fit_noalloc
//
// The same fit as slr_fit for callers that cannot allocate device memory:
// the bin sums live in this file-scope array instead of a caller workspace.
// Every GPU that loads the library holds these 26,624 bytes until exit.

namespace slrme {

namespace {

constexpr int kMaxDevices = 64;
static __device__ __align__(256) unsigned long long g_fit_scratch[kNbin * kNsum];
static std::mutex g_scratch_mu;
static void* g_scratch_addr[kMaxDevices];

// Device address of g_fit_scratch on the current device, looked up once per
// device (with that device current).  In host code the array's name is only a
// host-side stand-in, so kernels must be given this address, never the name.
int scratch_address(void** out) {
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) {
        set_error("slr_fit_noalloc: cudaGetDevice: %s", cudaGetErrorString(err));
        return SLRME_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("slr_fit_noalloc: device ordinal %d outside 0..%d", dev, kMaxDevices - 1);
        return SLRME_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        err = cudaGetSymbolAddress(&p, g_fit_scratch);
        if (err != cudaSuccess || !p) {
            set_error("slr_fit_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(err));
            return SLRME_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SLRME_OK;
}

}  // namespace

}  // namespace slrme

extern "C" int slr_fit_noalloc(const uint8_t* s_dec3, const uint8_t* m3, const uint8_t* e, int h, int w,
                               int gf_on, slrme_params* params, slrme_stream_t stream) {
    using namespace slrme;
    if (h < 0 || w < 0 || (int64_t)h * (int64_t)w >= ((int64_t)1 << 31)) {
        set_error("slr_fit_noalloc: image %d x %d outside the supported size (h, w >= 0, h*w < 2^31): "
                  "the fixed %d-byte scratch holds exact sums only up to that size",
                  h, w, (int)sizeof(g_fit_scratch));
        return SLRME_EINVAL;
    }
    if (gf_on != 0 && gf_on != 1) {
        set_error("slr_fit_noalloc: gf_on must be 0 or 1");
        return SLRME_EINVAL;
    }
    if (!params || (uintptr_t)params % 4 != 0) {
        set_error("slr_fit_noalloc: params must be a non-null, 4-byte aligned device pointer");
        return SLRME_EINVAL;
    }
    const int64_t n = (int64_t)h * w;
    if (n > 0 && !(s_dec3 && m3 && e)) {
        set_error("slr_fit_noalloc: null image pointer");
        return SLRME_EINVAL;
    }
    void* scratch = nullptr;
    int st = scratch_address(&scratch);
    if (st != SLRME_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's sums: clear it before accumulating
    if (cudaMemsetAsync(scratch, 0, sizeof(g_fit_scratch), s) != cudaSuccess)
        return cuda_status("slr_fit_noalloc memset");
    unsigned long long* bins = static_cast<unsigned long long*>(scratch);
    if (n > 0) {
        const bool fast = (w % 8 == 0) && ((uintptr_t)s_dec3 % 8 == 0) && ((uintptr_t)m3 % 8 == 0) &&
                          ((uintptr_t)e % 8 == 0);
        const StripLaunch L = strip_launch(h, w, 2);
        k_fit<<<fit_strip_blocks(L, h, w), kThreads, 0, s>>>(s_dec3, m3, e, h, w, gf_on, fast ? 1 : 0, L.rows, bins);
        st = cuda_status("slr_fit_noalloc launch");
        if (st != SLRME_OK) return st;
    }
    k_solve<<<kSolveBlocks, 32, 0, s>>>(reinterpret_cast<const int64_t*>(bins), params);
    return cuda_status("slr_fit_noalloc solve launch");
}

extern "C" int slrme_device_status(int* status, int clear) {
    using namespace slrme;
    if (!status) {
        set_error("slrme_device_status: null pointer");
        return SLRME_EINVAL;
    }
    if (cudaMemcpyFromSymbol(status, g_slrme_status, sizeof(int)) != cudaSuccess)
        return cuda_status("slrme_device_status read");
    if (clear) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_slrme_status, &zero, sizeof(int)) != cudaSuccess)
            return cuda_status("slrme_device_status clear");
    }
    return SLRME_OK;
}
