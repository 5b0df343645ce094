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
#include <cuda.h>

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
// bytes, the mantissa bytes of the three planes, the x pairs and the count
// (or, for a flushed run, its 13 sums and the tag 256 + E); the odd stride
// keeps the lanes' accesses on distinct banks.
constexpr int kQueueStride = 21;

// Per-warp state of the fit: one run per exponent parity (adjacent regions
// of a smooth exponent field differ by one, so a boundary through a lane's
// column feeds the two runs without flushing either) and the queue of
// segments that need per-pixel work.
struct FitWarp {
    RunAcc even, odd;
    uint32_t* Q;
    int queued;   // entries in the queue (warp-uniform)
};

// Adds one queued entry to the bins without branches on the exponents: a
// flushed run (tag 256 + E) as its 13 sums, or a segment (tag = pixel count,
// 1 .. 8) pixel by pixel, 19 reductions each (the count, x and y are below
// 2^12 and go to the low words alone; x y and x x take two words).
__device__ __noinline__ void drain_entry_flat(const uint32_t* q, uint32_t B) {
    const uint32_t tag = q[20];
    if (tag >= 256u) {
        uint32_t acc[kNsum];
#pragma unroll
        for (int j = 0; j < kNsum; ++j) acc[j] = q[j];
        bins_add32(B, (int)(tag - 256u), acc);
        return;
    }
    const uint32_t elo = q[0], ehi = q[1];
    const uint32_t mlo[3] = {q[2], q[3], q[4]}, mhi[3] = {q[5], q[6], q[7]};
    constexpr uint32_t kHi = 4u * kNbin * kNsum;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i < (int)tag) {
            const uint32_t lo = B + 4u * kNsum * byte_of(i < 4 ? elo : ehi, i & 3);
            red_add(lo, 1u);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const uint32_t x = (q[8 + 4 * c + (i >> 1)] >> (16 * (i & 1))) & 0xFFFFu;
                const uint32_t y = byte_of(i < 4 ? mlo[c] : mhi[c], i & 3);
                const uint32_t xy = x * y, xx = x * x, a = lo + 4u * (1 + 4 * c);
                red_add(a, x);
                red_add(a + 4u, y);
                red_add(a + 8u, xy & 0xFFFu);
                red_add(a + 8u + kHi, xy >> 12);
                red_add(a + 12u, xx & 0xFFFu);
                red_add(a + 12u + kHi, xx >> 12);
            }
        }
    }
}

// Drains the warp's queue, one entry per lane.
template <bool kUnroll = false>
__device__ __forceinline__ void fit_drain(FitWarp& st, SmemBins& bins, int lane) {
    if (lane < st.queued) drain_entry_flat(st.Q + lane * kQueueStride, smem_addr(&bins));
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

// The parameters as (a, b) pairs, [c][E], so one 8-byte load gets both;
// threads 0 .. nthreads - 1 take part.
__device__ __forceinline__ void load_params_ab(const slrme_params* __restrict__ P, float2* ab, int nthreads) {
    for (int i = threadIdx.x; i < 3 * kNbin; i += nthreads) ab[i] = make_float2((&P->a[0][0])[i], (&P->b[0][0])[i]);
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

// ====================================================================== tensor-map row pipeline
//
// For images whose rows are 16-byte aligned (w % 16 == 0, 16-byte aligned
// planes).  The image is cut into strips of kTileCols = 2048 columns, one
// 256-column slice per consumer warp (kTileWarps = 8 per CTA).  The rows of
// all strips, strip after strip, are split into one contiguous range per
// CTA, and a range becomes tasks of at most kTaskRows rows of one strip.
// A producer warp streams the range through two shared-memory rings with
// tensor-map bulk copies (cp.async.bulk.tensor): per S item, the S row of the
// three planes with 16 halo columns on each side (one 4-D box); per row, its
// other planes (M and E for the fit and the residual, R and E for the
// decoder: one 4-D box and one 4-D box of a single plane).  Row j of a task
// needs S items j, j + 1, j + 2 (rows y - 1, y, y + 1, clamped to the image
// by the producer, which replicates the edge rows).  A slot's full barrier
// completes on the bytes of its copies; its empty barrier completes when all
// consumer warps have arrived.  Box columns past the image are zero-filled by
// the copy and never read as pixels: edge columns replicate through the
// neighbour offsets.  Every wait is bounded (see tma.cuh).

constexpr int kTileWarps = 8;                              // consumer warps
constexpr int kTileThreads = (kTileWarps + 1) * 32;        // + one producer warp
constexpr int kTileCols = kTileWarps * kStripCols;         // 2048
constexpr int kTileSW = kTileCols + 32;                    // S row with halos, per plane
constexpr int kTaskRows = 256;
constexpr int kTileS = 5;                                  // S ring slots
constexpr int kTileA = 3;                                  // M / E ring slots (fit, residual)
constexpr uint32_t kTileSBytes = 3u * kTileSW;             // 6240
constexpr uint32_t kTileSStride = 6272;                    // slot stride, multiple of 128
static_assert(kTileSStride >= kTileSBytes && kTileSStride % 128 == 0, "S slot");
// Flush every run this often: a run then holds at most 8 * 16 pixels, which
// keeps its 32-bit sums exact (see kMaxStripRows).
constexpr int kRunRows = kMaxStripRows;

enum class TmaMode { kResidual = 0, kDecode = 1, kFit = 2 };

// Aux slot: planes 0-2 (1 or 2 bytes per pixel) then E.
template <TmaMode MODE>
struct TileAux {
    static constexpr uint32_t kElem = MODE == TmaMode::kDecode ? 2 : 1;
    static constexpr uint32_t kPlane = kElem * kTileCols;          // bytes per plane row
    static constexpr uint32_t kE = 3 * kPlane;                     // offset of the E row
    static constexpr uint32_t kBytes = kE + kTileCols;
    static constexpr uint32_t kStride = kBytes;                    // multiple of 128
    static_assert(kStride % 128 == 0, "aux slot");
    static constexpr int kSlots = kTileA;   // ring slots
    // CTAs per SM the kernel is built for (the residual kernel's registers
    // and shared memory allow three; the launch uses three on large images)
    static constexpr int kCtas = MODE == TmaMode::kResidual ? 3 : 2;
};

struct TileMaps {
    CUtensorMap s;   // u8 (16, w/16, h, 3): S planes
    CUtensorMap a;   // u8 (16, w/16, h, 3) M planes, or u16 (8, w/8, h, 3) R planes
    CUtensorMap e;   // u8 (16, w/16, h, 1): E plane
};

struct TileArgs {
    int h, w;
    int gf;
    int64_t total_rows;                      // strips * h
    int max_spins;
    const slrme_params* params;              // residual / decode
    int16_t* r3_out;                         // residual
    uint32_t* hist;                          // residual (may be null)
    uint32_t* out;                           // decode
    unsigned long long* gbins;               // fit
};

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Barrier among the consumer warps only (the producer warp may have left).
__device__ __forceinline__ void consumers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kTileWarps * 32) : "memory");
}

// The CTA's rows r .. end - 1 in (strip, row) order and its current task.
struct TileRange {
    int64_t r, end;
    int h;
    int y0, rows, xs;
    __device__ __forceinline__ bool next() {
        if (r >= end) return false;
        const int64_t c = r / h;
        y0 = (int)(r - c * h);
        rows = (int)min(min(end - r, (int64_t)(h - y0)), (int64_t)kTaskRows);
        xs = (int)c * kTileCols;
        r += rows;
        return true;
    }
};

__device__ __forceinline__ TileRange tile_range(int64_t total_rows, int h) {
    const int64_t G = gridDim.x, b = blockIdx.x;
    return TileRange{b * total_rows / G, (b + 1) * total_rows / G, h, 0, 0, 0};
}

// Shared-memory layout of a tile kernel: the two rings, then four barrier
// arrays, then the mode's own data at `extra`.
template <TmaMode MODE>
struct TileSmem {
    uint32_t s_ring, a_ring, bars, extra;
    __device__ __forceinline__ uint32_t sfull(int k) const { return bars + 8u * k; }
    __device__ __forceinline__ uint32_t sempty(int k) const { return bars + 8u * (kTileS + k); }
    __device__ __forceinline__ uint32_t afull(int k) const { return bars + 8u * (2 * kTileS + k); }
    __device__ __forceinline__ uint32_t aempty(int k) const {
        return bars + 8u * (2 * kTileS + TileAux<MODE>::kSlots + k);
    }
    __device__ __forceinline__ uint32_t sslot(uint32_t i) const { return s_ring + (i % kTileS) * kTileSStride; }
    __device__ __forceinline__ uint32_t aslot(uint32_t i) const {
        return a_ring + (i % TileAux<MODE>::kSlots) * TileAux<MODE>::kStride;
    }
    static constexpr uint32_t kRings = kTileS * kTileSStride + TileAux<MODE>::kSlots * TileAux<MODE>::kStride;
    static constexpr uint32_t kHead = kRings + 8u * 2 * (kTileS + TileAux<MODE>::kSlots);   // multiple of 16
};

template <TmaMode MODE>
__device__ __forceinline__ TileSmem<MODE> tile_smem(char* dyn) {
    const uint32_t base = (smem_addr(dyn) + 127u) & ~127u;
    TileSmem<MODE> L;
    L.s_ring = base;
    L.a_ring = base + kTileS * kTileSStride;
    L.bars = base + TileSmem<MODE>::kRings;
    L.extra = base + TileSmem<MODE>::kHead;
    return L;
}

template <TmaMode MODE>
__device__ __forceinline__ void tile_init_barriers(const TileSmem<MODE>& L) {
    if (threadIdx.x == 0) {
        for (int k = 0; k < kTileS; ++k) {
            mbar_init(L.sfull(k), 1);
            mbar_init(L.sempty(k), kTileWarps);
        }
        for (int k = 0; k < TileAux<MODE>::kSlots; ++k) {
            mbar_init(L.afull(k), 1);
            mbar_init(L.aempty(k), kTileWarps);
        }
        fence_async_shared();
    }
}

// The producer (one thread): items in the order the consumers use them.
// Returns false if a wait for a free slot gave up.
template <TmaMode MODE>
__device__ __noinline__ void tile_produce(const TileSmem<MODE>& L, const CUtensorMap* tm_s, const CUtensorMap* tm_a,
                                          const CUtensorMap* tm_e, const TileArgs& A) {
    TileRange P = tile_range(A.total_rows, A.h);
    uint32_t si = 0, ai = 0;
    bool ok = true;
    while (ok && P.next()) {
        for (int k = 0; k < P.rows + 2 && ok; ++k) {
            // S item k: row y0 - 1 + k, clamped (edge rows replicate)
            {
                const int slot = (int)(si % kTileS);
                if (si >= (uint32_t)kTileS)
                    ok = mbar_wait(L.sempty(slot), ((si / kTileS) - 1u) & 1u, &g_slrme_status, A.max_spins);
                if (!ok) break;
                const int ys = min(max(P.y0 - 1 + k, 0), A.h - 1);
                fence_async_shared();
                mbar_arrive_expect_tx(L.sfull(slot), kTileSBytes);
                tma_load_4d(L.sslot(si), tm_s, 0, P.xs / 16 - 1, ys, 0, L.sfull(slot));
                ++si;
            }
            if (k >= 2) {   // the other planes of row y0 + k - 2
                constexpr uint32_t KA = TileAux<MODE>::kSlots;
                const int slot = (int)(ai % KA);
                if (ai >= KA) ok = mbar_wait(L.aempty(slot), ((ai / KA) - 1u) & 1u, &g_slrme_status, A.max_spins);
                if (!ok) break;
                const int y = P.y0 + k - 2;
                const uint32_t dst = L.aslot(ai);
                fence_async_shared();
                mbar_arrive_expect_tx(L.afull(slot), TileAux<MODE>::kBytes);
                if constexpr (MODE == TmaMode::kDecode)
                    tma_load_4d(dst, tm_a, 0, P.xs / 8, y, 0, L.afull(slot));
                else
                    tma_load_4d(dst, tm_a, 0, P.xs / 16, y, 0, L.afull(slot));
                tma_load_4d(dst + TileAux<MODE>::kE, tm_e, 0, P.xs / 16, y, 0, L.afull(slot));
                ++ai;
            }
        }
    }
    // before leaving, wait (bounded) for the last copy into every slot, so
    // no copy is in flight if the consumers stopped early
    const int spins = ok ? A.max_spins : (1 << 10);
    for (uint32_t k = si > (uint32_t)kTileS ? si - kTileS : 0; k < si; ++k)
        mbar_wait(L.sfull((int)(k % kTileS)), (k / kTileS) & 1u, &g_slrme_status, spins);
    constexpr uint32_t KA = TileAux<MODE>::kSlots;
    for (uint32_t k = ai > KA ? ai - KA : 0; k < ai; ++k)
        mbar_wait(L.afull((int)(k % KA)), (k / KA) & 1u, &g_slrme_status, spins);
}

// A consumer warp is done with a slot (all lanes call after their last read).
__device__ __forceinline__ void tile_release(uint32_t empty_bar, int lane) {
    __syncwarp();
    if (lane == 0) mbar_arrive(empty_bar);
}

// One consumer warp's view of the rings: waits and releases by item index.
template <TmaMode MODE>
struct TileConsumer {
    TileSmem<MODE> L;
    int max_spins;
    __device__ __forceinline__ bool wait_s(uint32_t i) const {
        return mbar_wait(L.sfull((int)(i % kTileS)), (i / kTileS) & 1u, &g_slrme_status, max_spins);
    }
    __device__ __forceinline__ bool wait_a(uint32_t i) const {
        constexpr uint32_t KA = TileAux<MODE>::kSlots;
        return mbar_wait(L.afull((int)(i % KA)), (i / KA) & 1u, &g_slrme_status, max_spins);
    }
    // all lanes call after their last read of the items
    __device__ __forceinline__ void release_s(uint32_t i, int lane) const {
        __syncwarp();
        if (lane == 0) mbar_arrive(L.sempty((int)(i % kTileS)));
    }
    __device__ __forceinline__ void release_a(uint32_t i, int lane) const {
        __syncwarp();
        if (lane == 0) mbar_arrive(L.aempty((int)(i % TileAux<MODE>::kSlots)));
    }
};

// One lane's S row segment from an S slot (shared address): 8 bytes plus the
// neighbours at the given offsets.
__device__ __forceinline__ Row10 tile_seg(uint32_t row, int own, int offl, int offr) {
    Row10 R;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(R.lo), "=r"(R.hi) : "r"(row + own));
    uint32_t l, r;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(l) : "r"(row + offl));
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(r) : "r"(row + offr));
    R.l = l;
    R.r = r;
    return R;
}

__device__ __forceinline__ uint2 lds64(uint32_t a) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ uint4 lds128(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

// Per-lane geometry of a task: the lane's 8 columns and its S byte offsets.
struct LaneCols {
    int x0, own, offl, offr;
    bool inside;
    __device__ __forceinline__ LaneCols(int xs, int w, int warp, int lane) {
        x0 = xs + kStripCols * warp + 8 * lane;
        own = 16 + kStripCols * warp + 8 * lane;
        offl = x0 == 0 ? own : own - 1;
        offr = x0 + 8 >= w ? own + 7 : own + 8;
        inside = x0 < w;
    }
};

// x = 16 S* of channel c for the lane's 8 pixels, as 16-bit pairs.
__device__ __forceinline__ void tile_x(uint32_t sa, uint32_t sb, uint32_t sc, int c, const LaneCols& lc, bool gf,
                                       uint32_t (&X)[4]) {
    const uint32_t po = (uint32_t)c * kTileSW;
    if (gf) {
        gf_pairs(tile_seg(sa + po, lc.own, lc.offl, lc.offr), tile_seg(sb + po, lc.own, lc.offl, lc.offr),
                 tile_seg(sc + po, lc.own, lc.offl, lc.offr), true, X);
    } else {
        const Row10 r = tile_seg(sb + po, lc.own, lc.offl, lc.offr);
        gf_pairs(r, r, r, false, X);
    }
}

// ---------------------------------------------------------------- fit on the tile pipeline

// One channel of an 8-pixel segment added to a run: x pairs and y bytes
// already masked to the run's pixels.
__device__ __forceinline__ void chan_accum(const uint32_t (&x)[4], uint32_t yl, uint32_t yh, RunAcc& a, int c) {
    uint32_t sx = a.sx[c];
#pragma unroll
    for (int k = 0; k < 4; ++k) sx = __dp2a_lo(x[k], 0x0101u, sx);
    a.sx[c] = sx;
    a.sy[c] = __dp4a(yl, 0x01010101u, __dp4a(yh, 0x01010101u, a.sy[c]));
    uint32_t q = __dp2a_lo(x[0], yl, a.sxy[c]);
    q = __dp2a_hi(x[1], yl, q);
    q = __dp2a_lo(x[2], yh, q);
    a.sxy[c] = __dp2a_hi(x[3], yh, q);
    uint32_t r = a.sxx[c];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t lo16 = x[k] & 0xFFFFu, hi16 = x[k] >> 16;
        r += lo16 * lo16 + hi16 * hi16;
    }
    a.sxx[c] = r;
}

// Two per-warp queues: flushed runs (their sums) and segments that need
// per-pixel work (their pixels).  Each is drained by its own code path, one
// entry per lane, so draining runs -- the common case -- never pays for the
// per-pixel segment path.  A row queues at most one segment per lane, so the
// segment queue holds 32 (a row's segments are written piece by piece while
// the row is processed); runs, complete when queued, go in chunks that fit
// the 16-entry run queue, draining it in between.
constexpr int kRunQ = 16;
constexpr int kRunStride = 15;   // 13 sums, the region, a pad word (odd stride: distinct banks)
constexpr int kSegQ = 32;        // segment entries of kQueueStride words
struct FitQueues {
    uint32_t* R;   // run entries
    uint32_t* Q;   // segment entries
    int nr, nq;    // entries queued (warp-uniform)
};

__device__ __forceinline__ void drain_runs(FitQueues& fq, SmemBins& bins, int lane) {
    if (lane < fq.nr) {
        const uint32_t* q = fq.R + lane * kRunStride;
        uint32_t acc[kNsum];
#pragma unroll
        for (int j = 0; j < kNsum; ++j) acc[j] = q[j];
        bins_add32(smem_addr(&bins), (int)q[kNsum], acc);
    }
    __syncwarp();
    fq.nr = 0;
}

// Adds the eight pixels of a queued segment to their bins one by one, without
// branches: per pixel 19 reductions (the count, x and y are below 2^12 and
// have no high part under the split rule; x y and x x take two words).
__device__ __forceinline__ void drain_segment_pixels(const uint32_t* q, uint32_t B) {
    const uint32_t elo = q[0], ehi = q[1];
    uint32_t mlo[3] = {q[2], q[3], q[4]}, mhi[3] = {q[5], q[6], q[7]};
    uint32_t X[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) X[c][k] = q[8 + 4 * c + k];
    constexpr uint32_t kHi = 4u * kNbin * kNsum;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t lo = B + 4u * kNsum * byte_of(i < 4 ? elo : ehi, i & 3);
        red_add(lo, 1u);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint32_t x = (X[c][i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
            const uint32_t y = byte_of(i < 4 ? mlo[c] : mhi[c], i & 3);
            const uint32_t xy = x * y, xx = x * x;
            const uint32_t a = lo + 4u * (1 + 4 * c);
            red_add(a, x);
            red_add(a + 4u, y);
            red_add(a + 8u, xy & 0xFFFu);
            red_add(a + 8u + kHi, xy >> 12);
            red_add(a + 12u, xx & 0xFFFu);
            red_add(a + 12u + kHi, xx >> 12);
        }
    }
}

__device__ __forceinline__ void drain_segs(FitQueues& fq, SmemBins& bins, int lane) {
    if (lane < fq.nq) drain_segment_pixels(fq.Q + lane * kQueueStride, smem_addr(&bins));
    __syncwarp();
    fq.nq = 0;
}

// Queues the run of every lane with `want` set: the even run (all - odd,
// region all.E) or the odd run (odd, region odd.E), in chunks that fit.
template <bool kEven>
__device__ __forceinline__ void push_run(FitQueues& fq, bool want, const RunAcc& all, const RunAcc& odd,
                                         SmemBins& bins, int lane) {
    unsigned m = __ballot_sync(0xffffffffu, want);
    while (m) {
        if (fq.nr == kRunQ) drain_runs(fq, bins, lane);
        // the first kRunQ - nr lanes of m go now
        unsigned take = m;
        while (__popc(take) > kRunQ - fq.nr) take &= ~(1u << (31 - __clz(take)));
        if (take & (1u << lane)) {
            uint32_t* q = fq.R + (fq.nr + __popc(take & ((1u << lane) - 1u))) * kRunStride;
            if constexpr (kEven) {
                q[0] = all.n - odd.n;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    q[1 + 4 * c] = all.sx[c] - odd.sx[c];
                    q[2 + 4 * c] = all.sy[c] - odd.sy[c];
                    q[3 + 4 * c] = all.sxy[c] - odd.sxy[c];
                    q[4 + 4 * c] = all.sxx[c] - odd.sxx[c];
                }
                q[kNsum] = (uint32_t)all.E;
            } else {
                q[0] = odd.n;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    q[1 + 4 * c] = odd.sx[c];
                    q[2 + 4 * c] = odd.sy[c];
                    q[3 + 4 * c] = odd.sxy[c];
                    q[4 + 4 * c] = odd.sxx[c];
                }
                q[kNsum] = (uint32_t)odd.E;
            }
        }
        __syncwarp();
        fq.nr += __popc(take);
        m &= ~take;
    }
}

constexpr uint32_t kFitQueueBytes = sizeof(uint32_t) * kTileWarps * (kRunQ * kRunStride + kSegQ * kQueueStride);
constexpr uint32_t kFitExtra = sizeof(SmemBins) + kFitQueueBytes;
constexpr size_t kTileFitSmem = 128 + TileSmem<TmaMode::kFit>::kHead + kFitExtra;
static_assert(2 * (kTileFitSmem + 1024) <= 228 * 1024, "two fit CTAs per SM");

// Per lane: `all` holds the sums of both runs, `odd` those of the odd run;
// the even run is all - odd.  A run that changes region leaves through the
// warp's queue; a task's runs are flushed every kRunRows rows and at its end.
__global__ void __launch_bounds__(kTileThreads, TileAux<TmaMode::kFit>::kCtas) k_fit_tile(const __grid_constant__ CUtensorMap tm_s,
                                                               const __grid_constant__ CUtensorMap tm_a,
                                                               const __grid_constant__ CUtensorMap tm_e,
                                                               const TileArgs A) {
    extern __shared__ __align__(128) char dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TileSmem<TmaMode::kFit> L = tile_smem<TmaMode::kFit>(dyn);
    char* extra = dyn + (L.extra - smem_addr(dyn));
    SmemBins& bins = *reinterpret_cast<SmemBins*>(extra);
    uint32_t* queue = reinterpret_cast<uint32_t*>(extra + sizeof(SmemBins));
    tile_init_barriers(L);
    __syncthreads();

    if (warp == kTileWarps) {
        if (lane == 0) tile_produce(L, &tm_s, &tm_a, &tm_e, A);
        return;
    }
    // the consumers clear the bins while the first copies are in flight
    static_assert(sizeof(SmemBins) % 16 == 0 && TileSmem<TmaMode::kFit>::kHead % 16 == 0, "16-byte bin stores");
    for (int i = threadIdx.x; i < (int)(sizeof(SmemBins) / 16); i += kTileWarps * 32)
        reinterpret_cast<uint4*>(extra)[i] = make_uint4(0u, 0u, 0u, 0u);
    consumers_sync();
    const TileConsumer<TmaMode::kFit> C{L, A.max_spins};
    const int w = A.w;
    const bool gf = A.gf != 0;
    FitQueues fq;
    fq.R = queue + warp * (kRunQ * kRunStride + kSegQ * kQueueStride);
    fq.Q = fq.R + kRunQ * kRunStride;
    fq.nr = fq.nq = 0;
    RunAcc all, odd;
    TileRange T = tile_range(A.total_rows, A.h);
    uint32_t si = 0, ai = 0;
    bool ok = true;
    while (ok && T.next()) {
        const LaneCols lc(T.xs, w, warp, lane);
        run_reset(all, -1);
        run_reset(odd, -1);
        ok = C.wait_s(si) && C.wait_s(si + 1);
        for (int j = 0; j < T.rows && ok; ++j) {
            ok = C.wait_s(si + j + 2) && C.wait_a(ai + j);
            if (!ok) break;
            const uint32_t sa = L.sslot(si + j), sb = L.sslot(si + j + 1), sc = L.sslot(si + j + 2);
            const uint32_t as = L.aslot(ai + j) + kStripCols * warp + 8 * lane;
            const uint2 ev = lds64(as + TileAux<TmaMode::kFit>::kE);
            const uint32_t elo = ev.x, ehi = ev.y;
            // byte masks of the odd-exponent pixels and the two exponents
            const uint32_t olo = (elo & 0x01010101u) * 0xFFu, ohi = (ehi & 0x01010101u) * 0xFFu;
            const uint32_t Eo = max_byte(elo & olo, ehi & ohi);
            const uint32_t Ee = max_byte(elo & ~olo, ehi & ~ohi);
            const bool two = ((elo ^ (Eo * 0x01010101u)) & olo) == 0 && ((ehi ^ (Eo * 0x01010101u)) & ohi) == 0 &&
                             ((elo ^ (Ee * 0x01010101u)) & ~olo) == 0 &&
                             ((ehi ^ (Ee * 0x01010101u)) & ~ohi) == 0;
            const bool slow = lc.inside && !two;
            const bool take = lc.inside && two;
            const uint32_t po_n = take ? (uint32_t)(__popc(olo) + __popc(ohi)) >> 3 : 0u;
            const bool chg_o = po_n != 0u && (int)Eo != odd.E;
            const bool chg_e = take && po_n != 8u && (int)Ee != all.E;
            // a run whose region changes leaves first (the even run is all - odd)
            push_run<true>(fq, chg_e && all.E >= 0 && all.n != odd.n, all, odd, bins, lane);
            push_run<false>(fq, chg_o && odd.E >= 0 && odd.n != 0u, all, odd, bins, lane);
            if (chg_e) {
                const int keep = odd.E;
                all = odd;        // the even part leaves: all - odd = 0
                all.E = (int)Ee;
                odd.E = keep;
            }
            if (chg_o) {
                const int keep = all.E;
                run_minus(all, odd);
                all.E = keep;
                run_reset(odd, (int)Eo);
            }
            const unsigned want = __ballot_sync(0xffffffffu, slow);
            uint32_t* qe = nullptr;
            if (want) {
                if (fq.nq + __popc(want) > kSegQ) drain_segs(fq, bins, lane);
                qe = fq.Q + (fq.nq + __popc(want & ((1u << lane) - 1u))) * kQueueStride;
            }
            uint32_t k16[4];
            mask16(olo, ohi, k16);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                uint32_t X[4];
                tile_x(sa, sb, sc, c, lc, gf, X);
                const uint2 mv = lds64(as + (uint32_t)c * TileAux<TmaMode::kFit>::kPlane);
                if (take) {
                    uint32_t xo[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) xo[k] = X[k] & k16[k];
                    chan_accum(xo, mv.x & olo, mv.y & ohi, odd, c);
                    chan_accum(X, mv.x, mv.y, all, c);
                }
                if (slow) {
                    qe[2 + c] = mv.x;
                    qe[5 + c] = mv.y;
#pragma unroll
                    for (int k = 0; k < 4; ++k) qe[8 + 4 * c + k] = X[k];
                }
            }
            odd.n += po_n;
            all.n += take ? 8u : 0u;
            if (want) {
                if (slow) {
                    qe[0] = elo;
                    qe[1] = ehi;
                    qe[20] = 8u;
                }
                __syncwarp();
                fq.nq += __popc(want);
            }
            tile_release(L.sempty((int)((si + j) % kTileS)), lane);
            tile_release(L.aempty((int)((ai + j) % TileAux<TmaMode::kFit>::kSlots)), lane);
            if ((j + 1) % kRunRows == 0 || j + 1 == T.rows) {
                // bounded runs: flush both (the even run is all - odd)
                RunAcc e = all;
                run_minus(e, odd);
                e.E = all.E;
                warp_flush(e, bins, lane);
                warp_flush(odd, bins, lane);
                run_reset(all, -1);
                run_reset(odd, -1);
            }
        }
        if (!ok) break;
        tile_release(L.sempty((int)((si + T.rows) % kTileS)), lane);
        tile_release(L.sempty((int)((si + T.rows + 1) % kTileS)), lane);
        si += T.rows + 2;
        ai += T.rows;
    }
    if (ok) {
        drain_runs(fq, bins, lane);
        drain_segs(fq, bins, lane);
    }
    consumers_sync();
    for (int i = threadIdx.x; i < kNbin * kNsum; i += kTileWarps * 32) {
        const unsigned long long v = ((unsigned long long)bins.hi[i] << 12) + bins.lo[i];
        if (v) atomicAdd(A.gbins + i, v);
    }
}

// ---------------------------------------------------------------- residual / decode on the tile pipeline

template <TmaMode MODE>
constexpr size_t tile_rows_smem() {
    return 128 + TileSmem<MODE>::kHead + sizeof(float2) * 3 * kNbin +
           (MODE == TmaMode::kResidual ? sizeof(uint32_t) * 3 * kNres : 0);
}
static_assert(3 * (tile_rows_smem<TmaMode::kResidual>() + 1024) <= 228 * 1024, "three residual CTAs per SM");
static_assert(2 * (tile_rows_smem<TmaMode::kDecode>() + 1024) <= 228 * 1024, "two decode CTAs per SM");

// k_rows_tile<kResidual>: R = M - M* and histograms; k_rows_tile<kDecode>:
// M = R + M*, repacked with E.
template <TmaMode MODE>
__global__ void __launch_bounds__(kTileThreads, TileAux<MODE>::kCtas) k_rows_tile(const __grid_constant__ CUtensorMap tm_s,
                                                                const __grid_constant__ CUtensorMap tm_a,
                                                                const __grid_constant__ CUtensorMap tm_e,
                                                                const TileArgs A) {
    extern __shared__ __align__(128) char dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TileSmem<MODE> L = tile_smem<MODE>(dyn);
    char* extra = dyn + (L.extra - smem_addr(dyn));
    float2* ab = reinterpret_cast<float2*>(extra);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ab + 3 * kNbin);
    tile_init_barriers(L);
    __syncthreads();

    if (warp == kTileWarps) {
        if (lane == 0) tile_produce(L, &tm_s, &tm_a, &tm_e, A);
        return;
    }
    // the consumers fetch the parameters while the first copies are in flight
    load_params_ab(A.params, ab, kTileWarps * 32);
    if (MODE == TmaMode::kResidual && A.hist)
        for (int i = threadIdx.x; i < 3 * kNres; i += kTileWarps * 32) hist[i] = 0u;
    consumers_sync();
    const TileConsumer<MODE> C{L, A.max_spins};
    const int w = A.w;
    const int64_t n = (int64_t)A.h * w;
    const bool gf = A.gf != 0;
    TileRange T = tile_range(A.total_rows, A.h);
    uint32_t si = 0, ai = 0;
    bool ok = true;
    while (ok && T.next()) {
        const LaneCols lc(T.xs, w, warp, lane);
        ok = C.wait_s(si) && C.wait_s(si + 1);
        for (int j = 0; j < T.rows && ok; ++j) {
            ok = C.wait_s(si + j + 2) && C.wait_a(ai + j);
            if (!ok) break;
            const uint32_t sa = L.sslot(si + j), sb = L.sslot(si + j + 1), sc = L.sslot(si + j + 2);
            const uint32_t as = L.aslot(ai + j);
            const int y = T.y0 + j;
            if (lc.inside) {
                const uint2 ev = lds64(as + TileAux<MODE>::kE + kStripCols * warp + 8 * lane);
                if constexpr (MODE == TmaMode::kResidual) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        uint32_t X[4];
                        tile_x(sa, sb, sc, c, lc, gf, X);
                        const uint2 mv = lds64(as + (uint32_t)c * TileAux<MODE>::kPlane + kStripCols * warp + 8 * lane);
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
                        *reinterpret_cast<uint4*>(A.r3_out + c * n + (int64_t)y * w + lc.x0) = v;
                        if (A.hist) {
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
                        tile_x(sa, sb, sc, c, lc, gf, X);
                        const uint4 v =
                            lds128(as + (uint32_t)c * TileAux<MODE>::kPlane + 2u * (kStripCols * warp + 8 * lane));
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
                    uint4* o4 = reinterpret_cast<uint4*>(A.out + (int64_t)y * w + lc.x0);
                    o4[0] = make_uint4(word[0], word[1], word[2], word[3]);
                    o4[1] = make_uint4(word[4], word[5], word[6], word[7]);
                }
            }
            C.release_s(si + j, lane);
            C.release_a(ai + j, lane);
        }
        if (!ok) break;
        C.release_s(si + T.rows, lane);
        C.release_s(si + T.rows + 1, lane);
        si += T.rows + 2;
        ai += T.rows;
    }
    if (MODE == TmaMode::kResidual && A.hist) {
        consumers_sync();
        for (int i = threadIdx.x; i < 3 * kNres; i += kTileWarps * 32)
            if (hist[i]) atomicAdd(A.hist + i, hist[i]);
    }
}

bool tma_eligible(int w, std::initializer_list<const void*> ptrs) {
    if (w % 16 != 0) return false;
    for (const void* p : ptrs)
        if ((uintptr_t)p % 16 != 0) return false;
    return true;
}

// ---------------------------------------------------------------- tensor maps (host)

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Tensor map of `planes` planes of h x w pixels of `esize` bytes, viewed as
// (16-byte chunk, chunk, row, plane); a box is one row of `box_chunks` chunks
// of every plane.
bool plane_map(CUtensorMap* tm, const void* base, int esize, int h, int w, int planes, int box_chunks) {
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return false;
    }
    const cuuint64_t row = (cuuint64_t)w * esize;
    const cuuint64_t dims[4] = {(cuuint64_t)(16 / esize), row / 16, (cuuint64_t)h, (cuuint64_t)planes};
    const cuuint64_t strides[3] = {16, row, row * (cuuint64_t)h};
    const cuuint32_t box[4] = {(cuuint32_t)(16 / esize), (cuuint32_t)box_chunks, 1, (cuuint32_t)planes};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = enc(tm, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 4,
                           const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for a %d x %d plane map", (int)r, h, w);
        return false;
    }
    return true;
}

template <TmaMode MODE>
bool tile_maps(TileMaps& M, const uint8_t* s3, const void* aux, const uint8_t* e, int h, int w) {
    return plane_map(&M.s, s3, 1, h, w, 3, kTileSW / 16) &&
           plane_map(&M.a, aux, (int)TileAux<MODE>::kElem, h, w, 3, (int)(TileAux<MODE>::kElem * kTileCols / 16)) &&
           plane_map(&M.e, e, 1, h, w, 1, kTileCols / 16);
}

// Grid of a tile kernel: at least four rows per CTA; at most two CTAs per SM,
// or `per_sm` when every CTA still gets 16 rows or more (a short range
// spends proportionally more of its time filling the rings); for the fit at
// least total_rows / rows_max CTAs.
int64_t tile_grid(int64_t total_rows, int64_t rows_max, int per_sm) {
    if (total_rows < (int64_t)16 * per_sm * geometry().sms) per_sm = 2;
    int64_t g = (total_rows + 3) / 4;
    const int64_t cap = (int64_t)geometry().sms * per_sm;
    if (g > cap) g = cap;
    if (rows_max > 0 && g < (total_rows + rows_max - 1) / rows_max) g = (total_rows + rows_max - 1) / rows_max;
    return g < 1 ? 1 : g;
}

template <typename K>
int tile_smem_attr(K kernel, size_t bytes, bool* set) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cuda_status("tile kernel device");
    if (!set[dev]) {
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
            return cuda_status("tile kernel shared memory attribute");
        set[dev] = true;
    }
    return SLRME_OK;
}

template <TmaMode MODE>
int launch_rows_tile(const uint8_t* s3, const void* aux, const uint8_t* e, int h, int w, int gf_on,
                     const slrme_params* P, int16_t* r3_out, uint32_t* hist, uint32_t* out, cudaStream_t s) {
    static bool attr_set[64];
    constexpr size_t smem = tile_rows_smem<MODE>();
    int st = tile_smem_attr(k_rows_tile<MODE>, smem, attr_set);
    if (st != SLRME_OK) return st;
    TileMaps M;
    if (!tile_maps<MODE>(M, s3, aux, e, h, w)) return SLRME_ECUDA;
    const int64_t total_rows = (int64_t)((w + kTileCols - 1) / kTileCols) * h;
    TileArgs A{h, w, gf_on, total_rows, kMaxSpins, P, r3_out, hist, out, nullptr};
    k_rows_tile<MODE><<<(unsigned)tile_grid(total_rows, 0, TileAux<MODE>::kCtas), kTileThreads, smem, s>>>(M.s, M.a,
                                                                                                    M.e, A);
    return cuda_status(MODE == TmaMode::kResidual ? "residual_encode launch" : "residual_decode launch");
}

int launch_fit_tile(const uint8_t* s3, const uint8_t* m3, const uint8_t* e, int h, int w, int gf_on,
                    unsigned long long* bins, cudaStream_t s) {
    static bool attr_set[64];
    int st = tile_smem_attr(k_fit_tile, kTileFitSmem, attr_set);
    if (st != SLRME_OK) return st;
    TileMaps M;
    if (!tile_maps<TmaMode::kFit>(M, s3, m3, e, h, w)) return SLRME_ECUDA;
    const int64_t total_rows = (int64_t)((w + kTileCols - 1) / kTileCols) * h;
    // a CTA adds at most kMaxBlockPixels pixels to its bins
    const int64_t rows_max = kMaxBlockPixels / kTileCols;
    TileArgs A{h, w, gf_on, total_rows, kMaxSpins, nullptr, nullptr, nullptr, nullptr, bins};
    k_fit_tile<<<(unsigned)tile_grid(total_rows, rows_max, TileAux<TmaMode::kFit>::kCtas), kTileThreads, kTileFitSmem,
                 s>>>(M.s, M.a, M.e, A);
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
            st = launch_fit_tile(s3, m3, e, h, w, gf_on, reinterpret_cast<unsigned long long*>(bin_sums), s);
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
    if (tma_eligible(w, {s3, m3, e, r3}))
        return launch_rows_tile<TmaMode::kResidual>(s3, m3, e, h, w, gf_on, params, r3, hist, nullptr, s);
    const StripLaunch L = strip_launch(h, w, 2);
    k_residual<<<L.blocks, kThreads, 0, s>>>(s3, m3, e, h, w, gf_on, fast ? 1 : 0, L.rows, params, r3, hist);
    return cuda_status("residual_encode launch");
}

int launch_residual_decode(const uint8_t* s3, const uint8_t* e, const int16_t* r3, int h, int w, int gf_on,
                           const slrme_params* params, uint32_t* rgbe_out, cudaStream_t s) {
    const bool fast = (w % 8 == 0) && ((uintptr_t)s3 % 8 == 0) && ((uintptr_t)e % 8 == 0);
    if (tma_eligible(w, {s3, e, r3, rgbe_out}))
        return launch_rows_tile<TmaMode::kDecode>(s3, r3, e, h, w, gf_on, params, nullptr, nullptr, rgbe_out, s);
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
static void* g_status_addr[kMaxDevices];

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

// Device address of the status word g_slrme_status on the current device,
// looked up once per device, for kernels of other translation units.
int status_word_address(int** out) {
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) {
        set_error("status word: cudaGetDevice: %s", cudaGetErrorString(err));
        return SLRME_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("status word: device ordinal %d outside 0..%d", dev, kMaxDevices - 1);
        return SLRME_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_status_addr[dev]) {
        void* p = nullptr;
        err = cudaGetSymbolAddress(&p, g_slrme_status);
        if (err != cudaSuccess || !p) {
            set_error("status word: cudaGetSymbolAddress: %s", cudaGetErrorString(err));
            return SLRME_ECUDA;
        }
        g_status_addr[dev] = p;
    }
    *out = (int*)g_status_addr[dev];
    return SLRME_OK;
}

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

namespace slrme {
namespace {

// Self-test of the bounded waits: one warp waits for phase 0 of a
// shared-memory mbarrier with room for one arrival.  With `arrive` = 0
// nothing ever arrives: the wait gives up after max_spins polls, records
// the timeout in the device status word and the kernel returns (no copy is
// in flight, so nothing is left behind).  With arrive = 1 lane 0 arrives
// first and the wait completes.
__global__ void __launch_bounds__(32) k_wait_probe(int max_spins, int arrive) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        fence_async_shared();
    }
    __syncwarp();
    if (arrive && threadIdx.x == 0) mbar_arrive(b);
    __syncwarp();
    mbar_wait(b, 0u, &g_slrme_status, max_spins);
}

}  // namespace
}  // namespace slrme

extern "C" int slrme_wait_probe(int max_spins, int arrive, slrme_stream_t stream) {
    using namespace slrme;
    if (max_spins < 1 || max_spins > (1 << 20) || (arrive != 0 && arrive != 1)) {
        set_error("slrme_wait_probe: max_spins must be in 1..2^20 and arrive 0 or 1");
        return SLRME_EINVAL;
    }
    k_wait_probe<<<1, 32, 0, (cudaStream_t)stream>>>(max_spins, arrive);
    return cuda_status("slrme_wait_probe launch");
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
