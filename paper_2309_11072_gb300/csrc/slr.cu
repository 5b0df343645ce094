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

// ====================================================================== bulk-copy row pipeline
//
// For images whose rows are 16-byte aligned (w % 16 == 0, 16-byte aligned
// planes).  The image is cut into strips of kTileCols = 2048 columns, one
// 256-column slice per consumer warp (kTileWarps = 8 per CTA).  The rows of
// all strips, strip after strip, are split into one contiguous range per
// CTA, and a range becomes tasks of at most kTaskRows rows of one strip.
// A producer warp streams the range through two shared-memory rings with
// 1-D bulk copies (cp.async.bulk, one per plane row: 2 to 4 KB each; a
// tensor map would cut the 2 KB rows into 16-byte box lines, and moved the
// same bytes about 1.5 times slower): per S item, the S row of the three
// planes with 16 halo columns on each side; per row, its other planes (M
// and E for the fit and the residual, R and E for the decoder).  Row j of a
// task needs S rows y - 1, y, y + 1 (clamped to the image by the producer,
// which replicates the edge rows); the consumers keep the filtered rows
// y - 1 and y in registers, so each S item is read once and released at
// once, and the S ring runs two items ahead of the aux ring.  A slot's full
// barrier completes on the bytes of its copies; its empty barrier completes
// when all consumer warps have arrived.  Edge columns replicate through the
// neighbour offsets.  Every wait is bounded (see tma.cuh).

constexpr int kTileWarps = 8;                              // consumer warps
constexpr int kTileThreads = (kTileWarps + 1) * 32;        // + one producer warp
constexpr int kTileCols = kTileWarps * kStripCols;         // 2048
constexpr int kTileSW = kTileCols + 32;                    // S row with halos, per plane
static_assert(kTileColsBatch == kTileCols, "batch strips are tile strips");
constexpr int kTaskRows = 256;
constexpr uint32_t kTileSBytes = 3u * kTileSW;             // 6240
constexpr uint32_t kTileSStride = 6272;                    // slot stride, multiple of 128
static_assert(kTileSStride >= kTileSBytes && kTileSStride % 128 == 0, "S slot");

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
    // Ring slots: the aux ring (rows j) and the S ring (rows j + 1, so it
    // runs two items ahead of the aux ring and needs two slots more).  The
    // fit's bins and queues leave room for 3 aux rows; the residual and the
    // decoder take deeper rings to keep more bytes in flight per SM.
    static constexpr int kSlots = MODE == TmaMode::kFit ? 3 : (MODE == TmaMode::kResidual ? 5 : 4);
    static constexpr int kSSlots = kSlots + 2;
    // CTAs per SM the kernel is built for
    static constexpr int kCtas = 2;
};

// In-order position in a ring of K slots: the slot and the parity of its
// current use (item i is slot i % K, use i / K).
template <int K>
struct RingPos {
    uint32_t v;   // slot * 2 + phase
    __device__ __forceinline__ uint32_t slot() const { return v >> 1; }
    __device__ __forceinline__ uint32_t phase() const { return v & 1u; }
    __device__ __forceinline__ void advance() {
        v += 2u;
        if (v >= 2u * K) v = (v & 1u) ^ 1u;
    }
};

struct TileArgs {
    const uint8_t* s3;                       // S planes
    const void* aux;                         // M planes (fit, residual)
    const uint8_t* e;                        // E plane
    int h, w;
    int gf;
    int64_t total_rows;                      // strips * h
    int max_spins;
    const slrme_params* params;              // residual
    int16_t* r3_out;                         // residual
    uint32_t* hist;                          // residual (may be null)
    unsigned long long* gbins;               // fit
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Barrier among the consumer warps only (the producer warp may have left).
__device__ __forceinline__ void consumers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kTileWarps * 32) : "memory");
}

// The CTA's rows r .. end - 1 in (strip, row) order and its current task.
// Rows are counted in 32 bits: the tile kernels need w % 16 == 0, so
// strips * h <= h * w / 2048 + h < 2^31 for every image the ABI accepts.
struct TileRange {
    int r, end;
    int h;
    int y0, rows, xs;
    __device__ __forceinline__ bool next() {
        if (r >= end) return false;
        const int c = r / h;
        y0 = r - c * h;
        rows = min(min(end - r, h - y0), kTaskRows);
        xs = c * kTileCols;
        r += rows;
        return true;
    }
};

__device__ __forceinline__ TileRange tile_range(int64_t total_rows, int h) {
    const int64_t G = gridDim.x, b = blockIdx.x;
    return TileRange{(int)(b * total_rows / G), (int)((b + 1) * total_rows / G), h, 0, 0, 0};
}

// Shared-memory layout of a tile kernel: the two rings, then four barrier
// arrays, then the mode's own data at `extra`.
template <TmaMode MODE>
struct TileSmem {
    static constexpr int KS = TileAux<MODE>::kSSlots, KA = TileAux<MODE>::kSlots;
    uint32_t s_ring, a_ring, bars, extra;
    __device__ __forceinline__ uint32_t sfull(uint32_t k) const { return bars + 8u * k; }
    __device__ __forceinline__ uint32_t sempty(uint32_t k) const { return bars + 8u * (KS + k); }
    __device__ __forceinline__ uint32_t afull(uint32_t k) const { return bars + 8u * (2 * KS + k); }
    __device__ __forceinline__ uint32_t aempty(uint32_t k) const { return bars + 8u * (2 * KS + KA + k); }
    __device__ __forceinline__ uint32_t sslot_at(uint32_t k) const { return s_ring + k * kTileSStride; }
    __device__ __forceinline__ uint32_t aslot_at(uint32_t k) const { return a_ring + k * TileAux<MODE>::kStride; }
    static constexpr uint32_t kRings = KS * kTileSStride + KA * TileAux<MODE>::kStride;
    static constexpr uint32_t kHead = kRings + 8u * 2 * (KS + KA);   // multiple of 16
};

template <TmaMode MODE>
__device__ __forceinline__ TileSmem<MODE> tile_smem(char* dyn) {
    const uint32_t base = (smem_addr(dyn) + 127u) & ~127u;
    TileSmem<MODE> L;
    L.s_ring = base;
    L.a_ring = base + TileSmem<MODE>::KS * kTileSStride;
    L.bars = base + TileSmem<MODE>::kRings;
    L.extra = base + TileSmem<MODE>::kHead;
    return L;
}

template <TmaMode MODE>
__device__ __forceinline__ void tile_init_barriers(const TileSmem<MODE>& L) {
    if (threadIdx.x == 0) {
        for (int k = 0; k < TileSmem<MODE>::KS; ++k) {
            mbar_init(L.sfull(k), 1);
            mbar_init(L.sempty(k), kTileWarps);
        }
        for (int k = 0; k < TileSmem<MODE>::KA; ++k) {
            mbar_init(L.afull(k), 1);
            mbar_init(L.aempty(k), kTileWarps);
        }
        fence_async_shared();
    }
}

// The producer (one thread): items in the order the consumers use them,
// each as 1-D bulk copies of whole plane rows (one per plane; 16-byte
// aligned because w % 16 == 0 and the planes are 16-byte aligned).  An S
// item is row ys of the three S planes, columns xs - 16 .. xs + 2063 clipped
// to the image, at offset x - (xs - 16) of each plane's slot row; an aux item
// is row y of the three aux planes and of E, columns xs .. xs + 2047 clipped.
// Slot bytes past the image are never read as pixels.  Stops issuing if a
// wait for a free slot gave up.
template <TmaMode MODE>
__device__ __noinline__ void tile_produce(const TileSmem<MODE>& L, const TileArgs& A) {
    constexpr int KS = TileSmem<MODE>::KS, KA = TileSmem<MODE>::KA;
    constexpr uint32_t kEl = TileAux<MODE>::kElem;
    const int64_t n = (int64_t)A.h * A.w;
    const uint8_t* aux = static_cast<const uint8_t*>(A.aux);
    TileRange P = tile_range(A.total_rows, A.h);
    uint32_t si = 0, ai = 0;   // items issued
    RingPos<KS> sp{0u};
    RingPos<KA> ap{0u};
    bool ok = true;
    while (ok && P.next()) {
        const int xa = max(P.xs - 16, 0), xb = min(P.xs + kTileCols + 16, A.w);
        const uint32_t s_bytes = (uint32_t)(xb - xa), s_off = (uint32_t)(xa - (P.xs - 16));
        const uint32_t cols = (uint32_t)(min(P.xs + kTileCols, A.w) - P.xs);
        for (int k = 0; k < P.rows + 2 && ok; ++k) {
            // S item k: row y0 - 1 + k, clamped (edge rows replicate)
            {
                if (si >= (uint32_t)KS) ok = mbar_wait(L.sempty(sp.slot()), sp.phase() ^ 1u, &g_slrme_status, A.max_spins);
                if (!ok) break;
                const int ys = min(max(P.y0 - 1 + k, 0), A.h - 1);
                const uint32_t dst = L.sslot_at(sp.slot()) + s_off, bar = L.sfull(sp.slot());
                const uint8_t* src = A.s3 + (int64_t)ys * A.w + xa;
                fence_async_shared();
                mbar_arrive_expect_tx(bar, 3u * s_bytes);
#pragma unroll
                for (int c = 0; c < 3; ++c) tma_load_1d(dst + (uint32_t)c * kTileSW, src + c * n, s_bytes, bar);
                ++si;
                sp.advance();
            }
            if (k >= 2) {   // the other planes of row y0 + k - 2
                if (ai >= (uint32_t)KA) ok = mbar_wait(L.aempty(ap.slot()), ap.phase() ^ 1u, &g_slrme_status, A.max_spins);
                if (!ok) break;
                const int64_t row = (int64_t)(P.y0 + k - 2) * A.w + P.xs;
                const uint32_t dst = L.aslot_at(ap.slot()), bar = L.afull(ap.slot());
                fence_async_shared();
                mbar_arrive_expect_tx(bar, (3u * kEl + 1u) * cols);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    tma_load_1d(dst + (uint32_t)c * TileAux<MODE>::kPlane, aux + (c * n + row) * kEl, kEl * cols, bar);
                tma_load_1d(dst + TileAux<MODE>::kE, A.e + row, cols, bar);
                ++ai;
                ap.advance();
            }
        }
    }
    // before leaving, wait (bounded) for the last copy into every slot, so
    // no copy is in flight if the consumers stopped early
    const int spins = ok ? A.max_spins : (1 << 10);
    for (uint32_t k = si > (uint32_t)KS ? si - KS : 0; k < si; ++k)
        mbar_wait(L.sfull(k % KS), (k / KS) & 1u, &g_slrme_status, spins);
    for (uint32_t k = ai > (uint32_t)KA ? ai - KA : 0; k < ai; ++k)
        mbar_wait(L.afull(k % KA), (k / KA) & 1u, &g_slrme_status, spins);
}

// One consumer warp's view of the rings: it waits for, reads and releases
// the items of each ring in order.
template <TmaMode MODE>
struct TileConsumer {
    TileSmem<MODE> L;
    int max_spins;
    RingPos<TileSmem<MODE>::KS> s;
    RingPos<TileSmem<MODE>::KA> a;
    // the whole warp waits together (mbar_wait_warp), so every lane sees the
    // same outcome before the warp-wide steps that follow
    __device__ __forceinline__ bool wait_s() const {
        return mbar_wait_warp(L.sfull(s.slot()), s.phase(), &g_slrme_status, max_spins);
    }
    __device__ __forceinline__ bool wait_a() const {
        return mbar_wait_warp(L.afull(a.slot()), a.phase(), &g_slrme_status, max_spins);
    }
    __device__ __forceinline__ uint32_t s_addr() const { return L.sslot_at(s.slot()); }
    __device__ __forceinline__ uint32_t a_addr() const { return L.aslot_at(a.slot()); }
    // all lanes call after their last read of the current item
    __device__ __forceinline__ void release_s(int lane) {
        __syncwarp();
        if (lane == 0) mbar_arrive(L.sempty(s.slot()));
        s.advance();
    }
    __device__ __forceinline__ void release_a(int lane) {
        __syncwarp();
        if (lane == 0) mbar_arrive(L.aempty(a.slot()));
        a.advance();
    }
};

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

// ---------------------------------------------------------------- fit on the tile pipeline
//
// A consumer lane keeps, per channel, the horizontally filtered S rows y - 1
// and y as 16-bit pairs (the 3x3 binomial filter is separable: [1 2 1] along
// x, then [1 2 1] along y), so each S row is read from the ring once and
// released at once.  Its pixels' sums go to two runs per lane: `all` holds
// both exponent parities, `odd` the odd one; the even run is all - odd.  A run
// lives until its region changes or its task ends, at most kTaskRows rows of
// 8 pixels.  sum x x is kept in two parts, sum x (x & 255) and sum x (x >> 8),
// so every run word stays below 2^32 at that length.

struct Run2 {
    int E;            // region (the even one for `all`), -1 = none
    uint32_t n;
    uint32_t sx[3], sy[3], sxy[3], sxl[3], sxh[3];
};
static_assert(8ull * kTaskRows * 4080ull * 255ull < (1ull << 32), "run sums of x y exceed 32 bits");

__device__ __forceinline__ void run2_reset(Run2& a, int E) {
    a.E = E;
    a.n = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) a.sx[c] = a.sy[c] = a.sxy[c] = a.sxl[c] = a.sxh[c] = 0;
}

__device__ __forceinline__ void run2_sub(Run2& a, const Run2& b) {   // a -= b (E kept)
    a.n -= b.n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a.sx[c] -= b.sx[c];
        a.sy[c] -= b.sy[c];
        a.sxy[c] -= b.sxy[c];
        a.sxl[c] -= b.sxl[c];
        a.sxh[c] -= b.sxh[c];
    }
}

// One channel of an 8-pixel segment added to sums (sum x, sum y, sum x y,
// sum x (x & 255), sum x (x >> 8)): x as 16-bit pairs and the y bytes, both
// already masked to the run's pixels (21 operations).
__device__ __forceinline__ void seg_accum5(const uint32_t (&X)[4], uint32_t yl, uint32_t yh, uint32_t& sx,
                                           uint32_t& sy, uint32_t& sxy, uint32_t& sxl, uint32_t& sxh) {
    const uint32_t ps = X[0] + X[1] + X[2] + X[3];   // each half at most 4 * 4080
    sx = __dp2a_lo(ps, 0x0101u, sx);
    sy = __dp4a(yl, 0x01010101u, __dp4a(yh, 0x01010101u, sy));
    uint32_t q = __dp2a_lo(X[0], yl, sxy);
    q = __dp2a_hi(X[1], yl, q);
    q = __dp2a_lo(X[2], yh, q);
    sxy = __dp2a_hi(X[3], yh, q);
    // x x = x (x & 255) + 256 x (x >> 8): the low and high bytes of each x as
    // byte operands of the 16 x 8-bit dot products
    const uint32_t la = __byte_perm(X[0], X[1], 0x6420), ha = __byte_perm(X[0], X[1], 0x7531);
    const uint32_t lb = __byte_perm(X[2], X[3], 0x6420), hb = __byte_perm(X[2], X[3], 0x7531);
    uint32_t l = __dp2a_lo(X[0], la, sxl);
    l = __dp2a_hi(X[1], la, l);
    l = __dp2a_lo(X[2], lb, l);
    sxl = __dp2a_hi(X[3], lb, l);
    uint32_t g = __dp2a_lo(X[0], ha, sxh);
    g = __dp2a_hi(X[1], ha, g);
    g = __dp2a_lo(X[2], hb, g);
    sxh = __dp2a_hi(X[3], hb, g);
}

__device__ __forceinline__ void seg_accum(const uint32_t (&X)[4], uint32_t yl, uint32_t yh, Run2& r, int c) {
    seg_accum5(X, yl, yh, r.sx[c], r.sy[c], r.sxy[c], r.sxl[c], r.sxh[c]);
}

// Horizontal [1 2 1] of one row segment (its 8 bytes lo/hi and the bytes l, r
// left and right of it) as 16-bit pairs: H[k] = (h(2k), h(2k + 1)).
__device__ __forceinline__ void hfilter(uint32_t lo, uint32_t hi, uint32_t l, uint32_t r, uint32_t (&H)[4]) {
    const uint32_t P0 = __byte_perm(lo, 0, 0x4140), P1 = __byte_perm(lo, 0, 0x4342);
    const uint32_t P2 = __byte_perm(hi, 0, 0x4140), P3 = __byte_perm(hi, 0, 0x4342);
    const uint32_t L0 = __byte_perm(l, P0, 0x5410);    // (s[-1], s[0])
    const uint32_t L1 = __byte_perm(P0, P1, 0x5432);   // (s[1], s[2])
    const uint32_t L2 = __byte_perm(P1, P2, 0x5432);   // (s[3], s[4])
    const uint32_t L3 = __byte_perm(P2, P3, 0x5432);   // (s[5], s[6])
    const uint32_t L4 = __byte_perm(P3, r, 0x5432);    // (s[7], s[8])
    H[0] = L0 + 2u * P0 + L1;
    H[1] = L1 + 2u * P1 + L2;
    H[2] = L2 + 2u * P2 + L3;
    H[3] = L3 + 2u * P3 + L4;
}

// The bytes of one lane's segment of plane c of an S slot as 16-bit pairs
// (kGf: horizontally filtered; else unpacked).
template <bool kGf>
__device__ __forceinline__ void s_row_pairs(uint32_t slot, int c, const LaneCols& lc, uint32_t (&H)[4]) {
    const uint32_t row = slot + (uint32_t)c * kTileSW;
    const uint2 v = lds64(row + lc.own);
    if constexpr (kGf) {
        uint32_t l, r;
        asm volatile("ld.shared.u8 %0, [%1];" : "=r"(l) : "r"(row + lc.offl));
        asm volatile("ld.shared.u8 %0, [%1];" : "=r"(r) : "r"(row + lc.offr));
        hfilter(v.x, v.y, l, r, H);
    } else {
        H[0] = __byte_perm(v.x, 0, 0x4140);
        H[1] = __byte_perm(v.x, 0, 0x4342);
        H[2] = __byte_perm(v.y, 0, 0x4140);
        H[3] = __byte_perm(v.y, 0, 0x4342);
    }
}

// Two per-warp queues: flushed runs (their sums) and segments that need
// per-pixel work (their pixels).  Each is drained by its own code path, one
// entry per lane, so draining runs never pays for the per-pixel segment path.
// A row queues at most one segment per lane, so the segment queue holds 32 (a
// row's segments are written piece by piece while the row is processed); runs,
// complete when queued, go in chunks that fit the 16-entry run queue, draining
// it in between.  A run entry: N, then per channel sum x, sum y, sum x y,
// sum x (x & 255) and sum x (x >> 8), then the region (odd stride: distinct
// banks).
constexpr int kRunQ = 16;
constexpr int kRunWords = 1 + 5 * 3;
constexpr int kRunStride = kRunWords + 1;   // 17
constexpr int kSegQ = 32;                   // segment entries of kQueueStride words
struct FitQueues {
    uint32_t* R;   // run entries
    uint32_t* Q;   // segment entries
    int nr, nq;    // entries queued (warp-uniform)
};

// Exactness of the tile fit's shared bins: a run entry adds sum x x as two
// values (sum x (x & 255) and 256 sum x (x >> 8)), so a low word takes at most
// two additions per pixel; a CTA adds at most kTileFitMaxPixels pixels, which
// keeps every low word below 2^21 (2^12 - 1) < 2^32 and every high word below
// 2^19 4080^2 / 2^12 < 2^32.
constexpr int64_t kTileFitMaxPixels = (int64_t)1 << 19;
static_assert(2ull * kTileFitMaxPixels * 4095ull < (1ull << 32), "tile fit low words overflow");
static_assert((unsigned long long)kTileFitMaxPixels * 4080ull * 4080ull / 4096ull < (1ull << 32),
              "tile fit high words overflow");

__device__ __forceinline__ void drain_runs(FitQueues& fq, SmemBins& bins, int lane) {
    if (lane < fq.nr) {
        const uint32_t* q = fq.R + lane * kRunStride;
        const uint32_t B = smem_addr(&bins);
        const uint32_t lo = B + 4u * (uint32_t)(q[kRunWords] * kNsum), hi = lo + 4u * kNbin * kNsum;
        red_add(lo, q[0] & 0xFFFu);
        red_add(hi, q[0] >> 12);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint32_t* v = q + 1 + 5 * c;
            const uint32_t a = 4u * (1 + 4 * c);
            red_add(lo + a, v[0] & 0xFFFu);
            red_add(hi + a, v[0] >> 12);
            red_add(lo + a + 4u, v[1] & 0xFFFu);
            red_add(hi + a + 4u, v[1] >> 12);
            red_add(lo + a + 8u, v[2] & 0xFFFu);
            red_add(hi + a + 8u, v[2] >> 12);
            // sum x x = sxl + 256 sxh
            red_add(lo + a + 12u, v[3] & 0xFFFu);
            red_add(hi + a + 12u, v[3] >> 12);
            red_add(lo + a + 12u, (v[4] & 0xFu) << 8);
            red_add(hi + a + 12u, v[4] >> 4);
        }
    }
    __syncwarp();
    fq.nr = 0;
}

// Adds the eight pixels of a queued segment to their bins one by one, without
// branches: per pixel 19 reductions (the count, x and y are below 2^12 and
// have no high part under the split rule; x y and x x take two words).
__device__ __forceinline__ void drain_segment_pixels(const uint32_t* q, uint32_t B) {
    const uint32_t elo = q[0], ehi = q[1];
    const int cnt = (int)q[20];   // pixels of the segment (fewer than 8 at an image's right edge)
    uint32_t mlo[3] = {q[2], q[3], q[4]}, mhi[3] = {q[5], q[6], q[7]};
    uint32_t X[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) X[c][k] = q[8 + 4 * c + k];
    constexpr uint32_t kHi = 4u * kNbin * kNsum;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i < cnt) {
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
}

__device__ __forceinline__ void drain_segs(FitQueues& fq, SmemBins& bins, int lane) {
    if (lane < fq.nq) drain_segment_pixels(fq.Q + lane * kQueueStride, smem_addr(&bins));
    __syncwarp();
    fq.nq = 0;
}

// Queues the run of every lane with `want` set: the even run (all - odd,
// region all.E) or the odd run (odd, region odd.E), in chunks that fit.
template <bool kEven>
__device__ __forceinline__ void push_run(FitQueues& fq, bool want, const Run2& all, const Run2& odd,
                                         SmemBins& bins, int lane) {
    unsigned m = __ballot_sync(0xffffffffu, want);
    while (m) {
        if (fq.nr == kRunQ) drain_runs(fq, bins, lane);
        // the first kRunQ - nr lanes of m go now
        unsigned take = m;
        while (__popc(take) > kRunQ - fq.nr) take &= ~(1u << (31 - __clz(take)));
        if (take & (1u << lane)) {
            uint32_t* q = fq.R + (fq.nr + __popc(take & ((1u << lane) - 1u))) * kRunStride;
            q[0] = kEven ? all.n - odd.n : odd.n;   // even: all - odd; odd: odd
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if constexpr (kEven) {
                    q[1 + 5 * c] = all.sx[c] - odd.sx[c];
                    q[2 + 5 * c] = all.sy[c] - odd.sy[c];
                    q[3 + 5 * c] = all.sxy[c] - odd.sxy[c];
                    q[4 + 5 * c] = all.sxl[c] - odd.sxl[c];
                    q[5 + 5 * c] = all.sxh[c] - odd.sxh[c];
                } else {
                    q[1 + 5 * c] = odd.sx[c];
                    q[2 + 5 * c] = odd.sy[c];
                    q[3 + 5 * c] = odd.sxy[c];
                    q[4 + 5 * c] = odd.sxl[c];
                    q[5 + 5 * c] = odd.sxh[c];
                }
            }
            q[kRunWords] = (uint32_t)(kEven ? all.E : odd.E);
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

// x = 16 S* of channel c for the lane's 8 pixels as 16-bit pairs, from the
// window (rows y - 1 and y) and the new S row y + 1 in slot `sn`; the window
// moves down one row.
template <bool kGf>
__device__ __forceinline__ void window_x(uint32_t sn, int c, const LaneCols& lc, uint32_t (&Hm)[4],
                                         uint32_t (&H0)[4], uint32_t (&X)[4]) {
    uint32_t Hn[4];
    s_row_pairs<kGf>(sn, c, lc, Hn);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if constexpr (kGf) {
            X[k] = Hm[k] + 2u * H0[k] + Hn[k];
            Hm[k] = H0[k];
        } else {
            X[k] = H0[k] << 4;
        }
        H0[k] = Hn[k];
    }
}

// Moves a lane's runs to the region(s) of its next segment: a run whose
// region changes leaves through the queue first (the even run is all - odd).
// Ee / Eo: the segment's even / odd region; has_e / has_o: whether it has
// pixels of that parity.
__device__ __forceinline__ void runs_rekey(FitQueues& fq, Run2& all, Run2& odd, bool has_e, int Ee, bool has_o,
                                           int Eo, SmemBins& bins, int lane) {
    const bool chg_e = has_e && Ee != all.E;
    const bool chg_o = has_o && Eo != odd.E;
    if (!__any_sync(0xffffffffu, chg_e || chg_o)) return;
    push_run<true>(fq, chg_e && all.E >= 0 && all.n != odd.n, all, odd, bins, lane);
    push_run<false>(fq, chg_o && odd.E >= 0 && odd.n != 0u, all, odd, bins, lane);
    if (chg_e) {   // the even part left: all = odd
        const int keep = odd.E;
        all = odd;
        all.E = Ee;
        odd.E = keep;
    }
    if (chg_o) {   // the odd part left
        const int keep = all.E;
        run2_sub(all, odd);
        all.E = keep;
        run2_reset(odd, Eo);
    }
}

// The fit's consumer loop over the CTA's tasks.  Per row and lane: the
// exponent bytes decide, for the whole warp, between the fast path (every
// lane's 8 pixels in one region: one set of sums per channel, added to the
// run of the region's parity) and the general one (one even and one odd
// region per segment: the odd pixels' sums and all sums; anything else is
// queued for per-pixel work); then, channel by channel, the new S row moves
// the filter window and x = 16 S* is added.
template <bool kGf>
__device__ __forceinline__ bool fit_consume(const TileSmem<TmaMode::kFit>& L, const TileArgs& A, SmemBins& bins,
                                            uint32_t* queue, int warp, int lane) {
    TileConsumer<TmaMode::kFit> C{L, A.max_spins, {0u}, {0u}};
    const int w = A.w;
    FitQueues fq;
    fq.R = queue + warp * (kRunQ * kRunStride + kSegQ * kQueueStride);
    fq.Q = fq.R + kRunQ * kRunStride;
    fq.nr = fq.nq = 0;
    Run2 all, odd;
    TileRange T = tile_range(A.total_rows, A.h);
    bool ok = true;
    while (ok && T.next()) {
        const LaneCols lc(T.xs, w, warp, lane);
        run2_reset(all, -1);
        run2_reset(odd, -1);
        // the window: rows y0 - 1 and y0 (S items 0 and 1 of the task)
        uint32_t Hm[3][4], H0[3][4];
        ok = C.wait_s();
        if (!ok) break;
        if constexpr (kGf) {
#pragma unroll
            for (int c = 0; c < 3; ++c) s_row_pairs<kGf>(C.s_addr(), c, lc, Hm[c]);
        }
        C.release_s(lane);
        ok = C.wait_s();
        if (!ok) break;
#pragma unroll
        for (int c = 0; c < 3; ++c) s_row_pairs<kGf>(C.s_addr(), c, lc, H0[c]);
        C.release_s(lane);
        for (int j = 0; j < T.rows; ++j) {
            ok = C.wait_s() && C.wait_a();
            if (!ok) break;
            const uint32_t sn = C.s_addr();
            const uint32_t as = C.a_addr() + kStripCols * warp + 8 * lane;
            const uint2 ev = lds64(as + TileAux<TmaMode::kFit>::kE);
            const uint32_t elo = ev.x, ehi = ev.y;
            const uint32_t E1 = elo & 255u;
            const bool uni = elo == ehi && elo == E1 * 0x01010101u;
            if (__all_sync(0xffffffffu, uni || !lc.inside)) {
                // ---- fast path: one region per lane segment
                const bool isodd = (E1 & 1u) != 0u;
                runs_rekey(fq, all, odd, lc.inside && !isodd, (int)E1, lc.inside && isodd, (int)E1, bins, lane);
                const uint32_t mo = lc.inside && isodd ? 0xFFFFFFFFu : 0u;
                const uint32_t nadd = lc.inside ? 8u : 0u;
                all.n += nadd;
                odd.n += nadd & mo;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    uint32_t X[4];
                    window_x<kGf>(sn, c, lc, Hm[c], H0[c], X);
                    const uint2 mv = lds64(as + (uint32_t)c * TileAux<TmaMode::kFit>::kPlane);
                    if (lc.inside) {
                        uint32_t sx = 0u, sy = 0u, sxy = 0u, sxl = 0u, sxh = 0u;   // channel c of the segment
                        seg_accum5(X, mv.x, mv.y, sx, sy, sxy, sxl, sxh);
                        all.sx[c] += sx;
                        all.sy[c] += sy;
                        all.sxy[c] += sxy;
                        all.sxl[c] += sxl;
                        all.sxh[c] += sxh;
                        odd.sx[c] += sx & mo;
                        odd.sy[c] += sy & mo;
                        odd.sxy[c] += sxy & mo;
                        odd.sxl[c] += sxl & mo;
                        odd.sxh[c] += sxh & mo;
                    }
                }
            } else {
                // ---- general path: byte masks of the odd-exponent pixels; the
                // segment's odd (even) region is the OR of its odd (even) bytes,
                // which equals each of them exactly when they are all equal
                const uint32_t olo = (elo & 0x01010101u) * 0xFFu, ohi = (ehi & 0x01010101u) * 0xFFu;
                uint32_t eo = (elo & olo) | (ehi & ohi), ee = (elo & ~olo) | (ehi & ~ohi);
                eo |= eo >> 16;
                ee |= ee >> 16;
                const uint32_t Eo = (eo | (eo >> 8)) & 255u, Ee = (ee | (ee >> 8)) & 255u;
                const uint32_t Eo4 = Eo * 0x01010101u, Ee4 = Ee * 0x01010101u;
                const bool two = ((((elo ^ Eo4) & olo) | ((ehi ^ Eo4) & ohi) | ((elo ^ Ee4) & ~olo) |
                                   ((ehi ^ Ee4) & ~ohi)) == 0u);
                const bool slow = lc.inside && !two;
                const bool take = lc.inside && two;
                const uint32_t po_n = take ? (uint32_t)(__popc(olo) + __popc(ohi)) >> 3 : 0u;
                runs_rekey(fq, all, odd, take && po_n != 8u, (int)Ee, po_n != 0u, (int)Eo, bins, lane);
                const unsigned want = __ballot_sync(0xffffffffu, slow);
                uint32_t qe = 0u;   // word offset of this lane's segment entry
                if (want) {
                    if (fq.nq + __popc(want) > kSegQ) drain_segs(fq, bins, lane);
                    qe = (uint32_t)(fq.nq + __popc(want & ((1u << lane) - 1u))) * kQueueStride;
                }
                uint32_t k16[4];
                mask16(olo, ohi, k16);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    uint32_t X[4];
                    window_x<kGf>(sn, c, lc, Hm[c], H0[c], X);
                    const uint2 mv = lds64(as + (uint32_t)c * TileAux<TmaMode::kFit>::kPlane);
                    if (take) {
                        uint32_t xo[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) xo[k] = X[k] & k16[k];
                        seg_accum(xo, mv.x & olo, mv.y & ohi, odd, c);
                        seg_accum(X, mv.x, mv.y, all, c);
                    }
                    if (want) {   // warp-uniform: skipped when no lane queues a segment
                        if (slow) {
                            uint32_t* q = fq.Q + qe;
                            q[2 + c] = mv.x;
                            q[5 + c] = mv.y;
#pragma unroll
                            for (int k = 0; k < 4; ++k) q[8 + 4 * c + k] = X[k];
                        }
                    }
                }
                odd.n += po_n;
                all.n += take ? 8u : 0u;
                if (want) {
                    if (slow) {
                        uint32_t* q = fq.Q + qe;
                        q[0] = elo;
                        q[1] = ehi;
                        q[20] = 8u;
                    }
                    __syncwarp();
                    fq.nq += __popc(want);
                }
            }
            C.release_s(lane);
            C.release_a(lane);
        }
        if (!ok) break;
        // the task's runs leave
        push_run<true>(fq, all.E >= 0 && all.n != odd.n, all, odd, bins, lane);
        push_run<false>(fq, odd.E >= 0 && odd.n != 0u, all, odd, bins, lane);
    }
    if (ok) {
        drain_runs(fq, bins, lane);
        drain_segs(fq, bins, lane);
    }
    return ok;
}

template <bool kGf>
// The tile kernels hand their argument block by reference to the producer
// (a separate function): as a grid constant it stays in the parameter bank
// instead of being copied to each thread's stack, where every read of a field
// by the consumers would be a local-memory load.
__global__ void __launch_bounds__(kTileThreads, TileAux<TmaMode::kFit>::kCtas) k_fit_tile(const __grid_constant__ TileArgs A) {
    extern __shared__ __align__(128) char dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ int gave_up;   // a consumer's wait gave up: the CTA's bins are incomplete
    const TileSmem<TmaMode::kFit> L = tile_smem<TmaMode::kFit>(dyn);
    char* extra = dyn + (L.extra - smem_addr(dyn));
    SmemBins& bins = *reinterpret_cast<SmemBins*>(extra);
    uint32_t* queue = reinterpret_cast<uint32_t*>(extra + sizeof(SmemBins));
    tile_init_barriers(L);
    if (threadIdx.x == 0) gave_up = 0;
    __syncthreads();

    if (warp == kTileWarps) {
        if (lane == 0) tile_produce(L, A);
        return;
    }
    // the consumers clear the bins while the first copies are in flight
    static_assert(sizeof(SmemBins) % 16 == 0 && TileSmem<TmaMode::kFit>::kHead % 16 == 0, "16-byte bin stores");
    for (int i = threadIdx.x; i < (int)(sizeof(SmemBins) / 16); i += kTileWarps * 32)
        reinterpret_cast<uint4*>(extra)[i] = make_uint4(0u, 0u, 0u, 0u);
    consumers_sync();
    if (!fit_consume<kGf>(L, A, bins, queue, warp, lane) && lane == 0) atomicOr(&gave_up, 1);
    consumers_sync();
    // after a timeout (reported in the status word) the partial bins are not
    // added, so the sums hold only whole CTAs' pixels
    if (gave_up) return;
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
static_assert(TileAux<TmaMode::kResidual>::kCtas * (tile_rows_smem<TmaMode::kResidual>() + 1024) <= 228 * 1024,
              "residual CTAs per SM");
static_assert(TileAux<TmaMode::kDecode>::kCtas * (tile_rows_smem<TmaMode::kDecode>() + 1024) <= 228 * 1024,
              "decode CTAs per SM");

// The residual consumer loop: per row and lane, the new S row moves the
// filter window (as in the fit), then Eq. (8) per pixel and channel with the
// region's (a, b) pair from shared memory; R = M - M* is stored and counted.
// (The single-image decoder runs the batch form's row kernel on one image
// described inline, which was measured faster for it.)
template <TmaMode MODE, bool kGf>
__device__ __forceinline__ void rows_consume(const TileSmem<MODE>& L, const TileArgs& A, const float2* ab,
                                             uint32_t* hist, int warp, int lane) {
    static_assert(MODE == TmaMode::kResidual, "the single-image row kernel is the residual's");
    TileConsumer<MODE> C{L, A.max_spins, {0u}, {0u}};
    const int w = A.w;
    const int64_t n = (int64_t)A.h * w;
    TileRange T = tile_range(A.total_rows, A.h);
    bool ok = true;
    while (ok && T.next()) {
        const LaneCols lc(T.xs, w, warp, lane);
        uint32_t Hm[3][4], H0[3][4];
        ok = C.wait_s();
        if (!ok) break;
        if constexpr (kGf) {
#pragma unroll
            for (int c = 0; c < 3; ++c) s_row_pairs<kGf>(C.s_addr(), c, lc, Hm[c]);
        }
        C.release_s(lane);
        ok = C.wait_s();
        if (!ok) break;
#pragma unroll
        for (int c = 0; c < 3; ++c) s_row_pairs<kGf>(C.s_addr(), c, lc, H0[c]);
        C.release_s(lane);
        for (int j = 0; j < T.rows; ++j) {
            ok = C.wait_s() && C.wait_a();
            if (!ok) break;
            const uint32_t sn = C.s_addr();
            const uint32_t as = C.a_addr() + kStripCols * warp + 8 * lane;
            const int64_t pix = (int64_t)(T.y0 + j) * w + lc.x0;
            const uint2 ev = lds64(as + TileAux<MODE>::kE);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                uint32_t X[4];
                window_x<kGf>(sn, c, lc, Hm[c], H0[c], X);
                const uint2 mv = lds64(as + (uint32_t)c * TileAux<MODE>::kPlane);
                int rr[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int E = (int)byte_of(i < 4 ? ev.x : ev.y, i & 3);
                    // 0x4B000000 | M: the estimate's bias cancels in the difference
                    const int Mb = (int)__byte_perm(i < 4 ? mv.x : mv.y, 0x4B000000u, 0x7540u | (uint32_t)(i & 3));
                    const float2 p = ab[c * kNbin + E];
                    rr[i] = Mb - predict_bits(p.x, p.y, x_biased(X, i));
                }
                if (lc.inside) {
                    uint4 v;
                    v.x = __byte_perm((uint32_t)rr[0], (uint32_t)rr[1], 0x5410);
                    v.y = __byte_perm((uint32_t)rr[2], (uint32_t)rr[3], 0x5410);
                    v.z = __byte_perm((uint32_t)rr[4], (uint32_t)rr[5], 0x5410);
                    v.w = __byte_perm((uint32_t)rr[6], (uint32_t)rr[7], 0x5410);
                    *reinterpret_cast<uint4*>(A.r3_out + c * n + pix) = v;
                    if (hist) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) atomicAdd(&hist[c * kNres + rr[i] + 255], 1u);
                    }
                }
            }
            C.release_s(lane);
            C.release_a(lane);
        }
    }
}

// k_rows_tile<kResidual>: R = M - M* and histograms.
template <TmaMode MODE, bool kGf>
__global__ void __launch_bounds__(kTileThreads, TileAux<MODE>::kCtas) k_rows_tile(const __grid_constant__ TileArgs A) {
    extern __shared__ __align__(128) char dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TileSmem<MODE> L = tile_smem<MODE>(dyn);
    char* extra = dyn + (L.extra - smem_addr(dyn));
    float2* ab = reinterpret_cast<float2*>(extra);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ab + 3 * kNbin);
    tile_init_barriers(L);
    __syncthreads();

    if (warp == kTileWarps) {
        if (lane == 0) tile_produce(L, A);
        return;
    }
    // the consumers fetch the parameters while the first copies are in flight
    load_params_ab(A.params, ab, kTileWarps * 32);
    if (MODE == TmaMode::kResidual && A.hist)
        for (int i = threadIdx.x; i < 3 * kNres; i += kTileWarps * 32) hist[i] = 0u;
    consumers_sync();
    rows_consume<MODE, kGf>(L, A, ab, MODE == TmaMode::kResidual && A.hist ? hist : nullptr, warp, lane);
    if (MODE == TmaMode::kResidual && A.hist) {
        consumers_sync();
        for (int i = threadIdx.x; i < 3 * kNres; i += kTileWarps * 32)
            if (hist[i]) atomicAdd(A.hist + i, hist[i]);
    }
}


// ---------------------------------------------------------------- batch form on the row pipeline
//
// The same rings and consumers over many images: the rows of every image's
// 2048-column strips, image after image (row_prefix), are split into one
// contiguous range per CTA, so a CTA's tasks may belong to several images.
// Every plane of image i has the row pitch p_i (w_i rounded up to 16), so each
// row starts 16-byte aligned and the producer copies whole rows rounded up to
// 16 bytes.  A lane whose 8 columns cross the image's right edge (k < 8 valid
// pixels) replicates its last valid S byte into byte k before filtering and
// stores or adds only its k pixels.  At a change of image the consumer warps
// meet at a barrier to flush the CTA's shared bins or histograms to that
// image and reload the parameters; a warp whose wait gave up keeps walking
// the same task sequence (no waits, no work) so that every warp reaches every
// such barrier.

struct TileBatchArgs {
    BatchDev B;
    const uint8_t* s3b;          // S planes of the batch
    const uint8_t* auxb;         // M planes (fit, residual) or R planes (decode), as bytes
    const uint8_t* eb;           // E plane
    int64_t total_rows;          // rows of 2048-column strips over all images
    int max_spins;
    const slrme_params* params;  // [n_images]
    int16_t* r3b;                // residual planes (residual)
    uint32_t* hist;              // [n_images][3][511] (residual; may be null)
    uint32_t* outb;              // decoded words (decode)
    // one image described inline (B.img and B.row_prefix null): the
    // single-image decoder runs these kernels on its dense planes
    BatchImage one;
    int64_t one_rows;
};

__device__ __forceinline__ BatchImage batch_img(const TileBatchArgs& A, int i) {
    return A.B.img ? A.B.img[i] : A.one;
}
__device__ __forceinline__ int64_t batch_prefix(const TileBatchArgs& A, int i) {
    return A.B.row_prefix ? A.B.row_prefix[i] : (i == 0 ? 0 : A.one_rows);
}

// A CTA's range of global rows and its current task and image.
struct BatchRange {
    int64_t start;               // the CTA's first global row; the counters below are relative to it
    int r, end;
    int base, limit;             // rows of the current image: [base, limit)
    int img;
    const uint8_t* s3;
    const uint8_t* aux;
    const uint8_t* e;
    int64_t px;                  // first element of the image in the word planes
    int h, w, p, gf;
    int y0, rows, xs;
    __device__ __forceinline__ void set(const TileBatchArgs& A, int i, uint32_t elem) {
        img = i;
        // both within one image's rows of the CTA's range, so they fit 32 bits
        base = (int)(batch_prefix(A, i) - start);
        limit = (int)(batch_prefix(A, i + 1) - start);
        const BatchImage im = batch_img(A, i);
        h = im.h;
        w = im.w;
        p = im.pitch;
        gf = im.gf_on;
        px = im.px;
        s3 = A.s3b + 3 * im.px;
        aux = A.auxb + 3 * im.px * (int64_t)elem;
        e = A.eb + im.px;
    }
    __device__ __forceinline__ bool next(const TileBatchArgs& A, uint32_t elem) {
        if (r >= end) return false;
        if (r >= limit) {   // the next image with rows (images without rows have base == limit)
            int i = img;
            do {
                ++i;
            } while (batch_prefix(A, i + 1) - start <= (int64_t)r);
            set(A, i, elem);
        }
        const int local = r - base;
        const int c = local / h;
        y0 = local - c * h;
        rows = min(min(end - r, h - y0), kTaskRows);
        xs = c * kTileCols;
        r += rows;
        return true;
    }
};

__device__ __forceinline__ BatchRange batch_range(const TileBatchArgs& A, uint32_t elem) {
    const int64_t G = gridDim.x, b = blockIdx.x;
    BatchRange T;
    T.start = b * A.total_rows / G;
    T.r = 0;
    T.end = (int)((b + 1) * A.total_rows / G - T.start);
    T.img = -1;
    T.base = T.limit = 0;
    if (T.r < T.end) T.set(A, A.B.row_prefix ? batch_image_of(A.B.row_prefix, A.B.n, T.start) : 0, elem);
    return T;
}

// Per-lane geometry of a batch task: as LaneCols, plus the lane's valid
// pixels k and the byte selectors that copy byte k - 1 into byte k.
struct LaneColsB {
    int x0, own, offl, offr, k;
    uint32_t sel_lo, sel_hi;
    bool inside, full;
    __device__ __forceinline__ LaneColsB(int xs, int w, int warp, int lane) {
        x0 = xs + kStripCols * warp + 8 * lane;
        own = 16 + kStripCols * warp + 8 * lane;
        k = min(max(w - x0, 0), 8);
        inside = k > 0;
        full = k == 8;
        offl = x0 == 0 ? own : own - 1;
        offr = full && x0 + 8 < w ? own + 8 : own + max(k - 1, 0);
        // result byte j takes source byte j, except byte k (1 <= k <= 7), which takes k - 1
        const uint32_t id = 0x76543210u;
        const uint32_t sel = (k >= 1 && k <= 7) ? ((id & ~(0xFu << (4 * k))) | ((uint32_t)(k - 1) << (4 * k))) : id;
        sel_lo = sel & 0xFFFFu;
        sel_hi = sel >> 16;
    }
};

// x pairs of one S row of channel c for a batch lane (restoration per image).
__device__ __forceinline__ void s_row_pairs_b(uint32_t slot, int c, const LaneColsB& lc, bool gf, uint32_t (&H)[4]) {
    const uint32_t row = slot + (uint32_t)c * kTileSW;
    const uint2 v = lds64(row + lc.own);
    const uint32_t lo = __byte_perm(v.x, v.y, lc.sel_lo), hi = __byte_perm(v.x, v.y, lc.sel_hi);
    if (gf) {
        uint32_t l, r;
        asm volatile("ld.shared.u8 %0, [%1];" : "=r"(l) : "r"(row + lc.offl));
        asm volatile("ld.shared.u8 %0, [%1];" : "=r"(r) : "r"(row + lc.offr));
        hfilter(lo, hi, l, r, H);
    } else {
        H[0] = __byte_perm(lo, 0, 0x4140);
        H[1] = __byte_perm(lo, 0, 0x4342);
        H[2] = __byte_perm(hi, 0, 0x4140);
        H[3] = __byte_perm(hi, 0, 0x4342);
    }
}

__device__ __forceinline__ void window_x_b(uint32_t sn, int c, const LaneColsB& lc, bool gf, uint32_t (&Hm)[4],
                                           uint32_t (&H0)[4], uint32_t (&X)[4]) {
    uint32_t Hn[4];
    s_row_pairs_b(sn, c, lc, gf, Hn);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        X[k] = gf ? Hm[k] + 2u * H0[k] + Hn[k] : H0[k] << 4;
        Hm[k] = H0[k];
        H0[k] = Hn[k];
    }
}

// The batch producer: as tile_produce, over the images of the CTA's range,
// with each image's planes, pitch and width (copies rounded up to 16 bytes,
// which stay inside the pitched row).
template <TmaMode MODE>
__device__ __noinline__ void tile_produce_batch(const TileSmem<MODE>& L, const TileBatchArgs& A) {
    constexpr int KS = TileSmem<MODE>::KS, KA = TileSmem<MODE>::KA;
    constexpr uint32_t kEl = TileAux<MODE>::kElem;
    BatchRange P = batch_range(A, kEl);
    uint32_t si = 0, ai = 0;
    RingPos<KS> sp{0u};
    RingPos<KA> ap{0u};
    bool ok = true;
    while (ok && P.next(A, kEl)) {
        const int64_t n = (int64_t)P.h * P.p;
        const int xa = max(P.xs - 16, 0), xb = min(P.xs + kTileCols + 16, P.w);
        const uint32_t s_bytes = (uint32_t)(((xb + 15) & ~15) - xa), s_off = (uint32_t)(xa - (P.xs - 16));
        const uint32_t cols = (uint32_t)(((min(P.xs + kTileCols, P.w) - P.xs) + 15) & ~15);
        for (int k = 0; k < P.rows + 2 && ok; ++k) {
            {
                if (si >= (uint32_t)KS) ok = mbar_wait(L.sempty(sp.slot()), sp.phase() ^ 1u, &g_slrme_status, A.max_spins);
                if (!ok) break;
                const int ys = min(max(P.y0 - 1 + k, 0), P.h - 1);
                const uint32_t dst = L.sslot_at(sp.slot()) + s_off, bar = L.sfull(sp.slot());
                const uint8_t* src = P.s3 + (int64_t)ys * P.p + xa;
                fence_async_shared();
                mbar_arrive_expect_tx(bar, 3u * s_bytes);
#pragma unroll
                for (int c = 0; c < 3; ++c) tma_load_1d(dst + (uint32_t)c * kTileSW, src + c * n, s_bytes, bar);
                ++si;
                sp.advance();
            }
            if (k >= 2) {
                if (ai >= (uint32_t)KA) ok = mbar_wait(L.aempty(ap.slot()), ap.phase() ^ 1u, &g_slrme_status, A.max_spins);
                if (!ok) break;
                const int64_t row = (int64_t)(P.y0 + k - 2) * P.p + P.xs;
                const uint32_t dst = L.aslot_at(ap.slot()), bar = L.afull(ap.slot());
                fence_async_shared();
                mbar_arrive_expect_tx(bar, (3u * kEl + 1u) * cols);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    tma_load_1d(dst + (uint32_t)c * TileAux<MODE>::kPlane, P.aux + (c * n + row) * kEl, kEl * cols,
                                bar);
                tma_load_1d(dst + TileAux<MODE>::kE, P.e + row, cols, bar);
                ++ai;
                ap.advance();
            }
        }
    }
    const int spins = ok ? A.max_spins : (1 << 10);
    for (uint32_t k = si > (uint32_t)KS ? si - KS : 0; k < si; ++k)
        mbar_wait(L.sfull(k % KS), (k / KS) & 1u, &g_slrme_status, spins);
    for (uint32_t k = ai > (uint32_t)KA ? ai - KA : 0; k < ai; ++k)
        mbar_wait(L.afull(k % KA), (k / KA) & 1u, &g_slrme_status, spins);
}

// Adds the CTA's shared bins to image `img`'s sums and clears them (consumer
// threads; the caller brackets this with consumer barriers).
__device__ __forceinline__ void bins_flush_consumers(SmemBins& bins, unsigned long long* __restrict__ g, bool add) {
    for (int i = threadIdx.x; i < kNbin * kNsum; i += kTileWarps * 32) {
        const unsigned long long v = ((unsigned long long)bins.hi[i] << 12) + bins.lo[i];
        if (add && v) atomicAdd(g + i, v);
        bins.lo[i] = bins.hi[i] = 0u;
    }
}

// The fit over the batch.  The bins hold one image's sums of at most 256 rows
// of 2048 pixels (2^19 pixels, the bins' bound) between flushes.
// kGfMode: 0 every image without restoration, 1 every image with it, 2
// mixed (the flag read per image).
template <int kGfMode>
__device__ __forceinline__ void fit_consume_batch(const TileSmem<TmaMode::kFit>& L, const TileBatchArgs& A,
                                                  SmemBins& bins, uint32_t* queue, int* gave_up, int warp, int lane) {
    TileConsumer<TmaMode::kFit> C{L, A.max_spins, {0u}, {0u}};
    FitQueues fq;
    fq.R = queue + warp * (kRunQ * kRunStride + kSegQ * kQueueStride);
    fq.Q = fq.R + kRunQ * kRunStride;
    fq.nr = fq.nq = 0;
    Run2 all, odd;
    BatchRange T = batch_range(A, 1u);
    bool ok = true;
    int cur = -1, since = 0;
    auto flush = [&]() {
        if (ok) {
            drain_runs(fq, bins, lane);
            drain_segs(fq, bins, lane);
        }
        consumers_sync();
        bins_flush_consumers(bins, A.B.sums + (int64_t)cur * kNbin * kNsum, *gave_up == 0);
        consumers_sync();
    };
    while (T.next(A, 1u)) {
        if (T.img != cur || since + T.rows > kTaskRows) {
            if (cur >= 0) flush();
            cur = T.img;
            since = 0;
        }
        since += T.rows;
        if (!ok) continue;   // after a timeout: walk the tasks (and their barriers) without work
        const LaneColsB lc(T.xs, T.w, warp, lane);
        const bool gf = kGfMode == 2 ? T.gf != 0 : kGfMode == 1;
        run2_reset(all, -1);
        run2_reset(odd, -1);
        uint32_t Hm[3][4], H0[3][4];
        ok = C.wait_s();
        if (ok) {
#pragma unroll
            for (int c = 0; c < 3; ++c) s_row_pairs_b(C.s_addr(), c, lc, gf, Hm[c]);
            C.release_s(lane);
            ok = C.wait_s();
        }
        if (ok) {
#pragma unroll
            for (int c = 0; c < 3; ++c) s_row_pairs_b(C.s_addr(), c, lc, gf, H0[c]);
            C.release_s(lane);
        }
        for (int j = 0; j < T.rows && ok; ++j) {
            ok = C.wait_s() && C.wait_a();
            if (!ok) break;
            const uint32_t sn = C.s_addr();
            const uint32_t as = C.a_addr() + kStripCols * warp + 8 * lane;
            const uint2 ev = lds64(as + TileAux<TmaMode::kFit>::kE);
            const uint32_t elo = ev.x, ehi = ev.y;
            const uint32_t E1 = elo & 255u;
            const bool uni = elo == ehi && elo == E1 * 0x01010101u;
            if (__all_sync(0xffffffffu, (uni && lc.full) || !lc.inside)) {
                // fast path: every segment of the warp is whole and in one region
                const bool isodd = (E1 & 1u) != 0u;
                runs_rekey(fq, all, odd, lc.inside && !isodd, (int)E1, lc.inside && isodd, (int)E1, bins, lane);
                const uint32_t mo = lc.inside && isodd ? 0xFFFFFFFFu : 0u;
                const uint32_t nadd = lc.inside ? 8u : 0u;
                all.n += nadd;
                odd.n += nadd & mo;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    uint32_t X[4];
                    window_x_b(sn, c, lc, gf, Hm[c], H0[c], X);
                    const uint2 mv = lds64(as + (uint32_t)c * TileAux<TmaMode::kFit>::kPlane);
                    if (lc.inside) {
                        uint32_t sx = 0u, sy = 0u, sxy = 0u, sxl = 0u, sxh = 0u;
                        seg_accum5(X, mv.x, mv.y, sx, sy, sxy, sxl, sxh);
                        all.sx[c] += sx;
                        all.sy[c] += sy;
                        all.sxy[c] += sxy;
                        all.sxl[c] += sxl;
                        all.sxh[c] += sxh;
                        odd.sx[c] += sx & mo;
                        odd.sy[c] += sy & mo;
                        odd.sxy[c] += sxy & mo;
                        odd.sxl[c] += sxl & mo;
                        odd.sxh[c] += sxh & mo;
                    }
                }
                C.release_s(lane);
                C.release_a(lane);
                continue;
            }
            const uint32_t olo = (elo & 0x01010101u) * 0xFFu, ohi = (ehi & 0x01010101u) * 0xFFu;
            uint32_t eo = (elo & olo) | (ehi & ohi), ee = (elo & ~olo) | (ehi & ~ohi);
            eo |= eo >> 16;
            ee |= ee >> 16;
            const uint32_t Eo = (eo | (eo >> 8)) & 255u, Ee = (ee | (ee >> 8)) & 255u;
            const uint32_t Eo4 = Eo * 0x01010101u, Ee4 = Ee * 0x01010101u;
            const bool two = ((((elo ^ Eo4) & olo) | ((ehi ^ Eo4) & ohi) | ((elo ^ Ee4) & ~olo) |
                               ((ehi ^ Ee4) & ~ohi)) == 0u);
            // lanes cut by the image's right edge go to the per-pixel queue
            const bool slow = lc.inside && (!two || !lc.full);
            const bool take = lc.inside && two && lc.full;
            const uint32_t po_n = take ? (uint32_t)(__popc(olo) + __popc(ohi)) >> 3 : 0u;
            runs_rekey(fq, all, odd, take && po_n != 8u, (int)Ee, po_n != 0u, (int)Eo, bins, lane);
            const unsigned want = __ballot_sync(0xffffffffu, slow);
            uint32_t qe = 0u;
            if (want) {
                if (fq.nq + __popc(want) > kSegQ) drain_segs(fq, bins, lane);
                qe = (uint32_t)(fq.nq + __popc(want & ((1u << lane) - 1u))) * kQueueStride;
            }
            uint32_t k16[4];
            mask16(olo, ohi, k16);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                uint32_t X[4];
                window_x_b(sn, c, lc, gf, Hm[c], H0[c], X);
                const uint2 mv = lds64(as + (uint32_t)c * TileAux<TmaMode::kFit>::kPlane);
                if (take) {
                    uint32_t xo[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) xo[k] = X[k] & k16[k];
                    seg_accum(xo, mv.x & olo, mv.y & ohi, odd, c);
                    seg_accum(X, mv.x, mv.y, all, c);
                }
                if (want) {
                    if (slow) {
                        uint32_t* q = fq.Q + qe;
                        q[2 + c] = mv.x;
                        q[5 + c] = mv.y;
#pragma unroll
                        for (int k = 0; k < 4; ++k) q[8 + 4 * c + k] = X[k];
                    }
                }
            }
            odd.n += po_n;
            all.n += take ? 8u : 0u;
            if (want) {
                if (slow) {
                    uint32_t* q = fq.Q + qe;
                    q[0] = elo;
                    q[1] = ehi;
                    q[20] = (uint32_t)lc.k;
                }
                __syncwarp();
                fq.nq += __popc(want);
            }
            C.release_s(lane);
            C.release_a(lane);
        }
        if (!ok) {
            if (lane == 0) atomicOr(gave_up, 1);
            continue;
        }
        push_run<true>(fq, all.E >= 0 && all.n != odd.n, all, odd, bins, lane);
        push_run<false>(fq, odd.E >= 0 && odd.n != 0u, all, odd, bins, lane);
    }
    if (cur >= 0) flush();
}

template <int kGfMode>
__global__ void __launch_bounds__(kTileThreads, TileAux<TmaMode::kFit>::kCtas) k_fit_tile_batch(const __grid_constant__ TileBatchArgs A) {
    extern __shared__ __align__(128) char dyn[];
    __shared__ int gave_up;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TileSmem<TmaMode::kFit> L = tile_smem<TmaMode::kFit>(dyn);
    char* extra = dyn + (L.extra - smem_addr(dyn));
    SmemBins& bins = *reinterpret_cast<SmemBins*>(extra);
    uint32_t* queue = reinterpret_cast<uint32_t*>(extra + sizeof(SmemBins));
    tile_init_barriers(L);
    if (threadIdx.x == 0) gave_up = 0;
    __syncthreads();
    if (warp == kTileWarps) {
        if (lane == 0) tile_produce_batch(L, A);
        return;
    }
    for (int i = threadIdx.x; i < (int)(sizeof(SmemBins) / 16); i += kTileWarps * 32)
        reinterpret_cast<uint4*>(extra)[i] = make_uint4(0u, 0u, 0u, 0u);
    consumers_sync();
    fit_consume_batch<kGfMode>(L, A, bins, queue, &gave_up, warp, lane);
}

// Residual / decoder over the batch: the parameters (and, for the residual,
// the histograms) of the current image in shared memory, switched at image
// changes behind consumer barriers.
template <TmaMode MODE, int kGfMode>
__device__ __forceinline__ void rows_consume_batch(const TileSmem<MODE>& L, const TileBatchArgs& A, float2* ab,
                                                   uint32_t* hist, int warp, int lane) {
    constexpr uint32_t kEl = TileAux<MODE>::kElem;
    TileConsumer<MODE> C{L, A.max_spins, {0u}, {0u}};
    BatchRange T = batch_range(A, kEl);
    bool ok = true;
    int cur = -1;
    const bool with_hist = MODE == TmaMode::kResidual && A.hist != nullptr;
    while (T.next(A, kEl)) {
        if (T.img != cur) {
            consumers_sync();
            if (with_hist && cur >= 0)
                for (int i = threadIdx.x; i < 3 * kNres; i += kTileWarps * 32) {
                    if (hist[i]) atomicAdd(A.hist + (int64_t)cur * 3 * kNres + i, hist[i]);
                    hist[i] = 0u;
                }
            load_params_ab(A.params + T.img, ab, kTileWarps * 32);
            consumers_sync();
            cur = T.img;
        }
        if (!ok) continue;   // after a timeout: walk the tasks (and their barriers) without work
        const LaneColsB lc(T.xs, T.w, warp, lane);
        const bool gf = kGfMode == 2 ? T.gf != 0 : kGfMode == 1;
        const int64_t n = (int64_t)T.h * T.p;
        uint32_t Hm[3][4], H0[3][4];
        ok = C.wait_s();
        if (ok) {
#pragma unroll
            for (int c = 0; c < 3; ++c) s_row_pairs_b(C.s_addr(), c, lc, gf, Hm[c]);
            C.release_s(lane);
            ok = C.wait_s();
        }
        if (ok) {
#pragma unroll
            for (int c = 0; c < 3; ++c) s_row_pairs_b(C.s_addr(), c, lc, gf, H0[c]);
            C.release_s(lane);
        }
        for (int j = 0; j < T.rows && ok; ++j) {
            ok = C.wait_s() && C.wait_a();
            if (!ok) break;
            const uint32_t sn = C.s_addr();
            const uint32_t as = C.a_addr() + kStripCols * warp + 8 * lane;
            const int64_t pix = (int64_t)(T.y0 + j) * T.p + lc.x0;
            const uint2 ev = lds64(as + TileAux<MODE>::kE);
            if constexpr (MODE == TmaMode::kResidual) {
                int16_t* r3 = A.r3b + 3 * T.px;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    uint32_t X[4];
                    window_x_b(sn, c, lc, gf, Hm[c], H0[c], X);
                    const uint2 mv = lds64(as + (uint32_t)c * TileAux<MODE>::kPlane);
                    int rr[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int E = (int)byte_of(i < 4 ? ev.x : ev.y, i & 3);
                        // 0x4B000000 | M: the estimate's bias cancels in the difference
                        const int Mb = (int)__byte_perm(i < 4 ? mv.x : mv.y, 0x4B000000u, 0x7540u | (uint32_t)(i & 3));
                        const float2 p = ab[c * kNbin + E];
                        rr[i] = Mb - predict_bits(p.x, p.y, x_biased(X, i));
                    }
                    if (lc.full) {
                        uint4 v;
                        v.x = __byte_perm((uint32_t)rr[0], (uint32_t)rr[1], 0x5410);
                        v.y = __byte_perm((uint32_t)rr[2], (uint32_t)rr[3], 0x5410);
                        v.z = __byte_perm((uint32_t)rr[4], (uint32_t)rr[5], 0x5410);
                        v.w = __byte_perm((uint32_t)rr[6], (uint32_t)rr[7], 0x5410);
                        *reinterpret_cast<uint4*>(r3 + c * n + pix) = v;
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if (i < lc.k) r3[c * n + pix + i] = (int16_t)rr[i];
                    }
                    if (with_hist) {
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if (i < lc.k) atomicAdd(&hist[c * kNres + rr[i] + 255], 1u);
                    }
                }
            } else {
                uint32_t word[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) word[i] = __byte_perm(i < 4 ? ev.x : ev.y, 0u, 0x0444 | ((i & 3) << 12));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    uint32_t X[4];
                    window_x_b(sn, c, lc, gf, Hm[c], H0[c], X);
                    const uint4 v = lds128(as + (uint32_t)c * TileAux<MODE>::kPlane + (kStripCols * warp + 8 * lane));
                    const uint32_t q4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int rv = (int)(int16_t)((q4[i >> 1] >> (16 * (i & 1))) & 0xFFFFu);
                        const int E = (int)(word[i] >> 24);
                        const float2 p = ab[c * kNbin + E];
                        // the low byte of R + (0x4B000000 + M*) is M
                        const int M = rv + predict_bits(p.x, p.y, x_biased(X, i));
                        word[i] |= ((uint32_t)M & 255u) << (8 * c);
                    }
                }
                uint32_t* out = A.outb + T.px + pix;
                if (lc.full) {
                    uint4* o4 = reinterpret_cast<uint4*>(out);
                    __stcs(o4, make_uint4(word[0], word[1], word[2], word[3]));   // streaming stores: the codec never reads its decoded words back
                    __stcs(o4 + 1, make_uint4(word[4], word[5], word[6], word[7]));
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (i < lc.k) out[i] = word[i];
                }
            }
            C.release_s(lane);
            C.release_a(lane);
        }
    }
    if (with_hist && cur >= 0) {
        consumers_sync();
        for (int i = threadIdx.x; i < 3 * kNres; i += kTileWarps * 32)
            if (hist[i]) atomicAdd(A.hist + (int64_t)cur * 3 * kNres + i, hist[i]);
    }
}

template <TmaMode MODE, int kGfMode>
__global__ void __launch_bounds__(kTileThreads, TileAux<MODE>::kCtas) k_rows_tile_batch(const __grid_constant__ TileBatchArgs A) {
    extern __shared__ __align__(128) char dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TileSmem<MODE> L = tile_smem<MODE>(dyn);
    char* extra = dyn + (L.extra - smem_addr(dyn));
    float2* ab = reinterpret_cast<float2*>(extra);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ab + 3 * kNbin);
    tile_init_barriers(L);
    __syncthreads();
    if (warp == kTileWarps) {
        if (lane == 0) tile_produce_batch(L, A);
        return;
    }
    if (MODE == TmaMode::kResidual && A.hist)
        for (int i = threadIdx.x; i < 3 * kNres; i += kTileWarps * 32) hist[i] = 0u;
    rows_consume_batch<MODE, kGfMode>(L, A, ab, hist, warp, lane);
}

bool tma_eligible(int w, std::initializer_list<const void*> ptrs) {
    if (w % 16 != 0) return false;
    for (const void* p : ptrs)
        if ((uintptr_t)p % 16 != 0) return false;
    return true;
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
                     const slrme_params* P, int16_t* r3_out, uint32_t* hist, cudaStream_t s) {
    static bool attr_gf[64], attr_plain[64];
    constexpr size_t smem = tile_rows_smem<MODE>();
    auto kernel = gf_on ? k_rows_tile<MODE, true> : k_rows_tile<MODE, false>;
    int st = tile_smem_attr(kernel, smem, gf_on ? attr_gf : attr_plain);
    if (st != SLRME_OK) return st;
    const int64_t total_rows = (int64_t)((w + kTileCols - 1) / kTileCols) * h;
    TileArgs A{s3, aux, e, h, w, gf_on, total_rows, kMaxSpins, P, r3_out, hist, nullptr};
    kernel<<<(unsigned)tile_grid(total_rows, 0, TileAux<MODE>::kCtas), kTileThreads, smem, s>>>(A);
    return cuda_status("residual_encode launch");
}

int launch_fit_tile(const uint8_t* s3, const uint8_t* m3, const uint8_t* e, int h, int w, int gf_on,
                    unsigned long long* bins, cudaStream_t s) {
    static bool attr_gf[64], attr_plain[64];
    auto kernel = gf_on ? k_fit_tile<true> : k_fit_tile<false>;
    int st = tile_smem_attr(kernel, kTileFitSmem, gf_on ? attr_gf : attr_plain);
    if (st != SLRME_OK) return st;
    const int64_t total_rows = (int64_t)((w + kTileCols - 1) / kTileCols) * h;
    // a CTA adds at most kTileFitMaxPixels pixels to its bins
    const int64_t rows_max = kTileFitMaxPixels / kTileCols;
    TileArgs A{s3, m3, e, h, w, gf_on, total_rows, kMaxSpins, nullptr, nullptr, nullptr, bins};
    kernel<<<(unsigned)tile_grid(total_rows, rows_max, TileAux<TmaMode::kFit>::kCtas), kTileThreads, kTileFitSmem,
             s>>>(A);
    return cuda_status("slr_fit launch");
}


struct StripLaunch {
    int rows;     // strip height
    int blocks;   // CTAs
};


// Grid of the batch row stages: per_sm CTAs per SM, at most one per 4 rows.
int64_t batch_tile_grid(int64_t tile_rows, int per_sm) {
    int64_t g = (tile_rows + 3) / 4;
    const int64_t cap = (int64_t)geometry().sms * per_sm;
    if (g > cap) g = cap;
    return g < 1 ? 1 : g;
}

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
        return launch_rows_tile<TmaMode::kResidual>(s3, m3, e, h, w, gf_on, params, r3, hist, s);
    const StripLaunch L = strip_launch(h, w, 2);
    k_residual<<<L.blocks, kThreads, 0, s>>>(s3, m3, e, h, w, gf_on, fast ? 1 : 0, L.rows, params, r3, hist);
    return cuda_status("residual_encode launch");
}

int launch_decode_one(const TileBatchArgs& A, int64_t rows, int gf_on, cudaStream_t s);

int launch_residual_decode(const uint8_t* s3, const uint8_t* e, const int16_t* r3, int h, int w, int gf_on,
                           const slrme_params* params, uint32_t* rgbe_out, cudaStream_t s) {
    const bool fast = (w % 8 == 0) && ((uintptr_t)s3 % 8 == 0) && ((uintptr_t)e % 8 == 0);
    if (tma_eligible(w, {s3, e, r3, rgbe_out})) {
        // the row-pipeline decoder of the batch form, on one image described inline
        const int64_t rows = (int64_t)((w + kTileCols - 1) / kTileCols) * h;
        TileBatchArgs A{};
        A.s3b = s3;
        A.auxb = reinterpret_cast<const uint8_t*>(r3);
        A.eb = e;
        A.total_rows = rows;
        A.max_spins = kMaxSpins;
        A.params = params;
        A.outb = rgbe_out;
        A.B.n = 1;
        A.one = BatchImage{h, w, 0, gf_on, 0, w, 0};
        A.one_rows = rows;
        return launch_decode_one(A, rows, gf_on, s);
    }
    const StripLaunch L = strip_launch(h, w, 2);
    k_decode<<<L.blocks, kThreads, 0, s>>>(s3, e, r3, h, w, gf_on, fast ? 1 : 0, L.rows, params, rgbe_out);
    return cuda_status("residual_decode launch");
}


// ---------------------------------------------------------------- batch launchers

namespace {

template <int kGfMode>
int fit_batch_kernel(const TileBatchArgs& A, int64_t tile_rows, cudaStream_t s) {
    static bool attr_set[64];
    int st = tile_smem_attr(k_fit_tile_batch<kGfMode>, kTileFitSmem, attr_set);
    if (st != SLRME_OK) return st;
    k_fit_tile_batch<kGfMode><<<(unsigned)batch_tile_grid(tile_rows, TileAux<TmaMode::kFit>::kCtas), kTileThreads,
                                kTileFitSmem, s>>>(A);
    return cuda_status("batch fit launch");
}

template <TmaMode MODE, int kGfMode>
int rows_batch_kernel(const TileBatchArgs& A, int64_t tile_rows, cudaStream_t s) {
    static bool attr_set[64];
    constexpr size_t smem = tile_rows_smem<MODE>();
    int st = tile_smem_attr(k_rows_tile_batch<MODE, kGfMode>, smem, attr_set);
    if (st != SLRME_OK) return st;
    k_rows_tile_batch<MODE, kGfMode><<<(unsigned)batch_tile_grid(tile_rows, TileAux<MODE>::kCtas), kTileThreads, smem,
                                       s>>>(A);
    return cuda_status(MODE == TmaMode::kResidual ? "batch residual launch" : "batch decode launch");
}

template <TmaMode MODE>
int rows_batch(const TileBatchArgs& A, int64_t tile_rows, int gf_mode, cudaStream_t s) {
    return gf_mode == 0 ? rows_batch_kernel<MODE, 0>(A, tile_rows, s)
                        : (gf_mode == 1 ? rows_batch_kernel<MODE, 1>(A, tile_rows, s)
                                        : rows_batch_kernel<MODE, 2>(A, tile_rows, s));
}

}  // namespace

// gf_mode: 0 no image of the batch uses the restoration, 1 every image does,
// 2 mixed (each image's flag read on the device).
int launch_fit_batch(const BatchDev& B, int64_t tile_rows, int gf_mode, const uint8_t* s3, const uint8_t* m3,
                     const uint8_t* e, slrme_params* params, cudaStream_t s) {
    if (cudaMemsetAsync(B.sums, 0, sizeof(unsigned long long) * kNbin * kNsum * (size_t)B.n, s) != cudaSuccess)
        return cuda_status("batch fit memset");
    if (tile_rows > 0) {
        TileBatchArgs A{B, s3, m3, e, tile_rows, kMaxSpins, nullptr, nullptr, nullptr, nullptr};
        const int st = gf_mode == 0 ? fit_batch_kernel<0>(A, tile_rows, s)
                                    : (gf_mode == 1 ? fit_batch_kernel<1>(A, tile_rows, s)
                                                    : fit_batch_kernel<2>(A, tile_rows, s));
        if (st != SLRME_OK) return st;
    }
    k_solve_batch<<<dim3(kSolveBlocks, B.n), 32, 0, s>>>(B.sums, params);
    return cuda_status("batch solve launch");
}

int launch_residual_batch(const BatchDev& B, int64_t tile_rows, int gf_mode, const uint8_t* s3, const uint8_t* m3,
                          const uint8_t* e, const slrme_params* params, int16_t* r3, uint32_t* hist, cudaStream_t s) {
    if (hist && cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 3 * kNres * (size_t)B.n, s) != cudaSuccess)
        return cuda_status("batch residual memset");
    if (tile_rows == 0) return SLRME_OK;
    TileBatchArgs A{B, s3, m3, e, tile_rows, kMaxSpins, params, r3, hist, nullptr};
    return rows_batch<TmaMode::kResidual>(A, tile_rows, gf_mode, s);
}

int launch_decode_one(const TileBatchArgs& A, int64_t rows, int gf_on, cudaStream_t s) {
    if (rows == 0) return SLRME_OK;
    return rows_batch<TmaMode::kDecode>(A, rows, gf_on ? 1 : 0, s);
}

int launch_decode_batch(const BatchDev& B, int64_t tile_rows, int gf_mode, const uint8_t* s3, const uint8_t* e,
                        const int16_t* r3, const slrme_params* params, uint32_t* out, cudaStream_t s) {
    if (tile_rows == 0) return SLRME_OK;
    TileBatchArgs A{B, s3, reinterpret_cast<const uint8_t*>(r3), e, tile_rows, kMaxSpins, params, nullptr, nullptr,
                    out};
    return rows_batch<TmaMode::kDecode>(A, tile_rows, gf_mode, s);
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

// A device symbol's address, cached per device ordinal together with the
// context it was looked up in: if the current context differs (the device's
// primary context was reset and created again), the address is looked up
// again, so a cached address never outlives its context.
struct SymbolCache {
    void* ctx[kMaxDevices];
    void* addr[kMaxDevices];
};
static SymbolCache g_scratch_cache, g_status_cache;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    });
    return fn;
}

// Device address of `symbol` on the current device, looked up with that
// device current (in host code a __device__ variable's name is only a
// host-side stand-in, so kernels must be given this address, never the name).
int symbol_address(const void* symbol, SymbolCache& cache, const char* what, void** out) {
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) {
        set_error("%s: cudaGetDevice: %s", what, cudaGetErrorString(err));
        return SLRME_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("%s: device ordinal %d outside 0..%d", what, dev, kMaxDevices - 1);
        return SLRME_EINVAL;
    }
    CtxGetCurrentFn get = ctx_get_current();
    CUcontext ctx = nullptr;
    if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!cache.addr[dev] || !ctx || cache.ctx[dev] != (void*)ctx) {
        // the lookup makes the device's primary context current if it is not yet
        void* p = nullptr;
        err = cudaGetSymbolAddress(&p, symbol);
        if (err != cudaSuccess || !p) {
            set_error("%s: cudaGetSymbolAddress: %s", what, cudaGetErrorString(err));
            return SLRME_ECUDA;
        }
        if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
        cache.addr[dev] = p;
        cache.ctx[dev] = (void*)ctx;
    }
    *out = cache.addr[dev];
    return SLRME_OK;
}

int scratch_address(void** out) { return symbol_address(g_fit_scratch, g_scratch_cache, "slr_fit_noalloc", out); }

}  // namespace

// Device address of the status word g_slrme_status on the current device,
// for kernels of other translation units.
int status_word_address(int** out) {
    void* p = nullptr;
    const int st = symbol_address(&g_slrme_status, g_status_cache, "status word", &p);
    *out = static_cast<int*>(p);
    return st;
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
