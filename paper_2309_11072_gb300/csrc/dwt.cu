// Reversible LeGall 5/3 wavelet over int16 planes (the transform of JPEG
// 2000's lossless mode, which codes the paper's enhancement layer, Sec. IV).
//
// 1-D step over n samples, nH = floor(n/2) high-pass and nL = ceil(n/2)
// low-pass values, whole-sample symmetric extension (x[n] = x[n-2],
// d[-1] = d[0], and for odd n d[nL-1] = d[nL-2]):
//   d[i] = x[2i+1] - floor((x[2i] + x[2i+2]) / 2)
//   s[i] = x[2i]   + floor((d[i-1] + d[i] + 2) / 4)
// (a single sample is its own low-pass value).  A 2-D level transforms the
// rows, then the columns; the next level transforms the low-low band.  Each
// plane's output is subband-major: LL_L, then HL, LH, HH from level L down
// to 1, each band row-major (HL: high-pass along the rows).
//
// Kernels: a row pass per level (a CTA per 2,048-pair row segment, staged in
// shared memory) into a workspace holding each row as [low | high]; a
// column pass (a thread walks 64 pairs of one column, 32 adjacent columns
// per warp) that writes the three detail bands to their places and the
// low-low band to the next level's input (or, at the last level, to band 0),
// with per-band histograms of the values inside -255..255 kept in shared
// memory (one copy per warp) and added to the caller's array once per block.
// The inverse runs the column pass, then the row pass, level by level from
// the deepest.  Arithmetic shifts of
// negative int are floors (two's complement, as nvcc compiles >>).
#include <stdint.h>

#include <algorithm>

#include "slrme_internal.cuh"

namespace slrme {
namespace {

constexpr int kMaxLevels = SLRME_DWT_MAX_LEVELS;
constexpr int kMaxBands = 1 + 3 * kMaxLevels;

struct Bands {
    int n;
    int32_t rows[kMaxBands], cols[kMaxBands];
    int64_t off[kMaxBands];   // first element of each band in a plane's output
};

void band_layout(int h, int w, int levels, Bands* B) {
    int hs[kMaxLevels + 1], ws[kMaxLevels + 1];
    hs[0] = h;
    ws[0] = w;
    for (int l = 1; l <= levels; ++l) {
        hs[l] = (hs[l - 1] + 1) / 2;
        ws[l] = (ws[l - 1] + 1) / 2;
    }
    int b = 0;
    B->rows[b] = hs[levels];
    B->cols[b] = ws[levels];
    ++b;
    for (int l = levels; l >= 1; --l) {
        const int H = hs[l - 1], W = ws[l - 1];
        const int HL = (H + 1) / 2, HH = H / 2, WL = (W + 1) / 2, WH = W / 2;
        B->rows[b] = HL; B->cols[b] = WH; ++b;   // HL
        B->rows[b] = HH; B->cols[b] = WL; ++b;   // LH
        B->rows[b] = HH; B->cols[b] = WH; ++b;   // HH
    }
    B->n = b;
    int64_t at = 0;
    for (int i = 0; i < b; ++i) {
        B->off[i] = at;
        at += (int64_t)B->rows[i] * B->cols[i];
    }
}

// ---------------------------------------------------------------- row passes
// A CTA takes kSeg pairs of one row (pairs i0 .. i0+kSeg-1): it stages the
// samples they need (2 i0 - 2 .. 2 i0 + 2 kSeg) in shared memory with
// coalesced loads, computes the high-pass values d_(i0-1) .. d_(i0+kSeg-1)
// once each, then the low-pass values.
constexpr int kRowThreads = 256;
constexpr int kSeg = 2048;

__global__ void __launch_bounds__(kRowThreads) k_dwt_rows_fwd(const int16_t* __restrict__ in, int64_t in_plane,
                                                              int H, int W, int16_t* __restrict__ out,
                                                              int64_t out_plane) {
    __shared__ int16_t xs[2 * kSeg + 3];
    __shared__ int16_t ds[kSeg + 1];
    const int nH = W / 2, nL = W - nH;
    const int i0 = blockIdx.x * kSeg;
    const int16_t* x = in + blockIdx.z * in_plane + (int64_t)blockIdx.y * W;
    int16_t* o = out + blockIdx.z * out_plane + (int64_t)blockIdx.y * W;
    if (W == 1) {
        if (threadIdx.x == 0) o[0] = x[0];
        return;
    }
    const int k0 = 2 * i0 - 2;                           // sample of xs[0]
    const int k1 = min(W, 2 * (i0 + kSeg) + 1);         // one past the last sample needed
    for (int k = max(k0, 0) + threadIdx.x; k < k1; k += kRowThreads) xs[k - k0] = x[k];
    __syncthreads();
    const int j0 = max(i0 - 1, 0), j1 = min(nH, i0 + kSeg);   // high-pass values to compute
    for (int j = j0 + threadIdx.x; j < j1; j += kRowThreads) {
        const int l = xs[2 * j - k0];
        const int r = (2 * j + 2 <= W - 1) ? xs[2 * j + 2 - k0] : l;
        const int d = xs[2 * j + 1 - k0] - ((l + r) >> 1);
        ds[j - (i0 - 1)] = (int16_t)d;
        if (j >= i0) o[nL + j] = (int16_t)d;
    }
    __syncthreads();
    const int iend = min(nL, i0 + kSeg);
    for (int i = i0 + threadIdx.x; i < iend; i += kRowThreads) {
        const int dl = ds[max(i - 1, 0) - (i0 - 1)];
        const int dr = ds[min(i, nH - 1) - (i0 - 1)];
        o[i] = (int16_t)(xs[2 * i - k0] + ((dl + dr + 2) >> 2));
    }
}

// Row inverse over the same segments: the CTA stages s_(i0) .. s_(i0+kSeg)
// and d_(i0-1) .. d_(i0+kSeg), computes the even samples 2 i0 .. 2 (i0+kSeg)
// once each, then the odd ones.
__global__ void __launch_bounds__(kRowThreads) k_dwt_rows_inv(const int16_t* __restrict__ t, int64_t t_plane, int H,
                                                              int W, int16_t* __restrict__ out, int64_t out_plane) {
    __shared__ int16_t ss[kSeg + 1];
    __shared__ int16_t dd[kSeg + 2];
    __shared__ int16_t es[kSeg + 1];
    const int nH = W / 2, nL = W - nH;
    const int i0 = blockIdx.x * kSeg;
    const int16_t* row = t + blockIdx.z * t_plane + (int64_t)blockIdx.y * W;
    int16_t* o = out + blockIdx.z * out_plane + (int64_t)blockIdx.y * W;
    if (W == 1) {
        if (threadIdx.x == 0) o[0] = row[0];
        return;
    }
    const int s1 = min(nL, i0 + kSeg + 1);
    for (int i = i0 + threadIdx.x; i < s1; i += kRowThreads) ss[i - i0] = row[i];
    const int dj0 = max(i0 - 1, 0), dj1 = min(nH, i0 + kSeg + 1);
    for (int j = dj0 + threadIdx.x; j < dj1; j += kRowThreads) dd[j - (i0 - 1)] = row[nL + j];
    __syncthreads();
    for (int i = i0 + threadIdx.x; i < s1; i += kRowThreads) {
        const int dl = dd[max(i - 1, 0) - (i0 - 1)];
        const int dr = dd[min(i, nH - 1) - (i0 - 1)];
        const int e = ss[i - i0] - ((dl + dr + 2) >> 2);
        es[i - i0] = (int16_t)e;
        if (i < i0 + kSeg) o[2 * i] = (int16_t)e;
    }
    __syncthreads();
    const int oend = min(nH, i0 + kSeg);
    for (int i = i0 + threadIdx.x; i < oend; i += kRowThreads) {
        const int e0 = es[i - i0];
        const int e1 = (2 * i + 2 <= W - 1) ? es[i + 1 - i0] : e0;
        o[2 * i + 1] = (int16_t)(dd[i - (i0 - 1)] + ((e0 + e1) >> 1));
    }
}

// ---------------------------------------------------------------- column passes
// A thread walks `run` pairs of one column (32 adjacent columns per warp, so
// every load and store of the warp is one contiguous 64-byte run), keeping
// the previous even sample and high-pass value in registers: two loads and
// one high-pass computation per pair.
// Pairs per thread: up to 32, fewer on short columns so that every column
// still has about two dozen walkers.
int col_run(int pairs) {
    int run = 32;
    while (run > 4 && pairs < 24 * run) run >>= 1;
    return run;
}

struct ColDst {
    int16_t* ll;            // low-low destination, row pitch WL
    int64_t ll_plane;
    int16_t* coef;          // the caller's subband-major output
    int64_t coef_plane;
    int64_t off_hl, off_lh, off_hh;
    uint32_t* hist;         // [plane][band][511] or null
    int nb;                 // bands per plane
    int b_ll, b_hl;         // band of the low-low output (-1: not a band yet), of HL (LH, HH follow)
};

// Each warp counts into its own copy of the four local histograms (band-major
// key = band * 511 + value + 255), so only lanes of one warp meet on a bin.
constexpr int kHistCopy = 4 * kNres;

__device__ __forceinline__ void hist_add(uint32_t* sh, int key) {
    if (key >= 0) atomicAdd(sh + key, 1u);
}

__global__ void __launch_bounds__(256) k_dwt_cols_fwd(const int16_t* __restrict__ t, int64_t t_plane, int H, int W,
                                                      int run, ColDst D) {
    extern __shared__ uint32_t hsm[];    // [8 warps][4 local bands: 0 LL, 1 HL, 2 LH, 3 HH][511]
    const bool want = D.hist != nullptr;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    if (want)
        for (int k = tid; k < 8 * kHistCopy; k += 256) hsm[k] = 0u;
    __syncthreads();
    uint32_t* sh = hsm + threadIdx.y * kHistCopy;
    const int p = blockIdx.z;
    const int xr = blockIdx.x * 32 + threadIdx.x;
    const bool live = xr < W;
    const int x = live ? xr : W - 1;                     // lanes past the edge shadow the last column
    const int WL = (W + 1) / 2, WH = W / 2;
    const int nHc = H / 2, nLc = H - nHc;
    const bool lowc = x < WL;
    const int16_t* col = t + p * t_plane + x;
    auto at = [&](int k) { return (int)__ldg(col + (int64_t)k * W); };
    int16_t* sdst = lowc ? D.ll + p * D.ll_plane + x : D.coef + p * D.coef_plane + D.off_hl + (x - WL);
    int16_t* ddst = lowc ? D.coef + p * D.coef_plane + D.off_lh + x : D.coef + p * D.coef_plane + D.off_hh + (x - WL);
    const int spitch = lowc ? WL : WH;
    const int sband = lowc ? (D.b_ll >= 0 ? 0 : -1) : 1;
    const int dband = lowc ? 2 : 3;
    const int i0 = (blockIdx.y * 8 + threadIdx.y) * run;
    const int i1 = min(nLc, i0 + run);
    if (i0 < i1) {
        if (H == 1) {
            const int s = at(0);
            if (live) sdst[0] = (int16_t)s;
            if (want) hist_add(sh, (live && sband >= 0 && s >= -255 && s <= 255) ? sband * kNres + s + 255 : -1);
        } else {
            // the high-pass value before the run (d_(-1) = d_0 at the top)
            int e = at(2 * i0);
            int dprev = 0;
            if (i0 >= 1) {
                const int l = at(2 * i0 - 2);
                dprev = at(2 * i0 - 1) - ((l + e) >> 1);
            }
            // blocks of 8 pairs: the block's 16 samples are loaded before any
            // arithmetic, so the walk waits for memory once per block
            constexpr int kB = 8;
            for (int ib = i0; ib < i1; ib += kB) {
                int xo[kB], xe[kB];
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int i = ib + u;
                    xo[u] = (i < i1 && i < nHc) ? at(2 * i + 1) : 0;
                    xe[u] = (i < i1 && 2 * i + 2 <= H - 1) ? at(2 * i + 2) : 0;
                }
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int i = ib + u;
                    if (i >= i1) break;
                    int d, r = e;
                    if (i < nHc) {
                        if (2 * i + 2 <= H - 1) r = xe[u];
                        d = xo[u] - ((e + r) >> 1);
                    } else {
                        d = dprev;                       // odd H: the last even sample mirrors d_(nH-1)
                    }
                    const int dl = i == 0 ? d : dprev;
                    const int s = e + ((dl + d + 2) >> 2);
                    if (live) {
                        sdst[(int64_t)i * spitch] = (int16_t)s;
                        if (i < nHc) ddst[(int64_t)i * spitch] = (int16_t)d;
                    }
                    if (want) {
                        hist_add(sh, (live && sband >= 0 && s >= -255 && s <= 255) ? sband * kNres + s + 255 : -1);
                        hist_add(sh, (live && i < nHc && d >= -255 && d <= 255) ? dband * kNres + d + 255 : -1);
                    }
                    e = r;
                    dprev = d;
                }
            }
        }
    }
    if (!want) return;
    __syncthreads();
    for (int k = tid; k < kHistCopy; k += 256) {
        uint32_t v = 0;
#pragma unroll
        for (int w8 = 0; w8 < 8; ++w8) v += hsm[w8 * kHistCopy + k];
        if (!v) continue;
        const int lb = k / kNres, bin = k - lb * kNres;
        const int band = lb == 0 ? D.b_ll : D.b_hl + (lb - 1);
        atomicAdd(D.hist + ((int64_t)p * D.nb + band) * kNres + bin, v);
    }
}

struct ColSrc {
    const int16_t* ll;      // low-low input, row pitch WL
    int64_t ll_plane;
    const int16_t* coef;
    int64_t coef_plane;
    int64_t off_hl, off_lh, off_hh;
};

// Column inverse into t (H x W, rows as [low | high]), walking `run` pairs:
// the even sample of pair i + 1 is computed once and serves both odd
// samples beside it.
__global__ void __launch_bounds__(256) k_dwt_cols_inv(ColSrc S, int H, int W, int run, int16_t* __restrict__ t,
                                                      int64_t t_plane) {
    const int p = blockIdx.z;
    const int x = blockIdx.x * 32 + threadIdx.x;
    if (x >= W) return;
    const int WL = (W + 1) / 2, WH = W / 2;
    const int nHc = H / 2, nLc = H - nHc;
    const int i0 = (blockIdx.y * 8 + threadIdx.y) * run;
    const int i1 = min(nLc, i0 + run);
    if (i0 >= i1) return;
    const bool lowc = x < WL;
    const int16_t* lo = lowc ? S.ll + p * S.ll_plane + x : S.coef + p * S.coef_plane + S.off_hl + (x - WL);
    const int16_t* hi = lowc ? S.coef + p * S.coef_plane + S.off_lh + x : S.coef + p * S.coef_plane + S.off_hh + (x - WL);
    const int pitch = lowc ? WL : WH;
    int16_t* tp = t + p * t_plane + x;
    auto s_at = [&](int k) { return (int)__ldg(lo + (int64_t)k * pitch); };
    auto d_at = [&](int k) { return (int)__ldg(hi + (int64_t)k * pitch); };
    if (H == 1) {
        tp[0] = (int16_t)s_at(0);
        return;
    }
    // even sample 2k from s_k and d_(k-1), d_k (mirrored at both ends)
    int dprev = d_at(i0 >= 1 ? i0 - 1 : 0);
    int dcur = d_at(i0 < nHc ? i0 : nHc - 1);
    int e = s_at(i0) - ((dprev + dcur + 2) >> 2);
    constexpr int kB = 8;
    for (int ib = i0; ib < i1; ib += kB) {
        int sn[kB], dn[kB];   // s_(i+1), d_(i+1) (mirrored) of the block's pairs, loaded first
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int i = ib + u;
            const bool more = i < i1 && i < nHc && 2 * i + 2 <= H - 1;
            sn[u] = more ? s_at(i + 1) : 0;
            dn[u] = more ? d_at(i + 1 < nHc ? i + 1 : nHc - 1) : 0;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int i = ib + u;
            if (i >= i1) break;
            tp[(int64_t)(2 * i) * W] = (int16_t)e;
            if (i < nHc) {
                int en = e;
                int dnext = dcur;
                if (2 * i + 2 <= H - 1) {
                    dnext = dn[u];
                    en = sn[u] - ((dcur + dnext + 2) >> 2);
                }
                tp[(int64_t)(2 * i + 1) * W] = (int16_t)(dcur + ((e + en) >> 1));
                e = en;
                dcur = dnext;
            }
        }
    }
}

constexpr size_t kColFwdSmem = 8 * kHistCopy * sizeof(uint32_t);   // 65,408 bytes
bool g_col_attr[64];

bool aligned2(const void* p) {
    return ((uintptr_t)p & 1u) == 0;
}

int check_args(const char* who, int nplanes, int h, int w, int levels) {
    if (nplanes < 1 || nplanes > 65535 || h < 0 || h > 65535 || w < 0 || (int64_t)h * w >= (int64_t(1) << 31) ||
        levels < 1 || levels > kMaxLevels) {
        set_error("%s: need 1 <= nplanes <= 65535, 0 <= h <= 65535, 0 <= w, h*w < 2^31 and 1 <= levels <= %d", who,
                  kMaxLevels);
        return SLRME_EINVAL;
    }
    return SLRME_OK;
}

}  // namespace
}  // namespace slrme

extern "C" int dwt53_bands(int h, int w, int levels, int32_t* dims) {
    using namespace slrme;
    if (!dims || h < 0 || w < 0 || levels < 1 || levels > kMaxLevels) {
        set_error("dwt53_bands: need dims, 0 <= h, w and 1 <= levels <= %d", kMaxLevels);
        return SLRME_EINVAL;
    }
    Bands B;
    band_layout(h, w, levels, &B);
    for (int b = 0; b < B.n; ++b) {
        dims[2 * b] = B.rows[b];
        dims[2 * b + 1] = B.cols[b];
    }
    return B.n;
}

extern "C" size_t dwt53_workspace_bytes(int nplanes, int h, int w) {
    if (nplanes < 1 || h < 0 || w < 0) return 0;
    const int64_t n = (int64_t)h * w, q = (int64_t)((h + 1) / 2) * ((w + 1) / 2);
    const size_t bytes = (size_t)nplanes * (size_t)(n + q) * sizeof(int16_t);
    return (bytes + 255) & ~(size_t)255;
}

extern "C" int dwt53_forward(const int16_t* planes, int nplanes, int h, int w, int levels, int16_t* coef,
                             uint32_t* hist, void* ws, slrme_stream_t stream) {
    using namespace slrme;
    int rc = check_args("dwt53_forward", nplanes, h, w, levels);
    if (rc) return rc;
    if (!planes || !coef || !ws || !aligned2(planes) || !aligned2(coef) || ((uintptr_t)ws & 255u) ||
        (hist && ((uintptr_t)hist & 3u))) {
        set_error("dwt53_forward: null or misaligned pointer (planes, coef 2; hist 4; ws 256 bytes)");
        return SLRME_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Bands B;
    band_layout(h, w, levels, &B);
    if (hist && cudaMemsetAsync(hist, 0, (size_t)nplanes * B.n * kNres * sizeof(uint32_t), s) != cudaSuccess)
        return cuda_status("dwt53_forward hist clear");
    if ((int64_t)h * w == 0) return SLRME_OK;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cuda_status("dwt53_forward device");
        if (!g_col_attr[dev]) {
            if (cudaFuncSetAttribute(k_dwt_cols_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kColFwdSmem) !=
                cudaSuccess)
                return cuda_status("dwt53_forward shared memory attribute");
            g_col_attr[dev] = true;
        }
    }
    const int64_t plane = (int64_t)h * w;
    const int64_t qplane = (int64_t)((h + 1) / 2) * ((w + 1) / 2);
    int16_t* tmp = (int16_t*)ws;
    int16_t* A = tmp + (int64_t)nplanes * plane;
    const int16_t* in = planes;
    int64_t in_plane = plane;
    int H = h, W = w;
    for (int l = 1; l <= levels; ++l) {
        const int WL = (W + 1) / 2, HL = (H + 1) / 2;
        {
            const dim3 grid((unsigned)((WL + kSeg - 1) / kSeg), (unsigned)H, (unsigned)nplanes);
            k_dwt_rows_fwd<<<grid, kRowThreads, 0, s>>>(in, in_plane, H, W, tmp, plane);
        }
        const int bHL = 1 + 3 * (levels - l);
        ColDst D;
        const bool last = l == levels;
        D.ll = last ? coef : A;
        D.ll_plane = last ? plane : qplane;
        D.coef = coef;
        D.coef_plane = plane;
        D.off_hl = B.off[bHL];
        D.off_lh = B.off[bHL + 1];
        D.off_hh = B.off[bHL + 2];
        D.hist = hist;
        D.nb = B.n;
        D.b_ll = last ? 0 : -1;
        D.b_hl = bHL;
        const int run = col_run(HL);
        const dim3 grid((unsigned)((W + 31) / 32), (unsigned)((HL + 8 * run - 1) / (8 * run)), (unsigned)nplanes);
        k_dwt_cols_fwd<<<grid, dim3(32, 8), hist ? kColFwdSmem : 0, s>>>(tmp, plane, H, W, run, D);
        in = A;
        in_plane = qplane;
        H = HL;
        W = WL;
    }
    return cuda_status("dwt53_forward launch");
}

extern "C" int dwt53_inverse(const int16_t* coef, int nplanes, int h, int w, int levels, int16_t* planes, void* ws,
                             slrme_stream_t stream) {
    using namespace slrme;
    int rc = check_args("dwt53_inverse", nplanes, h, w, levels);
    if (rc) return rc;
    if (!planes || !coef || !ws || !aligned2(planes) || !aligned2(coef) || ((uintptr_t)ws & 255u)) {
        set_error("dwt53_inverse: null or misaligned pointer (planes, coef 2; ws 256 bytes)");
        return SLRME_EINVAL;
    }
    if ((int64_t)h * w == 0) return SLRME_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Bands B;
    band_layout(h, w, levels, &B);
    const int64_t plane = (int64_t)h * w;
    const int64_t qplane = (int64_t)((h + 1) / 2) * ((w + 1) / 2);
    int16_t* tmp = (int16_t*)ws;
    int16_t* A = tmp + (int64_t)nplanes * plane;
    int hs[kMaxLevels + 1], wsz[kMaxLevels + 1];
    hs[0] = h;
    wsz[0] = w;
    for (int l = 1; l <= levels; ++l) {
        hs[l] = (hs[l - 1] + 1) / 2;
        wsz[l] = (wsz[l - 1] + 1) / 2;
    }
    for (int l = levels; l >= 1; --l) {
        const int H = hs[l - 1], W = wsz[l - 1];
        const int HL = (H + 1) / 2, WL = (W + 1) / 2;
        const int bHL = 1 + 3 * (levels - l);
        ColSrc S;
        S.ll = l == levels ? coef : A;
        S.ll_plane = l == levels ? plane : qplane;
        S.coef = coef;
        S.coef_plane = plane;
        S.off_hl = B.off[bHL];
        S.off_lh = B.off[bHL + 1];
        S.off_hh = B.off[bHL + 2];
        const int run = col_run(HL);
        const dim3 cgrid((unsigned)((W + 31) / 32), (unsigned)((HL + 8 * run - 1) / (8 * run)), (unsigned)nplanes);
        k_dwt_cols_inv<<<cgrid, dim3(32, 8), 0, s>>>(S, H, W, run, tmp, plane);
        int16_t* out = l == 1 ? planes : A;
        const int64_t out_plane = l == 1 ? plane : qplane;
        const dim3 rgrid((unsigned)((WL + kSeg - 1) / kSeg), (unsigned)H, (unsigned)nplanes);
        k_dwt_rows_inv<<<rgrid, kRowThreads, 0, s>>>(tmp, plane, H, W, out, out_plane);
    }
    return cuda_status("dwt53_inverse launch");
}
