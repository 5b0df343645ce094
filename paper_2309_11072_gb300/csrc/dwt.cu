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
// Kernels: a row pass per level (one thread per output pair of a row) into
// a workspace holding each row as [low | high]; a column pass (one thread
// per output pair of a column, 32 adjacent columns per warp) that writes the
// three detail bands to their places and the low-low band to the next
// level's input (or, at the last level, to band 0), with per-band histograms
// of the values inside -255..255 kept in shared memory and added to the
// caller's array once per block.  The inverse runs the column pass, then
// the row pass, level by level from the deepest.  Arithmetic shifts of
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

// The high-pass value j of a row or column of n >= 2 samples read through `at`.
template <class F>
__device__ __forceinline__ int hp(const F& at, int n, int j) {
    const int l = at(2 * j);
    const int r = (2 * j + 2 <= n - 1) ? at(2 * j + 2) : l;
    return at(2 * j + 1) - ((l + r) >> 1);
}

// ---------------------------------------------------------------- forward
// Row pass: out row y = [s_0 .. s_{nL-1} | d_0 .. d_{nH-1}].
__global__ void k_dwt_rows_fwd(const int16_t* __restrict__ in, int64_t in_plane, int H, int W,
                               int16_t* __restrict__ out, int64_t out_plane) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nH = W / 2, nL = W - nH;
    if (i >= nL) return;
    const int16_t* x = in + blockIdx.z * in_plane + (int64_t)blockIdx.y * W;
    int16_t* o = out + blockIdx.z * out_plane + (int64_t)blockIdx.y * W;
    if (W == 1) {
        o[0] = x[0];
        return;
    }
    auto at = [&](int k) { return (int)__ldg(x + k); };
    const int dl = hp(at, W, i >= 1 ? i - 1 : 0);
    const int dr = hp(at, W, i < nH ? i : nH - 1);
    o[i] = (int16_t)(at(2 * i) + ((dl + dr + 2) >> 2));
    if (i < nH) o[nL + i] = (int16_t)dr;
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

constexpr int kColPairs = 8;   // pairs per thread in the column pass

__device__ __forceinline__ void hist_add(uint32_t* h, int v) {
    if (v >= -255 && v <= 255) atomicAdd(h + (v + 255), 1u);
}

// Column pass over the row-transformed array t (H x W): thread (x, pairs).
__global__ void __launch_bounds__(256) k_dwt_cols_fwd(const int16_t* __restrict__ t, int64_t t_plane, int H, int W,
                                                      ColDst D) {
    __shared__ uint32_t sh[4][kNres];   // local bands: 0 LL, 1 HL, 2 LH, 3 HH
    const bool want = D.hist != nullptr;
    if (want)
        for (int k = threadIdx.y * 32 + threadIdx.x; k < 4 * kNres; k += 256) (&sh[0][0])[k] = 0u;
    __syncthreads();
    const int p = blockIdx.z;
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int WL = (W + 1) / 2, WH = W / 2;
    const int nHc = H / 2, nLc = H - nHc;
    const int16_t* tp = t + p * t_plane;
    if (x < W) {
        auto at = [&](int k) { return (int)__ldg(tp + (int64_t)k * W + x); };
        const bool lowc = x < WL;
        for (int r = 0; r < kColPairs; ++r) {
            const int i = (blockIdx.y * kColPairs + r) * 8 + threadIdx.y;
            if (i >= nLc) break;
            int s, d = 0;
            if (H == 1) {
                s = at(0);
            } else {
                const int dl = hp(at, H, i >= 1 ? i - 1 : 0);
                const int dr = hp(at, H, i < nHc ? i : nHc - 1);
                s = at(2 * i) + ((dl + dr + 2) >> 2);
                d = dr;
            }
            if (lowc) {
                D.ll[p * D.ll_plane + (int64_t)i * WL + x] = (int16_t)s;
                if (want && D.b_ll >= 0) hist_add(sh[0], s);
                if (i < nHc) {
                    D.coef[p * D.coef_plane + D.off_lh + (int64_t)i * WL + x] = (int16_t)d;
                    if (want) hist_add(sh[2], d);
                }
            } else {
                D.coef[p * D.coef_plane + D.off_hl + (int64_t)i * WH + (x - WL)] = (int16_t)s;
                if (want) hist_add(sh[1], s);
                if (i < nHc) {
                    D.coef[p * D.coef_plane + D.off_hh + (int64_t)i * WH + (x - WL)] = (int16_t)d;
                    if (want) hist_add(sh[3], d);
                }
            }
        }
    }
    if (!want) return;
    __syncthreads();
    for (int k = threadIdx.y * 32 + threadIdx.x; k < 4 * kNres; k += 256) {
        const uint32_t v = (&sh[0][0])[k];
        if (!v) continue;
        const int lb = k / kNres, bin = k - lb * kNres;
        const int band = lb == 0 ? D.b_ll : D.b_hl + (lb - 1);
        atomicAdd(D.hist + ((int64_t)p * D.nb + band) * kNres + bin, v);
    }
}

// ---------------------------------------------------------------- inverse
struct ColSrc {
    const int16_t* ll;      // low-low input, row pitch WL
    int64_t ll_plane;
    const int16_t* coef;
    int64_t coef_plane;
    int64_t off_hl, off_lh, off_hh;
};

// Column inverse into t (H x W, rows as [low | high]).
__global__ void __launch_bounds__(256) k_dwt_cols_inv(ColSrc S, int H, int W, int16_t* __restrict__ t,
                                                      int64_t t_plane) {
    const int p = blockIdx.z;
    const int x = blockIdx.x * 32 + threadIdx.x;
    if (x >= W) return;
    const int WL = (W + 1) / 2, WH = W / 2;
    const int nHc = H / 2, nLc = H - nHc;
    const bool lowc = x < WL;
    const int16_t* lo = lowc ? S.ll + p * S.ll_plane + x : S.coef + p * S.coef_plane + S.off_hl + (x - WL);
    const int16_t* hi = lowc ? S.coef + p * S.coef_plane + S.off_lh + x : S.coef + p * S.coef_plane + S.off_hh + (x - WL);
    const int pitch = lowc ? WL : WH;
    int16_t* tp = t + p * t_plane + x;
    auto s_at = [&](int k) { return (int)__ldg(lo + (int64_t)k * pitch); };
    auto d_at = [&](int k) { return (int)__ldg(hi + (int64_t)k * pitch); };
    // even sample 2k from s_k and its two neighbouring high-pass values
    auto even = [&](int k) {
        const int dl = d_at(k >= 1 ? k - 1 : 0);
        const int dr = d_at(k < nHc ? k : nHc - 1);
        return s_at(k) - ((dl + dr + 2) >> 2);
    };
    for (int r = 0; r < kColPairs; ++r) {
        const int i = (blockIdx.y * kColPairs + r) * 8 + threadIdx.y;
        if (i >= nLc) break;
        if (H == 1) {
            tp[0] = (int16_t)s_at(0);
            continue;
        }
        const int e0 = even(i);
        tp[(int64_t)(2 * i) * W] = (int16_t)e0;
        if (i < nHc) {
            const int e1 = (2 * i + 2 <= H - 1) ? even(i + 1) : e0;
            tp[(int64_t)(2 * i + 1) * W] = (int16_t)(d_at(i) + ((e0 + e1) >> 1));
        }
    }
}

// Row inverse: row y of t = [s | d] back to samples.
__global__ void k_dwt_rows_inv(const int16_t* __restrict__ t, int64_t t_plane, int H, int W,
                               int16_t* __restrict__ out, int64_t out_plane) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nH = W / 2, nL = W - nH;
    if (i >= nL) return;
    const int16_t* row = t + blockIdx.z * t_plane + (int64_t)blockIdx.y * W;
    int16_t* o = out + blockIdx.z * out_plane + (int64_t)blockIdx.y * W;
    if (W == 1) {
        o[0] = row[0];
        return;
    }
    auto s_at = [&](int k) { return (int)__ldg(row + k); };
    auto d_at = [&](int k) { return (int)__ldg(row + nL + k); };
    auto even = [&](int k) {
        const int dl = d_at(k >= 1 ? k - 1 : 0);
        const int dr = d_at(k < nH ? k : nH - 1);
        return s_at(k) - ((dl + dr + 2) >> 2);
    };
    const int e0 = even(i);
    o[2 * i] = (int16_t)e0;
    if (i < nH) {
        const int e1 = (2 * i + 2 <= W - 1) ? even(i + 1) : e0;
        o[2 * i + 1] = (int16_t)(d_at(i) + ((e0 + e1) >> 1));
    }
}

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
            const dim3 grid((unsigned)((WL + 255) / 256), (unsigned)H, (unsigned)nplanes);
            k_dwt_rows_fwd<<<grid, 256, 0, s>>>(in, in_plane, H, W, tmp, plane);
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
        const dim3 grid((unsigned)((W + 31) / 32), (unsigned)((HL + 8 * kColPairs - 1) / (8 * kColPairs)),
                        (unsigned)nplanes);
        k_dwt_cols_fwd<<<grid, dim3(32, 8), 0, s>>>(tmp, plane, H, W, D);
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
        const dim3 cgrid((unsigned)((W + 31) / 32), (unsigned)((HL + 8 * kColPairs - 1) / (8 * kColPairs)),
                         (unsigned)nplanes);
        k_dwt_cols_inv<<<cgrid, dim3(32, 8), 0, s>>>(S, H, W, tmp, plane);
        int16_t* out = l == 1 ? planes : A;
        const int64_t out_plane = l == 1 ? plane : qplane;
        const dim3 rgrid((unsigned)((WL + 255) / 256), (unsigned)H, (unsigned)nplanes);
        k_dwt_rows_inv<<<rgrid, 256, 0, s>>>(tmp, plane, H, W, out, out_plane);
    }
    return cuda_status("dwt53_inverse launch");
}
