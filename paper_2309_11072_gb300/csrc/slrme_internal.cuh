// Internal declarations shared by the library's translation units.
// Device helpers, constant tables passed to kernels by value, and the
// launcher functions behind the C ABI in include/slrme.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/slrme.h"

namespace slrme {

constexpr int kNbin = SLRME_NBIN;
constexpr int kNsum = SLRME_NSUM;
constexpr int kNres = SLRME_NRES;

// ---------------------------------------------------------------- tables
// The constant tables (log2 LUT, gamma thresholds, key scales) are literals
// in tables.inc, included by each translation unit that reads them.

// Quantiser for one quality: steps q[v*8+u] and the reciprocal multipliers
// qm = ceil(2^24 / q), so floor(n / q) == umulhi(n << 8, qm) for 0 <= n < 4096.
struct QuantTable {
    int32_t q[64];
    uint32_t qm[64];
};

bool quant_table(int quality, QuantTable* out);          // T.81 Table K.1 (luminance), IJG-scaled
bool quant_table_chroma(int quality, QuantTable* out);   // T.81 Table K.2 (chrominance), IJG-scaled

// ---------------------------------------------------------------- batch plan (device side)
// One image of a batch.  Its planes start at pixel px of the batch planes:
// words rgbe[px..], mantissas m3[3 px + c h w ..], exponents e[px..], and so on.
struct BatchImage {
    int32_t h, w;
    int32_t quality;
    int32_t gf_on;
    int64_t px;
    int32_t pitch;      // row pitch of every plane (w rounded up to 16)
    int32_t reserved;
};

// Device views of a plan's workspace.  Prefix arrays have n + 1 entries:
// task k of a stage belongs to image i when prefix[i] <= k < prefix[i + 1].
struct BatchDev {
    const BatchImage* img;
    const QuantTable* quant;         // per image
    const int64_t* split_prefix;     // chunks of 4096 words
    const int64_t* base_prefix;      // CTA tasks of 8 band tasks (8 rows x 32 columns each)
    const int64_t* row_prefix;       // rows of 2048-column strips (strips x h per image)
    int64_t* lum_stats;              // [n][2]
    unsigned long long* sums;        // [n][256 * 13]
    int n;
};

// Image of task k by binary search over a prefix array (n is small).
__device__ __forceinline__ int batch_image_of(const int64_t* prefix, int n, int64_t k) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

constexpr int kSplitChunk = 4096;   // words per split task
constexpr int kTileColsBatch = 2048;  // columns per strip of the row stages

int launch_split_batch(const BatchDev& B, int64_t chunks, int ctas_per_sm, const uint32_t* rgbe, uint8_t* m3,
                       uint8_t* e, cudaStream_t s);
int launch_base_batch(const BatchDev& B, int64_t cta_tasks, int ctas_per_sm, const uint8_t* m3, const uint8_t* e,
                      uint8_t* s3, cudaStream_t s);
// gf_mode: 0 no image uses the restoration, 1 every image does, 2 mixed.
int launch_fit_batch(const BatchDev& B, int64_t tile_rows, int gf_mode, const uint8_t* s3, const uint8_t* m3,
                     const uint8_t* e, slrme_params* params, cudaStream_t s);
int launch_residual_batch(const BatchDev& B, int64_t tile_rows, int gf_mode, const uint8_t* s3, const uint8_t* m3,
                          const uint8_t* e, const slrme_params* params, int16_t* r3, uint32_t* hist, cudaStream_t s);
int launch_decode_batch(const BatchDev& B, int64_t tile_rows, int gf_mode, const uint8_t* s3, const uint8_t* e,
                        const int16_t* r3, const slrme_params* params, uint32_t* out, cudaStream_t s);

// ---------------------------------------------------------------- launch geometry
struct Geometry {
    int sms;
};
Geometry geometry();

// ---------------------------------------------------------------- error reporting
void set_error(const char* fmt, ...);
int cuda_status(const char* what);   // SLRME_OK or SLRME_ECUDA after a launch

// Device address of the library's status word (see slrme_device_status) on
// the current device; kernels OR their error bits into it.
int status_word_address(int** out);

// ---------------------------------------------------------------- launchers
int launch_split(const uint32_t* rgbe, int64_t n, uint8_t* m3, uint8_t* e,
                 int64_t* lum_stats, cudaStream_t s);
int launch_base(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats,
                const QuantTable& qt, uint8_t* s_dec3, uint8_t* sdr3, int16_t* levels3, cudaStream_t s);
int launch_white_point(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats, float* l_white,
                       cudaStream_t s);
int launch_base_white(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats,
                      const float* l_white, const QuantTable& qt, uint8_t* s_dec3, uint8_t* sdr3, cudaStream_t s);
int launch_base_420(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats,
                    const QuantTable& qy, const QuantTable& qc, uint8_t* s_dec3, int16_t* levels, uint8_t* ws,
                    cudaStream_t s);
int launch_fit(const uint8_t* s3, const uint8_t* m3, const uint8_t* e, int h, int w, int gf_on,
               int64_t* bin_sums, slrme_params* params, cudaStream_t s);
int launch_residual_encode(const uint8_t* s3, const uint8_t* m3, const uint8_t* e, int h, int w,
                           int gf_on, const slrme_params* params, int16_t* r3, uint32_t* hist,
                           cudaStream_t s);
int launch_residual_decode(const uint8_t* s3, const uint8_t* e, const int16_t* r3, int h, int w,
                           int gf_on, const slrme_params* params, uint32_t* rgbe_out, cudaStream_t s);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ int64_t floor_div64(int64_t a, int64_t b) {   // b > 0
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

// Key of the tone-mapping operator from the log-average statistic:
// j = floor((sum + 2048 n) / (4096 n)) = round-half-up(16 mu), j = 16 J + r.
__device__ __forceinline__ void key_from_stats(const int64_t* stats, int* J, int* r) {
    int64_t s = stats[0], n = stats[1];
    int64_t j = 0;
    if (n > 0) j = floor_div64(s + 2048 * n, 4096 * n);
    int64_t JJ = floor_div64(j, 16);
    *J = (int)JJ;
    *r = (int)(j - 16 * JJ);
}

__device__ __forceinline__ uint32_t byte_of(uint32_t w, int i) { return (w >> (8 * i)) & 255u; }

// Eq. (8): round(a x + b) clipped to [0, 255]; float32 multiply then add,
// half away from zero.  NaN and t <= 0 give 0.
//
// float(x) for 0 <= x < 2^23 is bits(0x4B000000 | x) - 2^23 exactly (the 2^23
// bias).  For the clipped t in [0, 255], round half away from zero is
// floor(t + 0.5); the sum rounded down keeps that floor exact (the exact sum
// is at least the rounded one, and an integer in between would have to be the
// rounded value itself), and adding 2^23 rounded down leaves floor(v) in the
// low mantissa bits.
// predict_bits: the same estimate as the biased word 0x4B000000 + M*, for
// callers that subtract it from (or add it to) another biased or masked value.
__device__ __forceinline__ int predict_bits(float a, float b, uint32_t xbits) {   // xbits = 0x4B000000 | x
    const float xf = __fsub_rn(__uint_as_float(xbits), 8388608.0f);
    float t = __fadd_rn(__fmul_rn(a, xf), b);
    t = fminf(fmaxf(t, 0.0f), 255.0f);
    const float v = __fadd_rd(t, 0.5f);
    return __float_as_int(__fadd_rd(v, 8388608.0f));
}

__device__ __forceinline__ int predict_biased(float a, float b, uint32_t xbits) {   // xbits = 0x4B000000 | x
    return predict_bits(a, b, xbits) - 0x4B000000;
}

__device__ __forceinline__ int predict(float a, float b, int x) {
    return predict_biased(a, b, 0x4B000000u | (uint32_t)x);
}

// The biased float bits 0x4B000000 | x of pixel i of a lane's x pairs (x in
// the low or high 16 bits of X[i / 2]): one byte permute.
__device__ __forceinline__ uint32_t x_biased(const uint32_t (&X)[4], int i) {
    return __byte_perm(X[i >> 1], 0x4B000000u, (i & 1) ? 0x7632 : 0x7610);
}

}  // namespace slrme
