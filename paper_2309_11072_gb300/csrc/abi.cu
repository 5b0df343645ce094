// C ABI entry points (include/slrme.h): argument checks, constant tables,
// error reporting.  Every step of the codec runs in the kernels launched
// from here; this file only validates, builds tables and launches.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "slrme_internal.cuh"

#define SLRME_TABLE static const
#include "tables.inc"
#undef SLRME_TABLE

namespace slrme {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_status(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
        return SLRME_ECUDA;
    }
    return SLRME_OK;
}

// ---------------------------------------------------------------- tables

// ITU-T T.81 Annex K, Table K.1 (luminance), row-major.
static const int kAnnexK1[64] = {
    16, 11, 10, 16, 24, 40, 51, 61,     12, 12, 14, 19, 26, 58, 60, 55,
    14, 13, 16, 24, 40, 57, 69, 56,     14, 17, 22, 29, 51, 87, 80, 62,
    18, 22, 37, 56, 68, 109, 103, 77,   24, 35, 55, 64, 81, 104, 113, 92,
    49, 64, 78, 87, 103, 121, 120, 101, 72, 92, 95, 98, 112, 100, 103, 99};

// ITU-T T.81 Annex K, Table K.2 (chrominance), row-major.
static const int kAnnexK2[64] = {
    17, 18, 24, 47, 99, 99, 99, 99,     18, 21, 26, 66, 99, 99, 99, 99,
    24, 26, 56, 99, 99, 99, 99, 99,     47, 66, 99, 99, 99, 99, 99, 99,
    99, 99, 99, 99, 99, 99, 99, 99,     99, 99, 99, 99, 99, 99, 99, 99,
    99, 99, 99, 99, 99, 99, 99, 99,     99, 99, 99, 99, 99, 99, 99, 99};

static bool build_quant_table(int quality, const int* base, QuantTable* out) {
    const int scale = quality < 50 ? 5000 / quality : 200 - 2 * quality;
    for (int i = 0; i < 64; ++i) {
        int v = (base[i] * scale + 50) / 100;
        v = v < 1 ? 1 : (v > 255 ? 255 : v);
        out->q[i] = v;
        out->qm[i] = (uint32_t)(((1u << 24) + (uint32_t)v - 1u) / (uint32_t)v);   // ceil(2^24 / v)
        // The reciprocal is exact for every numerator the kernel can form
        // (|F| + q/2 < 4096); check it rather than trust the bound.
        for (uint32_t n = 0; n < 4096; ++n) {
            uint32_t hi = (uint32_t)(((uint64_t)(n << 8) * out->qm[i]) >> 32);
            if (hi != n / (uint32_t)v) return false;
        }
    }
    return true;
}

static bool cached_table(int quality, const int* base, QuantTable* cache, int* state, std::mutex& mu,
                         QuantTable* out) {
    if (quality < 1 || quality > 100) return false;
    std::lock_guard<std::mutex> lock(mu);
    if (state[quality] == 0) state[quality] = build_quant_table(quality, base, &cache[quality]) ? 1 : -1;
    if (state[quality] < 0) return false;
    *out = cache[quality];
    return true;
}

bool quant_table(int quality, QuantTable* out) {
    static QuantTable cache[101];
    static int state[101];   // 0 = not built, 1 = valid, -1 = failed check
    static std::mutex mu;
    return cached_table(quality, kAnnexK1, cache, state, mu, out);
}

bool quant_table_chroma(int quality, QuantTable* out) {
    static QuantTable cache[101];
    static int state[101];
    static std::mutex mu;
    return cached_table(quality, kAnnexK2, cache, state, mu, out);
}

Geometry geometry() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 152;
    }
    return Geometry{sms};
}

}  // namespace slrme

using namespace slrme;

// ---------------------------------------------------------------- argument checks

static bool check_size(int h, int w) {
    if (h < 0 || w < 0) {
        set_error("image size must be non-negative (h=%d, w=%d)", h, w);
        return false;
    }
    if ((int64_t)h * (int64_t)w >= ((int64_t)1 << 31)) {
        set_error("image too large: h*w must be < 2^31 (h=%d, w=%d)", h, w);
        return false;
    }
    return true;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

#define REQUIRE(cond, ...)            \
    do {                              \
        if (!(cond)) {                \
            set_error(__VA_ARGS__);   \
            return SLRME_EINVAL;      \
        }                             \
    } while (0)

extern "C" {

const char* slrme_last_error(void) { return g_err; }

size_t slr_fit_workspace_bytes(void) { return sizeof(int64_t) * kNbin * kNsum; }

int rgbe_key_scale(const int64_t lum_stats[2], int32_t* J, int32_t* r) {
    REQUIRE(lum_stats && J && r, "rgbe_key_scale: null pointer");
    REQUIRE(lum_stats[1] >= 0, "rgbe_key_scale: negative pixel count");
    int64_t s = lum_stats[0], n = lum_stats[1];
    int64_t j = 0;
    if (n > 0) {
        int64_t a = s + 2048 * n, b = 4096 * n;
        j = a / b;
        if ((a % b) != 0 && a < 0) j -= 1;
    }
    int64_t JJ = j / 16;
    if ((j % 16) != 0 && j < 0) JJ -= 1;
    *J = (int32_t)JJ;
    *r = (int32_t)(j - 16 * JJ);
    return SLRME_OK;
}

int rgbe_split(const uint32_t* rgbe, int h, int w, uint8_t* m3, uint8_t* e, int64_t* lum_stats,
               slrme_stream_t stream) {
    if (!check_size(h, w)) return SLRME_EINVAL;
    const int64_t n = (int64_t)h * w;
    REQUIRE(lum_stats, "rgbe_split: lum_stats is null");
    REQUIRE(n == 0 || (rgbe && m3 && e), "rgbe_split: null image pointer");
    REQUIRE(aligned(rgbe, 4) && aligned(lum_stats, 8), "rgbe_split: rgbe must be 4-byte and lum_stats 8-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(lum_stats, 0, 2 * sizeof(int64_t), s) != cudaSuccess) return cuda_status("rgbe_split memset");
    if (n == 0) return SLRME_OK;
    return launch_split(rgbe, n, m3, e, lum_stats, s);
}

int sdri_base_roundtrip(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats,
                        int quality, uint8_t* s_dec3, uint8_t* sdr3, slrme_stream_t stream) {
    if (!check_size(h, w)) return SLRME_EINVAL;
    QuantTable qt;
    REQUIRE(quality >= 1 && quality <= 100, "sdri_base_roundtrip: quality %d outside 1..100", quality);
    REQUIRE(quant_table(quality, &qt), "sdri_base_roundtrip: quantiser table check failed");
    const int64_t n = (int64_t)h * w;
    if (n == 0) return SLRME_OK;
    REQUIRE(m3 && e && lum_stats && s_dec3, "sdri_base_roundtrip: null pointer");
    REQUIRE(aligned(lum_stats, 8), "sdri_base_roundtrip: lum_stats must be 8-byte aligned");
    return launch_base(m3, e, h, w, lum_stats, qt, s_dec3, sdr3, nullptr, (cudaStream_t)stream);
}

int sdri_white_point(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats, float* l_white,
                     slrme_stream_t stream) {
    if (!check_size(h, w)) return SLRME_EINVAL;
    REQUIRE(l_white && aligned(l_white, 4) && lum_stats && aligned(lum_stats, 8),
            "sdri_white_point: need a 4-byte aligned l_white and 8-byte aligned lum_stats");
    REQUIRE((int64_t)h * w == 0 || (m3 && e), "sdri_white_point: null image pointer");
    return launch_white_point(m3, e, h, w, lum_stats, l_white, (cudaStream_t)stream);
}

int sdri_base_roundtrip_white(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats,
                              const float* l_white, int quality, uint8_t* s_dec3, uint8_t* sdr3,
                              slrme_stream_t stream) {
    if (!check_size(h, w)) return SLRME_EINVAL;
    QuantTable qt;
    REQUIRE(quality >= 1 && quality <= 100, "sdri_base_roundtrip_white: quality %d outside 1..100", quality);
    REQUIRE(quant_table(quality, &qt), "sdri_base_roundtrip_white: quantiser table check failed");
    if ((int64_t)h * w == 0) return SLRME_OK;
    REQUIRE(m3 && e && lum_stats && s_dec3 && l_white, "sdri_base_roundtrip_white: null pointer");
    REQUIRE(aligned(lum_stats, 8) && aligned(l_white, 4),
            "sdri_base_roundtrip_white: lum_stats must be 8-byte and l_white 4-byte aligned");
    return launch_base_white(m3, e, h, w, lum_stats, l_white, qt, s_dec3, sdr3, (cudaStream_t)stream);
}

size_t sdri_base_420_workspace_bytes(int h, int w) {
    if (h < 0 || w < 0) return 0;
    const size_t n = (size_t)h * w, nc = (size_t)((h + 1) / 2) * ((w + 1) / 2);
    return (n + 2 * nc + 255) & ~(size_t)255;
}

int sdri_base_roundtrip_420(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats,
                            int quality, uint8_t* s_dec3, int16_t* levels, void* ws, slrme_stream_t stream) {
    if (!check_size(h, w)) return SLRME_EINVAL;
    REQUIRE(h <= 65535 * 2, "sdri_base_roundtrip_420: h must be at most 131070");
    QuantTable qy, qc;
    REQUIRE(quality >= 1 && quality <= 100, "sdri_base_roundtrip_420: quality %d outside 1..100", quality);
    REQUIRE(quant_table(quality, &qy) && quant_table_chroma(quality, &qc),
            "sdri_base_roundtrip_420: quantiser table check failed");
    const int64_t n = (int64_t)h * w;
    if (n == 0) return SLRME_OK;
    REQUIRE(m3 && e && lum_stats && s_dec3 && ws, "sdri_base_roundtrip_420: null pointer");
    REQUIRE(aligned(lum_stats, 8) && aligned(levels, 16),
            "sdri_base_roundtrip_420: lum_stats must be 8-byte and levels 16-byte aligned");
    return launch_base_420(m3, e, h, w, lum_stats, qy, qc, s_dec3, levels, (uint8_t*)ws, (cudaStream_t)stream);
}

int sdri_base_levels(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats, int quality,
                     uint8_t* s_dec3, int16_t* levels3, slrme_stream_t stream) {
    if (!check_size(h, w)) return SLRME_EINVAL;
    QuantTable qt;
    REQUIRE(quality >= 1 && quality <= 100, "sdri_base_levels: quality %d outside 1..100", quality);
    REQUIRE(quant_table(quality, &qt), "sdri_base_levels: quantiser table check failed");
    const int64_t n = (int64_t)h * w;
    if (n == 0) return SLRME_OK;
    REQUIRE(m3 && e && lum_stats && s_dec3 && levels3, "sdri_base_levels: null pointer");
    REQUIRE(aligned(lum_stats, 8) && aligned(levels3, 16),
            "sdri_base_levels: lum_stats must be 8-byte and levels3 16-byte aligned");
    return launch_base(m3, e, h, w, lum_stats, qt, s_dec3, nullptr, levels3, (cudaStream_t)stream);
}

int slr_fit(const uint8_t* s_dec3, const uint8_t* m3, const uint8_t* e, int h, int w, int gf_on,
            int64_t* bin_sums, slrme_params* params, slrme_stream_t stream) {
    if (!check_size(h, w)) return SLRME_EINVAL;
    REQUIRE(gf_on == 0 || gf_on == 1, "slr_fit: gf_on must be 0 or 1");
    REQUIRE(bin_sums && params, "slr_fit: null workspace or params");
    REQUIRE(aligned(bin_sums, 8) && aligned(params, 4), "slr_fit: bin_sums must be 8-byte and params 4-byte aligned");
    const int64_t n = (int64_t)h * w;
    REQUIRE(n == 0 || (s_dec3 && m3 && e), "slr_fit: null image pointer");
    return launch_fit(s_dec3, m3, e, h, w, gf_on, bin_sums, params, (cudaStream_t)stream);
}

int residual_encode(const uint8_t* s_dec3, const uint8_t* m3, const uint8_t* e, int h, int w, int gf_on,
                    const slrme_params* params, int16_t* r3, uint32_t* hist, slrme_stream_t stream) {
    if (!check_size(h, w)) return SLRME_EINVAL;
    REQUIRE(gf_on == 0 || gf_on == 1, "residual_encode: gf_on must be 0 or 1");
    const int64_t n = (int64_t)h * w;
    REQUIRE(aligned(hist, 4) && aligned(r3, 2) && aligned(params, 4),
            "residual_encode: hist and params must be 4-byte and r3 2-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (hist && cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 3 * kNres, s) != cudaSuccess)
        return cuda_status("residual_encode memset");
    if (n == 0) return SLRME_OK;
    REQUIRE(s_dec3 && m3 && e && params && r3, "residual_encode: null pointer");
    return launch_residual_encode(s_dec3, m3, e, h, w, gf_on, params, r3, hist, s);
}

int residual_decode(const uint8_t* s_dec3, const uint8_t* e, const int16_t* r3, int h, int w, int gf_on,
                    const slrme_params* params, uint32_t* rgbe_out, slrme_stream_t stream) {
    if (!check_size(h, w)) return SLRME_EINVAL;
    REQUIRE(gf_on == 0 || gf_on == 1, "residual_decode: gf_on must be 0 or 1");
    const int64_t n = (int64_t)h * w;
    if (n == 0) return SLRME_OK;
    REQUIRE(s_dec3 && e && r3 && params && rgbe_out, "residual_decode: null pointer");
    REQUIRE(aligned(r3, 2) && aligned(params, 4) && aligned(rgbe_out, 4),
            "residual_decode: r3 must be 2-byte, params and rgbe_out 4-byte aligned");
    return launch_residual_decode(s_dec3, e, r3, h, w, gf_on, params, rgbe_out, (cudaStream_t)stream);
}

int slrme_host_tables(int32_t* lut, float* gamma, float* kr, float* wr, int quality, int32_t* quant,
                      int32_t* dct) {
    if (lut) memcpy(lut, kLog2Lut, sizeof(int32_t) * 2048);
    if (gamma) memcpy(gamma, kGammaBits, sizeof(float) * 256);
    if (kr) memcpy(kr, kKrBits, sizeof(float) * 16);
    if (wr) memcpy(wr, kWrBits, sizeof(float) * 16);
    if (quant) {
        QuantTable qt;
        REQUIRE(quant_table(quality, &qt), "slrme_host_tables: quality %d outside 1..100", quality);
        memcpy(quant, qt.q, sizeof(int32_t) * 64);
    }
    if (dct) {
        // The constants the transform kernels use as immediates (base.cu).
        static const int32_t c[8][8] = {
            {1448, 1448, 1448, 1448, 1448, 1448, 1448, 1448},
            {2009, 1703, 1138, 400, -400, -1138, -1703, -2009},
            {1892, 784, -784, -1892, -1892, -784, 784, 1892},
            {1703, -400, -2009, -1138, 1138, 2009, 400, -1703},
            {1448, -1448, -1448, 1448, 1448, -1448, -1448, 1448},
            {1138, -2009, 400, 1703, -1703, -400, 2009, -1138},
            {784, -1892, 1892, -784, -784, 1892, -1892, 784},
            {400, -1138, 1703, -2009, 2009, -1703, 1138, -400}};
        memcpy(dct, c, sizeof(c));
    }
    return SLRME_OK;
}

}  // extern "C"
