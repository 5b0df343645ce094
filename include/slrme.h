/*
 * slrme.h -- C ABI of the GB300 (sm_103a) dual-layer lossless Radiance
 * (RGBE) coder with the simple linear regressive mantissa estimator
 * (SLRME) of Suzuki, Yukikata, Yang and Yoshida, "Lightning-Fast
 * Dual-Layer Lossless Coding for Radiance Format High Dynamic Range
 * Images" (arXiv 2309.11072).
 *
 * Encoder (Fig. 2, bottom):  rgbe_split -> sdri_base_roundtrip -> slr_fit
 *                            -> residual_encode
 * Decoder:                   residual_decode
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Images are h rows by w columns, row-major, row pitch = w elements.
 *   A packed RGBE word is R | G<<8 | B<<16 | E<<24 (the byte order of a
 *   Radiance file).  Colour planes are planar: plane c (R=0, G=1, B=2) of
 *   an "x3" buffer starts at element c*h*w.
 * - All image, workspace and parameter pointers are DEVICE pointers owned
 *   by the caller; the library allocates no memory.  Calls are asynchronous
 *   on `stream` (NULL = the legacy default stream) unless stated otherwise.
 * - 0 <= h, 0 <= w, h*w < 2^31.  An empty image (h*w == 0) is valid: the
 *   call only clears the outputs it documents as cleared.
 * - Typed buffers must be naturally aligned (uint32/float/int32: 4 bytes,
 *   int16: 2, int64: 8); a misaligned one is rejected with SLRME_EINVAL.
 *   Byte planes may start anywhere.  Planes aligned to 16 bytes with
 *   w % 16 == 0 take the tensor-map (TMA) kernels of slr_fit,
 *   residual_encode and residual_decode; 8-byte aligned planes with
 *   w % 8 == 0 take vectorised loads; others a scalar path.  Every path
 *   gives the same results.
 * - Return value: SLRME_OK, or a negative SLRME_E* code; the text of the
 *   last error of the calling thread is in slrme_last_error().
 *   SLRME_EINVAL is returned before anything is enqueued.  SLRME_ECUDA
 *   reports a launch error seen when the call returns (errors of the
 *   asynchronous execution surface at the caller's next synchronisation).
 */
#ifndef SLRME_H
#define SLRME_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SLRME_OK        0
#define SLRME_EINVAL   (-1)   /* bad argument: null pointer, size, quality, flag   */
#define SLRME_ECUDA    (-2)   /* CUDA launch / runtime error                        */

#define SLRME_NBIN      256   /* exponent regions: one per 8-bit exponent value E  */
#define SLRME_NSUM      13    /* per region: N_E, then per channel sum x, sum y,
                                 sum xy, sum xx                                     */
#define SLRME_NRES      511   /* residual values -255..255                          */

typedef struct CUstream_st* slrme_stream_t;   /* identical to cudaStream_t */

/* The transmitted SLRME parameters (Sec. III-C): one 32-bit slope a_E and one
 * 32-bit intercept b_E per colour channel and per used exponent region E.
 * The slope is per 1/16 grey level of the restored SDRI (x = 16 S*).
 * n[E] = N_E, the pixel count of region E; a region with N_E = 0 is unused
 * (a = b = 0) and is not transmitted.  7184 bytes, 4-byte aligned. */
typedef struct slrme_params {
    float   a[3][SLRME_NBIN];
    float   b[3][SLRME_NBIN];
    int32_t n[SLRME_NBIN];
    int32_t n_used;
    int32_t reserved[3];
} slrme_params;

/* RGBE split (Sec. II-A Fig. 1, Sec. III-A): separates the words into the
 * mantissa planes M_R, M_G, M_B (m3, uint8 [3][h][w]) and the exponent plane
 * E (e, uint8 [h][w]), and accumulates the log-average luminance statistic
 * of the tone-mapping operator into lum_stats (int64[2], device):
 *   lum_stats[0] = sum over pixels with E > 0 of l(p),  lum_stats[1] = their count,
 *   l = 65536 (E - 137 + k) + round(65536 log2 m),  Yq = 2126(2M_R+1) +
 *   7152(2M_G+1) + 722(2M_B+1), k = bitlen(Yq) - 12, m = Yq >> k,
 * i.e. l / 65536 approximates log2(10^4 Y) of the Eq. (3) floats.
 * lum_stats is cleared by the call before accumulation. */
int rgbe_split(const uint32_t* rgbe, int h, int w, uint8_t* m3, uint8_t* e,
               int64_t* lum_stats, slrme_stream_t stream);

/* Host helper, synchronous, no GPU: the key of the tone-mapping operator from
 * a host copy of lum_stats: j = round-half-up(16 mu), mu = lum_stats[0] /
 * (65536 lum_stats[1]) (j = 0 for an image without non-zero pixels), returned
 * as j = 16 J + r with 0 <= r < 16. */
int rgbe_key_scale(const int64_t lum_stats[2], int32_t* J, int32_t* r);

/* Base layer round trip (Sec. II-B, Fig. 2; JPEG at quality Q in Sec. IV):
 * tone maps M, E to the 8-bit SDRI with Reinhard's global operator
 * (key 0.18 over the log-average read from lum_stats on the device, float32
 * steps, gamma 2.2 by a threshold table), then runs every 8x8 block of each
 * colour plane through a fixed-point DCT (constants round(4096 D), rounding
 * shifts 9 and 15), quantisation with the T.81 Annex K.1 luminance table
 * scaled to `quality` (1..100, IJG rule), dequantisation and the inverse DCT,
 * and writes the decoded SDRI S (s_dec3, uint8 [3][h][w]).  Blocks at a
 * ragged edge replicate the last row/column.  sdr3 (uint8 [3][h][w]) receives
 * the tone-mapped SDRI before coding, or is NULL. */
int sdri_base_roundtrip(const uint8_t* m3, const uint8_t* e, int h, int w,
                        const int64_t* lum_stats, int quality,
                        uint8_t* s_dec3, uint8_t* sdr3, slrme_stream_t stream);

/* SLRME fit (Sec. III-B, Eqs. 9-10 from the normal equations 6-7 of Sec. II-C):
 * restores S with the 3x3 binomial Gaussian filter (gf_on = 1; x = 16 S* in
 * [0, 4080], edge replicated) or takes x = 16 S (gf_on = 0), accumulates per
 * exponent region E the exact int64 sums into bin_sums (workspace, int64
 * [256][13]: N_E, then per channel c sum x, sum y, sum xy, sum xx with y = M_c;
 * cleared by the call), and solves each (channel, region) on the device:
 *   D_xx = N sum xx - (sum x)^2, D_xy = N sum xy - sum x sum y  (int128),
 *   a_E = float(double(D_xy) / double(D_xx)),
 *   b_E = float((double(sum y) - double(a_E) double(sum x)) / N),
 * with a = 0, b = float(sum y / N) when D_xx = 0 and a = b = 0 when N_E = 0.
 * params receives the result (device, slrme_params). */
int slr_fit(const uint8_t* s_dec3, const uint8_t* m3, const uint8_t* e, int h, int w,
            int gf_on, int64_t* bin_sums, slrme_params* params, slrme_stream_t stream);

/* Bytes of the bin_sums workspace slr_fit needs (256 * 13 * 8). */
size_t slr_fit_workspace_bytes(void);

/* slr_fit for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a deployment variant).  Some callers hold no device
 * allocator of their own: a plugin whose host application owns all device
 * memory, a fixed-budget service that allocates nothing after start-up, or
 * C code that only receives device pointers from another framework.  They
 * cannot provide the bin_sums workspace, so this entry point keeps it in a
 * library-owned static device array of 26,624 bytes (256 regions x 13 int64
 * sums) that every GPU loading the library holds until exit.  It computes the
 * same params as slr_fit and calls no cudaMalloc / cudaFree.
 * - Sizes: the same as slr_fit (h, w >= 0, h*w < 2^31, the range in which the
 *   int64 sums are exact); anything else is rejected with SLRME_EINVAL.
 * - The first call on a device looks up the array's device address (with that
 *   device current); make that first call before any stream capture.  The
 *   address is kept with the context it belongs to and looked up again when
 *   the device's current context changes (after a device reset, say): the
 *   first call after such a change is again a first call.
 * - All calls share the one array: each call clears it on `stream` before
 *   use, and calls whose GPU work overlaps (other streams, other threads)
 *   race on it and give wrong parameters.  Serialise them. */
int slr_fit_noalloc(const uint8_t* s_dec3, const uint8_t* m3, const uint8_t* e, int h, int w,
                    int gf_on, slrme_params* params, slrme_stream_t stream);

/* Residual formation (Eq. 8, Sec. III-C): M*(q) = round(a_E S*(q) + b_E)
 * clipped to [0, 255] (float32 multiply then add, round half away from zero),
 * R = M - M* (r3, int16 [3][h][w]).  hist (uint32 [3][511], device, may be
 * NULL) is cleared and receives the count of each residual value per channel
 * (index R + 255), the statistics of the enhancement-layer rate. */
int residual_encode(const uint8_t* s_dec3, const uint8_t* m3, const uint8_t* e, int h, int w,
                    int gf_on, const slrme_params* params, int16_t* r3, uint32_t* hist,
                    slrme_stream_t stream);

/* Decoder (Sec. I and III-C): recomputes M* from the decoded SDRI, the
 * exponent plane and the transmitted parameters (no refitting), adds the
 * residual, M = R + M*, and repacks the RGBE words (rgbe_out, uint32 [h][w]).
 * For any params this inverts residual_encode exactly. */
int residual_decode(const uint8_t* s_dec3, const uint8_t* e, const int16_t* r3, int h, int w,
                    int gf_on, const slrme_params* params, uint32_t* rgbe_out,
                    slrme_stream_t stream);

/* Reinhard's operator with a white point (his Eq. 4 form: L_d = L (1 + L /
 * L_white^2) / (1 + L)), a variant of the operator of sdri_base_roundtrip
 * (Sec. IV names Reinhard's operator without its parameters).
 * sdri_white_point writes L_white (float, device, 4-byte aligned): the
 * largest scaled luminance L (as the operator computes it per pixel) over
 * the pixels with E > 0, 0 for an image without such pixels.
 * sdri_base_roundtrip_white is sdri_base_roundtrip with that operator: per
 * pixel, in float32 round-to-nearest, H = (num * (1 + L / (L_white *
 * L_white))) / den, each operation rounded once in that order (num, den and
 * L as in the plain operator); an infinite L_white^2 gives the plain
 * operator. */
int sdri_white_point(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats, float* l_white,
                     slrme_stream_t stream);
int sdri_base_roundtrip_white(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats,
                              const float* l_white, int quality, uint8_t* s_dec3, uint8_t* sdr3,
                              slrme_stream_t stream);

/* ===================================================================== base-layer entropy coding
 * Sec. IV codes the base layer with JPEG.  sdri_base_roundtrip models only
 * what changes S; these two calls give the base layer's coded size: the
 * quantised levels the round trip computes, and the size of their JPEG
 * baseline Huffman coding (T.81 Annex F.1.2) with the typical luminance
 * tables of Annex K.3 (Tables K.3, K.5), each colour plane a single-
 * component scan of its 8x8 blocks in raster order:
 *   DC: diff = level_DC - level_DC of the plane's previous block (0 before
 *       the first), category SSSS = bit length of |diff| (0..11), cost = DC
 *       code length of SSSS + SSSS;
 *   AC: zigzag positions 1..63 (T.81 Figure A.6); a nonzero level c after r
 *       zeros costs floor(r / 16) ZRL codes (symbol 0xF0), then the code of
 *       ((r mod 16) << 4) | SSSS(c) plus SSSS (1..10); trailing zeros cost
 *       one EOB code (symbol 0x00).
 * The size is the entropy-coded data in bits, before byte stuffing,
 * padding, markers and headers.
 * Levels layout: int16 [3][bh][bw][64], bh = ceil(h/8), bw = ceil(w/8);
 * within a block, coefficient (v vertical, u horizontal frequency) at
 * u*8 + v.  A level beyond the baseline categories (DC difference above
 * 2047, AC level above 1023 in magnitude) sets bit 2 (value 4) of the
 * status word and counts its size without a code. */

/* sdri_base_roundtrip (without the SDRI output) that also writes the levels
 * (levels3 device, 16-byte aligned). */
int sdri_base_levels(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats, int quality,
                     uint8_t* s_dec3, int16_t* levels3, slrme_stream_t stream);

/* Coded bits of each plane (bits3: uint64 [3], device, 8-byte aligned,
 * cleared first) and, if block_bits is not NULL, of each block (uint32
 * [3][bh*bw]).  Asynchronous on `stream`. */
int jpeg_huffman_bits(const int16_t* levels3, int h, int w, unsigned long long* bits3, uint32_t* block_bits,
                      slrme_stream_t stream);

/* Sizes of any planes of levels (up to 4): plane p has nblocks[p] blocks
 * (host array), its blocks following those of planes 0..p-1 in `levels`,
 * coded with the chrominance tables of Annex K.3 (Tables K.4, K.6) when
 * chroma[p] = 1 (host array) and the luminance tables when 0.  bits: uint64
 * [nplanes] (device, cleared first); block_bits (may be NULL): uint32 per
 * block in the same order. */
int jpeg_huffman_bits_planes(const int16_t* levels, int nplanes, const int64_t* nblocks, const int32_t* chroma,
                             unsigned long long* bits, uint32_t* block_bits, slrme_stream_t stream);

/* The base layer with a default JPEG encoder's colour handling (YCbCr 4:2:0):
 * the tone-mapped SDRI converted to YCbCr by T.871's equations in 16-bit
 * fixed point (weights round(65536 c), rounded half up, clamped):
 *   Y  = (19595 R + 38470 G + 7471 B + 32768) >> 16
 *   Cb = ((-11058 R - 21710 G + 32768 B + 32768) >> 16) + 128
 *   Cr = ((32768 R - 27439 G - 5329 B + 32768) >> 16) + 128,
 * chroma averaged over 2x2 pixels ((sum + 2) >> 2, edges replicated) into
 * planes of ceil(h/2) x ceil(w/2), each plane through the 8x8 round trip of
 * sdri_base_roundtrip (Y with Table K.1, Cb and Cr with Table K.2, both
 * IJG-scaled), chroma replicated back over its 2x2 pixels, and
 *   R = Y + ((91881 (Cr - 128) + 32768) >> 16)
 *   G = Y + ((-22554 (Cb - 128) - 46802 (Cr - 128) + 32768) >> 16)
 *   B = Y + ((116130 (Cb - 128) + 32768) >> 16), clamped, into s_dec3.
 * levels (may be NULL, 16-byte aligned): the Y plane's blocks, then Cb's,
 * then Cr's (each in raster order, 64 levels per block as above), for
 * jpeg_huffman_bits_planes with chroma = {0, 1, 1}.  ws: device workspace of
 * sdri_base_420_workspace_bytes(h, w) bytes.  h <= 131070. */
size_t sdri_base_420_workspace_bytes(int h, int w);
int sdri_base_roundtrip_420(const uint8_t* m3, const uint8_t* e, int h, int w, const int64_t* lum_stats,
                            int quality, uint8_t* s_dec3, int16_t* levels, void* ws, slrme_stream_t stream);

/* ===================================================================== enhancement-layer entropy coder
 * The enhancement layer carries the residuals R to the decoder through a
 * reversible coder (Sec. II-A: the enhancement layer's coders must be
 * reversible for lossless decoding; Sec. IV codes it with JPEG 2000's
 * lossless mode).  This coder is interleaved range asymmetric numeral
 * systems (rANS, Duda 2013) with one static frequency table per colour
 * channel:
 *   M = 2^14 (table total), state x in [2^16, 2^32), 16-bit words;
 *   symbol s = R + 255 (0..510), frequency f_s, cumulative c_s = sum_{t<s} f_t;
 *   encode, symbols of a stream in reverse order, from x = 2^16:
 *     if floor(x / 2^18) >= f_s: emit x mod 2^16, x = floor(x / 2^16);
 *     x = floor(x / f_s) M + (x mod f_s) + c_s;
 *   finally emit x mod 2^16, then floor(x / 2^16);
 *   decode: slot = x mod M, s with c_s <= slot < c_s + f_s,
 *     x = f_s floor(x / M) + slot - c_s, and if x < 2^16, x = 2^16 x + next word;
 *   the decoder reads the words in the reverse of their emission order and
 *   ends in the state 2^16 with every word read.
 * Layout for three residual planes of n symbols each (int16 [3][n], the
 * planes of residual_encode with n = h*w): chunks = ceil(n / 8192); chunk k
 * of plane c is coded as 32 streams, stream l taking symbols k*8192 + l + 32 j
 * (j = 0, 1, ...) of the plane.  Chunk k of plane c owns the block of
 * 32 * SLRME_RANS_CAP (258) uint16 words starting at word (c*chunks + k)*32*258
 * of `words`; its streams' words are packed from the start of the block,
 * stream l from the sum of the word counts of streams 0..l-1, each in decoding
 * order (the state's high word, its low word, then the renormalisation
 * words).  rans_encode writes nothing else of a block.
 * counts[(c*chunks + k)*32 + l] (uint32) is the number of words the stream
 * used (2..258, or 0 for a stream that could not be coded).
 * Errors found while a kernel runs (a value inside -255..255 with a zero
 * frequency, a table whose entries exceed M or do not sum to M, a stream
 * whose words do not decode back to the initial state) set bit 1 (value 2) of
 * the device status word (slrme_device_status); the affected outputs are then
 * unspecified but every access stays inside the documented buffers. */
#define SLRME_RANS_CHUNK  8192   /* symbols per chunk of a plane                 */
#define SLRME_RANS_LANES  32     /* interleaved streams per chunk                */
#define SLRME_RANS_CAP    258    /* uint16 words per stream region (256 + 2)     */
#define SLRME_RANS_M      16384  /* table total                                  */

/* Host, no GPU: uint16 words of `words` and uint32 entries of `counts` for
 * three planes of n symbols (0 for n <= 0). */
int64_t rans_words_capacity(int64_t n);
int64_t rans_counts_capacity(int64_t n);

/* Frequency tables freq3 (uint32 [3][511], device) from the residual
 * histograms hist3 (uint32 [3][511], device, as residual_encode writes them):
 * per channel with N = sum of its counts n_s > 0, f_s = max(1, floor(n_s M / N))
 * for every s with n_s > 0 and 0 otherwise; a shortfall M - sum f is added to
 * the most frequent symbol (smallest s on ties); an excess is removed one
 * unit at a time from the largest entry above 1 (smallest s on ties).  A
 * channel with N = 0 gets an all-zero table.  Asynchronous on `stream`. */
int rans_tables(const uint32_t* hist3, uint32_t* freq3, slrme_stream_t stream);

/* Encodes the residual planes r3 (int16 [3][n], device, 2-byte aligned) with
 * the tables freq3 (device) into words (device, rans_words_capacity(n) uint16,
 * 16-byte aligned) and counts (device, rans_counts_capacity(n) uint32).  0 <= n < 2^31; n = 0 enqueues nothing.
 * The table total M must hold for every channel with n > 0 symbols. */
int rans_encode(const int16_t* r3, int64_t n, const uint32_t* freq3, uint16_t* words, uint32_t* counts,
                slrme_stream_t stream);

/* Decodes words/counts (as rans_encode writes them; words 16-byte aligned)
 * with the same tables back into the residual planes r3 (int16 [3][n]).
 * Each chunk's packed words are read with one bulk copy whose wait is
 * bounded: a wait that gives up sets bit 0 of the status word and the kernel
 * stops. */
int rans_decode(const uint16_t* words, const uint32_t* counts, int64_t n, const uint32_t* freq3, int16_t* r3,
                slrme_stream_t stream);

/* Segments: a run of symbol arrays coded each with its own table, for the
 * wavelet coefficients below (one segment per plane and band).  The symbols
 * of segment g follow those of segments 0..g-1 in `sym`; freq holds one
 * table of 511 entries per segment (from rans_tables_n); segment g is cut
 * into ceil(len[g] / 8192) chunks whose blocks and counts follow those of
 * the segments before it.  A chunk holding a value outside -255..255 is
 * stored raw: its block holds the chunk's values (int16 bit patterns, in
 * order) and all 32 of its counts are SLRME_RANS_RAW.  The three-plane
 * calls above are this form with three segments of n symbols (a residual
 * outside -255..255 makes its chunk raw).  1 <= nseg <= SLRME_RANS_MAX_SEGMENTS,
 * len (host array) >= 0, total symbols < 2^31. */
#define SLRME_RANS_MAX_SEGMENTS 64
#define SLRME_RANS_RAW          0xFFFFFFFFu

/* Host: uint16 words and uint32 counts of a run of segments (0 on bad arguments). */
int64_t rans_segments_words_capacity(int nseg, const int64_t* len);
int64_t rans_segments_counts_capacity(int nseg, const int64_t* len);

/* rans_tables for `ntables` histograms (uint32 [ntables][511]) -> freq
 * (uint32 [ntables][511]); 1 <= ntables <= 65535. */
int rans_tables_n(const uint32_t* hist, int ntables, uint32_t* freq, slrme_stream_t stream);

int rans_encode_segments(const int16_t* sym, int nseg, const int64_t* len, const uint32_t* freq, uint16_t* words,
                         uint32_t* counts, slrme_stream_t stream);
int rans_decode_segments(const uint16_t* words, const uint32_t* counts, int nseg, const int64_t* len,
                         const uint32_t* freq, int16_t* sym, slrme_stream_t stream);

/* ===================================================================== reversible 5/3 wavelet
 * The transform of JPEG 2000's lossless mode, which codes the enhancement
 * layer in Sec. IV: integer lifting with whole-sample symmetric extension.
 * For a row or column of n >= 2 samples (nH = floor(n/2), nL = ceil(n/2)):
 *   d[i] = x[2i+1] - floor((x[2i] + x[2i+2]) / 2),   i < nH   (x[n] = x[n-2])
 *   s[i] = x[2i]   + floor((d[i-1] + d[i] + 2) / 4), i < nL   (d[-1] = d[0];
 *                                                  odd n: d[nL-1] = d[nL-2])
 * and a single sample is its own low-pass value.  One level transforms the
 * rows, then the columns; level l + 1 transforms level l's low-low band.
 * Output per plane, subband-major, each band row-major: LL_L, then HL, LH,
 * HH of level L, ..., of level 1 (HL: high-pass along the rows, low along
 * the columns; LH the reverse), 1 + 3L bands.  Each pass at most doubles the
 * largest magnitude: inputs in -255..255 stay within +-16320 at L = 3. */
#define SLRME_DWT_MAX_LEVELS 3

/* Host: band sizes in output order, dims[2b] rows and dims[2b+1] columns of
 * band b; returns the number of bands (1 + 3 levels) or SLRME_EINVAL. */
int dwt53_bands(int h, int w, int levels, int32_t* dims);

/* Device workspace bytes for nplanes planes of h x w. */
size_t dwt53_workspace_bytes(int nplanes, int h, int w);

/* Forward transform of nplanes planes (int16 [nplanes][h][w], device) into
 * coef (int16 [nplanes][h*w], device, each plane subband-major) and, if hist
 * is not NULL, the histograms of the values inside -255..255 of every band
 * (uint32 [nplanes][1 + 3 levels][511], value + 255; cleared first), the
 * tables' input for the segment coder.  1 <= levels <= 3, 1 <= nplanes <=
 * 65535, h <= 65535, h*w < 2^31; ws: dwt53_workspace_bytes, 256-byte
 * aligned.  Planes and coef must not overlap. */
int dwt53_forward(const int16_t* planes, int nplanes, int h, int w, int levels, int16_t* coef, uint32_t* hist,
                  void* ws, slrme_stream_t stream);

/* Inverse of dwt53_forward (coef -> planes). */
int dwt53_inverse(const int16_t* coef, int nplanes, int h, int w, int levels, int16_t* planes, void* ws,
                  slrme_stream_t stream);

/* ===================================================================== learned estimator
 * A small integer CNN that predicts the mantissas from the decoded SDRI and
 * the exponent plane, a learned alternative to Eq. (8) (the paper's estimator
 * is the regression; this one is chosen per image only where its residuals
 * cost fewer bits, and the residual / lossless decoding of Sec. III-C is
 * unchanged).  Definition:
 *   input a0 (4 planes, int8): S_c - 128 (c = R, G, B) and
 *     clamp(E - 137 - J, -128, 127), J the image's tone-mapping key
 *     (rgbe_key_scale), sent as side information with the network's residuals;
 *   layers l = 1..4: 3x3 convolution with zero padding, channels
 *     4 -> 16 -> 16 -> 16 -> 3, acc = b + sum w a (exact integer),
 *     a' = clamp(floor((acc * m + 2^(shift-1)) / 2^shift), 0, hi) with hi = 127
 *     for layers 1-3 and 255 for layer 4, whose planes y_R, y_G, y_B correct the
 *     regression: M^_c = clamp(M*_c + y_c - 128, 0, 255), M* from Eq. (8).
 * Weights are int8 in [-127, 127]; m > 0 and 1 <= shift <= 30 (checked by the
 * caller); |acc| stays below 2^24. */
typedef struct slrme_cnn_net {
    int8_t  w1[16][4][9];      /* [out][in][3x3 tap, row-major] */
    int8_t  w2[16][16][9];
    int8_t  w3[16][16][9];
    int8_t  w4[3][16][9];
    int32_t b1[16], b2[16], b3[16], b4[3];
    int32_t m1[16], m2[16], m3[16], m4[3];
    int32_t shift[4];
    int32_t reserved;
} slrme_cnn_net;   /* 6044 bytes, 4-byte aligned (device memory) */

/* Output planes y (uint8 [3][h][w]) of the network for one image. */
int cnn_infer(const uint8_t* s_dec3, const uint8_t* e, int h, int w, int32_t J, const slrme_cnn_net* net,
              uint8_t* mhat3, slrme_stream_t stream);

/* Residuals R = M - M^ (int16 [3][h][w]) of the refined estimate M^ (the
 * image's regression `params` with restoration gf_on, corrected by the
 * network) and, if hist is not NULL, their histograms (cleared first). */
int cnn_residual_encode(const uint8_t* s_dec3, const uint8_t* m3, const uint8_t* e, int h, int w, int32_t J,
                        const slrme_cnn_net* net, const slrme_params* params, int gf_on, int16_t* r3,
                        uint32_t* hist, slrme_stream_t stream);

/* Decoder of those residuals: M = R + M^, repacked with E into RGBE words. */
int cnn_residual_decode(const uint8_t* s_dec3, const uint8_t* e, const int16_t* r3, int h, int w, int32_t J,
                        const slrme_cnn_net* net, const slrme_params* params, int gf_on, uint32_t* rgbe_out,
                        slrme_stream_t stream);

/* Training of the network (float32, on the device), used to produce its
 * weights from (decoded SDRI, exponent, mantissa) triples of the codec itself.
 * Tensors are [B][C][H][W] float32 (B crops of H x W); theta is the flat
 * parameter vector: for l = 1..4, w_l[out][in][3][3] then b_l[out] (5667
 * floats).  quant = 1 trains with fake quantisation (weights to int8 steps per
 * output channel, hidden activations to multiples of 1/8 in [0, 127/8],
 * straight-through gradients); quant = 0 is the plain ReLU network.  All
 * reductions run in a fixed order (no float atomics): results are
 * reproducible bit for bit.  ws: device workspace of
 * cnn_train_workspace_bytes(B, H, W) bytes shared by forward and backward. */
size_t cnn_train_workspace_bytes(int B, int H, int W);

/* Forward pass: x [B][4][H][W] -> out [B][3][H][W]; keeps activations in ws. */
int cnn_train_forward(const float* theta, const float* x, int B, int H, int W, int quant, float* ws, float* out,
                      slrme_stream_t stream);

/* Backward pass after cnn_train_forward on the same ws: grad (5667 floats) of
 * the loss whose gradient w.r.t. out is dout [B][3][H][W]. */
int cnn_train_backward(const float* x, const float* dout, int B, int H, int W, int quant, float* ws, float* grad,
                       slrme_stream_t stream);

/* Mean absolute error of out against target (n values): *loss (device float)
 * and dout = sign(out - target) / n.  ws: ceil(n / 256) floats. */
int cnn_loss_l1(const float* out, const float* target, int64_t n, float* dout, float* loss, float* ws,
                slrme_stream_t stream);

/* One bias-corrected Adam update of theta (n values) at step >= 1. */
int cnn_adam_step(float* theta, const float* grad, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                  int step, slrme_stream_t stream);

/* Training crops from coded images: crops[6 k ..] = (pixel offset of the
 * image's planes as in the batch layout, h, row pitch, y0, x0, J) for crop k;
 * writes x[k] = (S - 128, clamp(E - 137 - J, -128, 127)) and target[k] =
 * R + 128 with R = M - M* the regression's residual, as floats of CH x CW. */
int cnn_gather_crops(const uint8_t* s3, const uint8_t* e, const int16_t* r3, const int64_t* crops, int ncrops, int CH,
                     int CW, float* x, float* target, slrme_stream_t stream);

/* ===================================================================== batch form
 * Many images of uneven sizes coded together: one persistent launch per stage
 * (split, base round trip, fit + solve, residual; decode), tiles chosen by an
 * autotuner, and the whole chain capturable as one CUDA graph.  The paper
 * codes one image at a time; the batch form computes, image by image, exactly
 * what the single-image entry points compute.
 *
 * Layout: all images share batch planes, and every plane of image i has the
 * row pitch pitch_i = w_i rounded up to a multiple of 16 (so every row of
 * every plane starts on a 16-byte boundary and the row stages can stream
 * whole rows with bulk copies).  With n_i = h_i pitch_i, image i occupies
 * elements [px_offset_i, px_offset_i + n_i) of the word planes (rgbe, e,
 * rgbe_out), pixel (y, x) at px_offset_i + y pitch_i + x, and
 * [3 px_offset_i, 3 px_offset_i + 3 n_i) of the three-plane buffers (m3, s3,
 * r3: plane c of the image at 3 px_offset_i + c n_i).  The words of the
 * padding columns x = w_i .. pitch_i - 1 of rgbe must be 0 (the zero word:
 * no pixel), so they add nothing to the log-average statistic; the outputs
 * hold no defined values there.  params[i] and hist[i * 3 * 511 ...] hold
 * image i's parameters and histograms. */
typedef struct slrme_batch_image {
    int32_t h, w;         /* size: h, w >= 0, h*w < 2^31 */
    int32_t quality;      /* base-layer quality 1..100 */
    int32_t gf_on;        /* Gaussian restoration, 0 or 1 */
    int64_t px_offset;    /* OUT (slrme_batch_plan_init): first element of the image in the word planes,
                             a multiple of 256 */
    int32_t pitch;        /* OUT (slrme_batch_plan_init): row pitch of every plane of the image */
    int32_t reserved;
} slrme_batch_image;

typedef struct slrme_batch_tiles {
    int32_t split_ctas_per_sm;  /* persistent CTAs per SM: split 1..8 */
    int32_t base_ctas_per_sm;   /* base round trip 1..3 */
} slrme_batch_tiles;

/* Host-side plan; the caller owns the struct, the images array (kept alive
 * while the plan is used) and the device workspace. */
typedef struct slrme_batch_plan {
    int32_t n_images;
    int64_t total_px;                   /* pixels of a word plane (images + alignment padding) */
    const slrme_batch_image* images;
    void* workspace;                    /* device, slrme_batch_workspace_bytes(n_images), 256-byte aligned */
    slrme_batch_tiles tiles;
    int64_t split_chunks, base_tasks, tile_rows;   /* task counts (tile_rows: rows of 2048-column strips) */
    void* graph;                        /* instantiated CUDA graph (cudaGraphExec_t) or NULL */
} slrme_batch_plan;

/* Device buffers of one batch (all device pointers, caller-owned).  The
 * planes (rgbe, m3, e, s3, r3, rgbe_out) must be 16-byte aligned, params and
 * hist 4-byte aligned.  Sizes: rgbe, e, rgbe_out: total_px elements; m3, s3,
 * r3: 3 total_px; params: n_images; hist: n_images * 3 * 511 (or NULL). */
typedef struct slrme_batch_buffers {
    const uint32_t* rgbe;
    uint8_t* m3;
    uint8_t* e;
    uint8_t* s3;
    int16_t* r3;
    slrme_params* params;
    uint32_t* hist;
    uint32_t* rgbe_out;
} slrme_batch_buffers;

/* Workspace bytes for n_images images (descriptors, quantiser tables, task
 * tables, per-image statistics and bin sums). */
size_t slrme_batch_workspace_bytes(int n_images);

/* Most images in one plan (the per-image solve runs as one grid row per image). */
#define SLRME_BATCH_MAX_IMAGES 65535

/* Lays the images out (sets images[i].px_offset), uploads descriptors and task
 * tables to the workspace with default tiles.  Synchronises `stream`.
 * SLRME_EINVAL for 1 > n_images or n_images > SLRME_BATCH_MAX_IMAGES. */
int slrme_batch_plan_init(slrme_batch_plan* plan, slrme_batch_image* images, int n_images, void* workspace,
                          slrme_stream_t stream);

/* Sets the tiles (validated) and re-uploads the task tables.  Synchronises `stream`. */
int slrme_batch_set_tiles(slrme_batch_plan* plan, const slrme_batch_tiles* tiles, slrme_stream_t stream);

/* Encoder over the batch: split, base round trip, fit + solve, residual
 * (hist may be NULL); asynchronous on `stream`. */
int slrme_batch_encode(const slrme_batch_plan* plan, const slrme_batch_buffers* bufs, slrme_stream_t stream);

/* Decoder over the batch (reads s3, e, r3, params; writes rgbe_out). */
int slrme_batch_decode(const slrme_batch_plan* plan, const slrme_batch_buffers* bufs, slrme_stream_t stream);

/* Times the split and base stages over candidate grid sizes on this batch
 * (`reps` runs each, best time) and keeps the fastest; synchronous,
 * overwrites the buffers' outputs.  The coded results never depend on the
 * tiles.  (The fit, residual and decoder stages stream whole rows through
 * shared-memory rings at a fixed two CTAs per SM.) */
int slrme_batch_autotune(slrme_batch_plan* plan, const slrme_batch_buffers* bufs, int reps, slrme_stream_t stream);

/* Copies the per-image log-average statistics of the last encode (int64
 * [n_images][2], as rgbe_split defines them) to host memory; synchronous. */
int slrme_batch_lum_stats(const slrme_batch_plan* plan, int64_t* stats_host, slrme_stream_t stream);

/* Captures encode + decode on `stream` (a created stream, not the legacy
 * default stream) into a CUDA graph bound to these buffers and instantiates
 * it into plan->graph, replacing any previous graph. */
int slrme_batch_graph_build(slrme_batch_plan* plan, const slrme_batch_buffers* bufs, slrme_stream_t stream);

/* Launches plan->graph on `stream`. */
int slrme_batch_graph_launch(const slrme_batch_plan* plan, slrme_stream_t stream);

/* Destroys plan->graph (if any). */
int slrme_batch_graph_destroy(slrme_batch_plan* plan);

/* Host, no GPU: copies the library's own constant tables (built by the
 * library's host code) for inspection: log2_lut[2048] = round(65536 log2(2048+i)),
 * gamma[256] thresholds (gamma[k] = float(((k-0.5)/255)^2.2), gamma[0] = 0),
 * kr[16] = float(0.18 2^(-r/16)), wr[16] = float(1800 2^(-r/16)),
 * quant[64] the steps for `quality` (row-major, vertical frequency first),
 * dct[64] = round(4096 alpha_u cos((2x+1) u pi / 16)) (row u).  Any pointer
 * may be NULL.  Returns SLRME_EINVAL for a quality outside 1..100. */
int slrme_host_tables(int32_t* log2_lut, float* gamma, float* kr, float* wr,
                      int quality, int32_t* quant, int32_t* dct);

/* Device status word of the current device (synchronous): 0, or a mask of
 * bit 0 (1): a kernel's wait for its own bulk copies gave up after its bound
 *   (the kernel then stopped and its outputs are incomplete);
 * bit 1 (2): the rANS coder met input outside its table or a corrupt stream;
 * bit 2 (4): jpeg_huffman_bits met a level beyond the baseline categories.
 * clear != 0 resets it. */
int slrme_device_status(int* status, int clear);

/* Self-test of the bounded waits the TMA-staged kernels use (the paper has
 * no counterpart): launches one warp that waits on a shared-memory mbarrier
 * for at most max_spins polls (1 .. 2^20).  arrive = 0: nothing arrives, so
 * the wait gives up, sets bit 0 of the device status word (see
 * slrme_device_status) and the kernel returns, leaving the context usable;
 * arrive = 1: the barrier completes and the status word is untouched.
 * Asynchronous on `stream`; SLRME_EINVAL for arguments out of range. */
int slrme_wait_probe(int max_spins, int arrive, slrme_stream_t stream);

/* Text of the last error reported to the calling thread ("" if none). */
const char* slrme_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SLRME_H */
