// Batch runtime: many images of uneven sizes coded with one persistent launch
// per stage, a tile autotuner, and CUDA-graph capture of the whole chain.
//
// A plan lays the images out in shared batch planes (each image's first pixel
// aligned to 256 pixels, every row of every plane to 16 bytes: the row pitch
// is w rounded up to 16), writes the device descriptors and the per-stage
// task prefix tables into a caller-provided workspace, and holds the tile
// choice.  Stage kernels (split.cu, base.cu, slr.cu) map their task index to
// an image by binary search over a prefix table.
#include <string.h>

#include <vector>

#include "slrme_internal.cuh"

namespace slrme {
namespace {

static_assert(sizeof(slrme_batch_image) == 32 && sizeof(slrme_batch_tiles) == 8, "batch ABI structs");
static_assert(sizeof(slrme_batch_plan) == 72 && sizeof(slrme_batch_buffers) == 64, "batch ABI structs");
static_assert(sizeof(BatchImage) == sizeof(slrme_batch_image), "device image descriptor");

constexpr int64_t kAlignPx = 256;
constexpr int kPitchAlign = 16;
constexpr size_t kSection = 256;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
    size_t img, quant, split_prefix, base_prefix, row_prefix, lum, sums, total;
};

Layout layout(int n) {
    Layout L;
    size_t o = 0;
    L.img = o;
    o = round_up(o + sizeof(BatchImage) * (size_t)n, kSection);
    L.quant = o;
    o = round_up(o + sizeof(QuantTable) * (size_t)n, kSection);
    L.split_prefix = o;
    o = round_up(o + sizeof(int64_t) * (size_t)(n + 1), kSection);
    L.base_prefix = o;
    o = round_up(o + sizeof(int64_t) * (size_t)(n + 1), kSection);
    L.row_prefix = o;
    o = round_up(o + sizeof(int64_t) * (size_t)(n + 1), kSection);
    L.lum = o;
    o = round_up(o + sizeof(int64_t) * 2 * (size_t)n, kSection);
    L.sums = o;
    o = round_up(o + sizeof(unsigned long long) * kNbin * kNsum * (size_t)n, kSection);
    L.total = o;
    return L;
}

BatchDev device_view(const slrme_batch_plan* p) {
    const Layout L = layout(p->n_images);
    char* base = static_cast<char*>(p->workspace);
    BatchDev B;
    B.img = reinterpret_cast<const BatchImage*>(base + L.img);
    B.quant = reinterpret_cast<const QuantTable*>(base + L.quant);
    B.split_prefix = reinterpret_cast<const int64_t*>(base + L.split_prefix);
    B.base_prefix = reinterpret_cast<const int64_t*>(base + L.base_prefix);
    B.row_prefix = reinterpret_cast<const int64_t*>(base + L.row_prefix);
    B.lum_stats = reinterpret_cast<int64_t*>(base + L.lum);
    B.sums = reinterpret_cast<unsigned long long*>(base + L.sums);
    B.n = p->n_images;
    return B;
}

bool tiles_valid(const slrme_batch_tiles& t) {
    return t.split_ctas_per_sm >= 1 && t.split_ctas_per_sm <= 8 && t.base_ctas_per_sm >= 1 &&
           t.base_ctas_per_sm <= 3;
}

int pitch_of(int w) { return (w + kPitchAlign - 1) / kPitchAlign * kPitchAlign; }

// Task prefix tables, uploaded synchronously: split chunks of 4096 words over
// each image's pitched plane, base CTA tasks of 8 bands of 8 x 32 pixels, and
// the rows of 2048-column strips of the row stages.
int upload_prefixes(slrme_batch_plan* p, cudaStream_t s) {
    const int n = p->n_images;
    std::vector<int64_t> sp(n + 1), bp(n + 1), rp(n + 1);
    sp[0] = bp[0] = rp[0] = 0;
    for (int i = 0; i < n; ++i) {
        const slrme_batch_image& im = p->images[i];
        const int64_t px = (int64_t)im.h * im.w;
        const int64_t words = (int64_t)im.h * pitch_of(im.w);
        const int64_t chunks = (words + kSplitChunk - 1) / kSplitChunk;
        const int64_t bands = (int64_t)((im.h + 7) / 8) * ((im.w + 31) / 32);
        const int64_t rows = px ? (int64_t)((im.w + kTileColsBatch - 1) / kTileColsBatch) * im.h : 0;
        sp[i + 1] = sp[i] + chunks;
        bp[i + 1] = bp[i] + (px ? (bands + 7) / 8 : 0);
        rp[i + 1] = rp[i] + rows;
    }
    const Layout L = layout(n);
    char* base = static_cast<char*>(p->workspace);
    if (cudaMemcpyAsync(base + L.split_prefix, sp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(base + L.base_prefix, bp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(base + L.row_prefix, rp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        return cuda_status("batch plan upload");
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_status("batch plan upload");
    p->split_chunks = sp[n];
    p->base_tasks = bp[n];
    p->tile_rows = rp[n];
    return SLRME_OK;
}

bool buffers_ok(const slrme_batch_plan* p, const slrme_batch_buffers* b, bool encode, bool decode) {
    if (!p || !b || !p->workspace || p->n_images < 1) {
        set_error("batch: null or uninitialised plan / buffers");
        return false;
    }
    if (p->total_px > 0) {
        if (encode && !(b->rgbe && b->m3 && b->e && b->s3 && b->r3)) {
            set_error("batch encode: null plane pointer");
            return false;
        }
        if (decode && !(b->s3 && b->e && b->r3 && b->rgbe_out)) {
            set_error("batch decode: null plane pointer");
            return false;
        }
    }
    auto a16 = [](const void* q) { return q == nullptr || (uintptr_t)q % 16 == 0; };
    if (!b->params || (uintptr_t)b->params % 4 || (b->hist && (uintptr_t)b->hist % 4) || !a16(b->rgbe) ||
        !a16(b->m3) || !a16(b->e) || !a16(b->s3) || !a16(b->r3) || !a16(b->rgbe_out)) {
        set_error("batch: params/hist must be 4-byte aligned, the planes 16-byte aligned");
        return false;
    }
    return true;
}

// Restoration over the batch's images with pixels: 0 none, 1 all, 2 mixed.
int gf_mode(const slrme_batch_plan* p) {
    bool any_on = false, any_off = false;
    for (int i = 0; i < p->n_images; ++i) {
        const slrme_batch_image& im = p->images[i];
        if ((int64_t)im.h * im.w == 0) continue;
        (im.gf_on ? any_on : any_off) = true;
    }
    return any_on && any_off ? 2 : (any_on ? 1 : 0);
}

int encode_stages(const slrme_batch_plan* p, const slrme_batch_buffers* b, cudaStream_t s) {
    const BatchDev B = device_view(p);
    const slrme_batch_tiles& t = p->tiles;
    int st = launch_split_batch(B, p->split_chunks, t.split_ctas_per_sm, b->rgbe, b->m3, b->e, s);
    if (st == SLRME_OK) st = launch_base_batch(B, p->base_tasks, t.base_ctas_per_sm, b->m3, b->e, b->s3, s);
    const int gm = gf_mode(p);
    if (st == SLRME_OK) st = launch_fit_batch(B, p->tile_rows, gm, b->s3, b->m3, b->e, b->params, s);
    if (st == SLRME_OK)
        st = launch_residual_batch(B, p->tile_rows, gm, b->s3, b->m3, b->e, b->params, b->r3, b->hist, s);
    return st;
}

int decode_stage(const slrme_batch_plan* p, const slrme_batch_buffers* b, cudaStream_t s) {
    const BatchDev B = device_view(p);
    return launch_decode_batch(B, p->tile_rows, gf_mode(p), b->s3, b->e, b->r3, b->params, b->rgbe_out, s);
}

}  // namespace
}  // namespace slrme

using namespace slrme;

extern "C" {

size_t slrme_batch_workspace_bytes(int n_images) { return n_images < 1 ? 0 : layout(n_images).total; }

int slrme_batch_plan_init(slrme_batch_plan* plan, slrme_batch_image* images, int n_images, void* workspace,
                          slrme_stream_t stream) {
    if (!plan || !images || !workspace || n_images < 1) {
        set_error("slrme_batch_plan_init: null pointer or no images");
        return SLRME_EINVAL;
    }
    if (n_images > SLRME_BATCH_MAX_IMAGES) {
        set_error("slrme_batch_plan_init: %d images, at most %d per plan", n_images, SLRME_BATCH_MAX_IMAGES);
        return SLRME_EINVAL;
    }
    if ((uintptr_t)workspace % kSection) {
        set_error("slrme_batch_plan_init: workspace must be 256-byte aligned");
        return SLRME_EINVAL;
    }
    std::vector<BatchImage> dev(n_images);
    std::vector<QuantTable> quant(n_images);
    int64_t px = 0;
    for (int i = 0; i < n_images; ++i) {
        slrme_batch_image& im = images[i];
        if (im.h < 0 || im.w < 0 || (int64_t)im.h * im.w >= ((int64_t)1 << 31) || (im.gf_on != 0 && im.gf_on != 1) ||
            !quant_table(im.quality, &quant[i])) {
            set_error("slrme_batch_plan_init: image %d has a bad size (%d x %d), quality (%d) or gf_on (%d)", i,
                      im.h, im.w, im.quality, im.gf_on);
            return SLRME_EINVAL;
        }
        im.px_offset = px;
        im.pitch = pitch_of(im.w);
        im.reserved = 0;
        dev[i] = BatchImage{im.h, im.w, im.quality, im.gf_on, px, im.pitch, 0};
        px += ((int64_t)im.h * im.pitch + kAlignPx - 1) / kAlignPx * kAlignPx;
    }
    plan->n_images = n_images;
    plan->total_px = px;
    plan->images = images;
    plan->workspace = workspace;
    plan->tiles = slrme_batch_tiles{4, 3};
    plan->graph = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    const Layout L = layout(n_images);
    char* base = static_cast<char*>(workspace);
    if (cudaMemcpyAsync(base + L.img, dev.data(), sizeof(BatchImage) * n_images, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(base + L.quant, quant.data(), sizeof(QuantTable) * n_images, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        return cuda_status("slrme_batch_plan_init upload");
    return upload_prefixes(plan, s);
}

int slrme_batch_set_tiles(slrme_batch_plan* plan, const slrme_batch_tiles* tiles, slrme_stream_t stream) {
    if (!plan || !tiles || !plan->workspace || !tiles_valid(*tiles)) {
        set_error("slrme_batch_set_tiles: bad plan or tiles");
        return SLRME_EINVAL;
    }
    plan->tiles = *tiles;
    return upload_prefixes(plan, (cudaStream_t)stream);
}

int slrme_batch_encode(const slrme_batch_plan* plan, const slrme_batch_buffers* bufs, slrme_stream_t stream) {
    if (!buffers_ok(plan, bufs, true, false)) return SLRME_EINVAL;
    return encode_stages(plan, bufs, (cudaStream_t)stream);
}

int slrme_batch_decode(const slrme_batch_plan* plan, const slrme_batch_buffers* bufs, slrme_stream_t stream) {
    if (!buffers_ok(plan, bufs, false, true)) return SLRME_EINVAL;
    return decode_stage(plan, bufs, (cudaStream_t)stream);
}

// Times the split and base stages over candidate grid sizes on the caller's
// batch and keeps the fastest; synchronous.  Results do not depend on the
// tiles, only speed.
int slrme_batch_autotune(slrme_batch_plan* plan, const slrme_batch_buffers* bufs, int reps, slrme_stream_t stream) {
    if (!buffers_ok(plan, bufs, true, true) || reps < 1) {
        if (reps < 1) set_error("slrme_batch_autotune: reps must be >= 1");
        return SLRME_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_status("slrme_batch_autotune events");
    int st = SLRME_OK;
    // best time of one stage function over `reps` runs
    auto timeit = [&](auto&& fn, float* best) -> int {
        *best = 1e30f;
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(e0, s);
            const int rc = fn();
            cudaEventRecord(e1, s);
            if (rc != SLRME_OK) return rc;
            if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_status("slrme_batch_autotune sync");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < *best) *best = ms;
        }
        return SLRME_OK;
    };
    slrme_batch_tiles best = plan->tiles;
    float t = 0.0f, tb;
    // split and base depend only on their own grid size
    tb = 1e30f;
    for (int c : {2, 4, 8}) {
        plan->tiles.split_ctas_per_sm = c;
        const BatchDev B = device_view(plan);
        st = timeit([&] { return launch_split_batch(B, plan->split_chunks, c, bufs->rgbe, bufs->m3, bufs->e, s); }, &t);
        if (st != SLRME_OK) goto done;
        if (t < tb) { tb = t; best.split_ctas_per_sm = c; }
    }
    plan->tiles.split_ctas_per_sm = best.split_ctas_per_sm;
    tb = 1e30f;
    for (int c : {1, 2, 3}) {
        const BatchDev B = device_view(plan);
        st = timeit([&] { return launch_base_batch(B, plan->base_tasks, c, bufs->m3, bufs->e, bufs->s3, s); }, &t);
        if (st != SLRME_OK) goto done;
        if (t < tb) { tb = t; best.base_ctas_per_sm = c; }
    }
    plan->tiles.base_ctas_per_sm = best.base_ctas_per_sm;
    st = slrme_batch_set_tiles(plan, &best, stream);
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SLRME_OK) slrme_batch_set_tiles(plan, &best, stream);
    return st;
}

int slrme_batch_lum_stats(const slrme_batch_plan* plan, int64_t* stats_host, slrme_stream_t stream) {
    if (!plan || !plan->workspace || !stats_host) {
        set_error("slrme_batch_lum_stats: null pointer");
        return SLRME_EINVAL;
    }
    const BatchDev B = device_view(plan);
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(stats_host, B.lum_stats, sizeof(int64_t) * 2 * (size_t)plan->n_images, cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_status("slrme_batch_lum_stats");
    return SLRME_OK;
}

// Captures encode + decode of the batch on `stream` (which must not be the
// legacy default stream) into a CUDA graph and instantiates it.
int slrme_batch_graph_build(slrme_batch_plan* plan, const slrme_batch_buffers* bufs, slrme_stream_t stream) {
    if (!buffers_ok(plan, bufs, true, true)) return SLRME_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) {
        set_error("slrme_batch_graph_build: needs a created stream (capture is not allowed on the legacy stream)");
        return SLRME_EINVAL;
    }
    slrme_batch_graph_destroy(plan);
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return cuda_status("slrme_batch_graph_build begin capture");
    int st = encode_stages(plan, bufs, s);
    if (st == SLRME_OK) st = decode_stage(plan, bufs, s);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    if (st != SLRME_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ec != cudaSuccess || !g) return cuda_status("slrme_batch_graph_build end capture");
    cudaGraphExec_t x = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return cuda_status("slrme_batch_graph_build instantiate");
    plan->graph = x;
    return SLRME_OK;
}

int slrme_batch_graph_launch(const slrme_batch_plan* plan, slrme_stream_t stream) {
    if (!plan || !plan->graph) {
        set_error("slrme_batch_graph_launch: no graph (call slrme_batch_graph_build)");
        return SLRME_EINVAL;
    }
    if (cudaGraphLaunch((cudaGraphExec_t)plan->graph, (cudaStream_t)stream) != cudaSuccess)
        return cuda_status("slrme_batch_graph_launch");
    return SLRME_OK;
}

int slrme_batch_graph_destroy(slrme_batch_plan* plan) {
    if (!plan) return SLRME_EINVAL;
    if (plan->graph) cudaGraphExecDestroy((cudaGraphExec_t)plan->graph);
    plan->graph = nullptr;
    return SLRME_OK;
}

}  // extern "C"
