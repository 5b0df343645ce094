// Training of the learned estimator on the GPU, in float32.
//
// The float network mirrors the integer one (4 -> 16 -> 16 -> 16 -> 3, 3x3,
// zero padding) with fake quantisation: weights to int8 steps per output
// channel (s = max|w| / 127), hidden activations to multiples of 1/8 in
// [0, 127/8], straight-through gradients inside the range.  quant = 0 turns
// the quantisers off (plain ReLU network) for gradient checks.
//
// Layout: tensors are [B][C][H][W] float32; the flat parameter vector holds,
// for l = 1..4, w_l[co][ci][3][3] then b_l[co] (5667 floats).  Every
// reduction (weight gradients, loss) runs in a fixed order, two passes, no
// float atomics, so a training run is bit-reproducible.
#include "slrme_internal.cuh"

namespace slrme {
namespace {

// channels at depth i: 4, 16, 16, 16, 3
__host__ __device__ constexpr int ch(int i) { return i == 0 ? 4 : (i == 4 ? 3 : 16); }
constexpr float kScaleA = 0.125f;
constexpr int kThreadsT = 256;
constexpr int kNParams = 5667;
constexpr int kNParamsCheck = kNParams;
constexpr int kChunkPx = 4096;   // pixels per partial of the weight-gradient reduction

__host__ __device__ constexpr int woff(int l) {   // offset of w_l (layer l = 0..3) in the flat vector
    return l == 0 ? 0 : woff(l - 1) + ch(l) * ch(l - 1) * 9 + ch(l);
}
__host__ __device__ constexpr int boff(int l) { return woff(l) + ch(l + 1) * ch(l) * 9; }
static_assert(boff(3) + 3 == kNParamsCheck, "flat parameter layout");

// Fake-quantised weights (or a copy) and biases: one thread per output channel.
__global__ void k_fq_weights(const float* __restrict__ theta, float* __restrict__ wq, int quant) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    int l = 0, co = t;
    while (l < 4 && co >= ch(l + 1)) {
        co -= ch(l + 1);
        ++l;
    }
    if (l >= 4) return;
    const int K = ch(l) * 9;
    const float* w = theta + woff(l) + co * K;
    float* q = wq + woff(l) + co * K;
    float s = 0.0f;
    for (int k = 0; k < K; ++k) s = fmaxf(s, fabsf(w[k]));
    s = s > 0.0f ? s / 127.0f : 1.0f;
    for (int k = 0; k < K; ++k) q[k] = quant ? rintf(w[k] / s) * s : w[k];
    wq[boff(l) + co] = theta[boff(l) + co];
}

__device__ __forceinline__ float act_fwd(float z, int quant) {
    if (!quant) return fmaxf(z, 0.0f);
    return fminf(fmaxf(rintf(z / kScaleA), 0.0f), 127.0f) * kScaleA;
}

__device__ __forceinline__ float act_mask(float z, int quant) {
    if (!quant) return z > 0.0f ? 1.0f : 0.0f;
    const float q = z / kScaleA;
    return (q > 0.0f && q < 127.5f) ? 1.0f : 0.0f;
}

// Forward of one layer: z = conv(in) + b; hidden layers also write a = act(z).
template <int CI, int CO, bool HIDDEN>
__global__ void __launch_bounds__(kThreadsT) k_conv_fwd(const float* __restrict__ in, const float* __restrict__ wq,
                                                        int l, int B, int H, int W, float* __restrict__ z,
                                                        float* __restrict__ a, int quant) {
    __shared__ float sw[CO * CI * 9], sb[CO];
    for (int i = threadIdx.x; i < CO * CI * 9; i += blockDim.x) sw[i] = wq[woff(l) + i];
    for (int i = threadIdx.x; i < CO; i += blockDim.x) sb[i] = wq[boff(l) + i];
    __syncthreads();
    const int64_t hw = (int64_t)H * W;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)B * hw) return;
    const int b = (int)(p / hw);
    const int y = (int)((p % hw) / W), x = (int)(p % W);
    float acc[CO];
#pragma unroll
    for (int o = 0; o < CO; ++o) acc[o] = sb[o];
    for (int c = 0; c < CI; ++c) {
        const float* plane = in + ((int64_t)b * CI + c) * hw;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
            const float v = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? plane[(int64_t)yy * W + xx] : 0.0f;
#pragma unroll
            for (int o = 0; o < CO; ++o) acc[o] = fmaf(sw[(o * CI + c) * 9 + t], v, acc[o]);
        }
    }
#pragma unroll
    for (int o = 0; o < CO; ++o) {
        const int64_t idx = ((int64_t)b * CO + o) * hw + (int64_t)y * W + x;
        z[idx] = acc[o];
        if (HIDDEN) a[idx] = act_fwd(acc[o], quant);
    }
}

// Gradient w.r.t. the layer input, times the previous layer's activation
// mask (so the result is the upstream gradient of the previous layer).
template <int CI, int CO>
__global__ void __launch_bounds__(kThreadsT) k_conv_bwd_data(const float* __restrict__ g, const float* __restrict__ wq,
                                                             int l, int B, int H, int W,
                                                             const float* __restrict__ zprev, int quant,
                                                             float* __restrict__ gprev) {
    __shared__ float sw[CO * CI * 9];
    for (int i = threadIdx.x; i < CO * CI * 9; i += blockDim.x) sw[i] = wq[woff(l) + i];
    __syncthreads();
    const int64_t hw = (int64_t)H * W;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)B * hw) return;
    const int b = (int)(p / hw);
    const int y = (int)((p % hw) / W), x = (int)(p % W);
    float acc[CI];
#pragma unroll
    for (int c = 0; c < CI; ++c) acc[c] = 0.0f;
    for (int o = 0; o < CO; ++o) {
        const float* plane = g + ((int64_t)b * CO + o) * hw;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = y - (t / 3 - 1), xx = x - (t % 3 - 1);
            const float v = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? plane[(int64_t)yy * W + xx] : 0.0f;
#pragma unroll
            for (int c = 0; c < CI; ++c) acc[c] = fmaf(sw[(o * CI + c) * 9 + t], v, acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < CI; ++c) {
        const int64_t idx = ((int64_t)b * CI + c) * hw + (int64_t)y * W + x;
        gprev[idx] = acc[c] * act_mask(zprev[idx], quant);
    }
}

// Partial weight and bias gradients of one chunk of pixels for one output
// channel and a group of 4 input channels: partial[chunk][co][ci][tap], and
// the bias partial in partial_b[chunk][co] (group 0 only).
template <int CI, int CO>
__global__ void __launch_bounds__(kThreadsT) k_conv_bwd_weight(const float* __restrict__ g,
                                                               const float* __restrict__ in, int B, int H, int W,
                                                               float* __restrict__ partial,
                                                               float* __restrict__ partial_b) {
    constexpr int G = CI < 4 ? CI : 4;
    const int chunk = blockIdx.x, co = blockIdx.y, c0 = blockIdx.z * G;
    const int64_t hw = (int64_t)H * W, total = (int64_t)B * hw;
    float acc[G * 9 + 1];
#pragma unroll
    for (int k = 0; k < G * 9 + 1; ++k) acc[k] = 0.0f;
    const int64_t p1 = min((int64_t)(chunk + 1) * kChunkPx, total);
    for (int64_t p = (int64_t)chunk * kChunkPx + threadIdx.x; p < p1; p += blockDim.x) {
        const int b = (int)(p / hw);
        const int y = (int)((p % hw) / W), x = (int)(p % W);
        const float gv = g[((int64_t)b * CO + co) * hw + (int64_t)y * W + x];
        acc[G * 9] += gv;
#pragma unroll
        for (int c = 0; c < G; ++c) {
            const float* plane = in + ((int64_t)b * CI + c0 + c) * hw;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
                const float v = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? plane[(int64_t)yy * W + xx] : 0.0f;
                acc[c * 9 + t] = fmaf(gv, v, acc[c * 9 + t]);
            }
        }
    }
    // block reduction in a fixed order: warp shuffles, then warps in order
    __shared__ float red[kThreadsT / 32][G * 9 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < G * 9 + 1; ++k) {
        float v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < G * 9 + 1; k += blockDim.x) {
        float v = 0.0f;
        for (int i = 0; i < kThreadsT / 32; ++i) v += red[i][k];
        if (k < G * 9) {
            const int c = k / 9, t = k % 9;
            partial[(((int64_t)chunk * CO + co) * CI + c0 + c) * 9 + t] = v;
        } else if (blockIdx.z == 0) {
            partial_b[(int64_t)chunk * CO + co] = v;
        }
    }
}

// Sums partials over chunks in chunk order: out[i] = sum_k partial[k][i].
__global__ void k_sum_chunks(const float* __restrict__ partial, int chunks, int n, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int k = 0; k < chunks; ++k) s += partial[(int64_t)k * n + i];
    out[i] = s;
}

// L1 loss: dout = sign(out - target) / n; per-block partial sums of |d|.
__global__ void __launch_bounds__(kThreadsT) k_loss_l1(const float* __restrict__ out, const float* __restrict__ tgt,
                                                       int64_t n, float* __restrict__ dout,
                                                       float* __restrict__ partial) {
    __shared__ float red[kThreadsT / 32];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float a = 0.0f;
    if (i < n) {
        const float d = out[i] - tgt[i];
        dout[i] = (d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f)) / (float)n;
        a = fabsf(d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int k = 0; k < kThreadsT / 32; ++k) s += red[k];
        partial[blockIdx.x] = s;
    }
}

__global__ void k_loss_final(const float* __restrict__ partial, int blocks, int64_t n, float* __restrict__ loss) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int k = 0; k < blocks; ++k) s += partial[k];
    *loss = (float)(s / (double)n);
}

__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Training crops: for crop k with origin (y0, x0) in image planes at pixel
// offset px (h x w, key J), x[k] = (S - 128, clamp(E - 137 - J)) and
// t[k] = R + 128 (the regression's residual, centred), as floats, CH x CW each.
__global__ void k_gather(const uint8_t* __restrict__ s3b, const uint8_t* __restrict__ eb,
                         const int16_t* __restrict__ r3b, const int64_t* __restrict__ crops, int ncrops, int CH,
                         int CW, float* __restrict__ x, float* __restrict__ t) {
    const int64_t hw = (int64_t)CH * CW;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)ncrops * hw) return;
    const int k = (int)(p / hw);
    const int yy = (int)((p % hw) / CW), xx = (int)(p % CW);
    const int64_t* c = crops + 6 * (int64_t)k;   // px, h, row pitch, y0, x0, J
    const int64_t px = c[0], h = c[1], w = c[2];
    const int64_t n = h * w, o = (c[3] + yy) * w + c[4] + xx;
    const uint8_t* s3 = s3b + 3 * px;
    const int16_t* r3 = r3b + 3 * px;
    int d = (int)eb[px + o] - 137 - (int)c[5];
    d = d < -128 ? -128 : (d > 127 ? 127 : d);
    float* xk = x + (int64_t)k * 4 * hw + (int64_t)yy * CW + xx;
    float* tk = t + (int64_t)k * 3 * hw + (int64_t)yy * CW + xx;
    for (int ch = 0; ch < 3; ++ch) {
        xk[ch * hw] = (float)((int)s3[ch * n + o] - 128);
        tk[ch * hw] = (float)((int)r3[ch * n + o] + 128);
    }
    xk[3 * hw] = (float)d;
}

// Workspace of a training step for batch B x H x W.
struct TrainWs {
    float *wq, *z[4], *a[3], *g0, *g1, *partial, *partial_b, *grad_tmp;
};

int64_t chunks_of(int B, int H, int W) { return ((int64_t)B * H * W + kChunkPx - 1) / kChunkPx; }

size_t ws_floats(int B, int H, int W) {
    const int64_t hw = (int64_t)B * H * W;
    return (size_t)kNParams + 16 * hw * 3 + 3 * hw + 16 * hw * 3 + 16 * hw * 2 +
           (size_t)chunks_of(B, H, W) * (16 * 16 * 9) + (size_t)chunks_of(B, H, W) * 16 + kNParams + 64;
}

TrainWs carve(float* ws, int B, int H, int W) {
    const int64_t hw = (int64_t)B * H * W;
    TrainWs T;
    float* p = ws;
    T.wq = p; p += kNParams;
    for (int l = 0; l < 3; ++l) { T.z[l] = p; p += 16 * hw; }
    T.z[3] = p; p += 3 * hw;
    for (int l = 0; l < 3; ++l) { T.a[l] = p; p += 16 * hw; }
    T.g0 = p; p += 16 * hw;
    T.g1 = p; p += 16 * hw;
    T.partial = p; p += chunks_of(B, H, W) * (16 * 16 * 9);
    T.partial_b = p; p += chunks_of(B, H, W) * 16;
    T.grad_tmp = p;
    return T;
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreadsT - 1) / kThreadsT); }

template <int CI, int CO>
int weight_grad(const float* g, const float* in, int l, int B, int H, int W, const TrainWs& T, float* grad,
                cudaStream_t s) {
    const int chunks = (int)chunks_of(B, H, W);
    constexpr int G = CI < 4 ? CI : 4;
    k_conv_bwd_weight<CI, CO><<<dim3(chunks, CO, CI / G), kThreadsT, 0, s>>>(g, in, B, H, W, T.partial, T.partial_b);
    k_sum_chunks<<<blocks_for(CO * CI * 9), kThreadsT, 0, s>>>(T.partial, chunks, CO * CI * 9, grad + woff(l));
    k_sum_chunks<<<1, kThreadsT, 0, s>>>(T.partial_b, chunks, CO, grad + boff(l));
    return cuda_status("cnn weight gradient launch");
}

}  // namespace
}  // namespace slrme

using namespace slrme;

extern "C" {

size_t cnn_train_workspace_bytes(int B, int H, int W) {
    if (B < 1 || H < 1 || W < 1) return 0;
    return sizeof(float) * ws_floats(B, H, W);
}

int cnn_train_forward(const float* theta, const float* x, int B, int H, int W, int quant, float* ws, float* out,
                      slrme_stream_t stream) {
    if (!theta || !x || !ws || !out || B < 1 || H < 1 || W < 1 || (int64_t)B * H * W >= ((int64_t)1 << 31)) {
        set_error("cnn_train_forward: bad arguments");
        return SLRME_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const TrainWs T = carve(ws, B, H, W);
    const int64_t n = (int64_t)B * H * W;
    k_fq_weights<<<1, 64, 0, s>>>(theta, T.wq, quant);
    k_conv_fwd<4, 16, true><<<blocks_for(n), kThreadsT, 0, s>>>(x, T.wq, 0, B, H, W, T.z[0], T.a[0], quant);
    k_conv_fwd<16, 16, true><<<blocks_for(n), kThreadsT, 0, s>>>(T.a[0], T.wq, 1, B, H, W, T.z[1], T.a[1], quant);
    k_conv_fwd<16, 16, true><<<blocks_for(n), kThreadsT, 0, s>>>(T.a[1], T.wq, 2, B, H, W, T.z[2], T.a[2], quant);
    k_conv_fwd<16, 3, false><<<blocks_for(n), kThreadsT, 0, s>>>(T.a[2], T.wq, 3, B, H, W, out, nullptr, quant);
    return cuda_status("cnn_train_forward launch");
}

int cnn_train_backward(const float* x, const float* dout, int B, int H, int W, int quant, float* ws, float* grad,
                       slrme_stream_t stream) {
    if (!x || !dout || !ws || !grad || B < 1 || H < 1 || W < 1 || (int64_t)B * H * W >= ((int64_t)1 << 31)) {
        set_error("cnn_train_backward: bad arguments");
        return SLRME_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const TrainWs T = carve(ws, B, H, W);
    const int64_t n = (int64_t)B * H * W;
    int st = weight_grad<16, 3>(dout, T.a[2], 3, B, H, W, T, grad, s);
    k_conv_bwd_data<16, 3><<<blocks_for(n), kThreadsT, 0, s>>>(dout, T.wq, 3, B, H, W, T.z[2], quant, T.g0);
    if (st == SLRME_OK) st = weight_grad<16, 16>(T.g0, T.a[1], 2, B, H, W, T, grad, s);
    k_conv_bwd_data<16, 16><<<blocks_for(n), kThreadsT, 0, s>>>(T.g0, T.wq, 2, B, H, W, T.z[1], quant, T.g1);
    if (st == SLRME_OK) st = weight_grad<16, 16>(T.g1, T.a[0], 1, B, H, W, T, grad, s);
    k_conv_bwd_data<16, 16><<<blocks_for(n), kThreadsT, 0, s>>>(T.g1, T.wq, 1, B, H, W, T.z[0], quant, T.g0);
    if (st == SLRME_OK) st = weight_grad<4, 16>(T.g0, x, 0, B, H, W, T, grad, s);
    if (st != SLRME_OK) return st;
    return cuda_status("cnn_train_backward launch");
}

int cnn_loss_l1(const float* out, const float* target, int64_t n, float* dout, float* loss, float* ws,
                slrme_stream_t stream) {
    if (!out || !target || !dout || !loss || !ws || n < 1 || n >= ((int64_t)1 << 31)) {
        set_error("cnn_loss_l1: bad arguments");
        return SLRME_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = blocks_for(n);
    k_loss_l1<<<blocks, kThreadsT, 0, s>>>(out, target, n, dout, ws);
    k_loss_final<<<1, 32, 0, s>>>(ws, (int)blocks, n, loss);
    return cuda_status("cnn_loss_l1 launch");
}

int cnn_adam_step(float* theta, const float* grad, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                  int step, slrme_stream_t stream) {
    if (!theta || !grad || !m || !v || n < 1 || step < 1) {
        set_error("cnn_adam_step: bad arguments");
        return SLRME_EINVAL;
    }
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<blocks_for(n), kThreadsT, 0, (cudaStream_t)stream>>>(theta, grad, m, v, n, lr, b1, b2, eps, c1, c2);
    return cuda_status("cnn_adam_step launch");
}

int cnn_gather_crops(const uint8_t* s3, const uint8_t* e, const int16_t* r3, const int64_t* crops, int ncrops, int CH,
                     int CW, float* x, float* target, slrme_stream_t stream) {
    if (!s3 || !e || !r3 || (uintptr_t)r3 % 2 || !crops || !x || !target || ncrops < 1 || CH < 1 || CW < 1 ||
        (int64_t)ncrops * CH * CW >= ((int64_t)1 << 31)) {
        set_error("cnn_gather_crops: bad arguments");
        return SLRME_EINVAL;
    }
    k_gather<<<blocks_for((int64_t)ncrops * CH * CW), kThreadsT, 0, (cudaStream_t)stream>>>(s3, e, r3, crops, ncrops,
                                                                                           CH, CW, x, target);
    return cuda_status("cnn_gather_crops launch");
}

}  // extern "C"
