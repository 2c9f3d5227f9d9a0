// k_mlp.cu -- the cost model's network: a 3-layer perceptron, FP32, hidden width 128.
//
//   z1 = x W1 + b1, h1 = relu(z1);  z2 = h1 W2 + b2, h2 = relu(z2);  y = h2 W3 + b3
//
// W1 is F x H, W2 is H x H, W3 is H x 1, all row-major with the input index first.  The
// parameters live in one flat FP32 array [W1 | b1 | W2 | b2 | W3 | b3].  Inputs are
// standardised on load, x' = (x - mu) * inv_sd, targets likewise, t' = (t - ym) * inv_ys.
//
// One CTA of 128 threads takes a tile of 32 rows; thread o owns hidden unit o.  The forward
// pass keeps z2 in registers and h1 in shared memory, so the backward pass of the tile runs
// in the same launch without storing activations.  Each CTA writes its whole gradient (all
// P parameters, plus its squared-error sum) to its own slot of a partial buffer; a second
// kernel sums the slots in a fixed order (deterministic) and either returns the gradient or
// applies one Adam step (Kingma & Ba, Algorithm 1) to the parameters.
#include <cuda_runtime.h>

#include <cstdio>

#include "qs_internal.h"

namespace qs {
namespace {

constexpr int kH = kMlpHidden;  // 128
constexpr int kR = 32;          // rows per tile
constexpr int kW2Pitch = kH + 1;

struct MlpOffsets {
    int w1, b1, w2, b2, w3, b3;
};

__host__ __device__ inline MlpOffsets mlp_offsets(int F)
{
    MlpOffsets o;
    o.w1 = 0;
    o.b1 = F * kH;
    o.w2 = o.b1 + kH;
    o.b2 = o.w2 + kH * kH;
    o.w3 = o.b2 + kH;
    o.b3 = o.w3 + kH;
    return o;
}

constexpr size_t tile_smem_bytes()
{
    return sizeof(float) * (size_t(kH) * kW2Pitch    // W2
                            + size_t(kR) * (kMlpMaxFeatures + 1)  // x tile
                            + size_t(kR) * kH        // h1
                            + size_t(kR) * kH        // d2 (backward) / scratch
                            + 4 * kR                 // per-warp row sums
                            + 2 * kR);               // y, dy
}

// TRAIN = false: write the tile's predictions (de-standardised) to y_out.
// TRAIN = true: write the tile's share of the gradient of the batch's mean squared error
// (standardised targets; scale = 2 / B) to partial[blockIdx.x * pstride + j] for every
// parameter j, and the tile's squared-error sum to slot nparams.
template <bool TRAIN>
__global__ void __launch_bounds__(kH) mlp_tile_kernel(MlpArgs a)
{
    extern __shared__ __align__(16) float sm[];
    float *W2s = sm;
    float *xs = W2s + kH * kW2Pitch;
    float *h1s = xs + kR * (kMlpMaxFeatures + 1);
    float *d2s = h1s + kR * kH;
    float *wsum = d2s + kR * kH;
    float *ys = wsum + 4 * kR;
    float *dys = ys + kR;
    const int o = threadIdx.x, F = a.F, xp = kMlpMaxFeatures + 1;
    const MlpOffsets off = mlp_offsets(F);
    const float *P = a.params;
    const int row0 = blockIdx.x * kR;

    if (TRAIN && a.step_counter && blockIdx.x == 0 && o == 0) *a.step_counter += 1;
    for (int i = o; i < kH * kH; i += kH) W2s[(i / kH) * kW2Pitch + (i % kH)] = P[off.w2 + i];
    for (int i = o; i < kR * F; i += kH) {
        const int r = i / F, f = i % F;
        const int row = row0 + r;
        xs[r * xp + f] = row < a.B ? (a.X[size_t(row) * F + f] - a.mu[f]) * a.inv_sd[f] : 0.f;
    }
    __syncthreads();

    // layer 1
    float acc[kR];
    {
        const float b = P[off.b1 + o];
#pragma unroll
        for (int r = 0; r < kR; ++r) acc[r] = b;
        for (int f = 0; f < F; ++f) {
            const float w = P[off.w1 + f * kH + o];
#pragma unroll
            for (int r = 0; r < kR; ++r) acc[r] = fmaf(xs[r * xp + f], w, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < kR; ++r) h1s[r * kH + o] = fmaxf(acc[r], 0.f);
    }
    __syncthreads();

    // layer 2 (z2 stays in registers)
    float z2[kR];
    {
        const float b = P[off.b2 + o];
#pragma unroll
        for (int r = 0; r < kR; ++r) z2[r] = b;
        for (int i = 0; i < kH; ++i) {
            const float w = W2s[i * kW2Pitch + o];
#pragma unroll
            for (int r = 0; r < kR; ++r) z2[r] = fmaf(h1s[r * kH + i], w, z2[r]);
        }
    }

    // layer 3: y[r] = b3 + sum_o relu(z2[r][o]) W3[o], reduced over the 128 threads
    const float w3 = P[off.w3 + o];
    {
        const int lane = o & 31, warp = o >> 5;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            float p = fmaxf(z2[r], 0.f) * w3;
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) p += __shfl_xor_sync(0xffffffffu, p, s);
            if (lane == 0) wsum[warp * kR + r] = p;
        }
        __syncthreads();
        if (o < kR) {
            const float y = P[off.b3] + ((wsum[o] + wsum[kR + o]) + (wsum[2 * kR + o] + wsum[3 * kR + o]));
            ys[o] = y;
            const int row = row0 + o;
            if (!TRAIN && row < a.B) a.y_out[row] = y * a.ys + a.ym;
            if (TRAIN) {
                const float e = row < a.B ? y - (a.T[row] - a.ym) * a.inv_ys : 0.f;
                dys[o] = e * a.scale;  // scale = 2 / B: d(mean sq. error)/dy
                float se = e * e;
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) se += __shfl_xor_sync(0xffffffffu, se, s);
                if (o == 0) a.partial[size_t(blockIdx.x) * a.pstride + a.nparams] = se;
            }
        }
    }
    if (!TRAIN) return;
    __syncthreads();

    float *G = a.partial + size_t(blockIdx.x) * a.pstride;
    // layer 3 gradients and d2 = relu'(z2) * W3 * dy
    {
        float gw3 = 0.f, gb2 = 0.f, gb3 = 0.f;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const float dy = dys[r];
            gw3 = fmaf(fmaxf(z2[r], 0.f), dy, gw3);
            gb3 += dy;
            const float d2 = z2[r] > 0.f ? w3 * dy : 0.f;
            z2[r] = d2;  // z2 now holds d2
            gb2 += d2;
            d2s[r * kH + o] = d2;
        }
        G[off.w3 + o] = gw3;
        G[off.b2 + o] = gb2;
        if (o == 0) G[off.b3] = gb3;
    }
    // dW2[i][o] = sum_r h1[r][i] d2[r][o]
    for (int i = 0; i < kH; ++i) {
        float s = 0.f;
#pragma unroll
        for (int r = 0; r < kR; ++r) s = fmaf(h1s[r * kH + i], z2[r], s);
        G[off.w2 + i * kH + o] = s;
    }
    __syncthreads();
    // d1[r][i] = relu'(z1[r][i]) * sum_o W2[i][o] d2[r][o]; thread o now plays unit i = o
    {
        const int i = o;
#pragma unroll
        for (int r = 0; r < kR; ++r) acc[r] = 0.f;
        for (int q = 0; q < kH; ++q) {
            const float w = W2s[i * kW2Pitch + q];
#pragma unroll
            for (int r = 0; r < kR; ++r) acc[r] = fmaf(w, d2s[r * kH + q], acc[r]);
        }
        float gb1 = 0.f;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            acc[r] = h1s[r * kH + i] > 0.f ? acc[r] : 0.f;
            gb1 += acc[r];
        }
        G[off.b1 + i] = gb1;
        for (int f = 0; f < F; ++f) {
            float s = 0.f;
#pragma unroll
            for (int r = 0; r < kR; ++r) s = fmaf(xs[r * xp + f], acc[r], s);
            G[off.w1 + f * kH + i] = s;
        }
    }
}

// Sum the per-tile partials in tile order.  update = 0: grad_out[j] = sum; the loss slot
// becomes loss_out[0] = sum / B.  update = 1: one Adam step on params with the summed
// gradient; step t is read from the counter the tile kernel just advanced.
__global__ void mlp_reduce_kernel(MlpArgs a, int ntiles, int update, float lr)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > a.nparams) return;
    float g = 0.f;
    for (int c = 0; c < ntiles; ++c) g += a.partial[size_t(c) * a.pstride + j];
    if (j == a.nparams) {
        if (a.loss_out) a.loss_out[0] = g / float(a.B);
        return;
    }
    if (!update) {
        a.grad_out[j] = g;
        return;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const int t = *a.step_counter;
    const float c1 = 1.f - powf(b1, float(t)), c2 = 1.f - powf(b2, float(t));
    const float m = b1 * a.adam_m[j] + (1.f - b1) * g;
    const float v = b2 * a.adam_v[j] + (1.f - b2) * g * g;
    a.adam_m[j] = m;
    a.adam_v[j] = v;
    a.params[j] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

bool g_attr_set[64] = {false};

int prepare(char *err, size_t errlen)
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !g_attr_set[dev]) {
        const int bytes = (int)tile_smem_bytes();
        cudaFuncSetAttribute(mlp_tile_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(mlp_tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        g_attr_set[dev] = true;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "MLP kernel set-up failed: %s", cudaGetErrorString(e));
        return QS_ECUDA;
    }
    return QS_OK;
}

int launched(const char *what, char *err, size_t errlen)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "%s launch failed: %s", what, cudaGetErrorString(e));
        return QS_ECUDA;
    }
    return QS_OK;
}

}  // namespace

int mlp_param_count(int F) { return mlp_offsets(F).b3 + 1; }

int mlp_tiles(int B) { return (B + kR - 1) / kR; }

int launch_mlp_forward(const MlpArgs &a, void *stream, char *err, size_t errlen)
{
    if (a.B <= 0) return QS_OK;
    int rc = prepare(err, errlen);
    if (rc) return rc;
    mlp_tile_kernel<false><<<mlp_tiles(a.B), kH, tile_smem_bytes(), (cudaStream_t)stream>>>(a);
    return launched("MLP forward", err, errlen);
}

int launch_mlp_train_step(const MlpArgs &a, int update, float lr, void *stream, char *err, size_t errlen)
{
    if (a.B <= 0) return QS_OK;
    int rc = prepare(err, errlen);
    if (rc) return rc;
    const int tiles = mlp_tiles(a.B);
    mlp_tile_kernel<true><<<tiles, kH, tile_smem_bytes(), (cudaStream_t)stream>>>(a);
    rc = launched("MLP forward/backward", err, errlen);
    if (rc) return rc;
    const int threads = 256, blocks = (a.nparams + 1 + threads - 1) / threads;
    mlp_reduce_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(a, tiles, update, lr);
    return launched("MLP gradient reduction", err, errlen);
}

}  // namespace qs
