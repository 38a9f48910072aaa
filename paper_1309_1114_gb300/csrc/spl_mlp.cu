// spl_mlp.cu -- the tile-cost network, its inference and training kernels.
//
// 32 -> 64 (ReLU) -> 1 in FP32: y = w2 . relu(W1 x + b1) + b2, trained on
// the render's own per-item timings to predict log(SM cycles).  Loss: mean
// squared error over a batch; gradients by the chain rule through the ReLU;
// optimiser: Adam (Kingma & Ba, Algorithm 1).  The paper has no counterpart:
// it only observes the load imbalance that this network's predictions are
// used to reduce (Sec. 4 Remarks).
#include <cmath>

#include "spl_internal.cuh"

namespace spl {

// y[b] for every sample, one thread each; weights in shared memory.
__global__ void __launch_bounds__(256) mlp_forward_kernel(const float *theta, const float *x,
                                                          int64_t B, float *y) {
    __shared__ float w[kNParam];
    for (int k = threadIdx.x; k < kNParam; k += blockDim.x) w[k] = theta[k];
    __syncthreads();
    const float *W1 = w, *b1 = w + kHid * kFeat, *w2 = b1 + kHid, *b2 = w2 + kHid;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x) {
        float xv[kFeat];
#pragma unroll
        for (int i = 0; i < kFeat; ++i) xv[i] = x[b * kFeat + i];
        float out = b2[0];
        for (int j = 0; j < kHid; ++j) {
            float z = b1[j];
#pragma unroll
            for (int i = 0; i < kFeat; ++i) z = fmaf(W1[j * kFeat + i], xv[i], z);
            if (z > 0.f) out = fmaf(w2[j], z, out);
        }
        y[b] = out;
    }
}

// Per sample: forward, residual, and the back-propagated quantities
// dy = 2 (y - t) / B, h = relu(z), dz = dy * w2 * [z > 0]; per-block partial
// sums of the squared residuals.
__global__ void __launch_bounds__(256) mlp_backprop_kernel(const float *theta, const float *x,
                                                           const float *t, int64_t B, float *dz,
                                                           float *h, float *dy, float *lpart) {
    __shared__ float w[kNParam];
    __shared__ float red[256];
    for (int k = threadIdx.x; k < kNParam; k += blockDim.x) w[k] = theta[k];
    __syncthreads();
    const float *W1 = w, *b1 = w + kHid * kFeat, *w2 = b1 + kHid, *b2 = w2 + kHid;
    float lsum = 0.f;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x) {
        float xv[kFeat];
#pragma unroll
        for (int i = 0; i < kFeat; ++i) xv[i] = x[b * kFeat + i];
        float out = b2[0];
        for (int j = 0; j < kHid; ++j) {
            float z = b1[j];
#pragma unroll
            for (int i = 0; i < kFeat; ++i) z = fmaf(W1[j * kFeat + i], xv[i], z);
            const float hj = z > 0.f ? z : 0.f;
            h[b * kHid + j] = hj;
            out = fmaf(w2[j], hj, out);
        }
        const float res = out - t[b];
        lsum = fmaf(res, res, lsum);
        const float d = 2.f * res / (float)B;
        dy[b] = d;
        for (int j = 0; j < kHid; ++j) dz[b * kHid + j] = h[b * kHid + j] > 0.f ? d * w2[j] : 0.f;
    }
    red[threadIdx.x] = lsum;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
}

// One thread per parameter, summing over the batch in a fixed order:
// dW1[j][i] = sum_b dz[b][j] x[b][i], db1[j] = sum_b dz[b][j],
// dw2[j] = sum_b dy[b] h[b][j], db2 = sum_b dy[b]; thread kNParam adds the
// loss partials.
__global__ void __launch_bounds__(256) mlp_reduce_kernel(const float *x, const float *dz,
                                                         const float *h, const float *dy,
                                                         int64_t B, const float *lpart, int nparts,
                                                         float *grad, float *loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kNParam) return;
    float acc = 0.f;
    if (p < kHid * kFeat) {
        const int j = p / kFeat, i = p % kFeat;
        for (int64_t b = 0; b < B; ++b) acc = fmaf(dz[b * kHid + j], x[b * kFeat + i], acc);
    } else if (p < kHid * kFeat + kHid) {
        const int j = p - kHid * kFeat;
        for (int64_t b = 0; b < B; ++b) acc += dz[b * kHid + j];
    } else if (p < kHid * kFeat + 2 * kHid) {
        const int j = p - kHid * kFeat - kHid;
        for (int64_t b = 0; b < B; ++b) acc = fmaf(dy[b], h[b * kHid + j], acc);
    } else if (p == kNParam - 1) {
        for (int64_t b = 0; b < B; ++b) acc += dy[b];
    } else {   // p == kNParam: the loss
        for (int k = 0; k < nparts; ++k) acc += lpart[k];
        if (loss) *loss = B > 0 ? acc / (float)B : 0.f;
        return;
    }
    grad[p] = acc;
}

constexpr int kBackpropBlocks = 256;

size_t mlp_work_floats(int64_t B) { return (size_t)B * (2 * kHid + 1) + kBackpropBlocks; }

void launch_mlp_forward(const float *theta, const float *x, int64_t B, float *y, cudaStream_t s) {
    if (B <= 0) return;
    int64_t blocks = (B + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    mlp_forward_kernel<<<(unsigned)blocks, 256, 0, s>>>(theta, x, B, y);
    ++g_launches;
}

void launch_mlp_loss_grad(const float *theta, const float *x, const float *t, int64_t B,
                          float *work, float *grad, float *loss, cudaStream_t s) {
    float *dz = work, *h = dz + B * kHid, *dy = h + B * kHid, *lpart = dy + B;
    mlp_backprop_kernel<<<kBackpropBlocks, 256, 0, s>>>(theta, x, t, B, dz, h, dy, lpart);
    ++g_launches;
    mlp_reduce_kernel<<<(kNParam + 1 + 255) / 256, 256, 0, s>>>(x, dz, h, dy, B, lpart,
                                                                  kBackpropBlocks, grad, loss);
}

// theta -= lr * m_hat / (sqrt(v_hat) + eps), step >= 1.
__global__ void mlp_adam_kernel(float *theta, const float *grad, float *m, float *v, int64_t np,
                                float c1, float c2, float lr, float b1, float b2, float eps) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < np;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float g = grad[k];
        const float mk = b1 * m[k] + (1.f - b1) * g;
        const float vk = b2 * v[k] + (1.f - b2) * g * g;
        m[k] = mk;
        v[k] = vk;
        theta[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

void launch_mlp_adam(float *theta, const float *grad, float *m, float *v, int64_t np, int64_t step,
                     float lr, float b1, float b2, float eps, cudaStream_t s) {
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)step));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)step));
    mlp_adam_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(theta, grad, m, v, np, c1, c2, lr,
                                                                   b1, b2, eps);
}

}  // namespace spl
