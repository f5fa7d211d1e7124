// zf_mlp.cu -- the learned selector: a 32 -> 64 -> 64 -> 12 perceptron
// (ReLU hidden layers, FP32) with hand-written forward, backward and Adam
// kernels, and the host loops that train it and use it in zf_plan.
//
// Parameters are one flat FP32 vector: W1[64][32], b1[64], W2[64][64], b2[64],
// W3[12][64], b3[12] (7,052 values).  The loss is the softmax cross-entropy
// over the classes each sample allows (others masked), averaged over the
// batch.  Gradients are computed per sample and summed in a fixed order, so
// training is deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "zf_internal.h"

namespace {

constexpr int IN = 32, HID = 64, OUT = 12;
constexpr int OW1 = 0, OB1 = OW1 + HID * IN, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
              OB3 = OW3 + OUT * HID, NP = OB3 + OUT;
static_assert(NP == 7052, "parameter layout");

// One CTA of 64 threads per sample: thread j owns hidden unit j.
__device__ __forceinline__ void forward_sample(const float* __restrict__ p, const float* x, float* h1, float* h2,
                                               float* z) {
    const int j = threadIdx.x;
    float a = p[OB1 + j];
    for (int i = 0; i < IN; i++) a += p[OW1 + j * IN + i] * x[i];
    h1[j] = fmaxf(a, 0.0f);
    __syncthreads();
    a = p[OB2 + j];
    for (int i = 0; i < HID; i++) a += p[OW2 + j * HID + i] * h1[i];
    h2[j] = fmaxf(a, 0.0f);
    __syncthreads();
    if (j < OUT) {
        a = p[OB3 + j];
        for (int i = 0; i < HID; i++) a += p[OW3 + j * HID + i] * h2[i];
        z[j] = a;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(HID) mlp_forward(const float* __restrict__ p, const float* __restrict__ X,
                                                   float* __restrict__ Z) {
    __shared__ float x[IN], h1[HID], h2[HID], z[OUT];
    const int b = blockIdx.x;
    if (threadIdx.x < IN) x[threadIdx.x] = X[(size_t)b * IN + threadIdx.x];
    __syncthreads();
    forward_sample(p, x, h1, h2, z);
    if (threadIdx.x < OUT) Z[(size_t)b * OUT + threadIdx.x] = z[threadIdx.x];
}

// Per-sample gradient of the batch-mean masked cross-entropy into G[b][NP],
// and the sample's loss into L[b].
__global__ void __launch_bounds__(HID) mlp_sample_grad(const float* __restrict__ p, const float* __restrict__ X,
                                                       const int32_t* __restrict__ Y, const uint8_t* __restrict__ MK,
                                                       uint32_t B, float* __restrict__ G, float* __restrict__ L) {
    __shared__ float x[IN], h1[HID], h2[HID], z[OUT], dz[OUT], dh2[HID], dh1[HID];
    const int b = blockIdx.x, j = threadIdx.x;
    if (j < IN) x[j] = X[(size_t)b * IN + j];
    __syncthreads();
    forward_sample(p, x, h1, h2, z);
    if (j == 0) {
        const int y = Y[b];
        float mx = -INFINITY;
        for (int k = 0; k < OUT; k++)
            if (MK[(size_t)b * OUT + k]) mx = fmaxf(mx, z[k]);
        float e[OUT], sum = 0.0f;
        for (int k = 0; k < OUT; k++) {
            e[k] = MK[(size_t)b * OUT + k] ? expf(z[k] - mx) : 0.0f;
            sum += e[k];
        }
        for (int k = 0; k < OUT; k++) dz[k] = (e[k] / sum - (k == y ? 1.0f : 0.0f)) / (float)B;
        L[b] = -logf(e[y] / sum);
    }
    __syncthreads();
    float* g = G + (size_t)b * NP;
    for (int k = 0; k < OUT; k++) g[OW3 + k * HID + j] = dz[k] * h2[j];
    if (j < OUT) g[OB3 + j] = dz[j];
    float a = 0.0f;
    for (int k = 0; k < OUT; k++) a += p[OW3 + k * HID + j] * dz[k];
    dh2[j] = h2[j] > 0.0f ? a : 0.0f;
    __syncthreads();
    for (int i = 0; i < HID; i++) g[OW2 + j * HID + i] = dh2[j] * h1[i];
    g[OB2 + j] = dh2[j];
    a = 0.0f;
    for (int i = 0; i < HID; i++) a += p[OW2 + i * HID + j] * dh2[i];
    dh1[j] = h1[j] > 0.0f ? a : 0.0f;
    __syncthreads();
    for (int c = 0; c < IN; c++) g[OW1 + j * IN + c] = dh1[j] * x[c];
    g[OB1 + j] = dh1[j];
}

// Forward pass and the argmax over each sample's allowed classes.
__global__ void __launch_bounds__(HID) mlp_predict(const float* __restrict__ p, const float* __restrict__ X,
                                                   const uint8_t* __restrict__ MK, int32_t* __restrict__ C) {
    __shared__ float x[IN], h1[HID], h2[HID], z[OUT];
    const int b = blockIdx.x;
    if (threadIdx.x < IN) x[threadIdx.x] = X[(size_t)b * IN + threadIdx.x];
    __syncthreads();
    forward_sample(p, x, h1, h2, z);
    if (threadIdx.x == 0) {
        int best = -1;
        for (int k = 0; k < OUT; k++)
            if (MK[(size_t)b * OUT + k] && (best < 0 || z[k] > z[best])) best = k;
        C[b] = best;
    }
}

// grad[i] = sum over samples in order; block 0's extra pass sums the losses.
__global__ void mlp_reduce(const float* __restrict__ G, const float* __restrict__ L, uint32_t B,
                           float* __restrict__ grad, float* __restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NP) {
        float s = 0.0f;
        for (uint32_t b = 0; b < B; b++) s += G[(size_t)b * NP + i];
        grad[i] = s;
    }
    if (i == 0 && loss) {
        float s = 0.0f;
        for (uint32_t b = 0; b < B; b++) s += L[b];
        *loss = s / (float)B;
    }
}

__global__ void mlp_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                         const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

uint64_t splitmix(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

double unit(uint64_t seed, uint64_t i) { return ((splitmix(seed ^ splitmix(i)) >> 11) + 0.5) / 9007199254740992.0; }

}  // namespace

struct zf_mlp {
    int device = 0;
    float* p = nullptr;       // parameters
    float* m = nullptr;       // Adam first moment
    float* v = nullptr;       // Adam second moment
    float* grad = nullptr;
    float* loss = nullptr;    // one float
    float* gs = nullptr;      // per-sample gradients
    float* ls = nullptr;      // per-sample losses
    uint32_t cap = 0;         // samples gs/ls hold
    uint32_t step = 0;
    // input standardization (x - mean) / std, fitted by zf_mlp_train on its
    // rows and applied by zf_mlp_train and zf_mlp_predict
    bool scaled = false;
    float mean[32] = {0}, sd[32] = {0};
};

namespace {
zf_status ensure_batch(zf_mlp* n, uint32_t B) {
    if (B <= n->cap) return ZF_OK;
    if (n->gs) cudaFree(n->gs);
    if (n->ls) cudaFree(n->ls);
    n->gs = n->ls = nullptr;
    n->cap = 0;
    if (cudaMalloc(&n->gs, (size_t)B * NP * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&n->ls, (size_t)B * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return ZF_ENOMEM;
    }
    n->cap = B;
    return ZF_OK;
}
}  // namespace

extern "C" {

zf_status zf_mlp_create(int device, uint64_t seed, zf_mlp** out) {
    zf::KeepDevice keep_device;
    if (!out) return ZF_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return ZF_ECUDA;
    auto* n = new zf_mlp();
    n->device = device;
    if (cudaMalloc(&n->p, NP * sizeof(float)) != cudaSuccess || cudaMalloc(&n->m, NP * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&n->v, NP * sizeof(float)) != cudaSuccess || cudaMalloc(&n->grad, NP * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&n->loss, sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        zf_mlp_destroy(n);
        return ZF_ENOMEM;
    }
    // He-normal weights (Box-Muller on a counter-based generator), zero biases
    std::vector<float> h(NP, 0.0f);
    auto fill = [&](int off, int rows, int cols) {
        for (int i = 0; i < rows * cols; i++) {
            const double u1 = unit(seed, 2ull * (off + i)), u2 = unit(seed, 2ull * (off + i) + 1);
            const double z = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
            h[off + i] = (float)(z * std::sqrt(2.0 / cols));
        }
    };
    fill(OW1, HID, IN);
    fill(OW2, HID, HID);
    fill(OW3, OUT, HID);
    zf_status st = zf_mlp_set_params(n, h.data());
    if (st) {
        zf_mlp_destroy(n);
        return st;
    }
    *out = n;
    return ZF_OK;
}

zf_status zf_mlp_destroy(zf_mlp* n) {
    zf::KeepDevice keep_device;
    if (!n) return ZF_OK;
    cudaSetDevice(n->device);
    for (float* q : {n->p, n->m, n->v, n->grad, n->loss, n->gs, n->ls})
        if (q) cudaFree(q);
    delete n;
    return ZF_OK;
}

zf_status zf_mlp_get_params(const zf_mlp* n, float* host) {
    zf::KeepDevice keep_device;
    if (!n || !host) return ZF_EINVAL;
    cudaSetDevice(n->device);
    return cudaMemcpy(host, n->p, NP * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess ? ZF_OK : ZF_ECUDA;
}

zf_status zf_mlp_set_params(zf_mlp* n, const float* host) {
    zf::KeepDevice keep_device;
    if (!n || !host) return ZF_EINVAL;
    cudaSetDevice(n->device);
    if (cudaMemcpy(n->p, host, NP * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(n->m, 0, NP * sizeof(float)) != cudaSuccess || cudaMemset(n->v, 0, NP * sizeof(float)) != cudaSuccess)
        return ZF_ECUDA;
    n->step = 0;
    n->scaled = false;   // parameters from elsewhere: inputs are taken as given
    return ZF_OK;
}

zf_status zf_mlp_forward(zf_mlp* n, const float* d_x, uint32_t batch, float* d_logits, void* stream) {
    if (!n || (batch && (!d_x || !d_logits))) return ZF_EINVAL;
    if (!batch) return ZF_OK;
    mlp_forward<<<batch, HID, 0, (cudaStream_t)stream>>>(n->p, d_x, d_logits);
    return cudaGetLastError() == cudaSuccess ? ZF_OK : ZF_ECUDA;
}

zf_status zf_mlp_grad(zf_mlp* n, const float* d_x, const int32_t* d_y, const uint8_t* d_mask, uint32_t batch,
                      float* d_grad, float* d_loss, void* stream) {
    if (!n || !batch || !d_x || !d_y || !d_mask || !d_grad) return ZF_EINVAL;
    zf_status st = ensure_batch(n, batch);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    mlp_sample_grad<<<batch, HID, 0, s>>>(n->p, d_x, d_y, d_mask, batch, n->gs, n->ls);
    mlp_reduce<<<(NP + 255) / 256, 256, 0, s>>>(n->gs, n->ls, batch, d_grad, d_loss);
    return cudaGetLastError() == cudaSuccess ? ZF_OK : ZF_ECUDA;
}

zf_status zf_mlp_adam(zf_mlp* n, const float* d_grad, float lr, void* stream) {
    if (!n || !d_grad) return ZF_EINVAL;
    n->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)n->step)), c2 = (float)(1.0 - std::pow(0.999, (double)n->step));
    mlp_adam<<<(NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n->p, n->m, n->v, d_grad, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? ZF_OK : ZF_ECUDA;
}

// Mini-batch training on the GPU: the sample order of every epoch is a
// seeded shuffle; each batch runs the gradient and Adam kernels.
zf_status zf_mlp_train(zf_mlp* n, const float* h_x, const int32_t* h_y, const uint8_t* h_mask, uint32_t count,
                       uint32_t epochs, uint32_t batch, float lr, uint64_t seed, float* h_losses) {
    zf::KeepDevice keep_device;
    if (!n || !h_x || !h_y || !h_mask || !count || !batch) return ZF_EINVAL;
    cudaSetDevice(n->device);
    float *dx = nullptr, *dl = nullptr;
    int32_t* dy = nullptr;
    uint8_t* dm = nullptr;
    auto done = [&](zf_status s) {
        for (void* q : {(void*)dx, (void*)dy, (void*)dm, (void*)dl})
            if (q) cudaFree(q);
        return s;
    };
    if (cudaMalloc(&dx, (size_t)count * IN * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&dy, (size_t)count * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&dm, (size_t)count * OUT) != cudaSuccess || cudaMalloc(&dl, sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return done(ZF_ENOMEM);
    }
    // per-feature mean and standard deviation of the training rows (a
    // constant feature keeps std 1), kept by the network for inference
    for (uint32_t f = 0; f < IN; f++) {
        double s1 = 0, s2 = 0;
        for (uint32_t r = 0; r < count; r++) {
            const double v = h_x[(size_t)r * IN + f];
            s1 += v;
            s2 += v * v;
        }
        const double mu = s1 / count, var = std::max(0.0, s2 / count - mu * mu);
        n->mean[f] = (float)mu;
        n->sd[f] = var > 0 ? (float)std::sqrt(var) : 1.0f;
    }
    n->scaled = true;
    std::vector<uint32_t> order(count);
    std::vector<float> bx((size_t)batch * IN);
    std::vector<int32_t> by(batch);
    std::vector<uint8_t> bm((size_t)batch * OUT);
    for (uint32_t e = 0; e < epochs; e++) {
        std::iota(order.begin(), order.end(), 0u);
        for (uint32_t i = count; i > 1; i--) {   // Fisher-Yates with the counter generator
            const uint32_t j = (uint32_t)(unit(seed + e, i) * i);
            std::swap(order[i - 1], order[std::min(j, i - 1)]);
        }
        double esum = 0;
        uint32_t nb = 0;
        for (uint32_t s0 = 0; s0 < count; s0 += batch) {
            const uint32_t B = std::min(batch, count - s0);
            for (uint32_t k = 0; k < B; k++) {
                const uint32_t r = order[s0 + k];
                for (uint32_t f = 0; f < IN; f++)
                    bx[(size_t)k * IN + f] = (h_x[(size_t)r * IN + f] - n->mean[f]) / n->sd[f];
                by[k] = h_y[r];
                memcpy(&bm[(size_t)k * OUT], h_mask + (size_t)r * OUT, OUT);
            }
            if (cudaMemcpy(dx, bx.data(), (size_t)B * IN * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(dy, by.data(), B * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(dm, bm.data(), (size_t)B * OUT, cudaMemcpyHostToDevice) != cudaSuccess)
                return done(ZF_ECUDA);
            zf_status st = zf_mlp_grad(n, dx, dy, dm, B, n->grad, dl, nullptr);
            if (st) return done(st);
            st = zf_mlp_adam(n, n->grad, lr, nullptr);
            if (st) return done(st);
            if (h_losses) {
                float l = 0;
                if (cudaMemcpy(&l, dl, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return done(ZF_ECUDA);
                esum += l;
                nb++;
            }
        }
        if (h_losses) h_losses[e] = (float)(esum / std::max(1u, nb));
    }
    return done(cudaDeviceSynchronize() == cudaSuccess ? ZF_OK : ZF_ECUDA);
}

// Class of each row of h_x (count x 32): the argmax of the logits over the
// classes h_mask allows (-1 if none), computed on the GPU.
zf_status zf_mlp_predict(zf_mlp* n, const float* h_x, const uint8_t* h_mask, uint32_t count, int32_t* h_class) {
    zf::KeepDevice keep_device;
    if (!n || !h_x || !h_mask || !h_class) return ZF_EINVAL;
    if (!count) return ZF_OK;
    cudaSetDevice(n->device);
    float* dx = nullptr;
    uint8_t* dm = nullptr;
    int32_t* dc = nullptr;
    auto done = [&](zf_status s) {
        for (void* q : {(void*)dx, (void*)dm, (void*)dc})
            if (q) cudaFree(q);
        return s;
    };
    if (cudaMalloc(&dx, (size_t)count * IN * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&dm, (size_t)count * OUT) != cudaSuccess || cudaMalloc(&dc, (size_t)count * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        return done(ZF_ENOMEM);
    }
    std::vector<float> xs;
    const float* src = h_x;
    if (n->scaled) {   // the standardization fitted by zf_mlp_train
        xs.resize((size_t)count * IN);
        for (size_t i = 0; i < xs.size(); i++) xs[i] = (h_x[i] - n->mean[i % IN]) / n->sd[i % IN];
        src = xs.data();
    }
    if (cudaMemcpy(dx, src, (size_t)count * IN * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dm, h_mask, (size_t)count * OUT, cudaMemcpyHostToDevice) != cudaSuccess)
        return done(ZF_ECUDA);
    mlp_predict<<<count, HID>>>(n->p, dx, dm, dc);
    if (cudaGetLastError() != cudaSuccess) return done(ZF_ECUDA);
    if (cudaMemcpy(h_class, dc, (size_t)count * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return done(ZF_ECUDA);
    return done(ZF_OK);
}

zf_status zf_mlp_get_scaling(const zf_mlp* n, float* mean, float* std_) {
    if (!n || !mean || !std_) return ZF_EINVAL;
    for (uint32_t f = 0; f < IN; f++) {
        mean[f] = n->scaled ? n->mean[f] : 0.0f;
        std_[f] = n->scaled ? n->sd[f] : 1.0f;
    }
    return ZF_OK;
}

}  // extern "C"
