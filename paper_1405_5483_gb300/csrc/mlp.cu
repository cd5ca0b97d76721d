// Learned cost model: an 8 -> 64 -> 64 -> 1 ReLU perceptron in FP32 that
// predicts ln(ms) of the batched scan for a pattern set and a parameter set
// (not in the paper, which fixes q from log_sigma(rm) and k by a closed form,
// Section 3.2).  Hand-written kernels:
//
//   mlp_forward_kernel  one thread per sample; the 4801 weights sit in
//                       shared memory and are read as broadcasts; the first
//                       hidden layer stays in registers, the second is
//                       streamed into the output.
//   mlp_grad_kernel     one block per tile of 64 samples: the forward pass
//                       keeps the tile's activations in shared memory (rows
//                       padded to 65 floats), then the backward pass forms
//                       dL/dz2, dL/dz1 and the tile's partial gradient as
//                       sums over the tile's samples, written to its own row.
//   mlp_reduce_kernel   one thread per parameter: sums the tiles' rows in
//                       tile order (so the result does not depend on
//                       scheduling) and either stores the gradient or applies
//                       Adam (Kingma and Ba, 2015) to the parameter.
//
// The loss is the mean squared error of the standardised output against the
// standardised target ln(ms).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "mpm.h"
#include "mpm_internal.h"

namespace {

constexpr int NI = MPM_MODEL_INPUTS;
constexpr int NH = MPM_MODEL_HIDDEN;
constexpr int NP = MPM_MODEL_PARAMS;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + NH * NI;  // 512
constexpr int OFF_W2 = OFF_B1 + NH;       // 576
constexpr int OFF_B2 = OFF_W2 + NH * NH;  // 4672
constexpr int OFF_W3 = OFF_B2 + NH;       // 4736
constexpr int OFF_B3 = OFF_W3 + NH;       // 4800
static_assert(OFF_B3 + 1 == NP, "parameter layout");
constexpr int NORM = 20;  // 8 means, 8 deviations, output mean, output deviation, padding

constexpr int kTile = 64;       // samples per gradient block
constexpr int kRow = NH + 1;    // padded activation row
constexpr int kGradThreads = 256;
constexpr size_t kGradSmem =
    sizeof(float) * (NP + NORM + kTile * NI + 4 * kTile * kRow + 2 * kTile);

__device__ __forceinline__ void load_weights(const float* theta, const float* norm, float* w,
                                             float* nm) {
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = theta[i];
    for (int i = threadIdx.x; i < NORM; i += blockDim.x) nm[i] = norm[i];
    __syncthreads();
}

__global__ void __launch_bounds__(128)
    mlp_forward_kernel(const float* __restrict__ theta, const float* __restrict__ norm,
                       const float* __restrict__ X, uint32_t N, float* __restrict__ y) {
    __shared__ float w[NP];
    __shared__ float nm[NORM];
    load_weights(theta, norm, w, nm);
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < N) {
        float x[NI];
#pragma unroll
        for (int c = 0; c < NI; c++) x[c] = (X[(size_t)s * NI + c] - nm[c]) / nm[NI + c];
        float h1[NH];
#pragma unroll
        for (int j = 0; j < NH; j++) {
            float z = w[OFF_B1 + j];
#pragma unroll
            for (int c = 0; c < NI; c++) z = fmaf(w[OFF_W1 + j * NI + c], x[c], z);
            h1[j] = fmaxf(z, 0.0f);
        }
        float f = w[OFF_B3];
#pragma unroll 1
        for (int j = 0; j < NH; j++) {
            float z = w[OFF_B2 + j];
#pragma unroll
            for (int i = 0; i < NH; i++) z = fmaf(w[OFF_W2 + j * NH + i], h1[i], z);
            f = fmaf(w[OFF_W3 + j], fmaxf(z, 0.0f), f);
        }
        y[s] = fmaf(nm[2 * NI + 1], f, nm[2 * NI]);
    }
}

// Samples begin + [blockIdx.x * 64, ...) of the (optionally permuted) list.
__global__ void __launch_bounds__(kGradThreads)
    mlp_grad_kernel(const float* __restrict__ theta, const float* __restrict__ norm,
                    const float* __restrict__ X, const float* __restrict__ Y,
                    const uint32_t* __restrict__ idx, uint32_t begin, uint32_t len,
                    float inv_count, float* __restrict__ partial,
                    float* __restrict__ partial_loss) {
    extern __shared__ float sm[];
    float* w = sm;
    float* nm = w + NP;
    float* Xs = nm + NORM;
    float* H1 = Xs + kTile * NI;
    float* H2 = H1 + kTile * kRow;
    float* D2 = H2 + kTile * kRow;
    float* D1 = D2 + kTile * kRow;
    float* dF = D1 + kTile * kRow;
    float* lossv = dF + kTile;
    load_weights(theta, norm, w, nm);
    const uint32_t s0 = blockIdx.x * kTile;
    const uint32_t ns = min((uint32_t)kTile, len - s0);
    const int tid = threadIdx.x;

    // forward: thread s takes sample s of the tile
    if (tid < kTile) {
        const int s = tid;
        float* h1r = H1 + s * kRow;
        float* h2r = H2 + s * kRow;
        if ((uint32_t)s < ns) {
            const uint32_t q = begin + s0 + (uint32_t)s;
            const size_t smp = idx ? idx[q] : q;
            float x[NI];
#pragma unroll
            for (int c = 0; c < NI; c++) {
                x[c] = (X[smp * NI + c] - nm[c]) / nm[NI + c];
                Xs[s * NI + c] = x[c];
            }
            float h1[NH];
#pragma unroll
            for (int j = 0; j < NH; j++) {
                float z = w[OFF_B1 + j];
#pragma unroll
                for (int c = 0; c < NI; c++) z = fmaf(w[OFF_W1 + j * NI + c], x[c], z);
                h1[j] = fmaxf(z, 0.0f);
                h1r[j] = h1[j];
            }
            float f = w[OFF_B3];
#pragma unroll 1
            for (int j = 0; j < NH; j++) {
                float z = w[OFF_B2 + j];
#pragma unroll
                for (int i = 0; i < NH; i++) z = fmaf(w[OFF_W2 + j * NH + i], h1[i], z);
                const float h2 = fmaxf(z, 0.0f);
                h2r[j] = h2;
                f = fmaf(w[OFF_W3 + j], h2, f);
            }
            const float yt = (Y[smp] - nm[2 * NI]) / nm[2 * NI + 1];
            const float d = f - yt;
            lossv[s] = d * d;
            dF[s] = 2.0f * d * inv_count;
        } else {
            for (int c = 0; c < NI; c++) Xs[s * NI + c] = 0.0f;
            for (int j = 0; j < NH; j++) h1r[j] = h2r[j] = 0.0f;
            lossv[s] = 0.0f;
            dF[s] = 0.0f;
        }
    }
    __syncthreads();
    // dL/dz2 = dL/df * w3, where the unit is active
    for (int p = tid; p < kTile * NH; p += kGradThreads) {
        const int s = p / NH, j = p % NH;
        D2[s * kRow + j] = H2[s * kRow + j] > 0.0f ? dF[s] * w[OFF_W3 + j] : 0.0f;
    }
    __syncthreads();
    // dL/dz1 = W2^T dL/dz2, where the unit is active
    for (int p = tid; p < kTile * NH; p += kGradThreads) {
        const int s = p / NH, i = p % NH;
        float acc = 0.0f;
        for (int j = 0; j < NH; j++) acc = fmaf(D2[s * kRow + j], w[OFF_W2 + j * NH + i], acc);
        D1[s * kRow + i] = H1[s * kRow + i] > 0.0f ? acc : 0.0f;
    }
    __syncthreads();
    // the tile's partial gradient: sums over its samples, in sample order
    float* g = partial + (size_t)blockIdx.x * NP;
    for (int p = tid; p < NH * NH; p += kGradThreads) {
        const int j = p / NH, i = p % NH;
        float acc = 0.0f;
        for (int s = 0; s < kTile; s++) acc = fmaf(D2[s * kRow + j], H1[s * kRow + i], acc);
        g[OFF_W2 + p] = acc;
    }
    for (int p = tid; p < NH * NI; p += kGradThreads) {
        const int i = p / NI, c = p % NI;
        float acc = 0.0f;
        for (int s = 0; s < kTile; s++) acc = fmaf(D1[s * kRow + i], Xs[s * NI + c], acc);
        g[OFF_W1 + p] = acc;
    }
    if (tid < NH) {
        float gb1 = 0.0f, gb2 = 0.0f, gw3 = 0.0f;
        for (int s = 0; s < kTile; s++) {
            gb1 += D1[s * kRow + tid];
            gb2 += D2[s * kRow + tid];
            gw3 = fmaf(dF[s], H2[s * kRow + tid], gw3);
        }
        g[OFF_B1 + tid] = gb1;
        g[OFF_B2 + tid] = gb2;
        g[OFF_W3 + tid] = gw3;
    } else if (tid == NH) {
        float gb3 = 0.0f, L = 0.0f;
        for (int s = 0; s < kTile; s++) {
            gb3 += dF[s];
            L += lossv[s];
        }
        g[OFF_B3] = gb3;
        partial_loss[blockIdx.x] = L;
    }
}

// mode 0: grad[p] = the sum of the tiles' rows; mode 1: Adam on theta[p].
// loss_acc (may be null) += the sum of the tiles' squared errors.
__global__ void __launch_bounds__(256)
    mlp_reduce_kernel(const float* __restrict__ partial, const float* __restrict__ partial_loss,
                      uint32_t tiles, int mode, float* __restrict__ grad, float* __restrict__ theta,
                      float* __restrict__ m, float* __restrict__ v, float lr, float beta1,
                      float beta2, float eps, float c1, float c2, float* __restrict__ loss_acc) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NP) {
        float g = 0.0f;
        for (uint32_t t = 0; t < tiles; t++) g += partial[(size_t)t * NP + p];
        if (mode == 0) {
            grad[p] = g;
        } else {
            const float mm = beta1 * m[p] + (1.0f - beta1) * g;
            const float vv = beta2 * v[p] + (1.0f - beta2) * g * g;
            m[p] = mm;
            v[p] = vv;
            theta[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
        }
    }
    if (p == 0 && loss_acc) {
        float L = 0.0f;
        for (uint32_t t = 0; t < tiles; t++) L += partial_loss[t];
        *loss_acc += L;
    }
}

uint64_t splitmix64(uint64_t& x) {
    // SplitMix64 (Steele, Lea and Flood, 2014)
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

using mpm::set_error;

}  // namespace

struct mpm_model {
    std::vector<float> theta, m, v;
    float norm[NORM];
    int64_t t = 0;
    int device = -1;
    bool dev_stale = true;   // the device copy is older than the host's
    bool host_stale = false; // the host copy is older than the device's
    float* d_theta = nullptr;
    float* d_m = nullptr;
    float* d_v = nullptr;
    float* d_norm = nullptr;
    float* d_partial = nullptr;
    float* d_ploss = nullptr;
    size_t partial_tiles = 0;
    float* d_grad = nullptr;
    float* d_loss = nullptr;
    size_t loss_cap = 0;
    float* d_in = nullptr;  // staged host inputs: X, then y / outputs
    size_t in_cap = 0;
    uint32_t* d_idx = nullptr;
    size_t idx_cap = 0;
    float* d_out = nullptr;  // predictions bound for the host
    size_t out_cap = 0;
};

namespace {

void free_device(mpm_model* md) {
    cudaFree(md->d_theta);
    cudaFree(md->d_m);
    cudaFree(md->d_v);
    cudaFree(md->d_norm);
    cudaFree(md->d_partial);
    cudaFree(md->d_ploss);
    cudaFree(md->d_grad);
    cudaFree(md->d_loss);
    cudaFree(md->d_in);
    cudaFree(md->d_idx);
    cudaFree(md->d_out);
}

// Host copy current (downloads after device work).
int sync_host(const mpm_model* cmd) {
    mpm_model* md = const_cast<mpm_model*>(cmd);
    if (!md->host_stale) return MPM_OK;
    if (cudaSetDevice(md->device) != cudaSuccess ||
        cudaMemcpy(md->theta.data(), md->d_theta, NP * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(md->m.data(), md->d_m, NP * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(md->v.data(), md->d_v, NP * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return MPM_ECUDA;
    }
    md->host_stale = false;
    return MPM_OK;
}

// Device copy current (allocates on first use).
int sync_device(mpm_model* md) {
    if (md->device < 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            return MPM_ECUDA;
        }
        md->device = dev;
        if (cudaMalloc(&md->d_theta, NP * 4) != cudaSuccess ||
            cudaMalloc(&md->d_m, NP * 4) != cudaSuccess ||
            cudaMalloc(&md->d_v, NP * 4) != cudaSuccess ||
            cudaMalloc(&md->d_norm, NORM * 4) != cudaSuccess ||
            cudaMalloc(&md->d_grad, NP * 4) != cudaSuccess ||
            cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kGradSmem) != cudaSuccess) {
            cudaGetLastError();
            return MPM_ENOMEM;
        }
        md->dev_stale = true;
    }
    if (cudaSetDevice(md->device) != cudaSuccess) {
        cudaGetLastError();
        return MPM_ECUDA;
    }
    if (md->dev_stale) {
        if (cudaMemcpy(md->d_theta, md->theta.data(), NP * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(md->d_m, md->m.data(), NP * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(md->d_v, md->v.data(), NP * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(md->d_norm, md->norm, NORM * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return MPM_ECUDA;
        }
        md->dev_stale = false;
    }
    return MPM_OK;
}

template <typename T>
int grow(T** p, size_t* cap, size_t need) {
    if (*cap >= need) return MPM_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, need * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return MPM_ENOMEM;
    }
    *cap = need;
    return MPM_OK;
}

int ensure_tiles(mpm_model* md, size_t tiles) {
    if (md->partial_tiles >= tiles) return MPM_OK;
    cudaFree(md->d_partial);
    cudaFree(md->d_ploss);
    md->d_partial = md->d_ploss = nullptr;
    md->partial_tiles = 0;
    if (cudaMalloc(&md->d_partial, tiles * NP * 4) != cudaSuccess ||
        cudaMalloc(&md->d_ploss, tiles * 4) != cudaSuccess) {
        cudaGetLastError();
        return MPM_ENOMEM;
    }
    md->partial_tiles = tiles;
    return MPM_OK;
}

// X (N x 8) and y (N, may be null) as device pointers, staged when on the host.
int stage_inputs(mpm_model* md, const float* X, const float* y, size_t N, const float** dX,
                 const float** dy) {
    const bool xd = on_device(X), yd = !y || on_device(y);
    size_t need = (xd ? 0 : N * NI) + (yd ? 0 : N);
    if (need) {
        int rc = grow(&md->d_in, &md->in_cap, need);
        if (rc) return rc;
    }
    float* at = md->d_in;
    if (xd) {
        *dX = X;
    } else {
        if (cudaMemcpy(at, X, N * NI * 4, cudaMemcpyHostToDevice) != cudaSuccess) return MPM_ECUDA;
        *dX = at;
        at += N * NI;
    }
    if (dy) {
        if (!y || yd) {
            *dy = y;
        } else {
            if (cudaMemcpy(at, y, N * 4, cudaMemcpyHostToDevice) != cudaSuccess) return MPM_ECUDA;
            *dy = at;
        }
    }
    return MPM_OK;
}

void bias_corrections(const mpm_model* md, float beta1, float beta2, float* c1, float* c2) {
    *c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)md->t)));
    *c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)md->t)));
}

struct TrainCfg {
    float lr, beta1, beta2, eps;
    int epochs, batch;
    uint64_t seed;
};

TrainCfg train_cfg(const mpm_train_opts* o) {
    TrainCfg c{1e-3f, 0.9f, 0.999f, 1e-8f, 200, 256, 0};
    if (o) {
        if (o->lr > 0) c.lr = o->lr;
        if (o->beta1 > 0) c.beta1 = o->beta1;
        if (o->beta2 > 0) c.beta2 = o->beta2;
        if (o->eps > 0) c.eps = o->eps;
        if (o->epochs > 0) c.epochs = o->epochs;
        if (o->batch > 0) c.batch = o->batch;
        c.seed = o->seed;
    }
    return c;
}

constexpr char kMagic[8] = {'M', 'P', 'M', 'M', 'L', 'P', '0', '1'};

}  // namespace

extern "C" {

mpm_model* mpm_model_create(uint64_t seed) {
    mpm_model* md = new (std::nothrow) mpm_model();
    if (!md) {
        set_error(MPM_ENOMEM);
        return nullptr;
    }
    md->theta.assign(NP, 0.0f);
    md->m.assign(NP, 0.0f);
    md->v.assign(NP, 0.0f);
    uint64_t x = seed;
    auto uniform = [&](float bound) {
        const double u = (double)(splitmix64(x) >> 40) * (1.0 / 16777216.0);
        return (float)((2.0 * u - 1.0) * bound);
    };
    // He-uniform: U(-sqrt(6 / fan_in), sqrt(6 / fan_in)); biases zero
    const float a1 = std::sqrt(6.0f / NI), a2 = std::sqrt(6.0f / NH);
    for (int i = 0; i < NH * NI; i++) md->theta[OFF_W1 + i] = uniform(a1);
    for (int i = 0; i < NH * NH; i++) md->theta[OFF_W2 + i] = uniform(a2);
    for (int i = 0; i < NH; i++) md->theta[OFF_W3 + i] = uniform(a2);
    for (int i = 0; i < NI; i++) {
        md->norm[i] = 0.0f;
        md->norm[NI + i] = 1.0f;
    }
    md->norm[2 * NI] = 0.0f;
    md->norm[2 * NI + 1] = 1.0f;
    md->norm[2 * NI + 2] = md->norm[2 * NI + 3] = 0.0f;
    set_error(MPM_OK);
    return md;
}

void mpm_model_free(mpm_model* md) {
    if (!md) return;
    if (md->device >= 0) {
        cudaSetDevice(md->device);
        free_device(md);
    }
    delete md;
}

int mpm_model_set_norm(mpm_model* md, const float* in_mean, const float* in_std, float out_mean,
                       float out_std) {
    if (!md || !in_mean || !in_std || !(out_std > 0.0f) || !std::isfinite(out_mean))
        return set_error(MPM_EINVAL);
    for (int i = 0; i < NI; i++)
        if (!(in_std[i] > 0.0f) || !std::isfinite(in_std[i]) || !std::isfinite(in_mean[i]))
            return set_error(MPM_EINVAL);
    int rc = sync_host(md);
    if (rc) return set_error(rc);
    for (int i = 0; i < NI; i++) {
        md->norm[i] = in_mean[i];
        md->norm[NI + i] = in_std[i];
    }
    md->norm[2 * NI] = out_mean;
    md->norm[2 * NI + 1] = out_std;
    md->dev_stale = true;
    return set_error(MPM_OK);
}

int mpm_model_get_norm(const mpm_model* md, float* in_mean, float* in_std, float* out_mean,
                       float* out_std) {
    if (!md || !in_mean || !in_std || !out_mean || !out_std) return set_error(MPM_EINVAL);
    for (int i = 0; i < NI; i++) {
        in_mean[i] = md->norm[i];
        in_std[i] = md->norm[NI + i];
    }
    *out_mean = md->norm[2 * NI];
    *out_std = md->norm[2 * NI + 1];
    return set_error(MPM_OK);
}

int mpm_model_get_params(const mpm_model* md, float* theta) {
    if (!md || !theta) return set_error(MPM_EINVAL);
    int rc = sync_host(md);
    if (rc) return set_error(rc);
    std::memcpy(theta, md->theta.data(), NP * 4);
    return set_error(MPM_OK);
}

int mpm_model_set_params(mpm_model* md, const float* theta) {
    if (!md || !theta) return set_error(MPM_EINVAL);
    std::memcpy(md->theta.data(), theta, NP * 4);
    std::fill(md->m.begin(), md->m.end(), 0.0f);
    std::fill(md->v.begin(), md->v.end(), 0.0f);
    md->t = 0;
    md->host_stale = false;
    md->dev_stale = true;
    return set_error(MPM_OK);
}

int mpm_model_predict(mpm_model* md, const float* X, size_t N, float* y) {
    if (!md || (N > 0 && (!X || !y)) || N >= (1ull << 31)) return set_error(MPM_EINVAL);
    if (N == 0) return set_error(MPM_OK);
    int rc = sync_device(md);
    if (rc) return set_error(rc);
    const float* dX = nullptr;
    rc = stage_inputs(md, X, nullptr, N, &dX, nullptr);
    if (rc) return set_error(rc);
    const bool yd = on_device(y);
    float* dY = y;
    if (!yd) {
        if ((rc = grow(&md->d_out, &md->out_cap, N))) return set_error(rc);
        dY = md->d_out;
    }
    const uint32_t blocks = (uint32_t)((N + 127) / 128);
    mlp_forward_kernel<<<blocks, 128>>>(md->d_theta, md->d_norm, dX, (uint32_t)N, dY);
    bool ok = cudaGetLastError() == cudaSuccess;
    if (!yd)
        ok = ok && cudaMemcpy(y, dY, N * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
    else
        ok = ok && cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return set_error(MPM_ECUDA);
    }
    return set_error(MPM_OK);
}

int mpm_model_loss_grad(mpm_model* md, const float* X, const float* y, size_t N, float* loss,
                        float* grad) {
    if (!md || !X || !y || N == 0 || N >= (1ull << 31)) return set_error(MPM_EINVAL);
    int rc = sync_device(md);
    if (rc) return set_error(rc);
    const float *dX = nullptr, *dY = nullptr;
    rc = stage_inputs(md, X, y, N, &dX, &dY);
    if (rc) return set_error(rc);
    const size_t tiles = (N + kTile - 1) / kTile;
    rc = ensure_tiles(md, tiles);
    if (rc) return set_error(rc);
    rc = grow(&md->d_loss, &md->loss_cap, 1);
    if (rc) return set_error(rc);
    cudaMemset(md->d_loss, 0, 4);
    mlp_grad_kernel<<<(uint32_t)tiles, kGradThreads, kGradSmem>>>(
        md->d_theta, md->d_norm, dX, dY, nullptr, 0, (uint32_t)N, (float)(1.0 / (double)N),
        md->d_partial, md->d_ploss);
    mlp_reduce_kernel<<<(NP + 255) / 256, 256>>>(md->d_partial, md->d_ploss, (uint32_t)tiles, 0,
                                                 md->d_grad, nullptr, nullptr, nullptr, 0.f, 0.f,
                                                 0.f, 0.f, 0.f, 0.f, md->d_loss);
    float L = 0.0f;
    bool ok = cudaGetLastError() == cudaSuccess &&
              cudaMemcpy(&L, md->d_loss, 4, cudaMemcpyDeviceToHost) == cudaSuccess &&
              (!grad || cudaMemcpy(grad, md->d_grad, NP * 4, cudaMemcpyDeviceToHost) == cudaSuccess);
    if (!ok) {
        cudaGetLastError();
        return set_error(MPM_ECUDA);
    }
    if (loss) *loss = (float)((double)L / (double)N);
    return set_error(MPM_OK);
}

int mpm_model_adam_step(mpm_model* md, const float* grad, const mpm_train_opts* opts) {
    if (!md || !grad) return set_error(MPM_EINVAL);
    const TrainCfg c = train_cfg(opts);
    int rc = sync_device(md);
    if (rc) return set_error(rc);
    rc = ensure_tiles(md, 1);
    if (rc) return set_error(rc);
    if (cudaMemcpy(md->d_partial, grad, NP * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return set_error(MPM_ECUDA);
    }
    md->t++;
    float c1, c2;
    bias_corrections(md, c.beta1, c.beta2, &c1, &c2);
    mlp_reduce_kernel<<<(NP + 255) / 256, 256>>>(md->d_partial, md->d_ploss, 1, 1, nullptr,
                                                 md->d_theta, md->d_m, md->d_v, c.lr, c.beta1,
                                                 c.beta2, c.eps, c1, c2, nullptr);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return set_error(MPM_ECUDA);
    }
    md->host_stale = true;
    return set_error(MPM_OK);
}

int mpm_model_train(mpm_model* md, const float* X, const float* y, size_t N,
                    const mpm_train_opts* opts, float* epoch_loss) {
    if (!md || !X || !y || N == 0 || N >= (1ull << 31)) return set_error(MPM_EINVAL);
    const TrainCfg c = train_cfg(opts);
    int rc = sync_device(md);
    if (rc) return set_error(rc);
    const float *dX = nullptr, *dY = nullptr;
    rc = stage_inputs(md, X, y, N, &dX, &dY);
    if (rc) return set_error(rc);
    const size_t B = std::min<size_t>((size_t)c.batch, N);
    const size_t tiles = (B + kTile - 1) / kTile;
    if ((rc = ensure_tiles(md, tiles)) || (rc = grow(&md->d_idx, &md->idx_cap, N)) ||
        (rc = grow(&md->d_loss, &md->loss_cap, (size_t)c.epochs)))
        return set_error(rc);
    cudaMemset(md->d_loss, 0, (size_t)c.epochs * 4);
    std::vector<uint32_t> perm(N);
    for (int e = 0; e < c.epochs; e++) {
        // the epoch's order: Fisher-Yates driven by SplitMix64(seed, epoch)
        uint64_t x = c.seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(e + 1));
        for (size_t i = 0; i < N; i++) perm[i] = (uint32_t)i;
        for (size_t i = N - 1; i > 0; i--) {
            const size_t j = (size_t)(splitmix64(x) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        if (cudaMemcpy(md->d_idx, perm.data(), N * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return set_error(MPM_ECUDA);
        }
        for (size_t b0 = 0; b0 < N; b0 += B) {
            const size_t len = std::min(B, N - b0);
            const uint32_t nt = (uint32_t)((len + kTile - 1) / kTile);
            mlp_grad_kernel<<<nt, kGradThreads, kGradSmem>>>(
                md->d_theta, md->d_norm, dX, dY, md->d_idx, (uint32_t)b0, (uint32_t)len,
                (float)(1.0 / (double)len), md->d_partial, md->d_ploss);
            md->t++;
            float c1, c2;
            bias_corrections(md, c.beta1, c.beta2, &c1, &c2);
            mlp_reduce_kernel<<<(NP + 255) / 256, 256>>>(
                md->d_partial, md->d_ploss, nt, 1, nullptr, md->d_theta, md->d_m, md->d_v, c.lr,
                c.beta1, c.beta2, c.eps, c1, c2, md->d_loss + e);
        }
        if (cudaGetLastError() != cudaSuccess) {
            md->host_stale = true;
            return set_error(MPM_ECUDA);
        }
    }
    std::vector<float> acc((size_t)c.epochs);
    md->host_stale = true;
    if (cudaMemcpy(acc.data(), md->d_loss, acc.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return set_error(MPM_ECUDA);
    }
    if (epoch_loss)
        for (int e = 0; e < c.epochs; e++) epoch_loss[e] = (float)((double)acc[e] / (double)N);
    return set_error(MPM_OK);
}

int mpm_model_save(const mpm_model* md, const char* path) {
    if (!md || !path) return set_error(MPM_EINVAL);
    int rc = sync_host(md);
    if (rc) return set_error(rc);
    FILE* f = std::fopen(path, "wb");
    if (!f) return set_error(MPM_EINVAL);
    const uint32_t np = NP;
    const int64_t t = md->t;
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&np, 4, 1, f) == 1 &&
              std::fwrite(md->norm, 4, NORM, f) == (size_t)NORM && std::fwrite(&t, 8, 1, f) == 1 &&
              std::fwrite(md->theta.data(), 4, NP, f) == (size_t)NP &&
              std::fwrite(md->m.data(), 4, NP, f) == (size_t)NP &&
              std::fwrite(md->v.data(), 4, NP, f) == (size_t)NP;
    ok = (std::fclose(f) == 0) && ok;
    return set_error(ok ? MPM_OK : MPM_EINVAL);
}

mpm_model* mpm_model_load(const char* path) {
    if (!path) {
        set_error(MPM_EINVAL);
        return nullptr;
    }
    FILE* f = std::fopen(path, "rb");
    if (!f) {
        set_error(MPM_EINVAL);
        return nullptr;
    }
    mpm_model* md = mpm_model_create(0);
    if (!md) {
        std::fclose(f);
        return nullptr;
    }
    char magic[8];
    uint32_t np = 0;
    int64_t t = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(&np, 4, 1, f) == 1 && np == (uint32_t)NP &&
              std::fread(md->norm, 4, NORM, f) == (size_t)NORM && std::fread(&t, 8, 1, f) == 1 &&
              std::fread(md->theta.data(), 4, NP, f) == (size_t)NP &&
              std::fread(md->m.data(), 4, NP, f) == (size_t)NP &&
              std::fread(md->v.data(), 4, NP, f) == (size_t)NP;
    std::fclose(f);
    if (!ok || t < 0) {
        mpm_model_free(md);
        set_error(MPM_EINVAL);
        return nullptr;
    }
    md->t = t;
    set_error(MPM_OK);
    return md;
}

int mpm_model_features(int sigma, double entropy, size_t m, size_t r, size_t n,
                       const mpm_params* params, size_t count, float* X) {
    if (!params || (count > 0 && !X) || m == 0 || r == 0 || n == 0) return set_error(MPM_EINVAL);
    for (size_t i = 0; i < count; i++) {
        const mpm_params& p = params[i];
        if (p.q < 1 || p.k < 1 || p.sigma_r < 2) return set_error(MPM_EINVAL);
        float* x = X + i * NI;
        x[0] = (float)sigma;
        x[1] = (float)entropy;
        x[2] = (float)std::log2((double)m);
        x[3] = (float)std::log10((double)r);
        x[4] = (float)std::log2((double)n);
        x[5] = (float)p.q;
        x[6] = (float)std::log2((double)p.sigma_r);
        x[7] = (float)p.k;
    }
    return set_error(MPM_OK);
}

int mpm_model_choose(mpm_model* md, const uint8_t* P, size_t r, size_t m, int sigma,
                     double entropy, size_t n, size_t max_table_bytes, mpm_params* best,
                     float* pred) {
    if (!md || !P || !best || n == 0) return set_error(MPM_EINVAL);
    size_t count = 0;
    int rc = mpm_model_grid(P, r, m, sigma, 32, nullptr, nullptr, 0, &count);
    if (rc) return set_error(rc);
    std::vector<mpm_params> all(count);
    std::vector<mpm_table_info> info(count);
    mpm_model_grid(P, r, m, sigma, 32, all.data(), info.data(), count, &count);
    std::vector<mpm_params> grid;
    for (size_t i = 0; i < count; i++)
        if (max_table_bytes == 0 || info[i].table_bytes <= max_table_bytes) grid.push_back(all[i]);
    count = grid.size();
    if (count == 0) return set_error(MPM_EINVAL);
    std::vector<float> X(count * NI), y(count);
    if ((rc = mpm_model_features(sigma, entropy, m, r, n, grid.data(), count, X.data())) ||
        (rc = mpm_model_predict(md, X.data(), count, y.data())))
        return set_error(rc);
    size_t at = 0;
    for (size_t i = 1; i < count; i++)
        if (y[i] < y[at]) at = i;
    *best = grid[at];
    if (pred) *pred = y[at];
    return set_error(MPM_OK);
}

}  // extern "C"
