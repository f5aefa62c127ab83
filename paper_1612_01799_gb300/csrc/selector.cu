// Learned grid selection: features of a coarse density sample and a small MLP that maps
// them to the predicted log10 error of the solver at each candidate grid size.
//
// Features (one block per density): the 32^3 sample's discrete Fourier transform, its
// power |F|^2 averaged over 64 radial shells of |k| in [0, 16 sqrt 3], as
// log10(P_b / P_0) clamped to [-30, 0].  The transform is three passes of 32-point DFTs
// over shared memory (x: real input, 17 bins kept; y and z: complex).
//
// MLP: 64 -> 64 -> 64 -> 64 -> K with ReLU on the hidden layers, FP32.  Parameters in one
// array: W1 (64x64), b1, W2 (64x64), b2, W3 (64x64), b3, W4 (K x 64), b4; W[j][i] multiplies
// input i into unit j.  Training kernels: forward (keeping the hidden activations), loss
// gradient of the mean squared error, backward (parameter gradients accumulated with
// atomics), Adam.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/poisson.h"
#include "solver.h"

namespace {

constexpr int kS = 32;        // sample points per axis
constexpr int kX = kS / 2 + 1;  // kept x bins of the real transform
constexpr int kBins = POISSON_FEATURES;
constexpr int kH = 64;        // hidden width
constexpr int kMaxK = POISSON_MAX_CANDIDATES;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(512) k_features(const float *__restrict__ sample, float *__restrict__ feat) {
    extern __shared__ float2 F[];  // [z][y][kx], kX bins of x
    __shared__ float2 W[kS];       // exp(-2 pi i m / 32)
    __shared__ float pw[kBins], cnt[kBins];
    const float *x = sample + (size_t)blockIdx.x * kS * kS * kS;
    for (int m = threadIdx.x; m < kS; m += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * m / kS, &sn, &cs);
        W[m] = make_float2((float)cs, (float)sn);
    }
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) pw[b] = cnt[b] = 0.f;
    __syncthreads();
    // x: each (y, z) row, real input -> bins 0..16.
    for (int i = threadIdx.x; i < kS * kS * kX; i += blockDim.x) {
        const int k = i % kX, row = i / kX;
        const float *r = x + (size_t)row * kS;
        float2 acc = make_float2(0.f, 0.f);
        for (int n = 0; n < kS; ++n) {
            const float2 w = W[(n * k) % kS];
            acc.x += r[n] * w.x;
            acc.y += r[n] * w.y;
        }
        F[i] = acc;
    }
    __syncthreads();
    // y: columns (z, kx) over y, in place through registers of the column.
    for (int c = threadIdx.x; c < kS * kX; c += blockDim.x) {
        const int z = c / kX, kx = c % kX;
        float2 col[kS];
        for (int y = 0; y < kS; ++y) col[y] = F[(z * kS + y) * kX + kx];
        for (int ky = 0; ky < kS; ++ky) {
            float2 acc = make_float2(0.f, 0.f);
            for (int y = 0; y < kS; ++y) {
                const float2 t = cmul(col[y], W[(y * ky) % kS]);
                acc.x += t.x;
                acc.y += t.y;
            }
            F[(z * kS + ky) * kX + kx] = acc;
        }
    }
    __syncthreads();
    // z: columns (ky, kx) over z; power into radial shells.
    const float kmax = 16.f * 1.7320508075688772f;
    for (int c = threadIdx.x; c < kS * kX; c += blockDim.x) {
        const int ky = c / kX, kx = c % kX;
        float2 col[kS];
        for (int z = 0; z < kS; ++z) col[z] = F[(z * kS + ky) * kX + kx];
        const int sky = ky < kS / 2 ? ky : ky - kS;
        const float wgt = (kx == 0 || kx == kS / 2) ? 1.f : 2.f;
        for (int kz = 0; kz < kS; ++kz) {
            float2 acc = make_float2(0.f, 0.f);
            for (int z = 0; z < kS; ++z) {
                const float2 t = cmul(col[z], W[(z * kz) % kS]);
                acc.x += t.x;
                acc.y += t.y;
            }
            const int skz = kz < kS / 2 ? kz : kz - kS;
            const float kr = sqrtf((float)(kx * kx + sky * sky + skz * skz));
            int b = (int)(kr / kmax * kBins);
            b = b < kBins ? b : kBins - 1;
            atomicAdd(&pw[b], wgt * (acc.x * acc.x + acc.y * acc.y));
            atomicAdd(&cnt[b], wgt);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) {
        const float p0 = pw[0] / fmaxf(cnt[0], 1.f);
        const float pb = cnt[b] > 0.f ? pw[b] / cnt[b] : 0.f;
        float v = log10f(pb / fmaxf(p0, 1e-37f) + 1e-30f);
        feat[(size_t)blockIdx.x * kBins + b] = fminf(fmaxf(v, -30.f), 0.f);
    }
}

// Offsets of the parameter blocks for K outputs.
__host__ __device__ inline int off_w(int l) { return l * (kH * kH + kH); }
__host__ __device__ inline int off_b(int l) { return l * (kH * kH + kH) + kH * kH; }
__host__ __device__ inline int nparams(int K) { return 3 * (kH * kH + kH) + K * kH + K; }

// One block (64 threads) per sample.  acts: B x 3 x 64 hidden activations (may be null).
__global__ void __launch_bounds__(kH) k_forward(const float *__restrict__ p, int K, const float *__restrict__ x,
                                                  float *__restrict__ y, float *__restrict__ acts) {
    __shared__ float h[2][kH];
    const int j = threadIdx.x, b = blockIdx.x;
    h[0][j] = x[(size_t)b * kH + j];
    __syncthreads();
    int cur = 0;
    for (int l = 0; l < 3; ++l) {
        const float *W = p + off_w(l);
        float a = p[off_b(l) + j];
        for (int i = 0; i < kH; ++i) a += W[j * kH + i] * h[cur][i];
        a = fmaxf(a, 0.f);
        if (acts) acts[((size_t)b * 3 + l) * kH + j] = a;
        h[1 - cur][j] = a;
        __syncthreads();
        cur = 1 - cur;
    }
    if (j < K) {
        const float *W = p + off_w(3);
        float a = p[off_w(3) + K * kH + j];
        for (int i = 0; i < kH; ++i) a += W[j * kH + i] * h[cur][i];
        y[(size_t)b * K + j] = a;
    }
}

// dy = 2 (y - t) / (B K) and the loss sum (y - t)^2 / (B K) (one block).
__global__ void k_loss(const float *__restrict__ y, const float *__restrict__ t, int n, float *__restrict__ dy,
                       float *__restrict__ loss) {
    __shared__ float s[256];
    float acc = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) {
        const float d = y[i] - t[i];
        dy[i] = 2.f * d / n;
        acc += d * d;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = s[0] / n;
}

// One block per sample; parameter gradients added into g.
__global__ void __launch_bounds__(kH) k_backward(const float *__restrict__ p, int K, const float *__restrict__ x,
                                                   const float *__restrict__ acts, const float *__restrict__ dy,
                                                   float *__restrict__ g) {
    __shared__ float a[4][kH];   // layer inputs: x, h1, h2, h3
    __shared__ float d[2][kH];   // deltas
    const int j = threadIdx.x, b = blockIdx.x;
    a[0][j] = x[(size_t)b * kH + j];
    for (int l = 0; l < 3; ++l) a[l + 1][j] = acts[((size_t)b * 3 + l) * kH + j];
    __syncthreads();
    // output layer
    const float *W4 = p + off_w(3);
    float *gW4 = g + off_w(3), *gb4 = g + off_w(3) + K * kH;
    for (int k = 0; k < K; ++k) {
        const float e = dy[(size_t)b * K + k];
        atomicAdd(&gW4[k * kH + j], e * a[3][j]);
        if (j == 0) atomicAdd(&gb4[k], e);
    }
    float acc = 0.f;
    for (int k = 0; k < K; ++k) acc += W4[k * kH + j] * dy[(size_t)b * K + k];
    d[0][j] = a[3][j] > 0.f ? acc : 0.f;
    __syncthreads();
    int cur = 0;
    for (int l = 2; l >= 0; --l) {
        const float *W = p + off_w(l);
        float *gW = g + off_w(l), *gb = g + off_b(l);
        const float dj = d[cur][j];
        for (int i = 0; i < kH; ++i) atomicAdd(&gW[j * kH + i], dj * a[l][i]);
        atomicAdd(&gb[j], dj);
        if (l > 0) {
            float s = 0.f;
            for (int k = 0; k < kH; ++k) s += W[k * kH + j] * d[cur][k];
            d[1 - cur][j] = a[l][j] > 0.f ? s : 0.f;
        }
        __syncthreads();
        cur = 1 - cur;
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int ok(cudaError_t e) {
    gsp::note_cuda_error(e);
    return e == cudaSuccess ? POISSON_OK : POISSON_ERR_CUDA;
}

}  // namespace

extern "C" int poisson_features32(const float *sample_d, int count, float *feat_d, void *stream) {
    if (count < 0 || (count > 0 && (!sample_d || !feat_d))) return POISSON_ERR_ARG;
    if (count == 0) return POISSON_OK;
    const size_t smem = (size_t)kS * kS * kX * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_features, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return ok(e);
    k_features<<<count, 512, smem, (cudaStream_t)stream>>>(sample_d, feat_d);
    return ok(cudaGetLastError());
}

extern "C" int poisson_mlp_nparams(int K) { return K >= 1 && K <= kMaxK ? nparams(K) : -1; }

extern "C" int poisson_mlp_forward(const float *params_d, int K, const float *x_d, int count, float *y_d,
                                   float *acts_d, void *stream) {
    if (K < 1 || K > kMaxK || count < 0 || (count > 0 && (!params_d || !x_d || !y_d))) return POISSON_ERR_ARG;
    if (count == 0) return POISSON_OK;
    k_forward<<<count, kH, 0, (cudaStream_t)stream>>>(params_d, K, x_d, y_d, acts_d);
    return ok(cudaGetLastError());
}

extern "C" int poisson_mlp_loss(const float *y_d, const float *target_d, int n, float *dy_d, float *loss_d,
                                void *stream) {
    if (n < 1 || !y_d || !target_d || !dy_d || !loss_d) return POISSON_ERR_ARG;
    k_loss<<<1, 256, 0, (cudaStream_t)stream>>>(y_d, target_d, n, dy_d, loss_d);
    return ok(cudaGetLastError());
}

extern "C" int poisson_mlp_backward(const float *params_d, int K, const float *x_d, const float *acts_d,
                                    int count, const float *dy_d, float *grad_d, void *stream) {
    if (K < 1 || K > kMaxK || count < 0 || (count > 0 && (!params_d || !x_d || !acts_d || !dy_d || !grad_d)))
        return POISSON_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(grad_d, 0, sizeof(float) * nparams(K), s);
    if (e != cudaSuccess || count == 0) return ok(e);
    k_backward<<<count, kH, 0, s>>>(params_d, K, x_d, acts_d, dy_d, grad_d);
    return ok(cudaGetLastError());
}

extern "C" int poisson_mlp_adam(float *params_d, const float *grad_d, float *m_d, float *v_d, int n, float lr,
                                float beta1, float beta2, float eps, int step, void *stream) {
    if (n < 1 || step < 1 || !params_d || !grad_d || !m_d || !v_d) return POISSON_ERR_ARG;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_adam<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params_d, grad_d, m_d, v_d, n, lr, beta1, beta2,
                                                               eps, c1, c2);
    return ok(cudaGetLastError());
}

// ---- selector objects -------------------------------------------------------------------
// File (little endian): "GSPSEL01", int32 K, int32 N[K], float margin, float feat_mean[64],
// float feat_std[64], float params[nparams(K)].  The network predicts log10 of the relative
// L2 error of a solve at each candidate N from the standardised features.

#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

struct poisson_selector_s {
    int K = 0;
    int N[kMaxK] = {};
    float margin = 0.f;
    int capacity = 0;
    float *params = nullptr, *mean = nullptr, *stdv = nullptr;  // device
    float *feat = nullptr, *pred = nullptr;                      // device, capacity rows
};

namespace {
__global__ void k_standardise(float *__restrict__ f, const float *__restrict__ mean, const float *__restrict__ sd,
                              int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = (f[i] - mean[i % kBins]) / sd[i % kBins];
}
void free_selector(poisson_selector s) {
    if (!s) return;
    float *bufs[] = {s->params, s->mean, s->stdv, s->feat, s->pred};
    for (float *b : bufs)
        if (b) cudaFree(b);
    delete s;
}
}  // namespace

extern "C" int poisson_selector_load(poisson_selector *out, const char *path, int capacity) {
    if (!out || !path || capacity < 1) return POISSON_ERR_ARG;
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return POISSON_ERR_ARG;
    char magic[8];
    poisson_selector s = new (std::nothrow) poisson_selector_s();
    if (!s) {
        std::fclose(f);
        return POISSON_ERR_ALLOC;
    }
    bool good = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "GSPSEL01", 8) == 0 &&
                std::fread(&s->K, 4, 1, f) == 1 && s->K >= 1 && s->K <= kMaxK &&
                std::fread(s->N, 4, s->K, f) == (size_t)s->K && std::fread(&s->margin, 4, 1, f) == 1;
    std::vector<float> mean(kBins), sd(kBins), params;
    if (good) {
        params.resize(nparams(s->K));
        good = std::fread(mean.data(), 4, kBins, f) == (size_t)kBins &&
               std::fread(sd.data(), 4, kBins, f) == (size_t)kBins &&
               std::fread(params.data(), 4, params.size(), f) == params.size();
    }
    std::fclose(f);
    if (!good) {
        delete s;
        return POISSON_ERR_ARG;
    }
    s->capacity = capacity;
    auto alloc = [&](float **p, size_t n) { return cudaMalloc(p, n * sizeof(float)) == cudaSuccess; };
    if (!alloc(&s->params, params.size()) || !alloc(&s->mean, kBins) || !alloc(&s->stdv, kBins) ||
        !alloc(&s->feat, (size_t)capacity * kBins) || !alloc(&s->pred, (size_t)capacity * s->K)) {
        free_selector(s);
        return POISSON_ERR_ALLOC;
    }
    if (cudaMemcpy(s->params, params.data(), params.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->mean, mean.data(), kBins * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->stdv, sd.data(), kBins * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        free_selector(s);
        return POISSON_ERR_CUDA;
    }
    *out = s;
    return POISSON_OK;
}

extern "C" int poisson_selector_destroy(poisson_selector s) {
    free_selector(s);
    return POISSON_OK;
}

extern "C" int poisson_select_n(poisson_selector s, const float *sample32_d, int count, double tol, int *N_out,
                                float *pred_out, void *stream) {
    if (!s || !sample32_d || !N_out || count < 1 || count > s->capacity || !(tol > 0.0)) return POISSON_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = poisson_features32(sample32_d, count, s->feat, stream);
    if (rc) return rc;
    const int n = count * kBins;
    k_standardise<<<(n + 255) / 256, 256, 0, st>>>(s->feat, s->mean, s->stdv, n);
    if ((rc = poisson_mlp_forward(s->params, s->K, s->feat, count, s->pred, nullptr, stream))) return rc;
    std::vector<float> pred((size_t)count * s->K);
    if (cudaMemcpyAsync(pred.data(), s->pred, pred.size() * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return POISSON_ERR_CUDA;
    const float goal = (float)std::log10(tol) - s->margin;
    for (int b = 0; b < count; ++b) {
        int pick = s->N[s->K - 1];
        for (int k = 0; k < s->K; ++k)
            if (pred[(size_t)b * s->K + k] <= goal) {
                pick = s->N[k];
                break;
            }
        N_out[b] = pick;
    }
    if (pred_out) std::memcpy(pred_out, pred.data(), pred.size() * 4);
    return POISSON_OK;
}
