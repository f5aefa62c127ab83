// poisson_compare: the final residual check, FP64-accumulated differences of two arrays.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/poisson.h"
#include "solver.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 1216;  // 8 per SM of a 152-SM part; grid-stride beyond

// Per-block partials (sum (a-b)^2, sum b^2, max |a-b|, max |b|); a second kernel folds them.
__device__ double g_part[kBlocks][4];
__device__ double g_out[4];
std::mutex g_mutex;

template <typename A, typename B>
__global__ void __launch_bounds__(kThreads) k_compare(const A *__restrict__ a, const B *__restrict__ b,
                                                      size_t n) {
    double d2 = 0.0, b2 = 0.0, dm = 0.0, bm = 0.0;
    for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kThreads) {
        const double x = (double)a[i], y = (double)b[i], d = x - y;
        d2 += d * d;
        b2 += y * y;
        dm = fmax(dm, fabs(d));
        bm = fmax(bm, fabs(y));
    }
    __shared__ double s[4][kThreads];
    s[0][threadIdx.x] = d2;
    s[1][threadIdx.x] = b2;
    s[2][threadIdx.x] = dm;
    s[3][threadIdx.x] = bm;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s[0][threadIdx.x] += s[0][threadIdx.x + o];
            s[1][threadIdx.x] += s[1][threadIdx.x + o];
            s[2][threadIdx.x] = fmax(s[2][threadIdx.x], s[2][threadIdx.x + o]);
            s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) g_part[blockIdx.x][threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k_fold(int nblocks) {
    if (threadIdx.x != 0) return;
    double r[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < nblocks; ++i) {  // fixed order: the result does not depend on timing
        r[0] += g_part[i][0];
        r[1] += g_part[i][1];
        r[2] = fmax(r[2], g_part[i][2]);
        r[3] = fmax(r[3], g_part[i][3]);
    }
    for (int k = 0; k < 4; ++k) g_out[k] = r[k];
}

template <typename A, typename B>
cudaError_t launch(const void *a, const void *b, size_t n, cudaStream_t s) {
    const size_t need = (n + kThreads - 1) / kThreads;
    const int blocks = (int)(need < (size_t)kBlocks ? (need > 0 ? need : 1) : kBlocks);
    k_compare<A, B><<<blocks, kThreads, 0, s>>>(static_cast<const A *>(a), static_cast<const B *>(b), n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_fold<<<1, 32, 0, s>>>(blocks);
    return cudaGetLastError();
}

}  // namespace

extern "C" int poisson_compare(const void *a_d, int a_dtype, const void *b_d, int b_dtype, size_t n,
                               double *rel_l2, double *rel_linf, void *stream) {
    if (!a_d || !b_d || !rel_l2 || !rel_linf) return POISSON_ERR_ARG;
    if ((a_dtype != POISSON_F32 && a_dtype != POISSON_F64) || (b_dtype != POISSON_F32 && b_dtype != POISSON_F64))
        return POISSON_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_mutex);
    cudaError_t e;
    if (a_dtype == POISSON_F32)
        e = b_dtype == POISSON_F32 ? launch<float, float>(a_d, b_d, n, s) : launch<float, double>(a_d, b_d, n, s);
    else
        e = b_dtype == POISSON_F32 ? launch<double, float>(a_d, b_d, n, s) : launch<double, double>(a_d, b_d, n, s);
    if (e != cudaSuccess) return POISSON_ERR_CUDA;
    double h[4];
    if ((e = cudaMemcpyFromSymbolAsync(h, g_out, sizeof(h), 0, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return POISSON_ERR_CUDA;
    *rel_l2 = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : (h[0] > 0.0 ? INFINITY : 0.0);
    *rel_linf = h[3] > 0.0 ? h[2] / h[3] : (h[2] > 0.0 ? INFINITY : 0.0);
    return POISSON_OK;
}
