// Synthetic inputs and exact potentials on the device, for the grid-selection pipeline.
//
// poisson_sample_gaussians   rho(x) = sum_g q_g prod_q (2 pi s_gq^2)^{-1/2}
//                              exp(-(x_q - c_gq)^2 / (2 s_gq^2)) on the cell-centred grid of
//                              [-L, L]^3 (the synthetic densities of the paper's Sec. 5 kind).
// poisson_gaussian_potential the exact potential of such a sum at chosen grid points:
//                              1/(4 pi r) = (1/(2 pi^{3/2})) int_0^inf exp(-r^2 s^2) ds turns
//                              the convolution with each normalised Gaussian into
//                              q/(2 pi^{3/2}) int_0^inf prod_q (1 + 2 s_q^2 s^2)^{-1/2}
//                              exp(-sum_q d_q^2 s^2 / (1 + 2 s_q^2 s^2)) ds,
//                              done by composite Gauss-Legendre after s = v / (1 - v).
// poisson_compare_points     FP64 relative L2 of a grid solution against reference values
//                              at those points.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/poisson.h"
#include "solver.h"

namespace {

constexpr int kMaxG = POISSON_MAX_GAUSSIANS;

struct Gaussians {
    int n;
    double c[kMaxG][3], s[kMaxG][3], q[kMaxG];
};

// Density on the grid: one block per z-plane; the 1-D factors of every Gaussian along x and
// y are tabulated in shared memory in FP64, then each point is a sum of products.
template <typename Real>
__global__ void k_sample(Gaussians G, int N, double L, Real *__restrict__ out) {
    extern __shared__ double f[];  // [g][x] then [g][y]
    const int z = blockIdx.x;
    const double h = 2.0 * L / N;
    const double rt2pi = 2.5066282746310005024;
    for (int i = threadIdx.x; i < G.n * N; i += blockDim.x) {
        const int g = i / N, x = i % N;
        const double px = -L + (x + 0.5) * h;
        const double dx = (px - G.c[g][0]) / G.s[g][0], dy = (px - G.c[g][1]) / G.s[g][1];
        f[i] = exp(-0.5 * dx * dx) / (rt2pi * G.s[g][0]);
        f[G.n * N + i] = exp(-0.5 * dy * dy) / (rt2pi * G.s[g][1]);
    }
    __shared__ double fz[kMaxG];
    if (threadIdx.x < G.n) {
        const int g = threadIdx.x;
        const double pz = -L + (z + 0.5) * h;
        const double dz = (pz - G.c[g][2]) / G.s[g][2];
        fz[g] = G.q[g] * exp(-0.5 * dz * dz) / (rt2pi * G.s[g][2]);
    }
    __syncthreads();
    Real *plane = out + (size_t)z * N * N;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        const int y = i / N, x = i % N;
        double acc = 0.0;
        for (int g = 0; g < G.n; ++g) acc += fz[g] * f[G.n * N + g * N + y] * f[g * N + x];
        plane[i] = (Real)acc;
    }
}

// Quadrature of the exact potential: nodes v and weights dv of composite Gauss-Legendre on
// [0, 1), panels graded geometrically towards both ends (filled once per device).
constexpr int kPanels = 40, kOrder = 16, kNodes = kPanels * kOrder;
__constant__ double c_s[kNodes], c_ds[kNodes];
bool g_nodes_ready[64];
std::mutex g_mutex;

void gl16(double *x, double *w) {
    const double pi = 3.141592653589793238462643383279502884;
    const int n = kOrder;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

cudaError_t ensure_nodes() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (g_nodes_ready[dev]) return cudaSuccess;
    double gx[kOrder], gw[kOrder], s[kNodes], ds[kNodes], edges[kPanels + 1];
    gl16(gx, gw);
    // edges: 0, then geometric towards 1/2 from 1e-7, mirrored towards 1.
    const int half = kPanels / 2;
    edges[0] = 0.0;
    for (int i = 1; i <= half; ++i) edges[i] = 0.5 * std::pow(1e-7, (double)(half - i) / (half - 1));
    for (int i = 1; i <= half; ++i) edges[half + i] = 1.0 - edges[half - i];
    for (int p = 0; p < kPanels; ++p) {
        const double a = edges[p], b = edges[p + 1];
        for (int i = 0; i < kOrder; ++i) {
            const double v = 0.5 * (a + b) + 0.5 * (b - a) * gx[i];
            s[p * kOrder + i] = v / (1.0 - v);
            ds[p * kOrder + i] = 0.5 * (b - a) * gw[i] / ((1.0 - v) * (1.0 - v));
        }
    }
    if ((e = cudaMemcpyToSymbol(c_s, s, sizeof(s))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_ds, ds, sizeof(ds))) != cudaSuccess) return e;
    g_nodes_ready[dev] = true;
    return cudaSuccess;
}

__global__ void k_potential(Gaussians G, int N, double L, int npts, const int *__restrict__ idx,
                            double *__restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    const double h = 2.0 * L / N;
    const double x[3] = {-L + (idx[3 * p] + 0.5) * h, -L + (idx[3 * p + 1] + 0.5) * h,
                         -L + (idx[3 * p + 2] + 0.5) * h};
    double u = 0.0;
    for (int g = 0; g < G.n; ++g) {
        double d2[3], s2[3];
        for (int a = 0; a < 3; ++a) {
            const double d = x[a] - G.c[g][a];
            d2[a] = d * d;
            s2[a] = 2.0 * G.s[g][a] * G.s[g][a];
        }
        double acc = 0.0;
        for (int k = 0; k < kNodes; ++k) {
            const double s = c_s[k], ss = s * s;
            const double e0 = 1.0 + s2[0] * ss, e1 = 1.0 + s2[1] * ss, e2 = 1.0 + s2[2] * ss;
            const double ex = d2[0] * ss / e0 + d2[1] * ss / e1 + d2[2] * ss / e2;
            acc += c_ds[k] * exp(-ex) * rsqrt(e0 * e1 * e2);
        }
        u += G.q[g] * acc;
    }
    out[p] = u / (2.0 * 5.568327996831707845);  // 2 pi^{3/2}
}

constexpr int kCmpThreads = 256;
__device__ double g_cmp[2];

template <typename Real>
__global__ void k_compare_points(const Real *__restrict__ u, int N, int npts, const int *__restrict__ idx,
                                 const double *__restrict__ ref) {
    __shared__ double s0[kCmpThreads], s1[kCmpThreads];
    double a = 0.0, b = 0.0;
    for (int p = threadIdx.x; p < npts; p += kCmpThreads) {  // one block: fixed summation order
        const size_t off = (size_t)idx[3 * p] + (size_t)N * ((size_t)idx[3 * p + 1] + (size_t)N * idx[3 * p + 2]);
        const double d = (double)u[off] - ref[p];
        a += d * d;
        b += ref[p] * ref[p];
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int o = kCmpThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s0[threadIdx.x] += s0[threadIdx.x + o];
            s1[threadIdx.x] += s1[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        g_cmp[0] = s0[0];
        g_cmp[1] = s1[0];
    }
}

bool read_gaussians(int ng, const double *params, Gaussians &G) {
    if (ng < 1 || ng > kMaxG || !params) return false;
    G.n = ng;
    for (int g = 0; g < ng; ++g) {
        for (int a = 0; a < 3; ++a) {
            G.c[g][a] = params[7 * g + a];
            G.s[g][a] = params[7 * g + 3 + a];
            if (!(G.s[g][a] > 0.0)) return false;
        }
        G.q[g] = params[7 * g + 6];
    }
    return true;
}

}  // namespace

extern "C" int poisson_sample_gaussians(int N, double L, int ng, const double *params, int dtype, void *out_d,
                                        void *stream) {
    Gaussians G;
    if (N < 1 || N > 1024 || !(L > 0.0) || !out_d || !read_gaussians(ng, params, G)) return POISSON_ERR_ARG;
    if (dtype != POISSON_F32 && dtype != POISSON_F64) return POISSON_ERR_ARG;
    const size_t smem = (size_t)2 * ng * N * sizeof(double);
    cudaStream_t s = (cudaStream_t)stream;
    // The kernel also has a little static shared memory: opt in above 32 KB of dynamic.
    cudaError_t ea = cudaSuccess;
    if (dtype == POISSON_F32) {
        if (smem > 32 * 1024)
            ea = cudaFuncSetAttribute(k_sample<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ea == cudaSuccess) k_sample<float><<<N, 256, smem, s>>>(G, N, L, static_cast<float *>(out_d));
    } else {
        if (smem > 32 * 1024)
            ea = cudaFuncSetAttribute(k_sample<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ea == cudaSuccess) k_sample<double><<<N, 256, smem, s>>>(G, N, L, static_cast<double *>(out_d));
    }
    if (ea != cudaSuccess) {
        gsp::note_cuda_error(ea);
        return POISSON_ERR_CUDA;
    }
    const cudaError_t e = cudaGetLastError();
    gsp::note_cuda_error(e);
    return e == cudaSuccess ? POISSON_OK : POISSON_ERR_CUDA;
}

extern "C" int poisson_gaussian_potential(int N, double L, int ng, const double *params, int npts,
                                          const int *idx_d, double *out_d, void *stream) {
    Gaussians G;
    if (N < 1 || !(L > 0.0) || npts < 0 || (npts > 0 && (!idx_d || !out_d)) || !read_gaussians(ng, params, G))
        return POISSON_ERR_ARG;
    if (npts == 0) return POISSON_OK;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        const cudaError_t e = ensure_nodes();
        gsp::note_cuda_error(e);
        if (e != cudaSuccess) return POISSON_ERR_CUDA;
    }
    k_potential<<<(npts + 127) / 128, 128, 0, (cudaStream_t)stream>>>(G, N, L, npts, idx_d, out_d);
    const cudaError_t e = cudaGetLastError();
    gsp::note_cuda_error(e);
    return e == cudaSuccess ? POISSON_OK : POISSON_ERR_CUDA;
}

extern "C" int poisson_compare_points(const void *u_d, int dtype, int N, int npts, const int *idx_d,
                                      const double *ref_d, double *rel_l2, void *stream) {
    if (!u_d || !idx_d || !ref_d || !rel_l2 || npts < 1 || N < 1) return POISSON_ERR_ARG;
    if (dtype != POISSON_F32 && dtype != POISSON_F64) return POISSON_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (dtype == POISSON_F32)
        k_compare_points<float><<<1, kCmpThreads, 0, s>>>(static_cast<const float *>(u_d), N, npts, idx_d, ref_d);
    else
        k_compare_points<double><<<1, kCmpThreads, 0, s>>>(static_cast<const double *>(u_d), N, npts, idx_d, ref_d);
    double h[2];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(h, g_cmp, sizeof(h), 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    gsp::note_cuda_error(e);
    if (e != cudaSuccess) return POISSON_ERR_CUDA;
    *rel_l2 = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : 0.0;
    return POISSON_OK;
}
