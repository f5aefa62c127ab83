// Plan setup on the device: the per-axis factors of the G-tensor (Sec. 2) and the symbol
// table of a rectangular box.  The per-axis factors (Sec. 2),
//   A_j(k) = 2 int_0^2 exp(-tau_j^2 t^2) cos(kappa_k t) dt,  kappa_k = pi k / 2,  k = 0..N,
// by the rule of the host setup (build_axis_table): the full-line closed form
// (sqrt(pi) / tau) exp(-kappa^2 / (4 tau^2)) for tau >= 3, where the Gaussian is below
// erfc(6) ~ 2e-17 of its mass at t = 2; otherwise the composite 16-point Gauss-Legendre
// rule with P = max(16, (N + 1) / 2) equal panels on [0, 2] and compensated (Neumaier)
// summation over the nodes in order, in FP64.
//
// Thread (j, k).  The block stages g_n = w_n exp(-tau_j^2 t_n^2) for every node n = 16 p + i
// (t_n = (2p + 1 + x_i) / P, w_n = v_i / P for the Gauss-Legendre nodes x_i and weights
// v_i).  For one node position i the cosines of successive panels differ by the angle
// 2 kappa / P, so each thread rotates (cos, sin) from panel to panel and takes them afresh
// from sincos every kReseed panels.
#include <cuda_runtime.h>

#include "fft_core.cuh"
#include "setup.h"
#include "solver.h"

namespace gsp {

namespace {
constexpr int kReseed = 16;
constexpr double kPiD = 3.141592653589793238462643383279502884;

__global__ void k_axis_table(const double *__restrict__ tau, const double *__restrict__ gl, int N, int P,
                             double *__restrict__ A) {
    extern __shared__ double g[];  // 16 P node weights of term j
    const int j = blockIdx.y, K = N + 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const double tj = tau[j];
    const double kap = 0.5 * kPiD * k;
    if (tj >= 3.0) {
        if (k < K) A[(size_t)j * K + k] = sqrt(kPiD) / tj * exp(-kap * kap / (4.0 * tj * tj));
        return;
    }
    const double *gx = gl, *gw = gl + 16;
    for (int n = threadIdx.x; n < 16 * P; n += blockDim.x) {
        const double t = (2.0 * (n >> 4) + 1.0 + gx[n & 15]) / P;
        g[n] = gw[n & 15] / P * exp(-tj * tj * t * t);
    }
    __syncthreads();
    if (k >= K) return;
    double sd, cd;
    sincos(2.0 * kap / P, &sd, &cd);
    double c[16], s[16];
    double acc = 0.0, comp = 0.0;
    for (int p = 0; p < P; ++p) {
        if (p % kReseed == 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) sincos(kap * ((2.0 * p + 1.0 + gx[i]) / P), &s[i], &c[i]);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const double term = g[16 * p + i] * c[i];
            const double sum = acc + term;
            comp += fabs(acc) >= fabs(term) ? (acc - sum) + term : (term - sum) + acc;
            acc = sum;
            const double cn = c[i] * cd - s[i] * sd;
            s[i] = s[i] * cd + c[i] * sd;
            c[i] = cn;
        }
    }
    A[(size_t)j * K + k] = 2.0 * (acc + comp);
}

// The symbol of a box [-l_1, l_1] x [-l_2, l_2] x [-l_3, l_3] (Sec. 2 standardised form):
// sum_j w_j Ax_j(kx) Ay_j(ky) Az_j(kz) with the per-axis factors of each axis (n_q + 1
// frequencies on axis q), and kappa_q = pi k_q / (2 l_q) in the correction (il2[q] = 1 / l_q^2);
// `literal` as in k_symbol_table.  The table is not symmetric: block (ky, kz) computes its
// whole kx line, sym[(kz * Ky + ky) * Ps + kx], and, when symT is set, writes it transposed,
// symT[(kx * Ky + ky) * Ps + kz], for the z warp forms, which read the table with kz
// innermost (those plans have Kx = Ky = Kz).
template <typename Real>
__global__ void k_symbol_box(Real *__restrict__ sym, Real *__restrict__ symT, const double *__restrict__ Ax,
                             const double *__restrict__ Ay, const double *__restrict__ Az, const double *__restrict__ w,
                             int nterms, int Kx, int Ky, int Ps, double C0, double C2, double scale, double il2x,
                             double il2y, double il2z, int literal) {
    extern __shared__ double cj[];
    const int b = blockIdx.x, c = blockIdx.y;
    for (int j = threadIdx.x; j < nterms; j += blockDim.x)
        cj[j] = w[j] * Ay[(long long)j * Ky + b] * Az[(long long)j * gridDim.y + c];
    __syncthreads();
    const double hp2 = 0.25 * 3.141592653589793238462643383279502884 * 3.141592653589793238462643383279502884;
    for (int a = threadIdx.x; a < Kx; a += blockDim.x) {
        double sum = 0.0;
        for (int j = 0; j < nterms; ++j) sum += cj[j] * Ax[(long long)j * Kx + a];
        const double k2 = (double)a * a * il2x + (double)b * b * il2y + (double)c * c * il2z;
        double v;
        if (!literal) v = sum + C0 - C2 * hp2 * k2;
        else v = ((a | b | c) & 1) ? sum : sum + 8.0 * (C0 - C2 * hp2 * k2);
        sym[((long long)c * Ky + b) * Ps + a] = (Real)(scale * v);
        if (symT) symT[((long long)a * Ky + b) * Ps + c] = (Real)(scale * v);
    }
}

template <typename Real>
cudaError_t symbol_table_box(const DevicePlan &p, const double *dA3, const double *dw, int nterms,
                             double C0, double C2, double scale, const double *l, int literal, cudaStream_t s) {
    const int Kx = (p.any ? p.n3[0] : p.N) + 1, Ky = (p.any ? p.n3[1] : p.N) + 1, Kz = (p.any ? p.n3[2] : p.N) + 1;
    const size_t bytes = (size_t)Kz * Ky * p.Ps * sizeof(Real);
    cudaError_t e = cudaMemsetAsync(p.sym, 0, bytes, s);
    if (e != cudaSuccess) return e;
    if (p.symT && (e = cudaMemsetAsync(p.symT, 0, bytes, s)) != cudaSuccess) return e;
    const double *Ax = dA3, *Ay = Ax + (size_t)nterms * Kx, *Az = Ay + (size_t)nterms * Ky;
    k_symbol_box<Real><<<dim3(Ky, Kz), 128, nterms * sizeof(double), s>>>(
        static_cast<Real *>(p.sym), static_cast<Real *>(p.symT), Ax, Ay, Az, dw, nterms, Kx, Ky, p.Ps, C0, C2,
        scale, 1.0 / (l[0] * l[0]), 1.0 / (l[1] * l[1]), 1.0 / (l[2] * l[2]), literal);
    return cudaGetLastError();
}
}  // namespace

cudaError_t symbol_table_box_f32(const DevicePlan &p, const double *dA3, const double *dw, int nterms,
                                 double C0, double C2, double scale, const double *l, int literal,
                                 cudaStream_t s) {
    return symbol_table_box<float>(p, dA3, dw, nterms, C0, C2, scale, l, literal, s);
}
cudaError_t symbol_table_box_f64(const DevicePlan &p, const double *dA3, const double *dw, int nterms,
                                 double C0, double C2, double scale, const double *l, int literal,
                                 cudaStream_t s) {
    return symbol_table_box<double>(p, dA3, dw, nterms, C0, C2, scale, l, literal, s);
}
cudaError_t symbol_table_box_df(const DevicePlan &p, const double *dA3, const double *dw, int nterms,
                                double C0, double C2, double scale, const double *l, int literal,
                                cudaStream_t s) {
    return symbol_table_box<DF>(p, dA3, dw, nterms, C0, C2, scale, l, literal, s);
}

cudaError_t launch_axis_table(const double *dtau, const double *dgl, int S, int N, double *dA, cudaStream_t s) {
    const int P = axis_table_panels(N);
    const size_t smem = (size_t)16 * P * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_axis_table, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const dim3 grid((N + 1 + 127) / 128, S);
    k_axis_table<<<grid, 128, smem, s>>>(dtau, dgl, N, P, dA);
    return cudaGetLastError();
}

}  // namespace gsp
