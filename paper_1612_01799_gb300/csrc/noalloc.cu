// poisson_solve_noalloc: a small-grid solve that allocates nothing.
//
// Who needs it: code that must solve while it may not allocate device memory, for example
// a real-time loop that must not enter an allocator (an allocation can take unbounded
// time), or a process whose device memory is already reserved by a framework's caching
// allocator (a cudaMalloc there fails or forces the framework to release its cache).  A
// plan (poisson_plan_create) allocates its tables and workspace; this entry point instead
// keeps everything, symbol table, twiddles, the three workspace buffers and its status
// word, in one file-scope static device array, and its host-side setup uses fixed static
// host arrays.  It calls no cudaMalloc, cudaFree, malloc/new or other allocating routine.
//
// The array is allocated with the module: every GPU that loads this library holds its
// POISSON_NOALLOC_SCRATCH_BYTES until the process exits.  All calls share it.
// Layout: the status word in the first 256 bytes (a fixed place, so that a set-up for other
// parameters does not clear a timeout not yet read), then the tables and the workspace of
// the current parameters.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/poisson.h"
#include "solver.h"

namespace {

constexpr int kMaxN = POISSON_NOALLOC_MAX_N;
constexpr size_t kScratchBytes = POISSON_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxTerms = 512;
constexpr int kOrder = 16;
constexpr int kMaxPanels = (kMaxN + 1) / 2 > 16 ? (kMaxN + 1) / 2 : 16;
constexpr int kMaxNodes = kOrder * kMaxPanels;
constexpr int kMaxDevices = 64;
constexpr int kNfit = 4096;
constexpr size_t kStatusBytes = 256;  // the status word's slot at the start of the array
const double kPi = 3.141592653589793238462643383279502884;

// The scratch of every call: symbol octant, twiddles, setup inputs and the workspace.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceState {
    bool have_addr = false;
    unsigned char *base = nullptr;  // device address of g_scratch on this device
    bool have_tables = false;       // tables of (N, L, tol, dtype) are in the array
    int N = 0, dtype = -1;
    double L = 0.0, tol = 0.0;
    gsp::DevicePlan dp;
};

DeviceState g_state[kMaxDevices];
std::mutex g_mutex;

// Host-side setup storage (static: the setup does not allocate).
double h_tau[kMaxTerms], h_w[kMaxTerms];
double h_A[kMaxTerms * (kMaxN + 1)];
double h_t[kMaxNodes], h_wt[kMaxNodes], h_g[kMaxNodes];
double h_cos[(kMaxN + 1) * kMaxNodes];
double h_gx[kOrder], h_gw[kOrder];
double h_tw[4 * kMaxN];
float h_twf[4 * kMaxN];
float h_tw4[8 * kMaxN];

double erfc_inv(double y) {
    double lo = -10.0, hi = 30.0;
    for (int it = 0; it < 200 && hi - lo > 0; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (std::erfc(mid) > y) lo = mid; else hi = mid;
    }
    double x = 0.5 * (lo + hi);
    double d = -2.0 / std::sqrt(kPi) * std::exp(-x * x);
    if (d != 0.0) x -= (std::erfc(x) - y) / d;
    return x;
}

// Gaussian sum by sinc quadrature (Sec. 2, eq. approx), the same rule as a plan's setup:
// trapezoid nodes s_j = j h with tails cut at eps/4 each, h the largest 2/m reaching a
// maximum relative error <= eps on 4096 log-spaced radii in [delta, r_max].
int gauss_sum(double eps, double delta, double r_max, int &S) {
    const double t_lo = eps * std::sqrt(kPi) / (8.0 * r_max);
    const double t_hi = erfc_inv(0.25 * eps) / delta;
    const double s_lo = std::log(t_lo), s_hi = std::log(t_hi);
    const double lr0 = std::log(delta), lr1 = std::log(r_max);
    const double norm = 1.0 / (2.0 * std::pow(kPi, 1.5));
    for (int m = 2; m < 4000; ++m) {
        const double hh = 2.0 / m;
        const long j0 = (long)std::floor(s_lo / hh), j1 = (long)std::ceil(s_hi / hh);
        if (j1 - j0 + 1 > kMaxTerms) return POISSON_ERR_NUMERIC;
        int n = 0;
        for (long j = j0; j <= j1; ++j, ++n) {
            double s = (double)j * hh;
            h_tau[n] = std::exp(s);
            h_w[n] = hh * std::exp(s) * norm;
        }
        double e = 0.0;
        for (int i = 0; i < kNfit; ++i) {
            double r = std::exp(lr0 + (lr1 - lr0) * i / (kNfit - 1));
            if (i == 0) r = delta;
            if (i == kNfit - 1) r = r_max;
            double acc = 0.0;
            for (int j = 0; j < n; ++j) {
                double a = r * h_tau[j];
                acc += h_w[j] * std::exp(-a * a);
            }
            e = std::fmax(e, std::fabs(4.0 * kPi * r * acc - 1.0));
        }
        if (e <= eps) {
            S = n;
            return POISSON_OK;
        }
    }
    return POISSON_ERR_NUMERIC;
}

void gauss_legendre() {
    const int n = kOrder;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
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
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        h_gx[i] = -z;
        h_gx[n - 1 - i] = z;
        h_gw[i] = h_gw[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// A_j(k) = 2 int_0^2 exp(-tau_j^2 t^2) cos(pi k t/2) dt (Sec. 2, G-tensor factors): the
// full-line closed form for tau >= 3, composite Gauss-Legendre otherwise.
void axis_table(int S, int N) {
    const int K = N + 1;
    gauss_legendre();
    const int P = (N + 1) / 2 > 16 ? (N + 1) / 2 : 16;
    const int T = P * kOrder;
    for (int p = 0; p < P; ++p) {
        double a = 2.0 * p / P, b = 2.0 * (p + 1) / P;
        for (int i = 0; i < kOrder; ++i) {
            h_t[p * kOrder + i] = 0.5 * (a + b) + 0.5 * (b - a) * h_gx[i];
            h_wt[p * kOrder + i] = 0.5 * (b - a) * h_gw[i];
        }
    }
    for (int k = 0; k < K; ++k) {
        double kap = 0.5 * kPi * k;
        for (int n = 0; n < T; ++n) h_cos[(size_t)k * T + n] = std::cos(kap * h_t[n]);
    }
    for (int j = 0; j < S; ++j) {
        if (h_tau[j] >= 3.0) {
            for (int k = 0; k < K; ++k) {
                double kap = 0.5 * kPi * k;
                h_A[(size_t)j * K + k] =
                    std::sqrt(kPi) / h_tau[j] * std::exp(-kap * kap / (4.0 * h_tau[j] * h_tau[j]));
            }
            continue;
        }
        double t2 = h_tau[j] * h_tau[j];
        for (int n = 0; n < T; ++n) h_g[n] = h_wt[n] * std::exp(-t2 * h_t[n] * h_t[n]);
        for (int k = 0; k < K; ++k) {
            const double *c = &h_cos[(size_t)k * T];
            double acc = 0.0, comp = 0.0;
            for (int n = 0; n < T; ++n) {
                const double term = h_g[n] * c[n];
                const double t = acc + term;
                comp += (std::fabs(acc) >= std::fabs(term)) ? (acc - t) + term : (term - t) + acc;
                acc = t;
            }
            h_A[(size_t)j * K + k] = 2.0 * (acc + comp);
        }
    }
}

double radial_moment(int p, double tau, double d) {
    double x = tau * d;
    if (x < 0.5) {
        double total = 0.0, fact = 1.0, t2n = 1.0;
        for (int n = 0; n < 80; ++n) {
            if (n > 0) {
                fact *= n;
                t2n *= -tau * tau;
            }
            double term = t2n * std::pow(d, 2 * n + p + 1) / (fact * (2 * n + p + 1));
            total += term;
            if (std::fabs(term) <= 1e-20 * std::fabs(total)) break;
        }
        return total;
    }
    double e = std::exp(-x * x), er = std::erf(x);
    if (p == 2) return std::sqrt(kPi) * er / (4.0 * tau * tau * tau) - d * e / (2.0 * tau * tau);
    return 3.0 * std::sqrt(kPi) * er / (8.0 * std::pow(tau, 5)) -
           e * (d * d * d / (2.0 * tau * tau) + 3.0 * d / (4.0 * std::pow(tau, 4)));
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return POISSON_OK;
    return e == cudaErrorMemoryAllocation ? POISSON_ERR_ALLOC : POISSON_ERR_CUDA;
}

// Tables for (N, L, tol, dtype) into the device array of `st` (the Sec. 3 setup phase).
int setup(DeviceState &st, int N, double L, double tol, int dtype, cudaStream_t s) {
    const double delta = std::fmax(2.0 * L / (50.0 * N), 1e-3);
    if (!(delta < 1.0)) return POISSON_ERR_ARG;
    const double eps = std::fmin(std::fmax(0.1 * tol, 1e-14), 1e-7);
    int S = 0;
    int rc = gauss_sum(eps, delta, 2.0 * std::sqrt(3.0), S);
    if (rc) return rc;
    axis_table(S, N);
    double s2 = 0.0, s4 = 0.0;
    for (int j = 0; j < S; ++j) {
        s2 += h_w[j] * radial_moment(2, h_tau[j], delta);
        s4 += h_w[j] * radial_moment(4, h_tau[j], delta);
    }
    const double C0 = 0.5 * delta * delta - 4.0 * kPi * s2;
    const double C2 = (0.25 * std::pow(delta, 4) - 4.0 * kPi * s4) / 6.0;
    const long double two_pi = 2.0L * std::acos(-1.0L);
    for (int e = 0; e < 2 * N; ++e) {
        long double a = two_pi * (long double)e / (long double)(2 * N);
        h_tw[2 * e] = (double)std::cos(a);
        h_tw[2 * e + 1] = (double)-std::sin(a);
        h_twf[2 * e] = (float)h_tw[2 * e];
        h_twf[2 * e + 1] = (float)h_tw[2 * e + 1];
        h_tw4[4 * e] = h_tw4[4 * e + 1] = h_twf[2 * e];
        h_tw4[4 * e + 2] = h_tw4[4 * e + 3] = h_twf[2 * e + 1];
    }

    // Layout of the array (256-byte aligned pieces).
    const size_t elem = dtype == POISSON_F32 ? 4 : 8, cx = 2 * elem;
    const size_t K = (size_t)N + 1;
    const int Px = gsp::pitch_for(N);
    const int Ps = gsp::sym_pitch_for(N);
    size_t off = kStatusBytes;
    auto take = [&](size_t bytes) {
        unsigned char *p = st.base + off;
        off = align256(off + bytes);
        return p;
    };
    gsp::DevicePlan dp;
    dp.N = N;
    dp.dtype = dtype;
    dp.Px = Px;
    dp.Ps = Ps;
    dp.sym = take(K * K * (size_t)Ps * elem);
    dp.tw = take((size_t)2 * N * cx);
    dp.twc = dtype == POISSON_F32 ? take((size_t)2 * N * 4 * sizeof(float)) : dp.tw;
    double *dA = reinterpret_cast<double *>(take((size_t)S * K * sizeof(double)));
    double *dw = reinterpret_cast<double *>(take((size_t)S * sizeof(double)));
    dp.w1 = take((size_t)N * N * Px * cx);
    dp.w2 = take((size_t)N * 2 * N * Px * cx);
    dp.w3 = take((size_t)N * 2 * N * Px * cx);
    dp.status = reinterpret_cast<int *>(st.base);
    if (off > kScratchBytes) return POISSON_ERR_UNSUPPORTED;
    if (gsp::encode_tma_maps(dp) != cudaSuccess) return POISSON_ERR_CUDA;

    cudaError_t e;
    // The workspace is cleared when the parameters change, so that no value left by a solve
    // of another size sits in its padding columns.  Nothing reads those columns, and every
    // element a pass reads was written by the pass before it in the same call, so no result
    // depends on this clearing.
    if ((e = cudaMemsetAsync(dp.w1, 0, (size_t)(st.base + off - (unsigned char *)dp.w1), s)))
        return map_cuda(e);
    if ((e = cudaMemcpyAsync(dA, h_A, (size_t)S * K * sizeof(double), cudaMemcpyHostToDevice, s)))
        return map_cuda(e);
    if ((e = cudaMemcpyAsync(dw, h_w, (size_t)S * sizeof(double), cudaMemcpyHostToDevice, s)))
        return map_cuda(e);
    if (dtype == POISSON_F32) {
        e = cudaMemcpyAsync(dp.tw, h_twf, (size_t)2 * N * cx, cudaMemcpyHostToDevice, s);
        if (e) return map_cuda(e);
        e = cudaMemcpyAsync(dp.twc, h_tw4, (size_t)2 * N * 4 * sizeof(float), cudaMemcpyHostToDevice, s);
    } else {
        e = cudaMemcpyAsync(dp.tw, h_tw, (size_t)2 * N * cx, cudaMemcpyHostToDevice, s);
    }
    if (e) return map_cuda(e);
    const double M = 2.0 * N;
    if ((e = gsp::launch_symbol_table(dp, dA, dw, S, C0, C2, L * L / (M * M * M), 0, s)))
        return map_cuda(e);
    // The host arrays are reused by the next setup: wait for the copies and the table.
    if ((e = cudaStreamSynchronize(s))) return map_cuda(e);
    st.dp = dp;
    st.N = N;
    st.L = L;
    st.tol = tol;
    st.dtype = dtype;
    st.have_tables = true;
    return POISSON_OK;
}

// The array's device address on the current device (looked up once per device, with that
// device current), or an error.  Called with g_mutex held.
int device_state(DeviceState *&out, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return map_cuda(e);
    if (dev < 0 || dev >= kMaxDevices) return POISSON_ERR_UNSUPPORTED;
    DeviceState &st = g_state[dev];
    if (!st.have_addr) {
        void *ptr = nullptr;
        if ((e = cudaGetSymbolAddress(&ptr, g_scratch)) != cudaSuccess) return map_cuda(e);
        // The status word must start at zero; it is cleared here once per device and then
        // only by poisson_noalloc_last_status.
        if ((e = cudaMemsetAsync(ptr, 0, kStatusBytes, s)) != cudaSuccess) return map_cuda(e);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return map_cuda(e);
        st.base = static_cast<unsigned char *>(ptr);
        st.have_addr = true;
    }
    out = &st;
    return POISSON_OK;
}

}  // namespace

extern "C" int poisson_solve_noalloc(int N, double L, double tol, int dtype, const void *rho_d,
                                     void *u_d, void *stream) {
    if (!rho_d || !u_d) return POISSON_ERR_ARG;
    if (dtype != POISSON_F32 && dtype != POISSON_F64) return POISSON_ERR_ARG;
    if (N < 4 || (N & 1) || !(L > 0.0) || !(tol > 0.0) || !std::isfinite(L) || !std::isfinite(tol))
        return POISSON_ERR_ARG;
    if (N > kMaxN || !gsp::n_supported(N)) return POISSON_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceState *st = nullptr;
    int rc = device_state(st, s);
    if (rc) return rc;
    if (!st->have_tables || st->N != N || st->L != L || st->tol != tol || st->dtype != dtype) {
        st->have_tables = false;
        rc = setup(*st, N, L, tol, dtype, s);
        if (rc) return rc;
    }
    gsp::PtrArray in, out;
    in.p[0] = rho_d;
    out.p[0] = u_d;
    for (int i = 1; i < gsp::kMaxBatch; ++i) in.p[i] = out.p[i] = nullptr;
    return map_cuda(gsp::launch_solve(st->dp, in, out, 1, s, nullptr));
}

extern "C" int poisson_noalloc_last_status(void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceState *st = nullptr;
    int rc = device_state(st, s);
    if (rc) return rc;
    static int h_status;  // static: the read allocates nothing; g_mutex serialises its use
    h_status = 0;
    cudaError_t e = cudaMemcpyAsync(&h_status, st->base, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return map_cuda(e);
    if (h_status == 0) return POISSON_OK;
    const int h = h_status;
    e = cudaMemsetAsync(st->base, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return map_cuda(e);
    return (h & gsp::kStatusTimeoutBit) ? POISSON_ERR_TIMEOUT : POISSON_ERR_CUDA;
}

extern "C" int poisson_noalloc_selftest_wait(long long polls, void *stream) {
    if (polls < 1 || polls > (1ll << 24)) return POISSON_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceState *st = nullptr;
    int rc = device_state(st, s);
    if (rc) return rc;
    static gsp::DevicePlan probe;  // only its status pointer is used
    probe.status = reinterpret_cast<int *>(st->base);
    return map_cuda(gsp::launch_wait_selftest(probe, polls, s));
}
