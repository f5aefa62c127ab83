// The five passes of one solve (Exl, arXiv:1612.01799, Sec. 2/3: zero-padded FFT
// convolution with the G-tensor plus the near-zone correction, crop to N^3), templated
// on the arithmetic type and N.  Included by one .cu file per type.
//
//   K1 x forward   rho [z][y][x] (N reals per row)  -> w1 [z][y][kx <= N]
//                  length-2N real DFT of the zero-padded row as an N-point complex FFT of
//                  the (even, odd) pairs (pruned: the upper N/2 pairs are zero), then the
//                  standard split into the N+1 Hermitian bins.
//   K2 y forward   w1 -> w2 [z][ky < 2N][kx]    length 2N, upper half of the input zero
//   K3 z fused     w2 -> w3 [z < N][ky][kx]     length 2N forward (upper half zero),
//                  product with the symbol G_tot(|kx|, |ky|, |kz|) scaled by
//                  lambda^2/(2N)^3, length 2N inverse keeping the lower half.  The
//                  (2N)^3 spectrum exists only in registers and shared memory: the
//                  inverse runs its radices in reverse order, so it starts from the
//                  forward's last-stage registers and the symbol is applied there.
//   K4 y inverse   w3 -> w1 [z][y < N][kx]      length 2N inverse, lower half kept
//   K5 x inverse   w1 -> u [z][y][x]            N+1 Hermitian bins -> N-point complex
//                  inverse FFT of the (even, odd) pairs, lower N/2 pairs kept (the crop).
//
// The column passes (K2-K4) of the FP32 path process two neighbouring columns per thread
// with packed FP32x2 arithmetic (type CV); the row passes and the FP64 path use one
// complex value per slot.
#pragma once
#include <mutex>
#include <type_traits>

#include "fft_core.cuh"
#include "solver.h"

namespace gsp {

// Per-thread element count E and radix sequence of a length-L transform.  The first and
// the last radix are even: the pruning rules (inputs r >= R/2 of stage 0 are zero, outputs
// r >= R/2 of the last stage are dropped) select exactly the rows >= L/2 only then.
template <int L> struct FftCfg;
#define GSP_FFT_CFG(LL, EE, ...)                  \
    template <> struct FftCfg<LL> {              \
        static constexpr int E = EE;             \
        using Rs = Radices<__VA_ARGS__>;         \
    }
GSP_FFT_CFG(4, 4, 4);
GSP_FFT_CFG(8, 8, 8);
GSP_FFT_CFG(16, 16, 16);
GSP_FFT_CFG(32, 8, 8, 4);
GSP_FFT_CFG(48, 12, 4, 3, 4);
GSP_FFT_CFG(64, 8, 8, 8);
GSP_FFT_CFG(80, 20, 4, 5, 4);
GSP_FFT_CFG(96, 24, 8, 3, 4);
GSP_FFT_CFG(128, 16, 16, 8);
GSP_FFT_CFG(160, 20, 4, 4, 5, 2);
GSP_FFT_CFG(192, 24, 8, 3, 8);
GSP_FFT_CFG(256, 16, 16, 16);
GSP_FFT_CFG(320, 20, 4, 4, 5, 4);
GSP_FFT_CFG(384, 24, 8, 8, 6);
GSP_FFT_CFG(512, 16, 16, 8, 4);
GSP_FFT_CFG(640, 20, 4, 4, 4, 5, 2);
GSP_FFT_CFG(768, 24, 8, 8, 6, 2);
GSP_FFT_CFG(1024, 16, 16, 16, 4);
GSP_FFT_CFG(2048, 16, 16, 16, 8);
#undef GSP_FFT_CFG

// The schedule a pass uses for its arithmetic: FftCfg, except in double-float, whose
// butterflies are about ten times longer in instructions: there the lengths that FftCfg
// does in radix 16 (16 values per thread) run in radices 8 and 4 with 8 values per thread
// (and 96, 384 and 768 with 12), so that a kernel's code stays within the instruction cache.
template <typename Real, int L> struct Cfg : FftCfg<L> {};
#define GSP_DF_CFG(LL, EE, ...)                  \
    template <> struct Cfg<DF, LL> {             \
        static constexpr int E = EE;             \
        using Rs = Radices<__VA_ARGS__>;         \
    }
GSP_DF_CFG(16, 4, 4, 4);
GSP_DF_CFG(96, 12, 4, 6, 4);
GSP_DF_CFG(128, 8, 8, 4, 4);
GSP_DF_CFG(256, 8, 8, 8, 4);
GSP_DF_CFG(384, 12, 4, 4, 6, 4);
GSP_DF_CFG(512, 8, 8, 8, 8);
GSP_DF_CFG(768, 12, 4, 4, 4, 6, 2);
GSP_DF_CFG(1024, 8, 8, 8, 4, 4);
GSP_DF_CFG(2048, 8, 8, 8, 8, 4);
#undef GSP_DF_CFG

// Complex types per arithmetic: CS for the row passes, CC (W columns per thread) for the
// column passes.
template <typename Real> struct Types;
template <> struct Types<float> {
    using CS = CF;
    using CC = CV;
    static constexpr int W = 2;
};
template <> struct Types<double> {
    using CS = CD;
    using CC = CD;
    static constexpr int W = 1;
};
// Double-float arithmetic (the FP64 path on the FP32 pipe): one complex value per slot.
template <> struct Types<DF> {
    using CS = CDF;
    using CC = CDF;
    static constexpr int W = 1;
};

// Columns per CTA of a column pass: 128-byte row segments (16 FP32 or 8 FP64 complex),
// halved until the block has <= 1024 threads and <= 128 KB of shared memory.
template <typename Real, int L> __host__ __device__ constexpr int col_tc() {
    const int W = Types<Real>::W;
    int tc = sizeof(Real) == 4 ? 16 : 8;
    const int P = L / Cfg<Real, L>::E;
    while (tc > W && ((tc / W) * P > 1024 || tc * L * 2 * (int)sizeof(Real) > 131072)) tc /= 2;
    return tc;
}
template <typename Real, int L> __host__ __device__ constexpr int col_threads() {
    return (col_tc<Real, L>() / Types<Real>::W) * (L / Cfg<Real, L>::E);
}
// Rows per CTA of an x pass (shared tile (N+1) x (TR+1) complex).
template <typename Real, int L> __host__ __device__ constexpr int row_tr() {
    int tr = sizeof(Real) == 4 ? 16 : 8;
    const int P = L / Cfg<Real, L>::E;
    while (tr > 1 && (tr * P > 1024 || (L + 1) * (tr + 1) * 2 * (int)sizeof(Real) > 163840)) tr /= 2;
    return tr;
}

// ---- loads and stores of W neighbouring complex values ---------------------------------
__device__ __forceinline__ CV ld_cc(const float2 *p) {
    const float4 f = __ldg(reinterpret_cast<const float4 *>(p));
    return {make_float2(f.x, f.z), make_float2(f.y, f.w)};
}
__device__ __forceinline__ void st_cc(float2 *p, CV x) {
    *reinterpret_cast<float4 *>(p) = make_float4(x.re.x, x.im.x, x.re.y, x.im.y);
}
__device__ __forceinline__ CD ld_cc(const double2 *p) {
    const double2 f = __ldg(p);
    return {f.x, f.y};
}
__device__ __forceinline__ void st_cc(double2 *p, CD x) { *p = make_double2(x.re, x.im); }
// Double-float workspace values: float4 (re.hi, re.lo, im.hi, im.lo).
__device__ __forceinline__ CDF ld_cc(const float4 *p) {
    const float4 f = __ldg(p);
    return {DF(f.x, f.y), DF(f.z, f.w)};
}
__device__ __forceinline__ void st_cc(float4 *p, CDF x) { *p = make_float4(x.re.hi, x.re.lo, x.im.hi, x.im.lo); }
__device__ __forceinline__ CF ld_cs(const float2 *p) {
    const float2 f = *p;
    return {f.x, f.y};
}
__device__ __forceinline__ CD ld_cs(const double2 *p) {
    const double2 f = *p;
    return {f.x, f.y};
}
// Symbol factors of the W columns.
__device__ __forceinline__ CV scale_sym(CV x, const float *s) {
    return cscale2(x, __ldg(reinterpret_cast<const float2 *>(s)));
}
__device__ __forceinline__ CD scale_sym(CD x, const double *s) { return cscale(x, __ldg(s)); }
__device__ __forceinline__ CDF scale_sym(CDF x, const DF *s) {
    const float2 f = __ldg(reinterpret_cast<const float2 *>(s));
    return cscale(x, DF(f.x, f.y));
}

// Storage of one complex workspace value (Cx2) and of a pair of consecutive real samples of
// the caller's density or potential (Ext2) for each arithmetic.  Double-float keeps its
// workspace in its own format and converts from and to FP64 only where the x passes read
// rho and write u.
template <typename Real> struct Store;
template <> struct Store<float> {
    using Ws = float2;
    using Ext = float2;
};
template <> struct Store<double> {
    using Ws = double2;
    using Ext = double2;
};
template <> struct Store<DF> {
    using Ws = float4;
    using Ext = double2;
};
template <typename Real> using Cx2 = typename Store<Real>::Ws;
template <typename Real> using Ext2 = typename Store<Real>::Ext;

__device__ __forceinline__ void st_ws(float2 *p, CF x) { *p = make_float2(x.re, x.im); }
__device__ __forceinline__ void st_ws(double2 *p, CD x) { *p = make_double2(x.re, x.im); }
__device__ __forceinline__ void st_ws(float4 *p, CDF x) { *p = make_float4(x.re.hi, x.re.lo, x.im.hi, x.im.lo); }
__device__ __forceinline__ CF ws_c(float2 f) { return {f.x, f.y}; }
__device__ __forceinline__ CD ws_c(double2 f) { return {f.x, f.y}; }
__device__ __forceinline__ CDF ws_c(float4 f) { return {DF(f.x, f.y), DF(f.z, f.w)}; }
__device__ __forceinline__ float2 c_ext(CF x) { return make_float2(x.re, x.im); }
__device__ __forceinline__ double2 c_ext(CD x) { return make_double2(x.re, x.im); }
__device__ __forceinline__ double2 c_ext(CDF x) { return make_double2(df_to_double(x.re), df_to_double(x.im)); }

// Twiddle tables of the runtime-length forms: exp(-2 pi i e / (2 n_q)) in the workspace
// storage of the arithmetic.
template <typename Real> using AnyTw = Cx2<Real>;

}  // namespace gsp
#include "passes_tma.cuh"
#include "passes_zwarp.cuh"
#include "passes_xy.cuh"
#include "passes_any.cuh"
namespace gsp {

// ---- K1: x forward (real, zero-padded to 2N) -------------------------------------------
// Rows (y, z) of all densities are numbered b N^2 + y + N z; a CTA's TR rows never straddle
// two densities (TR divides N^2).
template <typename Real, int N>
__global__ void __launch_bounds__(row_tr<Real, N>() * (N / Cfg<Real, N>::E))
k_x_forward(const PtrArray rho, Cx2<Real> *__restrict__ out, const Cx2<Real> *__restrict__ tw,
            int nrows, int Px) {
    using C = typename Types<Real>::CS;
    using T2 = Cx2<Real>;
    using X2 = Ext2<Real>;
    constexpr int E = Cfg<Real, N>::E, P = N / E, TR = row_tr<Real, N>(), SP = TR + 1, NT = TR * P;
    static_assert((N * N) % TR == 0, "row tiles stay inside one density");
    extern __shared__ __align__(16) unsigned char smraw[];
    griddep_wait();
    C *sm = reinterpret_cast<C *>(smraw);  // (N + 1) x SP
    const int t = threadIdx.x;
    const long long r0 = (long long)blockIdx.x * TR;
    const int nr = (int)min((long long)TR, (long long)nrows - r0);
    const int b = (int)(r0 / (N * N));
    // The tile is nr consecutive rows of N reals: contiguous N/2-pair chunks.
    const X2 *src = reinterpret_cast<const X2 *>(rho.p[b]) + (r0 - (long long)b * N * N) * (N / 2);
    for (int e = t; e < nr * (N / 2); e += NT) {
        const int r = e / (N / 2), m = e - r * (N / 2);
        const X2 f = __ldg(src + e);
        sm[m * SP + r] = C{f.x, f.y};
    }
    __syncthreads();
    const int c = t % TR, q = t / TR;
    C v[E];
    constexpr RunOpt opt{false, true, false, false, true};
    Stages<C, N, E, -1, 1, typename Cfg<Real, N>::Rs>::template run<opt>(
        v, q, c, sm, SP, tw, 2, [&](int row) { return sm[row * SP + c]; },
        [&](int row, C x) { sm[row * SP + c] = x; });
    __syncthreads();
    // C = FFT_N(pairs).  With Ev_k = (C_k + conj C_{N-k})/2 (DFT of the even samples) and
    // Od_k = (C_k - conj C_{N-k})/(2i) (odd samples): X_k = Ev_k + W_{2N}^k Od_k,
    // X_{N-k} = conj(Ev_k - W_{2N}^k Od_k), X_0 = Ev_0 + Od_0, X_N = Ev_0 - Od_0.
    for (int e = t; e < TR * (N / 2 + 1); e += NT) {
        const int r = e % TR, k = e / TR;
        if (r >= nr) continue;
        const C ck = sm[k * SP + r];
        const C cn = sm[((N - k) % N) * SP + r];
        const C ev = {(Real)0.5 * (ck.re + cn.re), (Real)0.5 * (ck.im - cn.im)};
        const C od = {(Real)0.5 * (ck.im + cn.im), (Real)0.5 * (cn.re - ck.re)};
        if (k == 0) {
            sm[r] = C{ev.re + od.re, (Real)0};
            sm[N * SP + r] = C{ev.re - od.re, (Real)0};
        } else {
            const C wo = twmul<-1>(od, __ldg(tw + k));
            sm[k * SP + r] = cadd(ev, wo);
            if (2 * k != N) {
                const C d = csub(ev, wo);
                sm[(N - k) * SP + r] = C{d.re, -d.im};
            }
        }
    }
    __syncthreads();
    T2 *dst = out + r0 * Px;
    for (int e = t; e < nr * (N + 1); e += NT) {
        const int r = e / (N + 1), k = e - r * (N + 1);
        st_ws(dst + (long long)r * Px + k, sm[k * SP + r]);
    }
}

// ---- K2 / K4: y transform over columns kx --------------------------------------------
// FWD: rows < L/2 of the input are nonzero, all L outputs stored.
// !FWD: all L inputs, outputs < L/2 stored.
template <typename Real, int L, bool FWD>
__global__ void __launch_bounds__(col_threads<Real, L>())
k_col(const Cx2<Real> *__restrict__ in, Cx2<Real> *__restrict__ out,
      const typename TwOf<typename Types<Real>::CC>::T *__restrict__ tw, int ncols, long long in_row,
      long long in_outer, long long out_row, long long out_outer) {
    using C = typename Types<Real>::CC;
    constexpr int W = Types<Real>::W, E = Cfg<Real, L>::E, TC = col_tc<Real, L>(), NG = TC / W;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);  // L x NG
    const int g = threadIdx.x % NG, q = threadIdx.x / NG;
    const int col = blockIdx.x * TC + W * g;
    const bool valid = col < ncols;
    const Cx2<Real> *src = in + (long long)blockIdx.y * in_outer + col;
    Cx2<Real> *dst = out + (long long)blockIdx.y * out_outer + col;
    C v[E];
    constexpr RunOpt opt{false, FWD, false, !FWD, false};
    Stages<C, L, E, FWD ? -1 : 1, 1, typename Cfg<Real, L>::Rs>::template run<opt>(
        v, q, g, sm, NG, tw, 1,
        [&](int row) { return valid ? ld_cc(src + row * in_row) : czero<C>(); },
        [&](int row, C x) {
            if (valid) st_cc(dst + row * out_row, x);
        });
}

// ---- K3: z forward, symbol, z inverse --------------------------------------------------
template <typename Real, int L>
__global__ void __launch_bounds__(col_threads<Real, L>())
k_z_symbol(const Cx2<Real> *__restrict__ in, Cx2<Real> *__restrict__ out, const Real *__restrict__ sym,
           const typename TwOf<typename Types<Real>::CC>::T *__restrict__ tw, int ncols, int Px,
           int Ps) {
    using C = typename Types<Real>::CC;
    using Rs = typename Cfg<Real, L>::Rs;
    constexpr int N = L / 2, W = Types<Real>::W, E = Cfg<Real, L>::E, TC = col_tc<Real, L>(), NG = TC / W;
    constexpr int P = L / E;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);  // L x NG
    const int g = threadIdx.x % NG, q = threadIdx.x / NG;
    const int col = blockIdx.x * TC + W * g;
    const bool valid = col < ncols;
    // Consecutive blocks take ky and its mirror 2N - ky, which read the same symbol rows.
    const int by = blockIdx.y;
    const int ky = (by & 1) ? L - ((by + 1) >> 1) : (by >> 1);
    const int kya = ky <= N ? ky : L - ky;
    const long long zs = (long long)L * Px;  // z stride of w2 / w3
    const Cx2<Real> *src = in + (long long)ky * Px + col;
    Cx2<Real> *dst = out + (long long)ky * Px + col;
    const long long plane = (long long)(N + 1) * Ps;
    const Real *srow = sym + (long long)kya * Ps + (valid ? col : 0);
    C v[E];
    constexpr RunOpt fwd{false, true, true, false, false};
    Stages<C, L, E, -1, 1, Rs>::template run<fwd>(
        v, q, g, sm, NG, tw, 1, [&](int row) { return valid ? ld_cc(src + row * zs) : czero<C>(); },
        [&](int, C) {});
    // The forward's last stage (radix RL) left row j + r L/RL of butterfly b in v[b RL + r].
    constexpr int RL = LastRadix<Rs>::v;
#pragma unroll
    for (int b = 0; b < E / RL; ++b) {
        const int j = q + P * b;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
            const int row = j + r * (L / RL);
            const int kz = row <= N ? row : L - row;
            v[b * RL + r] = scale_sym(v[b * RL + r], srow + kz * plane);
        }
    }
    constexpr RunOpt inv{true, false, false, true, false};
    Stages<C, L, E, 1, 1, Reverse<Rs>>::template run<inv>(
        v, q, g, sm, NG, tw, 1, [&](int) { return czero<C>(); },
        [&](int row, C x) {
            if (valid) st_cc(dst + row * zs, x);
        });
}

// ---- K5: x inverse (Hermitian N+1 bins -> N real samples) -------------------------------
template <typename Real, int N>
__global__ void __launch_bounds__(row_tr<Real, N>() * (N / Cfg<Real, N>::E))
k_x_inverse(const Cx2<Real> *__restrict__ in, const PtrArray u, const Cx2<Real> *__restrict__ tw,
            int nrows, int Px) {
    using C = typename Types<Real>::CS;
    using T2 = Cx2<Real>;
    using X2 = Ext2<Real>;
    constexpr int E = Cfg<Real, N>::E, P = N / E, TR = row_tr<Real, N>(), SP = TR + 1, NT = TR * P;
    extern __shared__ __align__(16) unsigned char smraw[];
    griddep_wait();
    C *sm = reinterpret_cast<C *>(smraw);  // (N + 1) x SP
    const int t = threadIdx.x;
    const long long r0 = (long long)blockIdx.x * TR;
    const int nr = (int)min((long long)TR, (long long)nrows - r0);
    const T2 *src = in + r0 * Px;
    // Loads in batches of up to 16 per thread, each batch issued before its stores.
    constexpr int NI = (TR * (N + 1) + NT - 1) / NT, NB = 16;
#pragma unroll
    for (int i0 = 0; i0 < NI; i0 += NB) {
        T2 f[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int e = t + (i0 + i) * NT;
            if (i0 + i < NI && e < nr * (N + 1)) f[i] = __ldg(src + (long long)(e / (N + 1)) * Px + e % (N + 1));
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int e = t + (i0 + i) * NT;
            if (i0 + i < NI && e < nr * (N + 1)) sm[(e % (N + 1)) * SP + e / (N + 1)] = ws_c(f[i]);
        }
    }
    __syncthreads();
    // Y_k, k = 0..N (Y_0, Y_N real) -> C_k = Ev_k + i Od_k with Ev_k = Y_k + conj Y_{N-k}
    // and Od_k = (Y_k - conj Y_{N-k}) W_{2N}^{-k}; the inverse N-point FFT of C gives
    // y_{2m} + i y_{2m+1}.  C_{N-k} = conj(Ev_k) + i conj(Od_k).
    for (int e = t; e < TR * (N / 2 + 1); e += NT) {
        const int r = e % TR, k = e / TR;
        if (r >= nr) continue;
        if (k == 0) {
            const Real y0 = sm[r].re, yn = sm[N * SP + r].re;
            sm[r] = C{y0 + yn, y0 - yn};
        } else {
            const C yk = sm[k * SP + r], yn = sm[(N - k) * SP + r];
            const C ev = {yk.re + yn.re, yk.im - yn.im};
            const C od = twmul<1>(C{yk.re - yn.re, yk.im + yn.im}, __ldg(tw + k));
            sm[k * SP + r] = add_rot<1>(ev, od);
            if (2 * k != N) sm[(N - k) * SP + r] = add_rot<1>(C{ev.re, -ev.im}, C{od.re, -od.im});
        }
    }
    __syncthreads();
    const int c = t % TR, q = t / TR;
    C v[E];
    constexpr RunOpt opt{false, false, false, true, true};
    Stages<C, N, E, 1, 1, typename Cfg<Real, N>::Rs>::template run<opt>(
        v, q, c, sm, SP, tw, 2, [&](int row) { return sm[row * SP + c]; },
        [&](int row, C x) { sm[row * SP + c] = x; });
    __syncthreads();
    const int b = (int)(r0 / (N * N));
    X2 *dst = reinterpret_cast<X2 *>(const_cast<void *>(u.p[b])) + (r0 - (long long)b * N * N) * (N / 2);
    for (int e = t; e < nr * (N / 2); e += NT) {
        const int r = e / (N / 2), m = e - r * (N / 2);
        dst[e] = c_ext(sm[m * SP + r]);
    }
}

// ---- symbol octant (setup, FP64 arithmetic) ---------------------------------------------
// sym[(kz * (N+1) + ky) * Ps + kx] for kx, ky, kz <= N; the pitch Ps (a multiple of 4)
// keeps the two-column loads of the FP32 z pass aligned.
//
// The near-field correction I_delta = C0 rho + C2 Laplace(rho) (Sec. 2) is placed in one of
// two ways.  literal = 0 (fused): C0 - C2 |kappa|^2 at every padded frequency, the
// Laplacian of the 2N-periodic series.  literal = 1 (the paper's order, where Laplace(rho)
// comes from an unpadded N^3 transform pair): the N-point DFT of rho is the padded DFT at
// even frequencies and kappa of N-point frequency k equals kappa of padded frequency 2k,
// so 8 (C0 - C2 |kappa|^2) at frequencies whose three indices are all even, 0 elsewhere,
// gives C0 rho + C2 Laplace_N(rho) on the kept N^3 points after the padded inverse (the 8
// turns its 1 / (2N)^3 into the unpadded 1 / N^3).
template <typename Real>
__global__ void k_symbol_table(Real *__restrict__ sym, const double *__restrict__ A,
                               const double *__restrict__ w, int nterms, int N, int Ps, double C0,
                               double C2, double scale, int literal) {
    // Block (b, c) with b <= c computes, for every a <= b, the entry at (kx, ky, kz) =
    // (a, b, c) and writes it to all six permutations: the symbol is symmetric in its
    // three indices, so each value is summed once (about a sixth of the terms) and the
    // table is exactly symmetric.  Entries kz >= ky >= kx keep this sum order:
    // (w_j A_j(ky) A_j(kz)) A_j(kx).
    extern __shared__ double cj[];
    const int b = blockIdx.x, c = blockIdx.y, K = N + 1;
    if (b > c) return;
    for (int j = threadIdx.x; j < nterms; j += blockDim.x)
        cj[j] = w[j] * A[(long long)j * K + b] * A[(long long)j * K + c];
    __syncthreads();
    const double hp2 = 0.25 * 3.141592653589793238462643383279502884 * 3.141592653589793238462643383279502884;
    for (int a = threadIdx.x; a <= b; a += blockDim.x) {
        double sum = 0.0;
        for (int j = 0; j < nterms; ++j) sum += cj[j] * A[(long long)j * K + a];
        const double k2 = (double)a * a + (double)b * b + (double)c * c;
        double v;
        if (!literal) v = sum + C0 - C2 * hp2 * k2;
        else v = ((a | b | c) & 1) ? sum : sum + 8.0 * (C0 - C2 * hp2 * k2);
        const Real g = (Real)(scale * v);
        auto put = [&](int z, int y, int x) { sym[((long long)z * K + y) * Ps + x] = g; };
        put(c, b, a);
        put(c, a, b);
        put(b, c, a);
        put(b, a, c);
        put(a, c, b);
        put(a, b, c);
    }
}

template <class K> static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define GSP_CHECK(x)                          \
    do {                                      \
        cudaError_t e_ = (x);                 \
        if (e_ != cudaSuccess) return e_;     \
    } while (0)

// Blocks of a persistent kernel: as many as fit on all SMs at once.  The occupancy of
// each kernel is queried once and cached by the kernel's address.
// Launch with programmatic dependent launch allowed: the kernel's CTAs may become resident
// and build their shared tables while the previous kernel on the stream finishes; every
// pass kernel calls griddep_wait before it touches memory that kernel writes or reads.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

template <class K> static int persistent_blocks(K kernel, int threads, size_t smem, int ntiles) {
    struct Entry {
        const void *fn;
        int dev, blocks;
    };
    static Entry cache[64];
    static int n = 0;
    static std::mutex mu;  // plans may launch from several host threads
    const void *fn = reinterpret_cast<const void *>(kernel);
    int dev = 0, blocks = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(mu);
        for (int i = 0; i < n; ++i)
            if (cache[i].fn == fn && cache[i].dev == dev) blocks = cache[i].blocks;
    }
    if (blocks == 0) {
        int sms = 1, per_sm = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        blocks = per_sm * (sms > 0 ? sms : 1);
        std::lock_guard<std::mutex> lock(mu);
        if (n < 64) cache[n++] = Entry{fn, dev, blocks};
    }
    return blocks < ntiles ? blocks : ntiles;
}

// Whether the warp form of the z pass exists (FP32, N = 256).
// The warp forms of the z and y passes and the half-warp x passes exist for FP32 at
// N = 16 E1, E1 in {16, 12, 10, 8, 6, 4}; the full-warp x passes at N = 512.
inline constexpr bool warp_n(int N) {
    return N == 256 || N == 192 || N == 160 || N == 128 || N == 96 || N == 64;
}
template <typename Real, int N> constexpr bool zwarp_form() { return std::is_same<Real, float>::value && warp_n(N); }
// The N = 512 warp form of the z pass (k_z_w512: one warp per column, unpacked).
template <typename Real, int N> constexpr bool zw512_form() { return std::is_same<Real, float>::value && N == ZW512::N; }
inline bool zwarp_available(int N) { return warp_n(N) || N == ZW512::N; }

// The fused z pass (K3) of B densities in the form p.zform selects: the length-2N
// transforms (0), the split into even and odd length-N transforms (1, where
// zsplit_available) or the warp form (2, zwarp_form); an absent form runs as form 0.
template <typename Real, int N>
cudaError_t z_pass(const DevicePlan &p, int B, cudaStream_t s, double *tail) {
    using T2 = Cx2<Real>;
    using TwC = typename TwOf<typename Types<Real>::CC>::T;
    constexpr int L = 2 * N;
    using L1 = TmaLayout<Real, L, 1>;
    const int ncols = N + 1;
    const int ntx = (ncols + L1::TC - 1) / L1::TC;
    const int nt = ntx * L * B;
    T2 *w3 = static_cast<T2 *>(p.w3);
    const TwC *twc = static_cast<const TwC *>(p.twc);
    if constexpr (zwarp_form<Real, N>()) {
        if (p.zform == 2) {
            using Z = ZWarp<N / 16>;
            const int ntxw = (ncols + Z::TC - 1) / Z::TC, ntw = ntxw * L * B;
            auto k = tail ? k_z_warp<N / 16, true> : k_z_warp<N / 16, false>;
            GSP_CHECK(set_smem(k, Z::SMEM));
            GSP_CHECK(launch_pdl(k, persistent_blocks(k, Z::NT, Z::SMEM, ntw), Z::NT, Z::SMEM, s,
                                 p.tm_zw_in, p.tm_zw_sym, p.tm_zw_out, static_cast<const float2 *>(p.tw), ntxw, ntw,
                                 ncols, p.status, tail));
            return cudaGetLastError();
        }
    }
    if constexpr (zw512_form<Real, N>()) {
        if (p.zform == 2) {
            using Z = ZW512;
            const int ntx5 = (ncols + Z::TC - 1) / Z::TC, nt5 = ntx5 * L * B;
            auto k = tail ? k_z_w512<true> : k_z_w512<false>;
            GSP_CHECK(set_smem(k, Z::SMEM));
            GSP_CHECK(launch_pdl(k, persistent_blocks(k, Z::NT, Z::SMEM, nt5), Z::NT, Z::SMEM, s,
                                 p.tm_zw_in, p.tm_zw_sym, p.tm_zw_out, static_cast<const float2 *>(p.tw), ntx5, nt5,
                                 ncols, p.status, tail));
            return cudaGetLastError();
        }
    }
    if constexpr (zsplit_available<L>() && !std::is_same<Real, DF>::value) {
        if (p.zform == 1) {
            auto k = tail ? k_z_split_tma<Real, L, true> : k_z_split_tma<Real, L, false>;
            constexpr int T = zsplit_threads<Real, L>();
            GSP_CHECK(set_smem(k, L1::SMEM));
            GSP_CHECK(launch_pdl(k, persistent_blocks(k, T, L1::SMEM, nt), T, L1::SMEM, s,
                                 p.tm_z_in, p.tm_z_sym, w3, twc, ntx, nt, ncols, p.Px, p.status, tail));
            return cudaGetLastError();
        }
    }
    auto k = tail ? k_z_symbol_tma<Real, L, true> : k_z_symbol_tma<Real, L, false>;
    constexpr int T = tma_threads<Real, L, 1>();
    GSP_CHECK(set_smem(k, L1::SMEM));
    GSP_CHECK(launch_pdl(k, persistent_blocks(k, T, L1::SMEM, nt), T, L1::SMEM, s,
                         p.tm_z_in, p.tm_z_sym, w3, twc, ntx, nt, ncols, p.Px, p.status, tail));
    return cudaGetLastError();
}

// The x passes (K1 forward, K5 inverse) of B densities in the form p.xform selects: 0 the
// block form (k_x_forward / k_x_inverse), 1 the warp form (FP32: k_x_warp_* at N = 256,
// k_x_warp2_* at N = 512).
template <typename Real, int N> constexpr bool xwarp_form() {
    return std::is_same<Real, float>::value && (warp_n(N) || N == XWarp2::N);
}

template <typename Real, int N>
cudaError_t x_pass(const DevicePlan &p, const PtrArray &rho, const PtrArray &u, int B, cudaStream_t s, bool fwd,
                   int rows = 0) {
    using T2 = Cx2<Real>;
    const int nrows = rows ? rows : B * N * N;
    if constexpr (xwarp_form<Real, N>()) {
        if (p.xform == 1) {
            const int npairs = nrows / 2;
            const float2 *tw = static_cast<const float2 *>(p.tw);
            if constexpr (N == XWarp2::N) {
                GSP_CHECK(set_smem(k_x_warp2_fwd<N>, XWarp2::SMEM));
                GSP_CHECK(set_smem(k_x_warp2_inv<N>, XWarp2::SMEM));
                const int nw = (npairs + XWarp2::NW - 1) / XWarp2::NW;
                constexpr int NT2 = XWarp2::NT, SM2 = XWarp2::SMEM;
                if (fwd)
                    GSP_CHECK(launch_pdl(k_x_warp2_fwd<N>, persistent_blocks(k_x_warp2_fwd<N>, NT2, SM2, nw), NT2, SM2,
                                         s, rho, static_cast<float2 *>(p.w1), tw, npairs, p.Px));
                else
                    GSP_CHECK(launch_pdl(k_x_warp2_inv<N>, persistent_blocks(k_x_warp2_inv<N>, NT2, SM2, nw), NT2, SM2,
                                         s, static_cast<const float2 *>(p.w1), u, tw, npairs, p.Px));
            } else {
                using X = XWarp<N>;
                GSP_CHECK(set_smem(k_x_warp_fwd<N>, X::SMEM));
                GSP_CHECK(set_smem(k_x_warp_inv<N>, X::SMEM));
                const int nw = (npairs + 15) / 16;
                if (fwd)
                    GSP_CHECK(launch_pdl(k_x_warp_fwd<N>,
                                         persistent_blocks(k_x_warp_fwd<N>, X::NT, X::SMEM, nw), X::NT, X::SMEM, s,
                                         rho, static_cast<float2 *>(p.w1), tw, npairs, p.Px));
                else
                    GSP_CHECK(launch_pdl(k_x_warp_inv<N>,
                                         persistent_blocks(k_x_warp_inv<N>, X::NT, X::SMEM, nw), X::NT, X::SMEM, s,
                                         static_cast<const float2 *>(p.w1), u, tw, npairs, p.Px));
            }
            return cudaGetLastError();
        }
    }
    constexpr int TR = row_tr<Real, N>(), PX1 = N / Cfg<Real, N>::E;
    const size_t smem_row = (size_t)(N + 1) * (TR + 1) * 2 * sizeof(Real);
    const dim3 grow((nrows + TR - 1) / TR);
    const T2 *tw = static_cast<const T2 *>(p.tw);
    if (fwd) {
        GSP_CHECK(set_smem(k_x_forward<Real, N>, smem_row));
        GSP_CHECK(launch_pdl(k_x_forward<Real, N>, grow, TR * PX1, smem_row, s,
                             rho, static_cast<T2 *>(p.w1), tw, nrows, p.Px));
    } else {
        GSP_CHECK(set_smem(k_x_inverse<Real, N>, smem_row));
        GSP_CHECK(launch_pdl(k_x_inverse<Real, N>, grow, TR * PX1, smem_row, s,
                             static_cast<const T2 *>(p.w1), u, tw, nrows, p.Px));
    }
    return cudaGetLastError();
}

// The y passes (K2 forward, K4 inverse) of B densities in the form p.yform selects: 0 the
// block form (k_col_tma), 1 the warp form (k_y_warp, ywarp_form); an absent form runs as 0.
template <typename Real, int N> constexpr bool ywarp_form() { return std::is_same<Real, float>::value && warp_n(N); }
template <typename Real, int N> constexpr bool yw512_form() { return std::is_same<Real, float>::value && N == ZW512::N; }

// planes z0 .. z0 + nz - 1 of the stacked densities (nz = 0: all B N planes).
template <typename Real, int N>
cudaError_t y_pass(const DevicePlan &p, int B, cudaStream_t s, bool fwd, int z0 = 0, int nz = 0) {
    using T2 = Cx2<Real>;
    using TwC = typename TwOf<typename Types<Real>::CC>::T;
    constexpr int L = 2 * N;
    const int ncols = N + 1;
    const int planes = nz ? nz : B * N;
    if constexpr (yw512_form<Real, N>()) {
        if (p.yform == 1) {
            using Z = ZW512;
            const int ntx = (ncols + Z::TC - 1) / Z::TC, nt = ntx * planes;
            auto k = fwd ? k_y_w512<true> : k_y_w512<false>;
            GSP_CHECK(set_smem(k, Z::SMEM));
            GSP_CHECK(launch_pdl(k, persistent_blocks(k, Z::NT, Z::SMEM, nt), Z::NT, Z::SMEM, s,
                                 fwd ? p.tm_yw1 : p.tm_yw3, fwd ? p.tm_yw2 : p.tm_yw1,
                                 static_cast<const float2 *>(p.tw), ntx, nt, ncols, p.status, z0));
            return cudaGetLastError();
        }
    }
    if constexpr (ywarp_form<Real, N>()) {
        if (p.yform == 1) {
            // The forward and inverse kernels take tiles of different widths (16 and 8 columns).
            auto launch = [&](auto kern, int tc, int nthreads, int smem, const CUtensorMap &tin,
                              const CUtensorMap &tout) -> cudaError_t {
                const int ntx = (ncols + tc - 1) / tc, nt = ntx * planes;
                GSP_CHECK(set_smem(kern, smem));
                GSP_CHECK(launch_pdl(kern, persistent_blocks(kern, nthreads, smem, nt), nthreads, smem, s, tin, tout,
                                     static_cast<const float2 *>(p.tw), ntx, nt, ncols, p.status, z0));
                return cudaGetLastError();
            };
            using YF = YWarp<N / 16, true>;
            using YI = YWarp<N / 16, false>;
            if (fwd) return launch(k_y_warp<N / 16, true>, YF::TC, YF::NT, YF::SMEM, p.tm_yw1, p.tm_yw2);
            return launch(k_y_warp<N / 16, false>, YI::TC, YI::NT, YI::SMEM, p.tm_ywi3, p.tm_ywi1);
        }
    }
    const TwC *twc = static_cast<const TwC *>(p.twc);
    const int Px = p.Px;
    if (fwd) {
        using L0 = TmaLayout<Real, L, 0>;
        const int ntx0 = (ncols + L0::TC - 1) / L0::TC, nt = ntx0 * planes;
        auto k = k_col_tma<Real, L, 0>;
        GSP_CHECK(set_smem(k, L0::SMEM));
        constexpr int NTC = tma_threads<Real, L, 0>();
        GSP_CHECK(launch_pdl(k, persistent_blocks(k, NTC, L0::SMEM, nt), NTC, L0::SMEM, s,
                             p.tm_y_in, static_cast<T2 *>(p.w2), twc, ntx0, nt, ncols, Px, (long long)L * Px, p.status, z0));
    } else {
        using L2 = TmaLayout<Real, L, 2>;
        const int ntx2 = (ncols + L2::TC - 1) / L2::TC, nt = ntx2 * planes;
        auto k = k_col_tma<Real, L, 2>;
        GSP_CHECK(set_smem(k, L2::SMEM));
        constexpr int NTC = tma_threads<Real, L, 2>();
        GSP_CHECK(launch_pdl(k, persistent_blocks(k, NTC, L2::SMEM, nt), NTC, L2::SMEM, s,
                             p.tm_yi_in, static_cast<T2 *>(p.w1), twc, ntx2, nt, ncols, Px, (long long)N * Px, p.status, z0));
    }
    return cudaGetLastError();
}

// The fused x and y passes (p.xyform == 1, k_xy_fwd / k_yx_inv): FP32 at the warp-form
// sizes, on plans that carry a counter block.  The ring lives in the workspace the pass does
// not touch otherwise: w3 on the way in, w2 on the way out (2N max_batch slots of N rows).
template <typename Real, int N> constexpr bool xy_fused_form() { return std::is_same<Real, float>::value && warp_n(N); }
template <typename Real, int N> bool xy_fused_on(const DevicePlan &p) {
    return xy_fused_form<Real, N>() && p.xyform == 1 && p.sync != nullptr;
}

template <typename Real, int N>
cudaError_t xy_pass(const DevicePlan &p, const PtrArray &rho, const PtrArray &u, int B, cudaStream_t s, bool fwd) {
    if constexpr (xy_fused_form<Real, N>()) {
        using X = XYWarp<N / 16>;
        const int P = B * N, S = X::NX + X::NY;
        const int smem = fwd ? X::SMEM_F : X::SMEM_I;
        int G;
        if (fwd) {
            GSP_CHECK(set_smem(k_xy_fwd<N / 16>, smem));
            G = persistent_blocks(k_xy_fwd<N / 16>, X::NT, smem, P * S);
        } else {
            GSP_CHECK(set_smem(k_yx_inv<N / 16>, smem));
            G = persistent_blocks(k_yx_inv<N / 16>, X::NT, smem, P * S);
        }
        // Steps (planes) the resident CTAs hold at once; the consumers trail the producers
        // by D steps so that a plane's producers have finished when its consumers start, and
        // a slot comes back R > D steps after its plane was produced.
        const int inflight = (G + S - 1) / S;
        const int R = std::min(std::min(kRingMax, 2 * N * p.max_batch), 3 * inflight + 4);
        const int D = std::min(std::min(inflight + inflight / 2 + 2, R - 1), P);
        const XYOrder ord{P, D, fwd ? X::NX : X::NY, fwd ? X::NY : X::NX};
        const float2 *tw = static_cast<const float2 *>(p.tw);
        if (fwd)
            GSP_CHECK(launch_pdl(k_xy_fwd<N / 16>, G, X::NT, smem, s,
                                 rho, static_cast<float2 *>(p.w3), p.tm_rf, p.tm_yw2, tw, ord, R, p.Px, p.sync,
                                 p.status));
        else
            GSP_CHECK(launch_pdl(k_yx_inv<N / 16>, G, X::NT, smem, s,
                                 p.tm_yw3, static_cast<float2 *>(p.w2), u, tw, ord, R, p.Px, p.sync, p.status));
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

// The x and y passes of planes z0 .. z0 + nz - 1 of one density (rho and u device
// pointers to the whole density): forward x then y, or inverse y then x, with the kernels
// of the plan's separate x and y forms on that slab of planes only.
template <typename Real, int N>
cudaError_t xy_slab(const DevicePlan &p, const void *rho, void *u, int z0, int nz, cudaStream_t s, bool fwd) {
    const long long row0 = (long long)z0 * N;
    DevicePlan q = p;
    q.w1 = static_cast<char *>(p.w1) + row0 * p.Px * 2 * (long long)sizeof(Real);
    PtrArray a{}, b{};
    a.p[0] = static_cast<const char *>(rho) + row0 * N * (long long)sizeof(Real);
    b.p[0] = static_cast<char *>(u) + row0 * N * (long long)sizeof(Real);
    if (fwd) {
        GSP_CHECK((x_pass<Real, N>(q, a, b, 1, s, true, nz * N)));
        return y_pass<Real, N>(p, 1, s, true, z0, nz);
    }
    GSP_CHECK((y_pass<Real, N>(p, 1, s, false, z0, nz)));
    return x_pass<Real, N>(q, a, b, 1, s, false, nz * N);
}

// The five passes.  With the fused x-y form the forward x and y passes are one launch
// (timed as the x forward, ev[1] and ev[2] recorded together) and so are the inverse y and
// x passes (timed as the y inverse).  skip: bit 0 leaves out the forward x and y passes
// (w2 already holds their output), bit 1 the inverse y and x passes (the caller runs them
// from w3, with xy_slab); not with the fused form.
template <typename Real, int N>
cudaError_t solve_n(const DevicePlan &p, const PtrArray &rho, const PtrArray &u, int B, cudaStream_t s,
                    cudaEvent_t *ev, double *tail, int skip) {
    const bool fused = xy_fused_on<Real, N>(p);
    if (fused && skip) return cudaErrorInvalidValue;
    if (ev) GSP_CHECK(cudaEventRecord(ev[0], s));
    if (fused) GSP_CHECK((xy_pass<Real, N>(p, rho, u, B, s, true)));
    else if (!(skip & 1)) GSP_CHECK((x_pass<Real, N>(p, rho, u, B, s, true)));
    if (ev) GSP_CHECK(cudaEventRecord(ev[1], s));

    if (!fused && !(skip & 1)) GSP_CHECK((y_pass<Real, N>(p, B, s, true)));
    if (ev) GSP_CHECK(cudaEventRecord(ev[2], s));

    GSP_CHECK((z_pass<Real, N>(p, B, s, tail)));
    if (ev) GSP_CHECK(cudaEventRecord(ev[3], s));

    if (fused) GSP_CHECK((xy_pass<Real, N>(p, rho, u, B, s, false)));
    else if (!(skip & 2)) GSP_CHECK((y_pass<Real, N>(p, B, s, false)));
    if (ev) GSP_CHECK(cudaEventRecord(ev[4], s));

    if (!fused && !(skip & 2)) GSP_CHECK((x_pass<Real, N>(p, rho, u, B, s, false)));
    if (ev) GSP_CHECK(cudaEventRecord(ev[5], s));
    return cudaSuccess;
}

// ---- TMA descriptors ----------------------------------------------------------------------
using TensorMapEncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                       const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                       const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                       CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline TensorMapEncodeFn tensor_map_encoder() {
    static TensorMapEncodeFn fn = []() -> TensorMapEncodeFn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<TensorMapEncodeFn>(f);
    }();
    return fn;
}

// 3-D tiled map: dims d (innermost first), byte strides of dims 1 and 2, box b.
inline cudaError_t encode_3d(CUtensorMap *m, CUtensorMapDataType dt, void *base, cuuint64_t d0,
                             cuuint64_t d1, cuuint64_t d2, cuuint64_t s1, cuuint64_t s2, cuuint32_t b0,
                             cuuint32_t b1, cuuint32_t b2,
                             CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_NONE,
                             CUtensorMapL2promotion l2 = CU_TENSOR_MAP_L2_PROMOTION_L2_256B) {
    TensorMapEncodeFn enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {s1, s2};
    const cuuint32_t box[3] = {b0, b1, b2};
    const cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, l2,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename Real, int N>
cudaError_t encode_n(DevicePlan &p) {
    constexpr int L = 2 * N;
    constexpr cuuint64_t u = 2 * sizeof(Real) / 8;            // 8-byte units per complex
    const cuuint64_t rowb = (cuuint64_t)p.Px * 2 * sizeof(Real);
    const CUtensorMapDataType U64 = CU_TENSOR_MAP_DATA_TYPE_UINT64;
    using L0 = TmaLayout<Real, L, 0>;
    using L1 = TmaLayout<Real, L, 1>;
    using L2 = TmaLayout<Real, L, 2>;
    const cuuint64_t BN = (cuuint64_t)p.max_batch * N;  // z of all densities, stacked
    GSP_CHECK(encode_3d(&p.tm_y_in, U64, p.w1, (N + 1) * u, N, BN, rowb, (cuuint64_t)N * rowb,
                        L0::ROWB / 8, L0::RPC, 1));
    GSP_CHECK(encode_3d(&p.tm_z_in, U64, p.w2, (N + 1) * u, L, BN, rowb, (cuuint64_t)L * rowb,
                        L1::ROWB / 8, 1, L1::RPC));
    const cuuint64_t srow = (cuuint64_t)p.Ps * sizeof(Real);
    GSP_CHECK(encode_3d(&p.tm_z_sym,
                        sizeof(Real) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                        p.sym, N + 1, N + 1, N + 1, srow, (cuuint64_t)(N + 1) * srow, L1::TC, 1, L1::SRC));
    GSP_CHECK(encode_3d(&p.tm_yi_in, U64, p.w3, (N + 1) * u, L, BN, rowb, (cuuint64_t)L * rowb,
                        L2::ROWB / 8, L2::RPC, 1));
    if constexpr (ywarp_form<Real, N>()) {
        // N-row boxes of w1, w2, w3 (16 columns x N rows of y or ky x 1 plane), 128-byte swizzle.
        GSP_CHECK(encode_3d(&p.tm_yw1, U64, p.w1, N + 1, N, BN, rowb, (cuuint64_t)N * rowb, YWarp<N / 16, true>::TC,
                            N, 1, CU_TENSOR_MAP_SWIZZLE_128B));
        GSP_CHECK(encode_3d(&p.tm_yw2, U64, p.w2, N + 1, L, BN, rowb, (cuuint64_t)L * rowb, YWarp<N / 16, true>::TC,
                            N, 1, CU_TENSOR_MAP_SWIZZLE_128B));
        GSP_CHECK(encode_3d(&p.tm_yw3, U64, p.w3, N + 1, L, BN, rowb, (cuuint64_t)L * rowb, YWarp<N / 16, true>::TC,
                            N, 1, CU_TENSOR_MAP_SWIZZLE_128B));
        // The warp-form y inverse: 8 columns x N rows of w3 (in) and w1 (out), 64-byte swizzle.
        GSP_CHECK(encode_3d(&p.tm_ywi3, U64, p.w3, N + 1, L, BN, rowb, (cuuint64_t)L * rowb, YWarp<N / 16, false>::TC,
                            N, 1, CU_TENSOR_MAP_SWIZZLE_64B));
        GSP_CHECK(encode_3d(&p.tm_ywi1, U64, p.w1, N + 1, N, BN, rowb, (cuuint64_t)N * rowb, YWarp<N / 16, false>::TC,
                            N, 1, CU_TENSOR_MAP_SWIZZLE_64B));
        // The fused forward pass's ring of N-row plane slots in w3.
        GSP_CHECK(encode_3d(&p.tm_rf, U64, p.w3, N + 1, N, 2 * BN, rowb, (cuuint64_t)N * rowb, YWarp<N / 16, true>::TC, N,
                            1, CU_TENSOR_MAP_SWIZZLE_128B));
    }
    if constexpr (zwarp_form<Real, N>()) {
        // Columns kx > N lie outside these maps: loads read zeros there, stores skip them.
        // Boxes of 8 columns x 1 ky x N z-rows (64-byte rows, 64-byte swizzle; L2 fills of 64 B).
        GSP_CHECK(encode_3d(&p.tm_zw_in, U64, p.w2, N + 1, L, BN, rowb, (cuuint64_t)L * rowb, ZWarp<N / 16>::TC, 1, N,
                            CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_64B));
        GSP_CHECK(encode_3d(&p.tm_zw_out, U64, p.w3, N + 1, L, BN, rowb, (cuuint64_t)L * rowb, ZWarp<N / 16>::TC, 1, N,
                            CU_TENSOR_MAP_SWIZZLE_64B));
        // The symbol octant read with its innermost index as kz (symmetric table): boxes of
        // 128 kz x 1 ky x 16 kx.
        GSP_CHECK(encode_3d(&p.tm_zw_sym, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, p.sym, N + 1, N + 1, N + 1, srow,
                            (cuuint64_t)(N + 1) * srow, ZWarp<N / 16>::SYM_KZB, 1, ZWarp<N / 16>::TC));
    }
    if constexpr (yw512_form<Real, N>()) {
        // 8 columns x 256 rows of y or ky x 1 plane of w1, w2, w3 (64-byte swizzle).
        GSP_CHECK(encode_3d(&p.tm_yw1, U64, p.w1, N + 1, N, BN, rowb, (cuuint64_t)N * rowb, ZW512::TC, 256, 1,
                            CU_TENSOR_MAP_SWIZZLE_64B));
        GSP_CHECK(encode_3d(&p.tm_yw2, U64, p.w2, N + 1, L, BN, rowb, (cuuint64_t)L * rowb, ZW512::TC, 256, 1,
                            CU_TENSOR_MAP_SWIZZLE_64B));
        GSP_CHECK(encode_3d(&p.tm_yw3, U64, p.w3, N + 1, L, BN, rowb, (cuuint64_t)L * rowb, ZW512::TC, 256, 1,
                            CU_TENSOR_MAP_SWIZZLE_64B));
    }
    if constexpr (zw512_form<Real, N>()) {
        // 8 columns x 1 ky x 256 z-rows of w2 and w3 (64-byte swizzle); the symbol octant
        // read with its innermost index as kz (the table is symmetric in its three indices):
        // 256 kz x 1 ky x 8 kx per box.
        // Rows of a box are 64 bytes: promote L2 fills to 64 B, not 256 B.
        GSP_CHECK(encode_3d(&p.tm_zw_in, U64, p.w2, N + 1, L, BN, rowb, (cuuint64_t)L * rowb, ZW512::TC, 1, N / 2,
                            CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_64B));
        GSP_CHECK(encode_3d(&p.tm_zw_out, U64, p.w3, N + 1, L, BN, rowb, (cuuint64_t)L * rowb, ZW512::TC, 1, N / 2,
                            CU_TENSOR_MAP_SWIZZLE_64B));
        GSP_CHECK(encode_3d(&p.tm_zw_sym, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, p.sym, N + 1, N + 1, N + 1, srow,
                            (cuuint64_t)(N + 1) * srow, ZW512::SYM_BOX, 1, ZW512::TC));
    }
    return cudaSuccess;
}

#define GSP_SUPPORTED_N(X) \
    X(4) X(8) X(16) X(32) X(48) X(64) X(80) X(96) X(128) X(160) X(192) X(256) X(320) X(384) X(512) X(1024)

// The per-N entry points are instantiated in separate translation units (a group of sizes
// each, compiled in parallel); the dispatch unit of a dtype sees them as extern.
#define GSP_SIZE_GROUP_A(X) X(4) X(8) X(16) X(32) X(48) X(64) X(80) X(96)
#define GSP_SIZE_GROUP_B(X) X(128) X(160) X(192) X(256)
#define GSP_SIZE_GROUP_C(X) X(320) X(384) X(512) X(1024)
// Double-float instantiations compile several times slower (their butterflies are long
// straight-line FP32 sequences), so they spread over more units, one to three sizes each.
#define GSP_DF_GROUP_1(X) X(4) X(8) X(16)
#define GSP_DF_GROUP_2(X) X(32) X(48)
#define GSP_DF_GROUP_3(X) X(64) X(80)
#define GSP_DF_GROUP_4(X) X(96) X(128)
#define GSP_DF_GROUP_5(X) X(160) X(192)
#define GSP_DF_GROUP_6(X) X(256)
#define GSP_DF_GROUP_7(X) X(320) X(384)
#define GSP_DF_GROUP_8(X) X(512)
#define GSP_DF_GROUP_9(X) X(1024)
#define GSP_DECLARE_N(EXT, Real, n)                                                                      \
    EXT template cudaError_t solve_n<Real, n>(const DevicePlan &, const PtrArray &, const PtrArray &, int, \
                                              cudaStream_t, cudaEvent_t *, double *, int);                 \
    EXT template cudaError_t xy_slab<Real, n>(const DevicePlan &, const void *, void *, int, int,           \
                                              cudaStream_t, bool);                                         \
    EXT template cudaError_t z_pass<Real, n>(const DevicePlan &, int, cudaStream_t, double *);             \
    EXT template cudaError_t y_pass<Real, n>(const DevicePlan &, int, cudaStream_t, bool, int, int);       \
    EXT template cudaError_t x_pass<Real, n>(const DevicePlan &, const PtrArray &, const PtrArray &, int,   \
                                             cudaStream_t, bool, int);                                     \
    EXT template cudaError_t xy_pass<Real, n>(const DevicePlan &, const PtrArray &, const PtrArray &, int,  \
                                              cudaStream_t, bool);                                         \
    EXT template cudaError_t encode_n<Real, n>(DevicePlan &);

// ---- runtime-length forms: launchers ----------------------------------------------------------
// Tiles sized so that the ping-pong pair of one CTA stays within about 64 KB of shared memory.
template <typename Real> int any_tile(int L, int cap, int extra = 0) {
    const int bytes = 2 * L * (int)sizeof(typename Types<Real>::CS);
    int t = cap;
    while (t > 1 && (t + extra) * bytes > 65536) t /= 2;
    return t;
}
inline int ilog2(int t) {
    int l = 0;
    while ((1 << (l + 1)) <= t) ++l;
    return l;
}

template <typename Real>
cudaError_t any_x(const DevicePlan &p, const PtrArray &rho, const PtrArray &u, int B, cudaStream_t s, bool fwd,
                  int rows = 0, void *w1 = nullptr) {
    const int nx = p.n3[0], ny = p.n3[1], nz = p.n3[2];
    const AnySched sc = any_sched(nx);
    const int rows_b = ny * nz, nrows = rows ? rows : B * rows_b;
    const int TR = any_tile<Real>(nx, 16, 1);  // pitch TR + 1
    const size_t smem = (size_t)2 * nx * (TR + 1) * sizeof(typename Types<Real>::CS);
    const AnyTw<Real> *tw = static_cast<const AnyTw<Real> *>(p.tw3[0]);
    Cx2<Real> *ws = static_cast<Cx2<Real> *>(w1 ? w1 : p.w1);
    const int grid = (nrows + TR - 1) / TR;
    if (fwd) {
        GSP_CHECK(set_smem(k_any_x_fwd<Real>, smem));
        GSP_CHECK(launch_pdl(k_any_x_fwd<Real>, grid, 256, smem, s, rho, ws, tw, sc, rows_b, nrows, p.Px, ilog2(TR)));
    } else {
        GSP_CHECK(set_smem(k_any_x_inv<Real>, smem));
        GSP_CHECK(launch_pdl(k_any_x_inv<Real>, grid, 256, smem, s, static_cast<const Cx2<Real> *>(ws), u, tw, sc,
                             rows_b, nrows, p.Px, ilog2(TR)));
    }
    return cudaGetLastError();
}

template <typename Real>
cudaError_t any_y(const DevicePlan &p, int B, cudaStream_t s, bool fwd, int z0 = 0, int nzs = 0) {
    const int nx = p.n3[0], ny = p.n3[1], nz = p.n3[2], L = 2 * ny;
    const AnySched sc = any_sched(L);
    const int TC = any_tile<Real>(L, 16), ncols = nx + 1, ntx = (ncols + TC - 1) / TC;
    const int planes = nzs ? nzs : B * nz;
    const size_t smem = (size_t)2 * L * TC * sizeof(typename Types<Real>::CS);
    const AnyTw<Real> *tw = static_cast<const AnyTw<Real> *>(p.tw3[1]);
    const long long Px = p.Px, w1p = (long long)ny * Px, w2p = (long long)L * Px;
    const Cx2<Real> *w1 = static_cast<const Cx2<Real> *>(p.w1), *w3 = static_cast<const Cx2<Real> *>(p.w3);
    Cx2<Real> *w1o = static_cast<Cx2<Real> *>(p.w1), *w2 = static_cast<Cx2<Real> *>(p.w2);
    if (fwd) {
        GSP_CHECK(set_smem(k_any_col<Real, true>, smem));
        GSP_CHECK(launch_pdl(k_any_col<Real, true>, ntx * planes, 256, smem, s, w1 + z0 * w1p, w2 + z0 * w2p, tw, sc,
                             ncols, ntx, ilog2(TC), Px, w1p, Px, w2p));
    } else {
        GSP_CHECK(set_smem(k_any_col<Real, false>, smem));
        GSP_CHECK(launch_pdl(k_any_col<Real, false>, ntx * planes, 256, smem, s, w3 + z0 * w2p, w1o + z0 * w1p, tw, sc,
                             ncols, ntx, ilog2(TC), Px, w2p, Px, w1p));
    }
    return cudaGetLastError();
}

// The z pass of lines ky0 <= ky < ky0 + nky (nky = 0: all 2 ny lines).  Runs on the tables of
// any plan: the compiled-length plans' symbol octant has the same layout as the box table
// and their twiddles W_{2N} are axis z's table.
template <typename Real>
cudaError_t any_z(const DevicePlan &p, int B, cudaStream_t s, double *tail, int ky0 = 0, int nky = 0) {
    const int nx = p.n3[0], ny = p.n3[1], nz = p.n3[2], L = 2 * nz;
    if (nky == 0) nky = 2 * ny;
    const AnySched sc = any_sched(L);
    const int TC = any_tile<Real>(L, 16), ncols = nx + 1, ntx = (ncols + TC - 1) / TC;
    const size_t smem = (size_t)2 * L * TC * sizeof(typename Types<Real>::CS);
    const AnyTw<Real> *tw = static_cast<const AnyTw<Real> *>(p.any ? p.tw3[2] : p.tw);
    const int grid = ntx * nky * B;
    auto k = tail ? k_any_z<Real, true> : k_any_z<Real, false>;
    GSP_CHECK(set_smem(k, smem));
    GSP_CHECK(launch_pdl(k, grid, 256, smem, s, static_cast<const Cx2<Real> *>(p.w2), static_cast<Cx2<Real> *>(p.w3),
                         static_cast<const Real *>(p.sym), tw, sc, nx, ny, ntx, ilog2(TC), p.Px, p.Ps, tail, ky0, nky));
    return cudaGetLastError();
}

template <typename Real>
cudaError_t solve_any(const DevicePlan &p, const PtrArray &rho, const PtrArray &u, int B, cudaStream_t s,
                      cudaEvent_t *ev, double *tail, int skip) {
    if (ev) GSP_CHECK(cudaEventRecord(ev[0], s));
    if (!(skip & 1)) GSP_CHECK(any_x<Real>(p, rho, u, B, s, true));
    if (ev) GSP_CHECK(cudaEventRecord(ev[1], s));
    if (!(skip & 1)) GSP_CHECK(any_y<Real>(p, B, s, true));
    if (ev) GSP_CHECK(cudaEventRecord(ev[2], s));
    GSP_CHECK(any_z<Real>(p, B, s, tail));
    if (ev) GSP_CHECK(cudaEventRecord(ev[3], s));
    if (!(skip & 2)) GSP_CHECK(any_y<Real>(p, B, s, false));
    if (ev) GSP_CHECK(cudaEventRecord(ev[4], s));
    if (!(skip & 2)) GSP_CHECK(any_x<Real>(p, rho, u, B, s, false));
    if (ev) GSP_CHECK(cudaEventRecord(ev[5], s));
    return cudaSuccess;
}

// The x and y passes of planes z0 .. z0 + nzs - 1 of one density (poisson_solve_host's slabs).
template <typename Real>
cudaError_t any_xy_slab(const DevicePlan &p, const void *rho, void *u, int z0, int nzs, cudaStream_t s, bool fwd) {
    const int nx = p.n3[0], ny = p.n3[1];
    const long long row0 = (long long)z0 * ny;
    void *w1 = static_cast<char *>(p.w1) + row0 * p.Px * (long long)sizeof(Cx2<Real>);
    PtrArray a{}, b{};
    a.p[0] = static_cast<const char *>(rho) + row0 * nx * (long long)sizeof(Ext2<Real>) / 2;
    b.p[0] = static_cast<char *>(u) + row0 * nx * (long long)sizeof(Ext2<Real>) / 2;
    if (fwd) {
        GSP_CHECK(any_x<Real>(p, a, b, 1, s, true, nzs * ny, w1));
        return any_y<Real>(p, 1, s, true, z0, nzs);
    }
    GSP_CHECK(any_y<Real>(p, 1, s, false, z0, nzs));
    return any_x<Real>(p, a, b, 1, s, false, nzs * ny, w1);
}

template <typename Real>
cudaError_t solve_dispatch(const DevicePlan &p, const PtrArray &rho, const PtrArray &u, int B,
                           cudaStream_t s, cudaEvent_t *ev, double *tail, int skip) {
    if (p.any) return solve_any<Real>(p, rho, u, B, s, ev, tail, skip);
    switch (p.N) {
#define GSP_CASE(n) \
    case n:         \
        return solve_n<Real, n>(p, rho, u, B, s, ev, tail, skip);
        GSP_SUPPORTED_N(GSP_CASE)
#undef GSP_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

template <typename Real>
cudaError_t z_pass_dispatch(const DevicePlan &p, cudaStream_t s) {
    if (p.any) return any_z<Real>(p, 1, s, nullptr);
    switch (p.N) {
#define GSP_CASE(n) \
    case n:         \
        return z_pass<Real, n>(p, 1, s, nullptr);
        GSP_SUPPORTED_N(GSP_CASE)
#undef GSP_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

template <typename Real>
cudaError_t y_pass_dispatch(const DevicePlan &p, cudaStream_t s) {
    if (p.any) {
        cudaError_t e = any_y<Real>(p, 1, s, true);
        return e != cudaSuccess ? e : any_y<Real>(p, 1, s, false);
    }
    switch (p.N) {
#define GSP_CASE(n)                                                   \
    case n: {                                                         \
        cudaError_t e = y_pass<Real, n>(p, 1, s, true);               \
        return e != cudaSuccess ? e : y_pass<Real, n>(p, 1, s, false); \
    }
        GSP_SUPPORTED_N(GSP_CASE)
#undef GSP_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

// The two x passes of one density on spare workspace (w2 as the density and the output),
// for timing the forms.
template <typename Real>
cudaError_t x_pass_dispatch(const DevicePlan &p, cudaStream_t s) {
    PtrArray a{};
    a.p[0] = p.w2;
    if (p.any) {
        cudaError_t e = any_x<Real>(p, a, a, 1, s, true);
        return e != cudaSuccess ? e : any_x<Real>(p, a, a, 1, s, false);
    }
    switch (p.N) {
#define GSP_CASE(n)                                                          \
    case n: {                                                                \
        cudaError_t e = x_pass<Real, n>(p, a, a, 1, s, true);                \
        return e != cudaSuccess ? e : x_pass<Real, n>(p, a, a, 1, s, false); \
    }
        GSP_SUPPORTED_N(GSP_CASE)
#undef GSP_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

// The forward and inverse x and y passes of one density on spare workspace, in the form
// p.xyform selects (for timing the forms): separately w2 -> w1 -> w2 and w3 -> w1 -> w2;
// fused w1 -> w2 (ring in w3) and w3 -> w1 (ring in w2).
template <typename Real>
cudaError_t xy_pass_dispatch(const DevicePlan &p, cudaStream_t s) {
    if (p.any) {
        PtrArray a{};
        a.p[0] = p.w2;
        cudaError_t e = any_x<Real>(p, a, a, 1, s, true);
        if (e == cudaSuccess) e = any_y<Real>(p, 1, s, true);
        if (e == cudaSuccess) e = any_y<Real>(p, 1, s, false);
        return e != cudaSuccess ? e : any_x<Real>(p, a, a, 1, s, false);
    }
    switch (p.N) {
#define GSP_CASE(n)                                                                  \
    case n: {                                                                        \
        PtrArray a{};                                                                \
        a.p[0] = xy_fused_on<Real, n>(p) ? p.w1 : p.w2;                              \
        if (xy_fused_on<Real, n>(p)) {                                               \
            cudaError_t e = xy_pass<Real, n>(p, a, a, 1, s, true);                   \
            return e != cudaSuccess ? e : xy_pass<Real, n>(p, a, a, 1, s, false);    \
        }                                                                            \
        cudaError_t e = x_pass<Real, n>(p, a, a, 1, s, true);                        \
        if (e == cudaSuccess) e = y_pass<Real, n>(p, 1, s, true);                    \
        if (e == cudaSuccess) e = y_pass<Real, n>(p, 1, s, false);                   \
        return e != cudaSuccess ? e : x_pass<Real, n>(p, a, a, 1, s, false);         \
    }
        GSP_SUPPORTED_N(GSP_CASE)
#undef GSP_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

template <typename Real>
cudaError_t z_lines_dispatch(const DevicePlan &p, int ky0, int nky, cudaStream_t s) {
    return any_z<Real>(p, 1, s, nullptr, ky0, nky);
}

template <typename Real>
cudaError_t xy_slab_dispatch(const DevicePlan &p, const void *rho, void *u, int z0, int nz, cudaStream_t s, bool fwd) {
    if (p.any) return any_xy_slab<Real>(p, rho, u, z0, nz, s, fwd);
    switch (p.N) {
#define GSP_CASE(n) \
    case n:         \
        return xy_slab<Real, n>(p, rho, u, z0, nz, s, fwd);
        GSP_SUPPORTED_N(GSP_CASE)
#undef GSP_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

inline bool zsplit_dispatch(int N) {
    switch (N) {
#define GSP_CASE(n) \
    case n:         \
        return zsplit_available<2 * n>();
        GSP_SUPPORTED_N(GSP_CASE)
#undef GSP_CASE
        default:
            return false;
    }
}

template <typename Real>
cudaError_t encode_dispatch(DevicePlan &p) {
    if (p.any) return cudaSuccess;  // the runtime-length forms use no TMA descriptors
    switch (p.N) {
#define GSP_CASE(n) \
    case n:         \
        return encode_n<Real, n>(p);
        GSP_SUPPORTED_N(GSP_CASE)
#undef GSP_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

template <typename Real>
cudaError_t symbol_table(const DevicePlan &p, const double *dA, const double *dw, int nterms,
                         double C0, double C2, double scale, int literal, cudaStream_t s) {
    const int K = p.N + 1;
    // Padding columns kx > N hold zeros (the kernel writes the octant entries only).
    GSP_CHECK(cudaMemsetAsync(p.sym, 0, (size_t)K * K * p.Ps * sizeof(Real), s));
    k_symbol_table<Real><<<dim3(K, K), 128, nterms * sizeof(double), s>>>(
        static_cast<Real *>(p.sym), dA, dw, nterms, p.N, p.Ps, C0, C2, scale, literal);
    return cudaGetLastError();
}


}  // namespace gsp
