// Register-resident mixed-radix FFT building blocks for sm_103a.
//
// A tile holds independent transforms ("columns") of length L.  Each column is served by
// P = L / E threads that each keep E complex values in registers.  A stage of radix R
// (Stockham autosort, decimation in time) makes every thread run E / R butterflies:
// butterfly j gathers x[j + r L/R] (r < R), multiplies by the twiddles
// W_{Ns R}^{r (j mod Ns)}, runs a length-R DFT in registers and scatters to
// y[(j / Ns) Ns R + (j mod Ns) + r Ns], Ns being the product of the earlier radices.
// Between stages the values go through shared memory, element (row, col) at
// sm[row * SP + col].  The first stage gathers through a caller functor (global or
// shared memory) or starts from values already in registers; the last stage scatters
// through a functor or leaves its values in registers, so a column pass touches HBM
// once per element.
//
// The complex type is a template parameter:
//   CF  one FP32 complex value,
//   CV  two FP32 complex values of two neighbouring columns, real parts in one float2 and
//       imaginary parts in another, so that the packed FP32x2 instructions of sm_100+
//       (__fadd2_rn, __fmul2_rn, __ffma2_rn) do two columns' arithmetic per instruction
//       and a product with +-i is a swap of the two registers,
//   CD  one FP64 complex value,
//   CDF one complex value in double-float arithmetic (type DF below: each real an
//       unevaluated sum hi + lo of two FP32 numbers), the FP32-pipe stand-in for CD.
//
// Pruning.  Stage 0 reads rows j + r L/R with j < L/R, so rows >= L/2 are exactly
// r >= R/2 when R is even: with prune_in those inputs are zero and never loaded (the zero
// half of the padded input).  The last stage writes rows j + r L/R (Ns R = L), so rows
// < L/2 are r < R/2: with prune_out only those are stored (the half cropped away).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "debug.cuh"

namespace gsp {

// ---- complex types and their arithmetic --------------------------------------------------

struct CF {
    float re, im;
};
struct CD {
    double re, im;
};
struct CV {
    float2 re, im;
};

// ---- double-float reals ------------------------------------------------------------------
// A real number held as hi + lo, two FP32 values: a 48-bit significand (unit roundoff
// 2^-48, about 3.6e-15) with FP32's exponent range, computed on the FP32 pipe.  Sums use a
// two-sum of the leading parts (the operands ordered by magnitude, then Dekker's fast
// two-sum), which yields the exact rounding error of that FP32 addition, and add it and
// both lo parts in FP32 without renormalising: the result's lo may exceed ulp(hi) / 2 by
// the few units a chain of operations collects.  Products use the exact product of an FP32
// multiplication that the fused multiply-add gives (fma(a, b, -ab) = the error of ab) and
// the cross terms hi x lo; a lone product renormalises (hi, lo) with a fast two-sum, the
// fused a b + c d of the complex products (df_sum_prod) leaves it unnormalised as well.
// The error of a sum is at most about 2^-47 (|a| + |b|) for operands whose lo holds a few
// units of ulp(hi), of a product about 2^-47 |a| |b| (the lo x lo term is dropped): the
// norm-wise error model of an FFT in FP64.  Leaving sums and the fused products
// unnormalised took the FP64 plan's solve at N = 256 from 2.43 to 2.05 ms, within the same
// 1e-12 bar against the oracle.  The _rn
// intrinsics keep the compiler from contracting or reassociating the error terms.
struct DF {
    float hi, lo;
    DF() = default;
    __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
    // The nearest double-float to d (exact for |d| in FP32's normal range to 48 bits).
    __host__ __device__ constexpr DF(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};
__host__ __device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ DF df_fast_two_sum(float s, float e) {  // needs |s| >= |e| or s = 0
    const float h = __fadd_rn(s, e);
    return DF(h, __fsub_rn(e, __fsub_rn(h, s)));
}
// s + e = x + y exactly, s = fl(x + y): the leading parts ordered by magnitude (selects on
// the ALU pipe), then Dekker's fast two-sum (three FP32 operations instead of the six of
// Knuth's branch-free two-sum; both give the same exact s and e).
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const bool sw = fabsf(b) > fabsf(a);
    const float x = sw ? b : a, y = sw ? a : b;
    const float s = __fadd_rn(x, y);
    return DF(s, __fsub_rn(y, __fsub_rn(s, x)));
}
__device__ __forceinline__ DF operator+(DF a, DF b) {
    const DF t = df_two_sum(a.hi, b.hi);
    return DF(t.hi, __fadd_rn(t.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

// a b + c d in one pass: the two leading products and their exact errors (FMA), one
// two-sum of the products, the cross terms hi x lo accumulated in FP32, no renormalisation:
// 13 FP32 operations and 3 selects, with the error bound of two products and a sum (the
// lo x lo terms dropped, about 2^-47 (|ab| + |cd|)).
__device__ __forceinline__ DF df_sum_prod(DF a, DF b, DF c, DF d) {
    const float p1 = __fmul_rn(a.hi, b.hi), p2 = __fmul_rn(c.hi, d.hi);
    const float e1 = __fmaf_rn(a.hi, b.hi, -p1), e2 = __fmaf_rn(c.hi, d.hi, -p2);
    const DF st = df_two_sum(p1, p2);
    const float s = st.hi;
    float t = __fadd_rn(st.lo, __fadd_rn(e1, e2));
    t = __fmaf_rn(a.hi, b.lo, t);
    t = __fmaf_rn(a.lo, b.hi, t);
    t = __fmaf_rn(c.hi, d.lo, t);
    t = __fmaf_rn(c.lo, d.hi, t);
    return DF(s, t);  // left unnormalised, as a sum's result
}

struct CDF {
    DF re, im;
};

template <typename C> struct CxReal;
template <> struct CxReal<CF> { using T = float; };
template <> struct CxReal<CD> { using T = double; };
template <> struct CxReal<CV> { using T = float; };
template <> struct CxReal<CDF> { using T = DF; };

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one packed FMA with -1 (the product is exact, so this rounds like a - b).
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2neg(float2 a) { return f2(-a.x, -a.y); }

template <typename C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ CF czero<CF>() { return {0.f, 0.f}; }
template <> __device__ __forceinline__ CD czero<CD>() { return {0.0, 0.0}; }
template <> __device__ __forceinline__ CV czero<CV>() { return {f2(0.f, 0.f), f2(0.f, 0.f)}; }
template <> __device__ __forceinline__ CDF czero<CDF>() { return {DF(0.f, 0.f), DF(0.f, 0.f)}; }

__device__ __forceinline__ CF cadd(CF a, CF b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ CF csub(CF a, CF b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ CD cadd(CD a, CD b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ CD csub(CD a, CD b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ CV cadd(CV a, CV b) { return {f2add(a.re, b.re), f2add(a.im, b.im)}; }
__device__ __forceinline__ CV csub(CV a, CV b) { return {f2sub(a.re, b.re), f2sub(a.im, b.im)}; }
__device__ __forceinline__ CDF cadd(CDF a, CDF b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ CDF csub(CDF a, CDF b) { return {a.re - b.re, a.im - b.im}; }

__device__ __forceinline__ CF cscale(CF a, float s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ CD cscale(CD a, double s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ CV cscale(CV a, float s) { return {f2mul(a.re, f2(s, s)), f2mul(a.im, f2(s, s))}; }
__device__ __forceinline__ CDF cscale(CDF a, DF s) { return {a.re * s, a.im * s}; }
// Lane-wise real scale (CV: one factor per column).
__device__ __forceinline__ CV cscale2(CV a, float2 s) { return {f2mul(a.re, s), f2mul(a.im, s)}; }

// a + i D b (D = +1 or -1): the product with +-i never materialises.
template <int D> __device__ __forceinline__ CF add_rot(CF a, CF b) {
    return D > 0 ? CF{a.re - b.im, a.im + b.re} : CF{a.re + b.im, a.im - b.re};
}
template <int D> __device__ __forceinline__ CD add_rot(CD a, CD b) {
    return D > 0 ? CD{a.re - b.im, a.im + b.re} : CD{a.re + b.im, a.im - b.re};
}
template <int D> __device__ __forceinline__ CV add_rot(CV a, CV b) {
    return D > 0 ? CV{f2sub(a.re, b.im), f2add(a.im, b.re)} : CV{f2add(a.re, b.im), f2sub(a.im, b.re)};
}
template <int D> __device__ __forceinline__ CDF add_rot(CDF a, CDF b) {
    return D > 0 ? CDF{a.re - b.im, a.im + b.re} : CDF{a.re + b.im, a.im - b.re};
}
// a - i D b
template <int D, typename C> __device__ __forceinline__ C sub_rot(C a, C b) { return add_rot<-D>(a, b); }

// Product with the constant exp(D 2 pi i m / R), given by its forward value (cr, ci) =
// exp(-2 pi i m / R): D < 0 multiplies by (cr, ci), D > 0 by (cr, -ci).
template <int D> __device__ __forceinline__ CF cmulk(CF a, float cr, float ci) {
    const float s = D < 0 ? ci : -ci;
    return {a.re * cr - a.im * s, a.re * s + a.im * cr};
}
template <int D> __device__ __forceinline__ CD cmulk(CD a, double cr, double ci) {
    const double s = D < 0 ? ci : -ci;
    return {a.re * cr - a.im * s, a.re * s + a.im * cr};
}
template <int D> __device__ __forceinline__ CDF cmulk(CDF a, DF cr, DF ci) {
    const DF s = D < 0 ? ci : -ci;
    return {df_sum_prod(a.re, cr, a.im, -s), df_sum_prod(a.re, s, a.im, cr)};
}
template <int D> __device__ __forceinline__ CV cmulk(CV a, float cr, float ci) {
    const float s = D < 0 ? ci : -ci;
    const float2 R = f2(cr, cr), S = f2(s, s), NS = f2(-s, -s);
    return {f2fma(a.im, NS, f2mul(a.re, R)), f2fma(a.re, S, f2mul(a.im, R))};
}

// Twiddle tables hold exp(-2 pi i e / TL): float2 / double2 (re, im) for CF / CD, and the
// lane-broadcast float4 (re, re, im, im) that the packed products of CV take directly.
template <typename C> struct TwOf;
template <> struct TwOf<CF> { using T = float2; };
template <> struct TwOf<CD> { using T = double2; };
template <> struct TwOf<CV> { using T = float4; };
template <> struct TwOf<CDF> { using T = float4; };  // (re.hi, re.lo, im.hi, im.lo)

// a times w (D < 0) or conj(w) (D > 0).
template <int D> __device__ __forceinline__ CF twmul(CF a, float2 w) {
    const float s = D < 0 ? w.y : -w.y;
    return {a.re * w.x - a.im * s, a.re * s + a.im * w.x};
}
template <int D> __device__ __forceinline__ CD twmul(CD a, double2 w) {
    const double s = D < 0 ? w.y : -w.y;
    return {a.re * w.x - a.im * s, a.re * s + a.im * w.x};
}
template <int D> __device__ __forceinline__ CDF twmul(CDF a, float4 w) {
    const DF wr(w.x, w.y), wi(w.z, w.w);
    const DF s = D < 0 ? wi : -wi;
    return {df_sum_prod(a.re, wr, a.im, -s), df_sum_prod(a.re, s, a.im, wr)};
}
template <int D> __device__ __forceinline__ CV twmul(CV a, float4 w) {
    const float2 R = f2(w.x, w.y), I = f2(w.z, w.w);
    if (D < 0) return {f2fma(f2neg(a.im), I, f2mul(a.re, R)), f2fma(a.re, I, f2mul(a.im, R))};
    return {f2fma(a.im, I, f2mul(a.re, R)), f2fma(f2neg(a.re), I, f2mul(a.im, R))};
}

// ---- length-R DFTs in registers: X_k = sum_n a_n exp(D 2 pi i n k / R) ----------------

template <int D, typename C> __device__ __forceinline__ void dft2(C &a0, C &a1) {
    C t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <int D, typename C> __device__ __forceinline__ void dft4(C &a0, C &a1, C &a2, C &a3) {
    C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = csub(a1, a3);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = add_rot<D>(t1, t3);
    a3 = sub_rot<D>(t1, t3);
}

template <int D, typename C> __device__ __forceinline__ void dft3(C &a0, C &a1, C &a2) {
    using R = typename CxReal<C>::T;
    const R h = (R)0.86602540378443864676;  // sqrt(3)/2
    C s = cadd(a1, a2);
    C d = cscale(csub(a1, a2), h);
    C m = csub(a0, cscale(s, (R)0.5));
    a0 = cadd(a0, s);
    a1 = add_rot<D>(m, d);
    a2 = sub_rot<D>(m, d);
}

template <int D, typename C> __device__ __forceinline__ void dft5(C &a0, C &a1, C &a2, C &a3, C &a4) {
    using R = typename CxReal<C>::T;
    const R c1 = (R)0.30901699437494742410;   // cos(2 pi / 5)
    const R c2 = (R)-0.80901699437494742410;  // cos(4 pi / 5)
    const R s1 = (R)0.95105651629515357212;   // sin(2 pi / 5)
    const R s2 = (R)0.58778525229247312917;   // sin(4 pi / 5)
    C b1 = cadd(a1, a4), b2 = cadd(a2, a3), d1 = csub(a1, a4), d2 = csub(a2, a3);
    C p1 = cadd(a0, cadd(cscale(b1, c1), cscale(b2, c2)));
    C p2 = cadd(a0, cadd(cscale(b1, c2), cscale(b2, c1)));
    C q1 = cadd(cscale(d1, s1), cscale(d2, s2));
    C q2 = csub(cscale(d1, s2), cscale(d2, s1));
    a0 = cadd(a0, cadd(b1, b2));
    a1 = add_rot<D>(p1, q1);
    a4 = sub_rot<D>(p1, q1);
    a2 = add_rot<D>(p2, q2);
    a3 = sub_rot<D>(p2, q2);
}

// Radix-2 combination of the half-length DFTs of the even (e) and odd (o) inputs:
// X_k = e_k + W^k o_k, X_{k+H} = e_k - W^k o_k, W = exp(D 2 pi i / (2H)).  (cs[k], sn[k])
// is the forward value of W^k; W^0 = 1 and W^{H/2} = i D are applied without products.
template <int D, int H, typename C, typename R>
__device__ __forceinline__ void combine2(const C *e, const C *o, C *out, const R *cs, const R *sn) {
#pragma unroll
    for (int k = 0; k < H; ++k) {
        if (k == 0) {
            out[0] = cadd(e[0], o[0]);
            out[H] = csub(e[0], o[0]);
        } else if (2 * k == H) {
            out[k] = add_rot<D>(e[k], o[k]);
            out[k + H] = sub_rot<D>(e[k], o[k]);
        } else {
            const C t = cmulk<D>(o[k], cs[k], sn[k]);
            out[k] = cadd(e[k], t);
            out[k + H] = csub(e[k], t);
        }
    }
}

template <int R, int D, typename C> __device__ __forceinline__ void dft(C *a) {
    using Re = typename CxReal<C>::T;
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        dft2<D>(a[0], a[1]);
    } else if constexpr (R == 3) {
        dft3<D>(a[0], a[1], a[2]);
    } else if constexpr (R == 4) {
        dft4<D>(a[0], a[1], a[2], a[3]);
    } else if constexpr (R == 5) {
        dft5<D>(a[0], a[1], a[2], a[3], a[4]);
    } else if constexpr (R == 6) {
        C e[3] = {a[0], a[2], a[4]}, o[3] = {a[1], a[3], a[5]};
        dft3<D>(e[0], e[1], e[2]);
        dft3<D>(o[0], o[1], o[2]);
        const Re cs[3] = {(Re)1, (Re)0.5, (Re)-0.5};
        const Re sn[3] = {(Re)0, (Re)-0.86602540378443864676, (Re)-0.86602540378443864676};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const C t = k == 0 ? o[0] : cmulk<D>(o[k], cs[k], sn[k]);
            a[k] = cadd(e[k], t);
            a[k + 3] = csub(e[k], t);
        }
    } else if constexpr (R == 8) {
        C e[4] = {a[0], a[2], a[4], a[6]}, o[4] = {a[1], a[3], a[5], a[7]};
        dft4<D>(e[0], e[1], e[2], e[3]);
        dft4<D>(o[0], o[1], o[2], o[3]);
        const Re r = (Re)0.70710678118654752440;
        const Re cs[4] = {(Re)1, r, (Re)0, -r}, sn[4] = {(Re)0, -r, (Re)-1, -r};
        combine2<D, 4>(e, o, a, cs, sn);
    } else if constexpr (R == 16) {
        C e[8], o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            e[i] = a[2 * i];
            o[i] = a[2 * i + 1];
        }
        dft<8, D>(e);
        dft<8, D>(o);
        const Re c1 = (Re)0.92387953251128675613, s1 = (Re)0.38268343236508977173;
        const Re r = (Re)0.70710678118654752440;
        const Re cs[8] = {(Re)1, c1, r, s1, (Re)0, -s1, -r, -c1};
        const Re sn[8] = {(Re)0, -s1, -r, -c1, (Re)-1, -c1, -r, -s1};
        combine2<D, 8>(e, o, a, cs, sn);
    } else {
        static_assert(R == 0, "unsupported radix");
    }
}

// ---- Stockham stages ------------------------------------------------------------------

template <int... Rs> struct Radices {};

// The radices in reverse order.
template <class A, class B> struct RevImpl;
template <int... Done> struct RevImpl<Radices<>, Radices<Done...>> { using T = Radices<Done...>; };
template <int R, int... Rest, int... Done>
struct RevImpl<Radices<R, Rest...>, Radices<Done...>> {
    using T = typename RevImpl<Radices<Rest...>, Radices<R, Done...>>::T;
};
template <class RL> using Reverse = typename RevImpl<RL, Radices<>>::T;

template <class RL> struct LastRadix;
template <int R> struct LastRadix<Radices<R>> { static constexpr int v = R; };
template <int R, int R2, int... Rs> struct LastRadix<Radices<R, R2, Rs...>> {
    static constexpr int v = LastRadix<Radices<R2, Rs...>>::v;
};

// Stage of a length-L transform, radix R, NS = product of the earlier radices.
// v holds E values: butterfly b of this thread at v[b*R .. b*R+R-1], butterfly index
// j = q + P b.
template <typename C, int L, int E, int D, int R, int NS>
struct Stage {
    static_assert(E % R == 0, "radix must divide the per-thread element count");
    static_assert(L % (NS * R) == 0, "radices must divide the length");
    static constexpr int NB = E / R;
    static constexpr int P = L / E;
    using Tw = typename TwOf<C>::T;

    template <bool PRUNE, class Ld>
    static __device__ __forceinline__ void gather(C *v, int q, Ld &&ld) {
        static_assert(!PRUNE || (NS == 1 && R % 2 == 0), "input pruning needs an even first radix");
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = q + P * b;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (PRUNE && 2 * r >= R)
                    v[b * R + r] = czero<C>();
                else
                    v[b * R + r] = ld(j + r * (L / R));
            }
        }
    }

    // tw: table of exp(-2 pi i e / TL), TL = L * twstride.
    static __device__ __forceinline__ void compute(C *v, int q, const Tw *__restrict__ tw, int twstride) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = q + P * b;
            if constexpr (NS > 1) {
                const int k = j % NS;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const int e = r * k * (L / (NS * R)) * twstride;
                    v[b * R + r] = twmul<D>(v[b * R + r], __ldg(tw + e));
                }
            }
            dft<R, D>(&v[b * R]);
        }
    }

    template <bool PRUNE, class St>
    static __device__ __forceinline__ void scatter(const C *v, int q, St &&st) {
        static_assert(!PRUNE || (NS * R == L && R % 2 == 0), "output pruning needs an even last radix");
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = q + P * b;
            const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!(PRUNE && 2 * r >= R)) st(base + r * NS, v[b * R + r]);
            }
        }
    }
};

// Options of a run of stages.
struct RunOpt {
    bool from_regs;  // stage 0 starts from v as it is (no gather)
    bool prune_in;
    bool to_regs;    // the last stage leaves its outputs in v (no scatter)
    bool prune_out;
    bool sync_last;  // barrier before the final scatter (it writes what the final gather read)
};

template <typename C, int L, int E, int D, int NS, class RL> struct Stages;

template <typename C, int L, int E, int D, int NS, int R, int... Rs>
struct Stages<C, L, E, D, NS, Radices<R, Rs...>> {
    using S = Stage<C, L, E, D, R, NS>;
    using Tw = typename TwOf<C>::T;
    static constexpr bool LAST = sizeof...(Rs) == 0;
    static_assert(!LAST || NS * R == L, "the radices must multiply to the length");

    // Runs this stage and the rest.  ld(row) gives stage-0 inputs, st(row, value) takes
    // last-stage outputs.  Intermediate values of this thread's column go through
    // sm[at(row)]; sync() orders the exchange among the threads that share the column
    // (every one of them must make the same calls).
    // After a to_regs run the last stage's butterfly b, output r of this thread (row
    // j + r L/R_last, j = q + P b) is v[b * R_last + r]: exactly what a run whose first
    // radix is R_last gathers, so a transform in the other direction with the radices in
    // reverse order can continue from_regs without a shared-memory exchange.
    template <RunOpt O, class Ld, class St, class At, class Sync>
    static __device__ __forceinline__ void run_with(C *v, int q, C *sm, const Tw *__restrict__ tw,
                                                    int twstride, Ld &&ld, St &&st, At &&at, Sync &&sync) {
        if constexpr (!O.from_regs) S::template gather<O.prune_in>(v, q, ld);
        S::compute(v, q, tw, twstride);
        if constexpr (LAST) {
            if constexpr (!O.to_regs) {
                if constexpr (O.sync_last) sync();
                S::template scatter<O.prune_out>(v, q, st);
            }
        } else {
            sync();  // every read of sm before this stage is done
            S::template scatter<false>(v, q, [&](int row, C x) { sm_st(sm + at(row), x); });
            sync();
            constexpr RunOpt next{false, false, O.to_regs, O.prune_out, O.sync_last};
            Stages<C, L, E, D, NS * R, Radices<Rs...>>::template run_with<next>(
                v, q, sm, tw, twstride, [&](int row) { return sm_ld(sm + at(row)); }, st, at, sync);
        }
    }

    // Block-wide form: column c at sm[row * SP + c], exchanges ordered by __syncthreads.
    template <RunOpt O, class Ld, class St>
    static __device__ __forceinline__ void run(C *v, int q, int c, C *sm, int SP,
                                               const Tw *__restrict__ tw, int twstride, Ld &&ld,
                                               St &&st) {
        run_with<O>(v, q, sm, tw, twstride, ld, st, [&](int row) { return row * SP + c; },
                    [] { __syncthreads(); });
    }
};

}  // namespace gsp
