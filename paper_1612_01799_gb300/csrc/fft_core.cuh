// Register-resident mixed-radix FFT building blocks for sm_103a.
//
// A tile holds NC independent transforms ("columns") of length L.  Each column is
// served by P = L / E threads that each keep E complex values in registers.  A stage of
// radix R (Stockham autosort, decimation in time) makes every thread run E / R
// butterflies: butterfly j gathers x[j + r L/R] (r < R), multiplies by the twiddles
// W_{Ns R}^{r (j mod Ns)}, runs a length-R DFT in registers and scatters to
// y[(j / Ns) Ns R + (j mod Ns) + r Ns], Ns being the product of the earlier radices.
// Between stages the values go through shared memory, element (row, col) at
// sm[row * SP + col].  The first stage gathers through a caller functor (global or
// shared memory) and the last stage scatters through one, so a column pass touches
// HBM once per element.
//
// Pruning.  Stage 0 reads rows j + r L/R with j < L/R, so rows >= L/2 are exactly
// r >= R/2: with PRUNE_IN those inputs are zero and never loaded (the zero half of the
// padded input).  The last stage writes rows j + r L/R (Ns R = L), so rows < L/2 are
// r < R/2: with PRUNE_OUT only those are stored (the half cropped away).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace gsp {

template <typename R> struct CxT;
template <> struct CxT<float> { using T = float2; };
template <> struct CxT<double> { using T = double2; };

template <typename T2> __device__ __forceinline__ T2 mk(decltype(T2::x) a, decltype(T2::x) b) {
    T2 r;
    r.x = a;
    r.y = b;
    return r;
}
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return mk<T2>(a.x + b.x, a.y + b.y); }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return mk<T2>(a.x - b.x, a.y - b.y); }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    return mk<T2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T2> __device__ __forceinline__ T2 cmulc(T2 a, T2 b) {
    return mk<T2>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T2> __device__ __forceinline__ T2 conj(T2 a) { return mk<T2>(a.x, -a.y); }
template <typename T2> __device__ __forceinline__ T2 cscale(T2 a, decltype(T2::x) s) { return mk<T2>(a.x * s, a.y * s); }
// i * D * a with D = +1 or -1 (the transform direction: -1 forward, +1 inverse).
template <int D, typename T2> __device__ __forceinline__ T2 rot(T2 a) {
    return D > 0 ? mk<T2>(-a.y, a.x) : mk<T2>(a.y, -a.x);
}
template <typename T2> __device__ __forceinline__ T2 czero() { return mk<T2>(0, 0); }

// Multiply by the twiddle w (forward) or conj(w) (inverse).
template <int D, typename T2> __device__ __forceinline__ T2 twid(T2 a, T2 w) {
    return D < 0 ? cmul(a, w) : cmulc(a, w);
}

// ---- length-R DFTs in registers: X_k = sum_n a_n exp(D 2 pi i n k / R) ----------------

template <int D, typename T2> __device__ __forceinline__ void dft2(T2 &a0, T2 &a1) {
    T2 t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <int D, typename T2> __device__ __forceinline__ void dft4(T2 &a0, T2 &a1, T2 &a2, T2 &a3) {
    T2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = rot<D>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <int D, typename T2> __device__ __forceinline__ void dft3(T2 &a0, T2 &a1, T2 &a2) {
    using R = decltype(T2::x);
    const R h = (R)0.86602540378443864676;  // sqrt(3)/2
    T2 s = cadd(a1, a2);
    T2 d = rot<D>(cscale(csub(a1, a2), h));
    T2 m = csub(a0, cscale(s, (R)0.5));
    a0 = cadd(a0, s);
    a1 = cadd(m, d);
    a2 = csub(m, d);
}

template <int D, typename T2>
__device__ __forceinline__ void dft5(T2 &a0, T2 &a1, T2 &a2, T2 &a3, T2 &a4) {
    using R = decltype(T2::x);
    const R c1 = (R)0.30901699437494742410;   // cos(2 pi / 5)
    const R c2 = (R)-0.80901699437494742410;  // cos(4 pi / 5)
    const R s1 = (R)0.95105651629515357212;   // sin(2 pi / 5)
    const R s2 = (R)0.58778525229247312917;   // sin(4 pi / 5)
    T2 b1 = cadd(a1, a4), b2 = cadd(a2, a3), d1 = csub(a1, a4), d2 = csub(a2, a3);
    T2 p1 = cadd(a0, cadd(cscale(b1, c1), cscale(b2, c2)));
    T2 p2 = cadd(a0, cadd(cscale(b1, c2), cscale(b2, c1)));
    T2 q1 = rot<D>(cadd(cscale(d1, s1), cscale(d2, s2)));
    T2 q2 = rot<D>(csub(cscale(d1, s2), cscale(d2, s1)));
    a0 = cadd(a0, cadd(b1, b2));
    a1 = cadd(p1, q1);
    a4 = csub(p1, q1);
    a2 = cadd(p2, q2);
    a3 = csub(p2, q2);
}

// Radix-2 combination of two half-length DFTs E (even inputs) and O (odd inputs):
// X_k = E_k + W^k O_k, X_{k+H} = E_k - W^k O_k, W = exp(D 2 pi i / (2H)).
template <int D, typename T2, int H>
__device__ __forceinline__ void combine2(T2 *e, T2 *o, T2 *out, const T2 *w) {
#pragma unroll
    for (int k = 0; k < H; ++k) {
        T2 t = (k == 0) ? o[k] : (D < 0 ? cmul(o[k], w[k]) : cmulc(o[k], w[k]));
        out[k] = cadd(e[k], t);
        out[k + H] = csub(e[k], t);
    }
}

template <int R, int D, typename T2> __device__ __forceinline__ void dft(T2 *a) {
    using Re = decltype(T2::x);
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
        // 6 = 2 x 3: DFT3 of even and odd inputs, then radix-2 with W6^k.
        T2 e[3] = {a[0], a[2], a[4]}, o[3] = {a[1], a[3], a[5]};
        dft3<D>(e[0], e[1], e[2]);
        dft3<D>(o[0], o[1], o[2]);
        const T2 w[3] = {mk<T2>((Re)1, (Re)0), mk<T2>((Re)0.5, (Re)-0.86602540378443864676),
                         mk<T2>((Re)-0.5, (Re)-0.86602540378443864676)};
        combine2<D, T2, 3>(e, o, a, w);
    } else if constexpr (R == 8) {
        T2 e[4] = {a[0], a[2], a[4], a[6]}, o[4] = {a[1], a[3], a[5], a[7]};
        dft4<D>(e[0], e[1], e[2], e[3]);
        dft4<D>(o[0], o[1], o[2], o[3]);
        const Re r = (Re)0.70710678118654752440;
        // forward twiddles exp(-2 pi i k / 8); combine2 conjugates them for D = +1
        const T2 w[4] = {mk<T2>((Re)1, (Re)0), mk<T2>(r, -r), mk<T2>((Re)0, (Re)-1), mk<T2>(-r, -r)};
        combine2<D, T2, 4>(e, o, a, w);
    } else if constexpr (R == 16) {
        T2 e[8], o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            e[i] = a[2 * i];
            o[i] = a[2 * i + 1];
        }
        dft<8, D>(e);
        dft<8, D>(o);
        const Re c1 = (Re)0.92387953251128675613, s1 = (Re)0.38268343236508977173;
        const Re r = (Re)0.70710678118654752440;
        const T2 w[8] = {mk<T2>((Re)1, (Re)0), mk<T2>(c1, -s1), mk<T2>(r, -r), mk<T2>(s1, -c1),
                         mk<T2>((Re)0, (Re)-1), mk<T2>(-s1, -c1), mk<T2>(-r, -r), mk<T2>(-c1, -s1)};
        combine2<D, T2, 8>(e, o, a, w);
    } else {
        static_assert(R == 0, "unsupported radix");
    }
}

// ---- Stockham stages ------------------------------------------------------------------

template <int... Rs> struct Radices {};

template <int R0, int... Rs> struct Prod { static constexpr int v = R0 * Prod<Rs...>::v; };
template <int R0> struct Prod<R0> { static constexpr int v = R0; };

// Stage s of a length-L transform, radix R, NS = product of the earlier radices.
// v holds E values: butterfly b of this thread at v[b*R .. b*R+R-1].
template <typename T2, int L, int E, int D, int R, int NS>
struct Stage {
    static_assert(E % R == 0, "radix must divide the per-thread element count");
    static_assert(L % (NS * R) == 0, "radices must divide the length");
    static constexpr int NB = E / R;
    static constexpr int P = L / E;

    template <bool PRUNE, class Ld>
    static __device__ __forceinline__ void gather(T2 *v, int q, Ld &&ld) {
        static_assert(!PRUNE || (NS == 1 && R % 2 == 0), "input pruning needs an even first radix");
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = q + P * b;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (PRUNE && 2 * r >= R)
                    v[b * R + r] = czero<T2>();
                else
                    v[b * R + r] = ld(j + r * (L / R));
            }
        }
    }

    // tw: table of W_TL^e = exp(-2 pi i e / TL), TL = L * twmul.
    static __device__ __forceinline__ void compute(T2 *v, int q, const T2 *__restrict__ tw, int twmul) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = q + P * b;
            if constexpr (NS > 1) {
                const int k = j % NS;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const int e = r * k * (L / (NS * R)) * twmul;
                    v[b * R + r] = twid<D>(v[b * R + r], tw[e]);
                }
            }
            dft<R, D>(&v[b * R]);
        }
    }

    template <bool PRUNE, class St>
    static __device__ __forceinline__ void scatter(const T2 *v, int q, St &&st) {
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

template <typename T2, int L, int E, int D, int NS, class RL> struct Stages;

template <typename T2, int L, int E, int D, int NS, int R, int... Rs>
struct Stages<T2, L, E, D, NS, Radices<R, Rs...>> {
    using S = Stage<T2, L, E, D, R, NS>;
    static constexpr bool LAST = sizeof...(Rs) == 0;
    static_assert(!LAST || NS * R == L, "the radices must multiply to the length");

    // Runs this stage and the rest.  ld(row) gives stage-0 inputs, st(row, value) takes
    // last-stage outputs.  Intermediate values go through sm[row * SP + c].  Every
    // thread of the block must call this (it synchronises the block between stages).
    // SYNC_LAST: the final scatter writes the same shared memory that the final gather
    // (or ld) read, so the block synchronises between the two.
    template <bool PRUNE_IN, bool PRUNE_OUT, bool SYNC_LAST, class Ld, class St>
    static __device__ __forceinline__ void run(T2 *v, int q, int c, T2 *sm, int SP,
                                               const T2 *__restrict__ tw, int twmul, Ld &&ld,
                                               St &&st) {
        S::template gather<PRUNE_IN>(v, q, ld);
        S::compute(v, q, tw, twmul);
        if constexpr (LAST) {
            if constexpr (SYNC_LAST) __syncthreads();
            S::template scatter<PRUNE_OUT>(v, q, st);
        } else {
            __syncthreads();  // all gathers of this stage are done before sm is overwritten
            S::template scatter<false>(v, q, [&](int row, T2 x) { sm[row * SP + c] = x; });
            __syncthreads();
            Stages<T2, L, E, D, NS * R, Radices<Rs...>>::template run<false, PRUNE_OUT, SYNC_LAST>(
                v, q, c, sm, SP, tw, twmul, [&](int row) { return sm[row * SP + c]; }, st);
        }
    }
};

}  // namespace gsp
