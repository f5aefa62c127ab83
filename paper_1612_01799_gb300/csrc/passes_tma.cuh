// Column passes (y forward, z fused, y inverse) with TMA-staged input tiles.
//
// Persistent CTAs walk the tiles of a pass (TC consecutive columns of one transform
// line).  A tile's input is one 3-D TMA box (TC columns x the nonzero input rows, split
// into copies of at most 256 rows) landing in shared memory and signalled on an mbarrier.
// As soon as every thread has pulled its stage-0 inputs out of the staging buffer into
// registers, one thread issues the TMA for the CTA's next tile into the same buffer, so
// the next tile's HBM read overlaps this tile's FFT stages and stores.  The FFT stages are
// the register/shared-memory Stockham stages of fft_core.cuh; outputs go straight from
// the last stage's registers to HBM.  The z pass also stages its symbol rows
// (TC columns x N+1 kz values of the octant) with a second TMA box per tile.
// All mbarrier waits are bounded (tma.cuh); on a timeout the whole CTA leaves.
#pragma once
#include "tma.cuh"

namespace gsp {

template <class RL> struct FirstRadix;
template <int R, int... Rs> struct FirstRadix<Radices<R, Rs...>> { static constexpr int v = R; };

// TMA copies of `rows` rows of row_bytes each, and rows per copy: at most 256 rows per
// copy (the box limit), and every copy's shared-memory destination 128-byte aligned (rows
// per copy a multiple of 128 / row_bytes).  Rows past the tensor's end are zero-filled by
// the TMA unit.
__host__ __device__ constexpr int tma_row_align(int row_bytes) { return row_bytes >= 128 ? 1 : 128 / row_bytes; }
__host__ __device__ constexpr int tma_rpc_for(int rows, int nc, int row_bytes) {
    return ((rows + nc - 1) / nc + tma_row_align(row_bytes) - 1) / tma_row_align(row_bytes) *
           tma_row_align(row_bytes);
}
__host__ __device__ constexpr int tma_ncopy(int rows, int row_bytes) {
    int nc = (rows + 255) / 256;
    while (tma_rpc_for(rows, nc, row_bytes) > 256) ++nc;
    return nc;
}
__host__ __device__ constexpr int tma_rows_per_copy(int rows, int row_bytes) {
    return tma_rpc_for(rows, tma_ncopy(rows, row_bytes), row_bytes);
}

// Shared memory of a TMA column pass with tile width tc (KIND 0: y forward, 1: z fused,
// 2: y inverse): 128 bytes of alignment slack, the staged input rows, the L-row exchange
// buffer and the z pass's symbol rows.
template <typename Real, int L, int KIND> __host__ __device__ constexpr int tma_smem(int tc) {
    const int s = (int)sizeof(Real);
    const int lin = KIND == 2 ? L : L / 2;
    const int rb = tc * 2 * s, sb = tc * s;
    const int in_rows = tma_ncopy(lin, rb) * tma_rows_per_copy(lin, rb);
    const int srows = KIND == 1 ? tma_ncopy(L / 2 + 1, sb) * tma_rows_per_copy(L / 2 + 1, sb) : 0;
    const int bytes = 128 + in_rows * rb + L * tc * 2 * s + srows * sb;
    return (bytes + 15) / 16 * 16 + 16;
}

// Columns per CTA of the TMA column passes: 128-byte tile rows (16 FP32 or 8 FP64 complex),
// half that for the y inverse (it stages all L input rows next to its L-row exchange
// buffer), narrowed until the block has <= 1024 threads and its shared memory fits in
// 227 KB.  The narrowest tile keeps every TMA box row a multiple of 16 bytes (symbol
// rows: tc * sizeof(Real)).
template <typename Real, int L, int KIND> __host__ __device__ constexpr int tma_tc() {
    int tc = sizeof(Real) == 4 ? 16 : 8;
    if (KIND == 2) tc /= 2;
    const int W = Types<Real>::W;
    const int P = L / Cfg<Real, L>::E;
    const int tc_min = sizeof(Real) == 4 ? 4 : 2;
    while (tc > tc_min && ((tc / W) * P > 1024 || tma_smem<Real, L, KIND>(tc) > 232448)) tc /= 2;
    return tc;
}
template <typename Real, int L, int KIND> __host__ __device__ constexpr int tma_threads() {
    return (tma_tc<Real, L, KIND>() / Types<Real>::W) * (L / Cfg<Real, L>::E);
}

template <typename Real, int L, int KIND> struct TmaLayout {
    static constexpr int N = L / 2;
    static constexpr int TC = tma_tc<Real, L, KIND>();
    static constexpr int W = Types<Real>::W;
    static constexpr int NG = TC / W;                                  // column groups (16 B each)
    static constexpr int P = L / Cfg<Real, L>::E;                      // threads per group
    static constexpr int ROWB = TC * 2 * (int)sizeof(Real);            // bytes of one tile row
    static constexpr int LIN = KIND == 2 ? L : N;                      // input rows per tile
    static constexpr int NCP = tma_ncopy(LIN, ROWB);
    static constexpr int RPC = tma_rows_per_copy(LIN, ROWB);
    static constexpr int IN_ROWS = NCP * RPC;
    static constexpr int SROWS_N = N + 1;                              // symbol rows (kz <= N)
    static constexpr int SROWB = TC * (int)sizeof(Real);               // bytes of one symbol row
    static constexpr int NCS = tma_ncopy(SROWS_N, SROWB);
    static constexpr int SRC = tma_rows_per_copy(SROWS_N, SROWB);
    static constexpr int S_ROWS = KIND == 1 ? NCS * SRC : 0;
    static constexpr int IN_BYTES = IN_ROWS * ROWB;
    static constexpr int XB_BYTES = L * NG * (int)sizeof(typename Types<Real>::CC);
    static constexpr int S_BYTES = S_ROWS * SROWB;
    static constexpr int OFF_XB = IN_BYTES;                             // from the aligned base
    static constexpr int OFF_S = OFF_XB + XB_BYTES;
    static constexpr int OFF_BAR = (OFF_S + S_BYTES + 15) / 16 * 16;
    static constexpr int SMEM = 128 + OFF_BAR + 16;
    static_assert(SMEM == tma_smem<Real, L, KIND>(TC), "layout and size agree");
    static_assert(SMEM <= 232448, "shared memory of one CTA");
    static_assert(NG * P <= 1024, "threads of one CTA");
    static_assert(ROWB % 16 == 0 && SROWB % 16 == 0, "16-byte TMA box rows");
    static_assert((RPC * ROWB) % 128 == 0 && IN_BYTES % 128 == 0, "128-byte aligned input copies");
    static_assert(OFF_S % 128 == 0 && (KIND != 1 || (SRC * SROWB) % 128 == 0), "128-byte aligned symbol copies");
    static_assert(RPC <= 256 && SRC <= 256, "TMA box rows");
};

template <typename C> __device__ __forceinline__ C ld_sm_cc(const unsigned char *p);
template <> __device__ __forceinline__ CV ld_sm_cc<CV>(const unsigned char *p) {
    const float4 f = sm_ld(reinterpret_cast<const float4 *>(p));
    return {make_float2(f.x, f.z), make_float2(f.y, f.w)};
}
template <> __device__ __forceinline__ CD ld_sm_cc<CD>(const unsigned char *p) {
    const double2 f = sm_ld(reinterpret_cast<const double2 *>(p));
    return {f.x, f.y};
}
template <> __device__ __forceinline__ CDF ld_sm_cc<CDF>(const unsigned char *p) {
    const float4 f = sm_ld(reinterpret_cast<const float4 *>(p));
    return {DF(f.x, f.y), DF(f.z, f.w)};
}
__device__ __forceinline__ CV scale_sym_sm(CV x, const float *s) {
    return cscale2(x, sm_ld(reinterpret_cast<const float2 *>(s)));
}
__device__ __forceinline__ CD scale_sym_sm(CD x, const double *s) { return cscale(x, sm_ld(s)); }
__device__ __forceinline__ CDF scale_sym_sm(CDF x, const DF *s) { return cscale(x, sm_ld(s)); }

// Blocks per SM requested from the compiler: a register budget of 64 per thread for E <= 8
// values per thread, 128 otherwise.
template <int T, int E> __host__ __device__ constexpr int min_blocks_for() {
    // Bounded by the SM's 65536 registers, 2048 threads and 32 resident blocks.
    const int regs = E <= 8 ? 64 : 128;
    const int by_regs = 65536 / (T * regs), by_threads = 2048 / T;
    const int b = by_regs < by_threads ? by_regs : by_threads;
    return b > 32 ? 32 : b > 0 ? b : 1;
}

// ---- K2 / K4 -----------------------------------------------------------------------------
// KIND 0 (y forward): tile = (tx, z); input rows y < N of w1, outputs all 2N rows of w2.
// KIND 2 (y inverse): tile = (tx, z); input rows ky < 2N of w3, outputs y < N of w1.
// Thread t serves column group g = t mod NG (16 bytes of each row: two FP32 or one FP64
// column) as its q = t / NG-th thread, so the lanes of a warp cover consecutive groups of
// the same rows and every global store of a warp is a contiguous row segment.
template <typename Real, int L, int KIND>
__global__ void __launch_bounds__(tma_threads<Real, L, KIND>(), min_blocks_for<tma_threads<Real, L, KIND>(), Cfg<Real, L>::E>())
k_col_tma(const __grid_constant__ CUtensorMap tin, Cx2<Real> *__restrict__ out,
          const typename TwOf<typename Types<Real>::CC>::T *__restrict__ tw, int ntx, int ntiles,
          int ncols, long long out_row, long long out_outer, int *__restrict__ status, int z0) {
    using C = typename Types<Real>::CC;
    using Lay = TmaLayout<Real, L, KIND>;
    using Rs = typename Cfg<Real, L>::Rs;
    constexpr bool FWD = KIND == 0;
    constexpr int E = Cfg<Real, L>::E, W = Lay::W, TC = Lay::TC, R0 = FirstRadix<Rs>::v;
    constexpr int TCU = Lay::ROWB / 8;  // box width in 8-byte units
    extern __shared__ __align__(16) unsigned char smraw[];
    griddep_wait();
    unsigned char *base = smraw + ((128 - (smem_addr(smraw) & 127)) & 127);
    unsigned char *inb = base;
    C *xb = reinterpret_cast<C *>(base + Lay::OFF_XB);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + Lay::OFF_BAR);
    constexpr int NG = Lay::NG;
    const int g = threadIdx.x % NG, q = threadIdx.x / NG;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        const int tx = t % ntx, outer = z0 + t / ntx;
        mbar_arrive_expect_tx(bar, Lay::IN_BYTES);
#pragma unroll
        for (int c = 0; c < Lay::NCP; ++c)
            tma_load_3d(inb + c * Lay::RPC * Lay::ROWB, &tin, bar, tx * TCU, c * Lay::RPC, outer);
    };
    int t = blockIdx.x;
    if (threadIdx.x == 0 && t < ntiles) issue(t);
    uint32_t phase = 0;
    for (; t < ntiles; t += gridDim.x) {
        const int tx = t % ntx, outer = z0 + t / ntx;
        const int col = tx * TC + W * g;
        const bool valid = col < ncols;
        const bool ok = mbar_wait(bar, phase, status);
        if (__syncthreads_or(!ok)) return;
        phase ^= 1;
        C v[E];
        Stage<C, L, E, FWD ? -1 : 1, R0, 1>::template gather<FWD>(v, q, [&](int row) {
            return ld_sm_cc<C>(inb + row * Lay::ROWB + g * 16);
        });
        __syncthreads();  // the staging buffer is free: fetch the next tile behind this one
        if (threadIdx.x == 0 && t + (int)gridDim.x < ntiles) {
            fence_proxy_async();
            issue(t + gridDim.x);
        }
        Cx2<Real> *dst = out + (long long)outer * out_outer + col;
        constexpr RunOpt opt{true, false, false, !FWD, false};
        Stages<C, L, E, FWD ? -1 : 1, 1, Rs>::template run<opt>(
            v, q, g, xb, NG, tw, 1, [&](int) { return czero<C>(); },
            [&](int row, C x) {
                if (valid) st_cc(dst + row * out_row, x);
            });
    }
}

// ---- K3 ----------------------------------------------------------------------------------
// Tile = (tx, ky, b): input z < N rows of density b in w2, symbol rows kz <= N of the
// octant at |ky|, output z < N rows of density b in w3.
// Energy |F|^2 of the padded spectrum in the registers of one element (both lanes of CV),
// weighted by column (kx = 0 and N once, 0 < kx < N twice for the mirrored -kx, kx > N
// padding not at all).
__device__ __forceinline__ float2 cenergy(CV x) { return f2fma(x.re, x.re, f2mul(x.im, x.im)); }
__device__ __forceinline__ float cenergy(CD x) { return (float)(x.re * x.re + x.im * x.im); }
__device__ __forceinline__ float cenergy(CF x) { return x.re * x.re + x.im * x.im; }
__device__ __forceinline__ float cenergy(CDF x) {
    const float r = x.re.hi + x.re.lo, i = x.im.hi + x.im.lo;  // the value, whatever the split
    return r * r + i * i;
}

// With TAIL, the forward spectrum's energy in the outer shell max(|kx|,|ky|,|kz|) >= 7N/8
// and its total energy are added (FP32 per thread, FP64 per tile) to tail[2 b], tail[2 b + 1]
// for density b: the a-posteriori indicator of the density's resolution.
template <typename Real, int L, bool TAIL>
__global__ void __launch_bounds__(tma_threads<Real, L, 1>(), min_blocks_for<tma_threads<Real, L, 1>(), Cfg<Real, L>::E>())
k_z_symbol_tma(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tsym,
               Cx2<Real> *__restrict__ out,
               const typename TwOf<typename Types<Real>::CC>::T *__restrict__ tw, int ntx, int ntiles,
               int ncols, int Px, int *__restrict__ status, double *__restrict__ tail) {
    using C = typename Types<Real>::CC;
    using Lay = TmaLayout<Real, L, 1>;
    using Rs = typename Cfg<Real, L>::Rs;
    using Rv = Reverse<Rs>;
    constexpr int N = L / 2, E = Cfg<Real, L>::E, W = Lay::W, TC = Lay::TC, P = Lay::P;
    constexpr int RL = LastRadix<Rs>::v, R0 = FirstRadix<Rs>::v;
    constexpr int TCU = Lay::ROWB / 8;
    extern __shared__ __align__(16) unsigned char smraw[];
    griddep_wait();
    unsigned char *base = smraw + ((128 - (smem_addr(smraw) & 127)) & 127);
    unsigned char *inb = base;
    C *xb = reinterpret_cast<C *>(base + Lay::OFF_XB);
    Real *sb = reinterpret_cast<Real *>(base + Lay::OFF_S);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + Lay::OFF_BAR);  // [0] input, [1] symbol
    constexpr int NG = Lay::NG;
    const int g = threadIdx.x % NG, q = threadIdx.x / NG;
    const long long zs = (long long)L * Px;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        fence_mbar_init();
    }
    __syncthreads();
    // Consecutive tiles take ky and its mirror 2N - ky, which read the same symbol rows.
    auto ky_of = [&](int by) { return (by & 1) ? L - ((by + 1) >> 1) : (by >> 1); };
    auto issue_in = [&](int t) {
        const int tx = t % ntx, ky = ky_of((t / ntx) % L), b = t / (ntx * L);
        mbar_arrive_expect_tx(bar, Lay::IN_BYTES);
#pragma unroll
        for (int c = 0; c < Lay::NCP; ++c)
            tma_load_3d(inb + c * Lay::RPC * Lay::ROWB, &tin, bar, tx * TCU, ky, b * N + c * Lay::RPC);
    };
    auto issue_sym = [&](int t) {
        const int tx = t % ntx, ky = ky_of((t / ntx) % L);
        const int kya = ky <= N ? ky : L - ky;
        mbar_arrive_expect_tx(bar + 1, Lay::S_BYTES);
#pragma unroll
        for (int c = 0; c < Lay::NCS; ++c)
            tma_load_3d(reinterpret_cast<unsigned char *>(sb) + c * Lay::SRC * Lay::SROWB, &tsym, bar + 1,
                        tx * TC, kya, c * Lay::SRC);
    };
    int t = blockIdx.x;
    if (threadIdx.x == 0 && t < ntiles) {
        issue_in(t);
        issue_sym(t);
    }
    uint32_t phase = 0;
    for (; t < ntiles; t += gridDim.x) {
        const int tx = t % ntx, ky = ky_of((t / ntx) % L), bb = t / (ntx * L);
        const int col = tx * TC + W * g;
        const bool valid = col < ncols;
        const bool more = t + (int)gridDim.x < ntiles;
        bool ok = mbar_wait(bar, phase, status);
        if (__syncthreads_or(!ok)) return;
        C v[E];
        Stage<C, L, E, -1, R0, 1>::template gather<true>(v, q, [&](int row) {
            return ld_sm_cc<C>(inb + row * Lay::ROWB + g * 16);
        });
        __syncthreads();
        if (threadIdx.x == 0 && more) {
            fence_proxy_async();
            issue_in(t + gridDim.x);
        }
        constexpr RunOpt fwd{true, false, true, false, false};
        Stages<C, L, E, -1, 1, Rs>::template run<fwd>(
            v, q, g, xb, NG, tw, 1, [&](int) { return czero<C>(); }, [&](int, C) {});
        if constexpr (TAIL) {
            const int kya = ky <= N ? ky : L - ky;
            constexpr int SHELL = N - N / 8;
            float w[W], eshell = 0.f, etot = 0.f;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const int kx = col + i;
                w[i] = kx > N || !valid ? 0.f : (kx == 0 || kx == N) ? 1.f : 2.f;
            }
#pragma unroll
            for (int b = 0; b < E / RL; ++b) {
                const int j = q + P * b;
#pragma unroll
                for (int r = 0; r < RL; ++r) {
                    const int row = j + r * (L / RL);
                    const int kz = row <= N ? row : L - row;
                    float e;
                    if constexpr (W == 2) {
                        const float2 en = cenergy(v[b * RL + r]);
                        e = w[0] * en.x + w[1] * en.y;
                        if ((kz >= SHELL || kya >= SHELL) || col >= SHELL) eshell += e;
                        else if (col + 1 >= SHELL) eshell += w[1] * en.y;
                    } else {
                        e = w[0] * cenergy(v[b * RL + r]);
                        if (kz >= SHELL || kya >= SHELL || col >= SHELL) eshell += e;
                    }
                    etot += e;
                }
            }
            // Tile sum: warp shuffles, then one FP64 atomic per warp (blocks of fewer than 32
            // threads, at the smallest sizes, add per thread).
            if constexpr (tma_threads<Real, L, 1>() >= 32) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    eshell += __shfl_xor_sync(0xffffffffu, eshell, o);
                    etot += __shfl_xor_sync(0xffffffffu, etot, o);
                }
            }
            if (tma_threads<Real, L, 1>() < 32 || (threadIdx.x & 31) == 0) {
                atomicAdd(tail + 2 * bb, (double)eshell);
                atomicAdd(tail + 2 * bb + 1, (double)etot);
            }
        }
        ok = mbar_wait(bar + 1, phase, status);
        if (__syncthreads_or(!ok)) return;
        phase ^= 1;
        // The forward's last stage (radix RL) left row j + r L/RL of butterfly b in v[b RL + r].
#pragma unroll
        for (int b = 0; b < E / RL; ++b) {
            const int j = q + P * b;
#pragma unroll
            for (int r = 0; r < RL; ++r) {
                const int row = j + r * (L / RL);
                const int kz = row <= N ? row : L - row;
                v[b * RL + r] = scale_sym_sm(v[b * RL + r], sb + kz * TC + W * g);
            }
        }
        __syncthreads();  // the symbol buffer is free
        if (threadIdx.x == 0 && more) {
            fence_proxy_async();
            issue_sym(t + gridDim.x);
        }
        Cx2<Real> *dst = out + ((long long)bb * N * L + ky) * Px + col;
        constexpr RunOpt inv{true, false, false, true, false};
        Stages<C, L, E, 1, 1, Rv>::template run<inv>(
            v, q, g, xb, NG, tw, 1, [&](int) { return czero<C>(); },
            [&](int row, C x) {
                if (valid) st_cc(dst + row * zs, x);
            });
    }
}

// ---- K3, split form ------------------------------------------------------------------------
// The pruned length-2N forward transform of a column splits by the parity of the output
// index: X[2m] is the length-N DFT of x, X[2m+1] the length-N DFT of x_n W_{2N}^n (the
// inputs x_n, n < N, are the nonzero half).  The kept inverse outputs split the same way:
// u_z = A_z + conj(W_{2N}^z) B_z for z < N, with A and B the length-N inverse DFTs of the
// even and odd halves of the spectrum.  Half h of the threads of a column group runs the
// length-N transforms of parity h.  Where the length-N schedule has one stage fewer than
// the length-2N one, this saves one shared-memory exchange per direction, for the price of
// reading the staged input twice and one half-size exchange that adds A and B.
template <class RL> struct NumStages;
template <int... Rs> struct NumStages<Radices<Rs...>> { static constexpr int v = sizeof...(Rs); };

template <int L> __host__ __device__ constexpr bool zsplit_available() {
    if constexpr (L < 8) {
        return false;
    } else {
        using Rh = typename FftCfg<L / 2>::Rs;
        return NumStages<Rh>::v < NumStages<typename FftCfg<L>::Rs>::v && FirstRadix<Rh>::v % 2 == 0;
    }
}
template <typename Real, int L> __host__ __device__ constexpr int zsplit_threads() {
    return TmaLayout<Real, L, 1>::NG * 2 * ((L / 2) / FftCfg<L / 2>::E);
}

template <typename Real, int L, bool TAIL>
__global__ void __launch_bounds__(zsplit_threads<Real, L>(), min_blocks_for<zsplit_threads<Real, L>(), FftCfg<L / 2>::E>())
k_z_split_tma(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tsym,
              Cx2<Real> *__restrict__ out,
              const typename TwOf<typename Types<Real>::CC>::T *__restrict__ tw, int ntx, int ntiles,
              int ncols, int Px, int *__restrict__ status, double *__restrict__ tail) {
    using C = typename Types<Real>::CC;
    using Lay = TmaLayout<Real, L, 1>;
    constexpr int N = L / 2;
    using Rs = typename FftCfg<N>::Rs;
    using Rv = Reverse<Rs>;
    constexpr int E = FftCfg<N>::E, PH = N / E, W = Lay::W, TC = Lay::TC, NG = Lay::NG;
    constexpr int R0 = FirstRadix<Rs>::v, RL = LastRadix<Rs>::v;
    constexpr int TCU = Lay::ROWB / 8;
    constexpr int NT = zsplit_threads<Real, L>();
    static_assert(R0 % 2 == 0, "the A + B exchange splits the first radix's outputs in halves");
    static_assert(NT <= 1024, "threads of one CTA");
    extern __shared__ __align__(16) unsigned char smraw[];
    griddep_wait();
    unsigned char *base = smraw + ((128 - (smem_addr(smraw) & 127)) & 127);
    unsigned char *inb = base;
    C *xb = reinterpret_cast<C *>(base + Lay::OFF_XB);
    Real *sb = reinterpret_cast<Real *>(base + Lay::OFF_S);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + Lay::OFF_BAR);  // [0] input, [1] symbol
    const int g = threadIdx.x % NG, q = threadIdx.x / NG;
    const int h = q / PH, qh = q - h * PH;  // parity of this thread's half, index within it
    C *xh = xb + h * N * NG;                // the half's exchange rows
    const long long zs = (long long)L * Px;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto ky_of = [&](int by) { return (by & 1) ? L - ((by + 1) >> 1) : (by >> 1); };
    auto issue_in = [&](int t) {
        const int tx = t % ntx, ky = ky_of((t / ntx) % L), b = t / (ntx * L);
        mbar_arrive_expect_tx(bar, Lay::IN_BYTES);
#pragma unroll
        for (int c = 0; c < Lay::NCP; ++c)
            tma_load_3d(inb + c * Lay::RPC * Lay::ROWB, &tin, bar, tx * TCU, ky, b * N + c * Lay::RPC);
    };
    auto issue_sym = [&](int t) {
        const int tx = t % ntx, ky = ky_of((t / ntx) % L);
        const int kya = ky <= N ? ky : L - ky;
        mbar_arrive_expect_tx(bar + 1, Lay::S_BYTES);
#pragma unroll
        for (int c = 0; c < Lay::NCS; ++c)
            tma_load_3d(reinterpret_cast<unsigned char *>(sb) + c * Lay::SRC * Lay::SROWB, &tsym, bar + 1,
                        tx * TC, kya, c * Lay::SRC);
    };
    int t = blockIdx.x;
    if (threadIdx.x == 0 && t < ntiles) {
        issue_in(t);
        issue_sym(t);
    }
    uint32_t phase = 0;
    for (; t < ntiles; t += gridDim.x) {
        const int tx = t % ntx, ky = ky_of((t / ntx) % L), bb = t / (ntx * L);
        const int col = tx * TC + W * g;
        const bool valid = col < ncols;
        const bool more = t + (int)gridDim.x < ntiles;
        bool ok = mbar_wait(bar, phase, status);
        if (__syncthreads_or(!ok)) return;
        C v[E];
        Stage<C, N, E, -1, R0, 1>::template gather<false>(v, qh, [&](int row) {
            return ld_sm_cc<C>(inb + row * Lay::ROWB + g * 16);
        });
        __syncthreads();
        if (threadIdx.x == 0 && more) {
            fence_proxy_async();
            issue_in(t + gridDim.x);
        }
        if (h) {  // odd outputs: transform x_n W_{2N}^n
#pragma unroll
            for (int b = 0; b < E / R0; ++b) {
                const int j = qh + PH * b;
#pragma unroll
                for (int r = 0; r < R0; ++r) v[b * R0 + r] = twmul<-1>(v[b * R0 + r], __ldg(tw + j + r * (N / R0)));
            }
        }
        constexpr RunOpt fwd{true, false, true, false, false};
        Stages<C, N, E, -1, 1, Rs>::template run<fwd>(
            v, qh, g, xh, NG, tw, 2, [&](int) { return czero<C>(); }, [&](int, C) {});
        // v[b RL + r] = X[2m + h], m = qh + PH b + r N/RL.
        if constexpr (TAIL) {
            const int kya = ky <= N ? ky : L - ky;
            constexpr int SHELL = N - N / 8;
            float w[W], eshell = 0.f, etot = 0.f;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const int kx = col + i;
                w[i] = kx > N || !valid ? 0.f : (kx == 0 || kx == N) ? 1.f : 2.f;
            }
#pragma unroll
            for (int b = 0; b < E / RL; ++b) {
#pragma unroll
                for (int r = 0; r < RL; ++r) {
                    const int k = 2 * (qh + PH * b + r * (N / RL)) + h;
                    const int kz = k <= N ? k : L - k;
                    float e;
                    if constexpr (W == 2) {
                        const float2 en = cenergy(v[b * RL + r]);
                        e = w[0] * en.x + w[1] * en.y;
                        if ((kz >= SHELL || kya >= SHELL) || col >= SHELL) eshell += e;
                        else if (col + 1 >= SHELL) eshell += w[1] * en.y;
                    } else {
                        e = w[0] * cenergy(v[b * RL + r]);
                        if (kz >= SHELL || kya >= SHELL || col >= SHELL) eshell += e;
                    }
                    etot += e;
                }
            }
            if constexpr (NT >= 32) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    eshell += __shfl_xor_sync(0xffffffffu, eshell, o);
                    etot += __shfl_xor_sync(0xffffffffu, etot, o);
                }
            }
            if (NT < 32 || (threadIdx.x & 31) == 0) {
                atomicAdd(tail + 2 * bb, (double)eshell);
                atomicAdd(tail + 2 * bb + 1, (double)etot);
            }
        }
        ok = mbar_wait(bar + 1, phase, status);
        if (__syncthreads_or(!ok)) return;
        phase ^= 1;
#pragma unroll
        for (int b = 0; b < E / RL; ++b) {
#pragma unroll
            for (int r = 0; r < RL; ++r) {
                const int k = 2 * (qh + PH * b + r * (N / RL)) + h;
                const int kz = k <= N ? k : L - k;
                v[b * RL + r] = scale_sym_sm(v[b * RL + r], sb + kz * TC + W * g);
            }
        }
        __syncthreads();  // the symbol buffer is free
        if (threadIdx.x == 0 && more) {
            fence_proxy_async();
            issue_sym(t + gridDim.x);
        }
        constexpr RunOpt inv{true, false, true, false, false};
        Stages<C, N, E, 1, 1, Rv>::template run<inv>(
            v, qh, g, xh, NG, tw, 2, [&](int) { return czero<C>(); }, [&](int, C) {});
        // v[b R0 + r] = A_z (h = 0) or B_z (h = 1), z = qh + PH b + r N/R0.  Half 0 keeps the
        // rows z < N/2 (r < R0/2) and half 1 the rest; each sends the other half its rows.
        if (h) {
#pragma unroll
            for (int b = 0; b < E / R0; ++b) {
                const int j = qh + PH * b;
#pragma unroll
                for (int r = 0; r < R0; ++r) v[b * R0 + r] = twmul<1>(v[b * R0 + r], __ldg(tw + j + r * (N / R0)));
            }
        }
        __syncthreads();  // every read of the inverse's exchanges is done
#pragma unroll
        for (int b = 0; b < E / R0; ++b) {
            const int j = qh + PH * b;
#pragma unroll
            for (int r = 0; r < R0; ++r)
                if ((2 * r < R0) == (h != 0)) sm_st(xb + (j + r * (N / R0)) * NG + g, v[b * R0 + r]);
        }
        __syncthreads();
        Cx2<Real> *dst = out + ((long long)bb * N * L + ky) * Px + col;
#pragma unroll
        for (int b = 0; b < E / R0; ++b) {
            const int j = qh + PH * b;
#pragma unroll
            for (int r = 0; r < R0; ++r) {
                if ((2 * r < R0) == (h == 0)) {
                    const int z = j + r * (N / R0);
                    const C x = cadd(v[b * R0 + r], xb[z * NG + g]);
                    if (valid) st_cc(dst + z * zs, x);
                }
            }
        }
    }
}

}  // namespace gsp
