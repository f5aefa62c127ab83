// Warp forms of the passes, FP32.  The fused z pass (K3) at N = 16 E1, L = 2N = 32 E1 for a
// first-stage length E1 (N = 256, 192, 160, 128, 96, 64); the y passes (K2, K4) on its
// transform halves; the x passes (K1, K5) at N = 16 E1 with a half-warp per row pair and at
// N = 512 with a warp per row pair (E1 in {4, 6, 8, 10, 12, 16}: N = 64 ... 256).  The
// description below is for E1 = 16; for E1 < 16
// the first stage is a pruned E1-point DFT (E1 / 2 nonzero inputs), the lane-pair radix 2
// pairs the halves of its outputs the same way, and only the 2 E1 lanes l with
// (l & 7) < E1 / 2 gather after the exchange (the others idle through the 16-point DFTs).
//
// Same operation as k_z_symbol_tma: per column (kx, ky) of w2, the pruned length-2N forward
// DFT along z, the product with the symbol G(|kx|, |ky|, |kz|), the inverse DFT and the crop
// to z < N (Sec. 2: convolution with the G-tensor on the zero-padded grid, I_delta folded
// into the symbol).  Here one warp owns one pair of neighbouring columns (packed FP32x2,
// type CV), so the exchanges of the transform are warp-local and no block barrier sits
// inside the transforms.
//
// Decomposition of the length-512 forward transform of a column x (x_n = 0 for n >= 256),
// lane q = q' + 16 s (q' < 16, s < 2), register j < 16:
//   F1  lane q: A_q[k1] = sum_{r<8} x[q + 32 r] W_16^{r k1}  (16-point DFT, 8 nonzero inputs)
//   F2  B_q[k1] = A_q[k1] W_512^{q k1}
//   F3  radix 2 over s between lanes q' and q' + 16 (shuffle):
//       V[q'][k1][0] = B_q'[k1] + B_{q'+16}[k1],  V[q'][k1][1] = (B_q'[k1] - B_{q'+16}[k1]) W_32^{q'}
//   F5  exchange through shared memory: lane l = k1 + 16 t gathers V[q'][k1][t], q' < 16
//   F6  16-point DFT over q':  X[k1 + 16 t + 32 k2] = sum_q' V[q'][k1][t] W_16^{q' k2}
// so lane l holds X[l + 32 k2] in register k2.  Every step is linear, and the inverse
// transform is the adjoint: the conjugate transpose of each step in reverse order, which
// moves data along the same paths and returns the z < N outputs to the lanes and registers
// the inputs came from.
//
// Register maps.  After F1, register j holds k1 = kappa0(j) = 2j (j < 8) or 2(j-8)+1 for
// the lower half-warp; the upper half holds kappa0(j) ^ 8, obtained by negating its odd
// inputs (X[k + 8] of a 16-point DFT with 8 nonzero inputs is X[k] of the inputs times
// (-1)^r).  Then the registers j in K = {0..3, 8..11} of both halves hold k1 values that
// pair with the partner's register j + 4, and F3 runs the same instructions on every lane:
// keep v[j], receive the partner's v[j + 4].  The upper half's difference comes out
// negated; its F3 twiddle carries the sign (-W_32^{q'}).
//
// Shared memory (one CTA = one tile of 8 columns x 1 ky x the N input rows, 4 warps; four
// CTAs per SM, so 16 warps from four independent tiles share it):
//   B   16 KB: the TMA input tile (256 rows x 64 B, 64-byte swizzle), then the tile's
//       symbol lines (boxes of 128 kz x 8 kx, kz innermost: the octant table is symmetric
//       in (kx, ky, kz), so read with its innermost index as kz each column's kz values
//       lie contiguous and the lanes read consecutive floats), then the next tile's input;
//   XO  32 KB: 512 rows of 64 B; warp g owns the 16-byte chunk g ^ ((row >> 1) & 3) of
//       every row, for its exchange slots (all 512 rows) and for its outputs (rows z < 256),
//       so the first 16 KB is the output tile in the TMA store's 64-byte swizzle;
//   T   4 KB: twiddles W_512^{q k1} as T[k1][q];
//   three mbarriers (input, symbol, XO free) and three arrival counters.
// The last warp to finish with B (input read, symbol read) issues the next TMA load into
// it; the last warp to write its outputs issues the TMA store of the tile and, once the
// store has read XO, frees XO for the next tile's exchange.  All waits are bounded.
//
// Exchange slots: reader lane l takes position p from row 16 l + (p ^ (l & 7)).  The bank
// group (row mod 8, with the warp's chunk) differs across the eight lanes of every
// quarter-warp access in both directions, and both addresses are a lane constant XOR a
// compile-time constant (bits 4-9) plus a compile-time offset.  (The y warp forms use the
// same slots in 128-byte rows, eight warps to a row.)
#pragma once
#include "tma.cuh"

namespace gsp {

template <int E1> struct ZWarp {
    static constexpr int H = E1 / 2, N = 16 * E1, L = 2 * N, TC = 8, NW = 4, NT = 128, ROWB = TC * 8;
    static constexpr int MINB = 4;  // CTAs per SM: 16 warps, 128 registers a thread
    // Symbol lines: boxes of SYM_KZB kz values (innermost) x 1 ky x TC kx; kz <= N.
    static constexpr int SYM_KZB = 128, SYM_NCP = (N + 1 + SYM_KZB - 1) / SYM_KZB;
    static constexpr int IN_BYTES = N * TC * 8;
    static constexpr int SYM_BYTES = SYM_NCP * SYM_KZB * TC * 4;
    static constexpr int B_BYTES = IN_BYTES > SYM_BYTES ? IN_BYTES : SYM_BYTES;
    static constexpr int XO_BYTES = 512 * ROWB;  // the exchange slots (512 rows), then the output tile
    static constexpr int OFF_B = 0, OFF_XO = (B_BYTES + 1023) / 1024 * 1024, OFF_T = OFF_XO + XO_BYTES;
    static constexpr int OFF_BAR = OFF_T + E1 * 32 * 8;
    static constexpr int SMEM = 1024 + OFF_BAR + 64;  // 1 KB alignment slack
    static_assert(E1 == 16 || E1 == 12 || E1 == 10 || E1 == 8 || E1 == 6 || E1 == 4,
                  "first stage: a pruned DFT of E1 / 2 inputs");
    static_assert(SYM_BYTES <= IN_BYTES, "the symbol lines fit the input buffer");
};

// CV times the scalar twiddle w = (re, im) (D < 0) or its conjugate (D > 0).
template <int D> __device__ __forceinline__ CV zw_twmul(CV a, float2 w) {
    const float2 R = f2(w.x, w.x);
    const float2 I = f2(w.y, w.y), NI = f2(-w.y, -w.y);
    if (D < 0) return {f2fma(a.im, NI, f2mul(a.re, R)), f2fma(a.re, I, f2mul(a.im, R))};
    return {f2fma(a.im, I, f2mul(a.re, R)), f2fma(a.re, NI, f2mul(a.im, R))};
}
__device__ __forceinline__ CV zw_neg(CV a) { return {f2mul(a.re, f2(-1.f, -1.f)), f2mul(a.im, f2(-1.f, -1.f))}; }
// a exp(D i pi / 2)
template <int D> __device__ __forceinline__ CV zw_rot(CV a) {
    return D < 0 ? CV{a.im, f2neg(a.re)} : CV{f2neg(a.im), a.re};
}

// exp(-2 pi i r / E) = (zw_cw, zw_sw), r < E / 2, E in {4, 6, 8, 10, 12, 16}.
__host__ __device__ constexpr float zw_cw(int E, int r) {
    return E == 4 ? (r == 0 ? 1.f : 0.f)
         : E == 6 ? (r == 0 ? 1.f : r == 1 ? 0.5f : -0.5f)
         : E == 8 ? (r == 0 ? 1.f : r == 1 ? 0.70710678118654752440f : r == 2 ? 0.f : -0.70710678118654752440f)
         : E == 16 ? (r == 0 ? 1.f : r == 1 ? 0.92387953251128675613f : r == 2 ? 0.70710678118654752440f
                      : r == 3 ? 0.38268343236508977173f : r == 4 ? 0.f : r == 5 ? -0.38268343236508977173f
                      : r == 6 ? -0.70710678118654752440f : -0.92387953251128675613f)
         : E == 12 ? (r == 0 ? 1.f : r == 1 ? 0.86602540378443864676f : r == 2 ? 0.5f : r == 3 ? 0.f
                      : r == 4 ? -0.5f : -0.86602540378443864676f)
                   : (r == 0 ? 1.f : r == 1 ? 0.80901699437494742410f : r == 2 ? 0.30901699437494742410f
                      : r == 3 ? -0.30901699437494742410f : -0.80901699437494742410f);
}
__host__ __device__ constexpr float zw_sw(int E, int r) {
    return E == 4 ? (r == 0 ? 0.f : -1.f)
         : E == 6 ? (r == 0 ? 0.f : -0.86602540378443864676f)
         : E == 8 ? (r == 0 ? 0.f : r == 1 ? -0.70710678118654752440f : r == 2 ? -1.f : -0.70710678118654752440f)
         : E == 16 ? (r == 0 ? 0.f : r == 1 ? -0.38268343236508977173f : r == 2 ? -0.70710678118654752440f
                      : r == 3 ? -0.92387953251128675613f : r == 4 ? -1.f : r == 5 ? -0.92387953251128675613f
                      : r == 6 ? -0.70710678118654752440f : -0.38268343236508977173f)
         : E == 12 ? (r == 0 ? 0.f : r == 1 ? -0.5f : r == 2 ? -0.86602540378443864676f : r == 3 ? -1.f
                      : r == 4 ? -0.86602540378443864676f : -0.5f)
                   : (r == 0 ? 0.f : r == 1 ? -0.58778525229247312917f : r == 2 ? -0.95105651629515357212f
                      : r == 3 ? -0.95105651629515357212f : -0.58778525229247312917f);
}

// Register maps of the first stage (E1 outputs, H = E1 / 2): register j holds
// k1 = kappa0(j) on the lower half-warp (2j for j < H, 2(j - H) + 1 otherwise); the keep
// set K holds kappa0 < H, and partner(j) is the register holding kappa0(j) + H.
template <int E1> struct ZwMap {
    static constexpr int H = E1 / 2;
    __host__ __device__ static constexpr int kappa0(int j) { return j < H ? 2 * j : 2 * (j - H) + 1; }
    __host__ __device__ static constexpr bool inK(int j) { return kappa0(j) < H; }
    __host__ __device__ static constexpr int partner(int j) {
        return (kappa0(j) + H) % 2 == 0 ? (kappa0(j) + H) / 2 : H + (kappa0(j) + H - 1) / 2;
    }
};

// F1: forward E1-point DFT of v[0..H-1] (inputs H..E1-1 zero): v[m] = X[2m], v[H+m] = X[2m+1]
// (X[2m] = DFT_H(a)[m], X[2m+1] = DFT_H(a_r W_E1^r)[m]).
template <int E1> __device__ __forceinline__ void zw_f1(CV *v) {
    constexpr int H = E1 / 2;
#pragma unroll
    for (int r = 0; r < H; ++r) {
        if (r == 0) v[H] = v[0];
        else if (4 * r == E1) v[H + r] = zw_rot<-1>(v[r]);
        else v[H + r] = cmulk<-1>(v[r], zw_cw(E1, r), zw_sw(E1, r));
    }
    dft<H, -1>(v);
    dft<H, -1>(v + H);
}
// Adjoint of F1: y_r = IDFT_H(v[0..H-1])[r] + conj(W_E1^r) IDFT_H(v[H..E1-1])[r], r < H, in v[0..H-1].
template <int E1> __device__ __forceinline__ void zw_f1_adj(CV *v) {
    constexpr int H = E1 / 2;
    dft<H, 1>(v);
    dft<H, 1>(v + H);
#pragma unroll
    for (int r = 0; r < H; ++r) {
        const CV o = r == 0 ? v[H] : 4 * r == E1 ? zw_rot<1>(v[H + r]) : cmulk<1>(v[H + r], zw_cw(E1, r), zw_sw(E1, r));
        v[r] = cadd(v[r], o);
    }
}

// Byte offset of row `row` of warp g in a 128-byte-swizzled region.
__device__ __forceinline__ int zw_sw128(int row, int g) { return row * 128 + ((g ^ (row & 7)) << 4); }
// The same in a region of RB-byte rows (RB = 128, or 64 with the TMA's 64-byte swizzle: chunk
// g ^ ((row >> 1) & 3) of four).
template <int RB> __device__ __forceinline__ int zw_swz(int row, int g) {
    return RB == 128 ? zw_sw128(row, g) : row * 64 + ((g ^ ((row >> 1) & 3)) << 4);
}

// Exchange slots by shared-memory address (layout re.x, re.y, im.x, im.y).
__device__ __forceinline__ void zw_sts(uint32_t a, CV x) {
    if (!dbg_smem_ok(a, 16)) return;
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x.re.x), "f"(x.re.y), "f"(x.im.x),
                 "f"(x.im.y)
                 : "memory");
}
__device__ __forceinline__ CV zw_lds(uint32_t a) {
    if (!dbg_smem_ok(a, 16)) return czero<CV>();
    float4 f;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(f.x), "=f"(f.y), "=f"(f.z), "=f"(f.w)
                 : "r"(a)
                 : "memory");
    return {f2(f.x, f.y), f2(f.z, f.w)};
}
__device__ __forceinline__ CV zw_shfl16(CV x) {
    return {f2(__shfl_xor_sync(0xffffffffu, x.re.x, 16), __shfl_xor_sync(0xffffffffu, x.re.y, 16)),
            f2(__shfl_xor_sync(0xffffffffu, x.im.x, 16), __shfl_xor_sync(0xffffffffu, x.im.y, 16))};
}


// Per-lane constants of the warp-form transform (lane q = q' + 16 s of warp g, exchange
// region at shared address xo with warp g owning chunk g ^ (row & 7) of its 512 rows; with
// RB = 64, rows of 64 bytes and chunk g ^ ((row >> 1) & 3)).  Slot row of the value
// V[q'][k1][t] (k1 = k0 + 8 s): 256 t + 128 s + 16 k0 + (q' ^ k0); within every quarter-warp
// access the row mod 8 differs from lane to lane, so the chunks hit distinct bank groups.
struct ZwLane {
    float2 tw32;   // F3 twiddle sgn W_32^{q'} (sgn = -1 on the upper half-warp)
    int tkb, tnb;  // twiddle-table bases of the registers in K (k1 = kappa0 + H s) and outside
    float sg;      // sign of the odd inputs / outputs of the upper half-warp
    uint32_t aw;   // exchange writer base: position q' of reader l = kappa0 + 8 s + 16 t
    uint32_t ar;   // exchange reader base: reader q, row 16 q + (p ^ (q & 7))
    bool rd;       // lane q gathers after the exchange ((q & 7) < H)
};
// tw: W_L^e (twstride 1) or W_2L^e (twstride 2), L = 32 E1.
template <int E1, int RB = 128>
__device__ __forceinline__ ZwLane zw_lane(const float2 *__restrict__ tw, uint32_t xo, int g, int q, int twstride = 1) {
    constexpr int H = E1 / 2;
    const int s = q >> 4, qp = q & 15;
    ZwLane z;
    z.tw32 = tw[E1 * qp * twstride];
    if (s) z.tw32 = f2(-z.tw32.x, -z.tw32.y);
    z.tkb = q + 32 * H * s;
    z.tnb = q - 32 * H * s;
    z.sg = s ? -1.f : 1.f;
    if (RB == 128) {
        z.aw = xo + 16384 * s + 128 * qp + 16 * (g ^ (qp & 7));
        z.ar = xo + 2048 * q + 128 * (q & 7) + 16 * (g ^ (q & 7));
    } else {
        z.aw = xo + 8192 * s + 64 * qp + 16 * (g ^ ((qp >> 1) & 3));
        z.ar = xo + 1024 * q + 64 * (q & 7) + 16 * (g ^ ((q >> 1) & 3));
    }
    z.rd = (q & 7) < H;
    return z;
}
__device__ __forceinline__ CV cconj_cv(CV a) { return {a.re, f2neg(a.im)}; }
__device__ __forceinline__ CV zw_sign(CV x, float sg) { return {f2mul(x.re, f2(sg, sg)), f2mul(x.im, f2(sg, sg))}; }

// F1 (inputs v[0..H-1], odd ones already signed), F2 and F3 with its twiddle.
template <int E1> __device__ __forceinline__ void zw_front(CV *v, const ZwLane &z, const float2 *T) {
    using M = ZwMap<E1>;
    zw_f1<E1>(v);
#pragma unroll
    for (int j = 0; j < E1; ++j) v[j] = zw_twmul<-1>(v[j], sm_ld(T + (M::inK(j) ? z.tkb : z.tnb) + 32 * M::kappa0(j)));
#pragma unroll
    for (int j = 0; j < E1; ++j) {
        if (!M::inK(j)) continue;
        const CV rcv = zw_shfl16(v[M::partner(j)]);
        const CV a = v[j];
        v[j] = cadd(a, rcv);
        v[M::partner(j)] = zw_twmul<-1>(csub(a, rcv), z.tw32);
    }
}
// Exchange slot addresses: writer slot of k0 (t = 0; t = 1 lies RB * 256 further) and reader
// position p, for RB-byte rows.
template <int RB> __device__ __forceinline__ uint32_t zw_wslot(const ZwLane &z, int k0) {
    return RB == 128 ? (z.aw ^ (144 * k0)) + 2048 * k0 : (z.aw ^ (64 * k0 + 16 * ((k0 >> 1) & 3))) + 1024 * k0;
}
template <int RB> __device__ __forceinline__ uint32_t zw_rslot(const ZwLane &z, int p) {
    return RB == 128 ? (z.ar ^ (144 * (p & 7))) + 1024 * (p >> 3)
                     : (z.ar ^ (64 * (p & 7) + 16 * ((p >> 1) & 3))) + 512 * (p >> 3);
}
// F5: write the values this lane holds as writer, gather its 16 as reader (reader lanes).
template <int E1, int RB = 128> __device__ __forceinline__ void zw_exchange(CV *v, const ZwLane &z) {
    using M = ZwMap<E1>;
#pragma unroll
    for (int j = 0; j < E1; ++j) {
        if (!M::inK(j)) continue;
        const int k0 = M::kappa0(j);
        zw_sts(zw_wslot<RB>(z, k0), v[j]);
        zw_sts(zw_wslot<RB>(z, k0) + 256 * RB, v[M::partner(j)]);
    }
    __syncwarp();
    if (z.rd) {
#pragma unroll
        for (int p = 0; p < 16; ++p) v[p] = zw_lds(zw_rslot<RB>(z, p));
    }
}
// Adjoint of F5.
template <int E1, int RB = 128> __device__ __forceinline__ void zw_exchange_adj(CV *v, const ZwLane &z) {
    using M = ZwMap<E1>;
    if (z.rd) {
#pragma unroll
        for (int p = 0; p < 16; ++p) zw_sts(zw_rslot<RB>(z, p), v[p]);
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < E1; ++j) {
        if (!M::inK(j)) continue;
        const int k0 = M::kappa0(j);
        v[j] = zw_lds(zw_wslot<RB>(z, k0));
        v[M::partner(j)] = zw_lds(zw_wslot<RB>(z, k0) + 256 * RB);
    }
}
// Adjoints of F3 (with its twiddle), F2 and F1: the outputs r < H in v[0..H-1], odd ones
// still to be signed.
template <int E1> __device__ __forceinline__ void zw_back(CV *v, const ZwLane &z, const float2 *T) {
    using M = ZwMap<E1>;
#pragma unroll
    for (int j = 0; j < E1; ++j) {
        if (!M::inK(j)) continue;
        const CV b = zw_twmul<1>(v[M::partner(j)], z.tw32);
        const CV a = v[j];
        v[j] = cadd(a, b);
        v[M::partner(j)] = zw_shfl16(csub(a, b));
    }
#pragma unroll
    for (int j = 0; j < E1; ++j) v[j] = zw_twmul<1>(v[j], sm_ld(T + (M::inK(j) ? z.tkb : z.tnb) + 32 * M::kappa0(j)));
    zw_f1_adj<E1>(v);
}

// Tile t = (tx, ky, b): tx the 8-column block, consecutive tiles take ky and its mirror
// 2N - ky (same symbol rows), b the density.  With TAIL the forward spectrum's shell and
// total energies are added to tail[2 b], tail[2 b + 1] (as in k_z_symbol_tma).
template <int E1, bool TAIL>
__global__ void __launch_bounds__(ZWarp<E1>::NT, ZWarp<E1>::MINB)
k_z_warp(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tsym,
         const __grid_constant__ CUtensorMap tout, const float2 *__restrict__ tw, int ntx, int ntiles,
         int ncols, int *__restrict__ status, double *__restrict__ tail) {
    using Z = ZWarp<E1>;
    constexpr int L = Z::L, N = Z::N, NW = Z::NW, H = Z::H;
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned char *base = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    unsigned char *Bb = base + Z::OFF_B;
    unsigned char *xo = base + Z::OFF_XO;
    float2 *T = reinterpret_cast<float2 *>(base + Z::OFF_T);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + Z::OFF_BAR);  // input, symbol, XO free
    int *cnt = reinterpret_cast<int *>(bar + 3);                       // input, symbol, output
    const int g = threadIdx.x >> 5, q = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        mbar_init(bar + 2, 1);
        cnt[0] = cnt[1] = cnt[2] = 0;
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < E1 * 32; i += Z::NT) T[i] = tw[(i & 31) * (i >> 5)];
    __syncthreads();
    griddep_wait();  // the previous pass has finished: its outputs are readable

    auto ky_of = [&](int by) { return (by & 1) ? L - ((by + 1) >> 1) : (by >> 1); };
    auto issue_in = [&](int t) {
        const int tx = t % ntx, ky = ky_of((t / ntx) % L), b = t / (ntx * L);
        mbar_arrive_expect_tx(bar, Z::IN_BYTES);
        tma_load_3d(Bb, &tin, bar, tx * Z::TC, ky, b * N);
    };
    auto issue_sym = [&](int t) {
        const int tx = t % ntx, ky = ky_of((t / ntx) % L);
        const int kya = ky <= N ? ky : L - ky;
        mbar_arrive_expect_tx(bar + 1, Z::SYM_BYTES);
#pragma unroll
        for (int c = 0; c < Z::SYM_NCP; ++c)
            tma_load_3d(Bb + c * Z::SYM_KZB * Z::TC * 4, &tsym, bar + 1, c * Z::SYM_KZB, kya, tx * Z::TC);
    };
    // Arrival of this warp on counter c; true on the lane-0 thread of the tile's last warp.
    auto last_arrival = [&](int c) {
        __syncwarp();
        bool last = false;
        if (q == 0) {
            __threadfence_block();
            last = atomicAdd(cnt + c, 1) % NW == NW - 1;
            if (last) {
                __threadfence_block();
                fence_proxy_async();
            }
        }
        return last;
    };
    if (threadIdx.x == 0) {
        mbar_arrive(bar + 2);  // XO starts free
        if ((int)blockIdx.x < ntiles) issue_in(blockIdx.x);
    }

    constexpr int RB = Z::ROWB;
    const ZwLane zl = zw_lane<E1, RB>(tw, smem_addr(xo), g, q);
    // Input/output rows q + 32 r of this warp's 16-byte chunk.
    const int io = zw_swz<RB>(q, g);
    // Symbol: reader q holds kz = kb + 2 E1 k2 (k2 < 8) and 2N - kb - 2 E1 k2 (k2 >= 8); its
    // columns 2g and 2g + 1 have kz lines SYM_KZB floats apart in every box.
    const int kb = (q & 7) + H * ((q >> 3) & 1) + E1 * (q >> 4);
    const unsigned char *symg = Bb + 2 * g * Z::SYM_KZB * 4;
    bool stored = false;
    uint32_t ph = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ph ^= 1) {
        if (t + (int)gridDim.x >= ntiles) griddep_launch();  // this CTA's last tile
        const int tx = t % ntx, ky = ky_of((t / ntx) % L), bb = t / (ntx * L);
        const int kya = ky <= N ? ky : L - ky;
        const int col = tx * Z::TC + 2 * g;
        const bool valid = col < ncols;
        CV v[16];
        if (!mbar_wait(bar, ph, status)) return;
        if (valid) {
#pragma unroll
            for (int r = 0; r < H; ++r) {
                const float4 f = sm_ld(reinterpret_cast<const float4 *>(Bb + io + 32 * RB * r));
                v[r] = {f2(f.x, f.z), f2(f.y, f.w)};
                if (r & 1) v[r] = zw_sign(v[r], zl.sg);
            }
        }
        if (last_arrival(0)) issue_sym(t);
        if (valid) zw_front<E1>(v, zl, T);
        if (!mbar_wait(bar + 2, ph, status)) return;  // the previous tile's store has read XO
        if (valid) {
            zw_exchange<E1, RB>(v, zl);
            if (zl.rd) dft<16, -1>(v);  // v[k2] = X[kb + 2 E1 k2]
        }
        if constexpr (TAIL) {
            constexpr int SHELL = N - N / 8;
            float eshell = 0.f, etot = 0.f;
            if (valid && zl.rd) {
                const float w0 = (col == 0 || col == N) ? 1.f : 2.f;
                const float w1 = col + 1 > N ? 0.f : (col + 1 == N) ? 1.f : 2.f;
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) {
                    const int kz = k2 < 8 ? kb + 2 * E1 * k2 : L - kb - 2 * E1 * k2;
                    const float2 en = cenergy(v[k2]);
                    const bool sh = kz >= SHELL || kya >= SHELL;
                    etot += w0 * en.x + w1 * en.y;
                    if (sh || col >= SHELL) eshell += w0 * en.x;
                    if (sh || col + 1 >= SHELL) eshell += w1 * en.y;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                eshell += __shfl_xor_sync(0xffffffffu, eshell, o);
                etot += __shfl_xor_sync(0xffffffffu, etot, o);
            }
            if (valid && q == 0) {
                atomicAdd(tail + 2 * bb, (double)eshell);
                atomicAdd(tail + 2 * bb + 1, (double)etot);
            }
        }
        if (!mbar_wait(bar + 1, ph, status)) return;
        if (valid && zl.rd) {
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const int kz = k2 < 8 ? kb + 2 * E1 * k2 : L - kb - 2 * E1 * k2;
                const unsigned char *sp = symg + (kz >> 7) * (Z::SYM_KZB * Z::TC * 4) + 4 * (kz & (Z::SYM_KZB - 1));
                v[k2] = cscale2(v[k2], f2(sm_ld(reinterpret_cast<const float *>(sp)),
                                          sm_ld(reinterpret_cast<const float *>(sp + Z::SYM_KZB * 4))));
            }
        }
        if (last_arrival(1) && t + (int)gridDim.x < ntiles) issue_in(t + gridDim.x);
        if (valid) {
            if (zl.rd) dft<16, 1>(v);
            zw_exchange_adj<E1, RB>(v, zl);
            zw_back<E1>(v, zl, T);
        }
        __syncwarp();  // every lane's exchange reads are done: the slots take the outputs
        if (valid) {
#pragma unroll
            for (int r = 0; r < H; ++r) {
                CV x = v[r];
                if (r & 1) x = zw_sign(x, zl.sg);
                sm_st(reinterpret_cast<float4 *>(xo + io + 32 * RB * r), make_float4(x.re.x, x.im.x, x.re.y, x.im.y));
            }
        }
        fence_proxy_async();
        if (last_arrival(2)) {
            tma_store_3d(&tout, xo, tx * Z::TC, ky, bb * N);
            bulk_commit();
            bulk_wait_read0();
            stored = true;
            mbar_arrive(bar + 2);
        }
    }
    if (stored) bulk_wait0();
}

}  // namespace gsp

namespace gsp {

// ---- K2 / K4, warp form (FP32, N = 256) -------------------------------------------------
// The y passes with the transform halves of k_z_warp: the forward half (F1..F6) alone for
// the y forward (N input rows, all 2N output rows kept), the adjoint half alone for the
// y inverse (2N input rows, rows y < N kept).  Tile t = (tx, zz): TC columns kx, plane
// zz = b N + z, planes in descending order: the x forward pass writes its rows in ascending
// order and the x inverse reads them so, so each y pass starts on (or ends with) the planes
// that L2 still holds.  As in k_z_warp, warp g owns one 16-byte chunk of each row of the
// exchange/output buffer (g ^ (row & 7) in 128-byte rows, g ^ ((row >> 1) & 3) in 64-byte
// rows), so a warp exchanges and writes its outputs in its own chunks without waiting for
// the other warps; the last warp to finish a tile issues the TMA store.
//   y forward: 16 columns, 8 warps, two CTAs per SM; a 32 KB input buffer (prefetched for
//     the CTA's next tile as soon as every warp has read its inputs) and a 64 KB
//     exchange/output buffer (2N rows of 128 B), freed for the next tile's exchange once
//     the store has read it;
//   y inverse: 8 columns, 4 warps, four CTAs per SM; one 32 KB buffer for the 2N input
//     rows of 64 B, the exchange and the N output rows; the next tile's load follows the
//     store's read of it, so four independent CTAs per SM cover each other's loads (with
//     16-column tiles, two CTAs per SM, the pass took 80 us at N = 256 against 74).
template <int E1, bool FWD> struct YWarp {
    static constexpr int H = E1 / 2, N = 16 * E1, L = 2 * N;
    static constexpr int TC = FWD ? 16 : 8, NW = TC / 2, NT = 32 * NW, RB = 8 * TC, MINB = FWD ? 2 : 4;
    static constexpr int T_BYTES = E1 * 32 * 8;
    static constexpr int F_IN = 0, F_XB = (N * RB + 1023) / 1024 * 1024, F_T = F_XB + 512 * RB;
    static constexpr int F_BAR = F_T + T_BYTES;
    static constexpr int I_XB = 0, I_T = 512 * RB, I_BAR = I_T + T_BYTES;
    static constexpr int SMEM = 1024 + (FWD ? F_BAR : I_BAR) + 64;
    static_assert((N * RB) % 1024 == 0, "the second half of a 2N-row tile starts 1024-byte aligned");
};

// y forward of warp g's column pair, first half: its N input rows from the swizzled tile of
// RB-byte rows at inb (row y at inb + io + 32 RB (y / 32) for lane y % 32), F1 to F3.
template <int E1, int RB>
__device__ __forceinline__ void yw_fwd_front(CV *v, const unsigned char *inb, int io, const ZwLane &zl, const float2 *T) {
#pragma unroll
    for (int r = 0; r < E1 / 2; ++r) {
        const float4 f = sm_ld(reinterpret_cast<const float4 *>(inb + io + 32 * RB * r));
        v[r] = {f2(f.x, f.z), f2(f.y, f.w)};
        if (r & 1) v[r] = zw_sign(v[r], zl.sg);
    }
    zw_front<E1>(v, zl, T);
}
// Second half: the exchange through xb, the 16-point DFTs, and the 2N spectrum rows to xb
// (reader lane with base kb holds rows kb + 2 E1 k2, in warp g's chunk of each row).
template <int E1, int RB>
__device__ __forceinline__ void yw_fwd_back(CV *v, const ZwLane &zl, unsigned char *xb, int kb, int g) {
    zw_exchange<E1, RB>(v, zl);
    if (zl.rd) dft<16, -1>(v);  // v[k2] = X[kb + 2 E1 k2]
    __syncwarp();
    if (zl.rd) {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2)
            sm_st(reinterpret_cast<float4 *>(xb + zw_swz<RB>(kb + 2 * E1 * k2, g)),
                  make_float4(v[k2].re.x, v[k2].im.x, v[k2].re.y, v[k2].im.y));
    }
}
// y inverse of warp g's column pair: the 2N spectrum rows from xb, the N kept rows back to xb
// in the input tile's layout (row y at xb + io + 32 RB (y / 32)).
template <int E1, int RB>
__device__ __forceinline__ void yw_inv(CV *v, const ZwLane &zl, unsigned char *xb, int kb, int io, int g,
                                       const float2 *T) {
    if (zl.rd) {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            const float4 f = sm_ld(reinterpret_cast<const float4 *>(xb + zw_swz<RB>(kb + 2 * E1 * k2, g)));
            v[k2] = {f2(f.x, f.z), f2(f.y, f.w)};
        }
        dft<16, 1>(v);
    }
    __syncwarp();  // every lane has read its inputs: its chunks take exchange slots
    zw_exchange_adj<E1, RB>(v, zl);
    zw_back<E1>(v, zl, T);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < E1 / 2; ++r) {
        CV x = v[r];
        if (r & 1) x = zw_sign(x, zl.sg);
        sm_st(reinterpret_cast<float4 *>(xb + io + 32 * RB * r), make_float4(x.re.x, x.im.x, x.re.y, x.im.y));
    }
}

template <int E1, bool FWD>
__global__ void __launch_bounds__(YWarp<E1, FWD>::NT, YWarp<E1, FWD>::MINB)
k_y_warp(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
         const float2 *__restrict__ tw, int ntx, int ntiles, int ncols, int *__restrict__ status, int z0) {
    using Y = YWarp<E1, FWD>;
    constexpr int RB = Y::RB;
    constexpr int NW = Y::NW, N = Y::N, H = Y::H;
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned char *base = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    unsigned char *inb = base + (FWD ? Y::F_IN : Y::I_XB);
    unsigned char *xb = base + (FWD ? Y::F_XB : Y::I_XB);
    float2 *T = reinterpret_cast<float2 *>(base + (FWD ? Y::F_T : Y::I_T));
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + (FWD ? Y::F_BAR : Y::I_BAR));  // input, buffer free
    int *cnt = reinterpret_cast<int *>(bar + 2);                                         // inputs read, outputs
    const int g = threadIdx.x >> 5, q = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        cnt[0] = cnt[1] = 0;
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < E1 * 32; i += Y::NT) T[i] = tw[(i & 31) * (i >> 5)];
    __syncthreads();
    griddep_wait();  // the previous pass has finished: its outputs are readable
    auto issue_in = [&](int t) {
        const int tx = t % ntx, zz = z0 + (ntiles / ntx - 1 - t / ntx);
        mbar_arrive_expect_tx(bar, (FWD ? 1 : 2) * N * RB);
        tma_load_3d(inb, &tin, bar, tx * Y::TC, 0, zz);
        if (!FWD) tma_load_3d(inb + N * RB, &tin, bar, tx * Y::TC, N, zz);
    };
    auto last_arrival = [&](int c) {
        __syncwarp();
        bool last = false;
        if (q == 0) {
            __threadfence_block();
            last = atomicAdd(cnt + c, 1) % NW == NW - 1;
            if (last) {
                __threadfence_block();
                fence_proxy_async();
            }
        }
        return last;
    };
    if (threadIdx.x == 0) {
        if (FWD) mbar_arrive(bar + 1);  // the exchange/output buffer starts free
        if ((int)blockIdx.x < ntiles) issue_in(blockIdx.x);
    }
    const ZwLane zl = zw_lane<E1, RB>(tw, smem_addr(xb), g, q);
    const int io = zw_swz<RB>(q, g);
    // Rows of the 2N-point spectrum a reader holds: kb + 2 E1 k2.
    const int kb = (q & 7) + H * ((q >> 3) & 1) + E1 * (q >> 4);
    bool stored = false;
    uint32_t ph = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ph ^= 1) {
        if (t + (int)gridDim.x >= ntiles) griddep_launch();  // this CTA's last tile
        const int tx = t % ntx, zz = z0 + (ntiles / ntx - 1 - t / ntx);
        const bool valid = tx * Y::TC + 2 * g < ncols;
        const bool more = t + (int)gridDim.x < ntiles;
        CV v[16];
        if (!mbar_wait(bar, ph, status)) return;
        if constexpr (FWD) {
            if (valid) yw_fwd_front<E1, RB>(v, inb, io, zl, T);
            if (last_arrival(0) && more) issue_in(t + gridDim.x);
            if (!mbar_wait(bar + 1, ph, status)) return;  // the previous tile's store has read xb
            if (valid) yw_fwd_back<E1, RB>(v, zl, xb, kb, g);
        } else {
            if (valid) yw_inv<E1, RB>(v, zl, xb, kb, io, g, T);
        }
        fence_proxy_async();
        if (last_arrival(1)) {
            tma_store_3d(&tout, xb, tx * Y::TC, 0, zz);
            if (FWD) tma_store_3d(&tout, xb + N * RB, tx * Y::TC, N, zz);
            bulk_commit();
            bulk_wait_read0();
            stored = true;
            if (FWD) mbar_arrive(bar + 1);
            else if (more) issue_in(t + gridDim.x);
        }
    }
    if (stored) bulk_wait0();
}

}  // namespace gsp

namespace gsp {

// ---- K1 / K5, warp form (FP32, N = 256) -------------------------------------------------
// The x passes with one half-warp per pair of adjacent rows (2i, 2i+1) in the two lanes of
// a packed FP32x2 value.  The length-2N real transform of a row is, as in k_x_forward, the
// N-point complex FFT of its (even, odd) sample pairs z_m (m < N/2 nonzero) and the
// Hermitian split.  N = 256 = 16 x 16: lane q' holds z[q' + 16 r] (r < 8); F1 (pruned
// 16-point DFT), F2 (twiddles W_256^{q' k1}), a half-warp exchange through shared memory
// (lane k1 gathers position q' from slot 16 k1 + (q' ^ (k1 & 7))), F6 (16-point DFT):
// lane k1 holds C[k1 + 16 k2] in register k2.  The split pairs C_k with C_{N-k} through the
// same slots (slot k), so each lane computes X_k and X_{N-k} for its k <= N/2.  The inverse
// runs the same steps backwards: the combine of (Y_k, Y_{N-k}) into (C_k, C_{N-k}), the
// slots, then the adjoint transform (F6^H, exchange, F2^H, F1^H keeping z[m], m < N/2).
// Rows are read and written straight from HBM: 16 lanes x 8 bytes = one 128-byte line per
// row and instruction.  Persistent CTAs; the x forward loads the next row pair while it
// transforms the current one.
template <int N> struct XWarp {
    static constexpr int E1 = N / 16, H = E1 / 2, NT = 256;
    static constexpr int OFF_X = 0, OFF_T = OFF_X + 16 * 4096, OFF_T2 = OFF_T + E1 * 16 * 8;
    static constexpr int SMEM = OFF_T2 + (N / 2 + 1) * 8;
    static_assert(E1 == 16 || E1 == 12 || E1 == 10 || E1 == 8 || E1 == 6 || E1 == 4,
                  "N = 16 E1 with a pruned first stage of E1 / 2 inputs");
};

// Twiddle tables of the x passes from W_2N^e: T[k1 * 16 + q'] = W_N^{q' k1}, T2[k] = W_2N^k
// (k <= N/2).
template <int N> __device__ __forceinline__ void xw_tables(float2 *T, float2 *T2, const float2 *__restrict__ tw) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) T[i] = tw[2 * (i & 15) * (i >> 4)];
    for (int i = threadIdx.x; i <= N / 2; i += blockDim.x) T2[i] = tw[i];
}

// Lane qq's samples of row pair i (rows 2i, 2i+1 of the stacked densities): f[2r], f[2r+1]
// are the pairs z[qq + 16 r] of the two rows.
template <int N> __device__ __forceinline__ void xw_load(const PtrArray &rho, int i, int qq, float2 *f) {
    constexpr int H = N / 32, NN = N * N;
    const int b = (2 * i) / NN;
    const float2 *s = reinterpret_cast<const float2 *>(rho.p[b]) + (long long)(2 * i - b * NN) * (N / 2) + qq;
#pragma unroll
    for (int r = 0; r < H; ++r) {
        f[2 * r] = __ldg(s + 16 * r);
        f[2 * r + 1] = __ldg(s + N / 2 + 16 * r);
    }
}

// Forward x transform of one loaded row pair by a half-warp (lane qq, 4 KB of exchange slots
// at shared address xs): the N+1 Hermitian bins X_k of both rows to d0[k], d1[k].
template <int N>
__device__ __forceinline__ void xw_fwd_pair(const float2 *f, uint32_t xs, int qq, const float2 *T, const float2 *T2,
                                            float2 *d0, float2 *d1) {
    using M = ZwMap<N / 16>;
    constexpr int E1 = N / 16, H = E1 / 2;
    const uint32_t aw = xs + 16 * qq, ar = xs + 256 * qq + 16 * (qq & 7);
    const bool rd = qq < E1;  // lane qq gathers k1 = qq after the exchange
    CV v[16];
#pragma unroll
    for (int r = 0; r < H; ++r) v[r] = {f2(f[2 * r].x, f[2 * r + 1].x), f2(f[2 * r].y, f[2 * r + 1].y)};
    zw_f1<E1>(v);
#pragma unroll
    for (int j = 0; j < E1; ++j) v[j] = zw_twmul<-1>(v[j], T[M::kappa0(j) * 16 + qq]);
#pragma unroll
    for (int j = 0; j < E1; ++j) {
        const int k0 = M::kappa0(j);
        zw_sts((aw ^ (16 * (k0 & 7))) + 256 * k0, v[j]);
    }
    __syncwarp();
    if (rd) {
#pragma unroll
        for (int p = 0; p < 16; ++p) v[p] = zw_lds((ar ^ (16 * (p & 7))) + 16 * (p & 8));
        dft<16, -1>(v);  // v[k2] = C[qq + E1 k2]
    }
    __syncwarp();
    if (rd) {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) zw_sts(xs + 16 * (qq + E1 * k2), v[k2]);
    }
    __syncwarp();
    const float2 h = f2(0.5f, 0.5f);
#pragma unroll
    for (int k2 = 0; k2 < 9; ++k2) {
        const int k = qq + E1 * k2;
        if (!rd || k > N / 2) continue;
        const CV ck = v[k2], cn = zw_lds(xs + 16 * (k == 0 ? 0 : N - k));
        const CV ev = {f2mul(h, f2add(ck.re, cn.re)), f2mul(h, f2sub(ck.im, cn.im))};
        const CV od = {f2mul(h, f2add(ck.im, cn.im)), f2mul(h, f2sub(cn.re, ck.re))};
        if (k == 0) {
            const float2 x0 = f2add(ev.re, od.re), xn = f2sub(ev.re, od.re);
            d0[0] = f2(x0.x, 0.f);
            d1[0] = f2(x0.y, 0.f);
            d0[N] = f2(xn.x, 0.f);
            d1[N] = f2(xn.y, 0.f);
        } else {
            const CV t = zw_twmul<-1>(od, T2[k]);
            const CV xk = cadd(ev, t);
            d0[k] = f2(xk.re.x, xk.im.x);
            d1[k] = f2(xk.re.y, xk.im.y);
            if (2 * k != N) {
                const CV xn = csub(ev, t);
                d0[N - k] = f2(xn.re.x, -xn.im.x);
                d1[N - k] = f2(xn.re.y, -xn.im.y);
            }
        }
    }
    __syncwarp();  // the slots are read before the next pair's exchange writes them
}

template <int N>
__global__ void __launch_bounds__(XWarp<N>::NT, 2)
k_x_warp_fwd(const PtrArray rho, float2 *__restrict__ out, const float2 *__restrict__ tw, int npairs, int Px) {
    using X = XWarp<N>;
    constexpr int H = X::H;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *T = reinterpret_cast<float2 *>(smraw + X::OFF_T);
    float2 *T2 = reinterpret_cast<float2 *>(smraw + X::OFF_T2);
    xw_tables<N>(T, T2, tw);
    __syncthreads();
    griddep_wait();  // the previous pass has finished: its outputs are readable
    const int lane = threadIdx.x & 31, hw = threadIdx.x >> 4, qq = lane & 15;
    const uint32_t xs = smem_addr(smraw + X::OFF_X) + 4096 * hw;
    const int stride = gridDim.x * (X::NT / 16);
    int i = blockIdx.x * (X::NT / 16) + hw;
    float2 f[2 * H], g[2 * H];
    if (i < npairs) xw_load<N>(rho, i, qq, f);
    for (; i < npairs; i += stride) {
        if (i + stride >= npairs) griddep_launch();  // this half-warp's last row pair
#pragma unroll
        for (int r = 0; r < 2 * H; ++r) g[r] = f[r];
        if (i + stride < npairs) xw_load<N>(rho, i + stride, qq, f);
        float2 *d0 = out + (long long)(2 * i) * Px;
        xw_fwd_pair<N>(g, xs, qq, T, T2, d0, d0 + Px);
    }
}

// Load of a value of the x passes' input rows: through the read-only path (ldg) for rows no
// kernel writes while they are read, else through L2 only (rows rewritten during the kernel).
template <bool CG> __device__ __forceinline__ float2 xw_ld(const float2 *p) { return CG ? __ldcg(p) : __ldg(p); }

// Inverse x transform of one row pair by a half-warp: the N+1 bins of rows s0, s1 to the
// N/2 sample pairs of both rows (lane qq writes pairs qq + 16 r of row 0 at d[16 r] and of
// row 1 at d[N/2 + 16 r]).  The bins are loaded in batches of NB per lane and row.
template <int N, bool CG, int NB = 5>
__device__ __forceinline__ void xw_inv_pair(const float2 *s0, const float2 *s1, uint32_t xs, int qq, const float2 *T,
                                            const float2 *T2, float2 *d) {
    using M = ZwMap<N / 16>;
    constexpr int E1 = N / 16, H = E1 / 2;
    const uint32_t aw = xs + 16 * qq, ar = xs + 256 * qq + 16 * (qq & 7);
    const bool rd = qq < E1;  // lane qq gathers k1 = qq after the exchange
    CV v[16];
    // (Y_k, Y_{N-k}) -> (C_k, C_{N-k}) for k = qq + E1 k2 <= N/2, in batches of loads.
#pragma unroll
    for (int k20 = 0; k20 < 9; k20 += NB) {
        float2 yk0[NB], yk1[NB], yn0[NB], yn1[NB];
#pragma unroll
        for (int d2 = 0; d2 < NB; ++d2) {
            const int k2 = k20 + d2, k = qq + E1 * k2;
            if (k2 > 8 || !rd || k > N / 2) continue;
            yk0[d2] = xw_ld<CG>(s0 + k);
            yk1[d2] = xw_ld<CG>(s1 + k);
            yn0[d2] = xw_ld<CG>(s0 + (N - k));
            yn1[d2] = xw_ld<CG>(s1 + (N - k));
        }
#pragma unroll
        for (int d2 = 0; d2 < NB; ++d2) {
            const int k2 = k20 + d2, k = qq + E1 * k2;
            if (k2 > 8 || !rd || k > N / 2) continue;
            if (k == 0) {
                v[0] = {f2(yk0[0].x + yn0[0].x, yk1[0].x + yn1[0].x), f2(yk0[0].x - yn0[0].x, yk1[0].x - yn1[0].x)};
            } else {
                const CV yk = {f2(yk0[d2].x, yk1[d2].x), f2(yk0[d2].y, yk1[d2].y)};
                const CV yn = {f2(yn0[d2].x, yn1[d2].x), f2(yn0[d2].y, yn1[d2].y)};
                const CV ev = {f2add(yk.re, yn.re), f2sub(yk.im, yn.im)};
                const CV od = zw_twmul<1>(CV{f2sub(yk.re, yn.re), f2add(yk.im, yn.im)}, T2[k]);
                v[k2] = add_rot<1>(ev, od);
                if (2 * k != N) zw_sts(xs + 16 * (N - k), add_rot<1>(cconj_cv(ev), cconj_cv(od)));
            }
        }
    }
    __syncwarp();
    if (rd) {
#pragma unroll
        for (int k2 = 8; k2 < 16; ++k2) {
            const int k = qq + E1 * k2;
            if (k != N / 2) v[k2] = zw_lds(xs + 16 * k);
        }
    }
    __syncwarp();
    if (rd) {
        dft<16, 1>(v);
#pragma unroll
        for (int p = 0; p < 16; ++p) zw_sts((ar ^ (16 * (p & 7))) + 16 * (p & 8), v[p]);
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < E1; ++j) {
        const int k0 = M::kappa0(j);
        v[j] = zw_lds((aw ^ (16 * (k0 & 7))) + 256 * k0);
    }
#pragma unroll
    for (int j = 0; j < E1; ++j) v[j] = zw_twmul<1>(v[j], T[M::kappa0(j) * 16 + qq]);
    zw_f1_adj<E1>(v);
#pragma unroll
    for (int r = 0; r < H; ++r) {
        d[16 * r] = f2(v[r].re.x, v[r].im.x);
        d[N / 2 + 16 * r] = f2(v[r].re.y, v[r].im.y);
    }
    __syncwarp();  // the slots are read before the next pair writes them
}

template <int N>
__global__ void __launch_bounds__(XWarp<N>::NT, 2)
k_x_warp_inv(const float2 *__restrict__ in, const PtrArray u, const float2 *__restrict__ tw, int npairs, int Px) {
    using X = XWarp<N>;
    constexpr int NN = N * N;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *T = reinterpret_cast<float2 *>(smraw + X::OFF_T);
    float2 *T2 = reinterpret_cast<float2 *>(smraw + X::OFF_T2);
    xw_tables<N>(T, T2, tw);
    __syncthreads();
    griddep_wait();  // the previous pass has finished: its outputs are readable
    const int lane = threadIdx.x & 31, hw = threadIdx.x >> 4, qq = lane & 15;
    const uint32_t xs = smem_addr(smraw + X::OFF_X) + 4096 * hw;
    const int stride = gridDim.x * (X::NT / 16);
    for (int i = blockIdx.x * (X::NT / 16) + hw; i < npairs; i += stride) {
        if (i + stride >= npairs) griddep_launch();  // this half-warp's last row pair
        const float2 *s0 = in + (long long)(2 * i) * Px;
        const int b = (2 * i) / NN;
        float2 *d = reinterpret_cast<float2 *>(const_cast<void *>(u.p[b])) + (long long)(2 * i - b * NN) * (N / 2) + qq;
        xw_inv_pair<N, false>(s0, s0 + Px, xs, qq, T, T2, d);
    }
}

}  // namespace gsp

namespace gsp {

// ---- K1 / K5, warp form at N = 512 (FP32) -------------------------------------------------
// The same row-pair scheme as k_x_warp_fwd / k_x_warp_inv with one full warp per pair of
// rows: the N = 512-point complex FFT of the (even, odd) sample pairs (256 nonzero) is the
// pruned length-512 transform of the z pass's warp form (F1..F6: lane q ends with
// C[q + 32 k2] in register k2), and the Hermitian split pairs C_k with C_{N-k} through the
// warp's 512 slots (slot k in row k, chunk g ^ (k & 7)).  The inverse combines
// (Y_k, Y_{N-k}) into (C_k, C_{N-k}) and runs the adjoint half.  The twiddle table of the
// plan is W_1024^e here.
struct XWarp2 {
    static constexpr int N = 512, NW = 8, NT = 256;
    static constexpr int OFF_XO = 0, OFF_T = 65536, OFF_T2 = OFF_T + 16 * 32 * 8;
    static constexpr int SMEM = 1024 + OFF_T2 + 257 * 8;
};

template <int N>
__global__ void __launch_bounds__(XWarp2::NT, 2)
k_x_warp2_fwd(const PtrArray rho, float2 *__restrict__ out, const float2 *__restrict__ tw, int npairs, int Px) {
    static_assert(N == XWarp2::N, "one warp per row pair: 512 = 16 x 2 x 16");
    constexpr long long NN = (long long)N * N;
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned char *base = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    unsigned char *xo = base + XWarp2::OFF_XO;
    float2 *T = reinterpret_cast<float2 *>(base + XWarp2::OFF_T);
    float2 *T2 = reinterpret_cast<float2 *>(base + XWarp2::OFF_T2);
    for (int i = threadIdx.x; i < 512; i += XWarp2::NT) T[i] = tw[2 * (i & 31) * (i >> 5)];
    for (int i = threadIdx.x; i <= N / 2; i += XWarp2::NT) T2[i] = tw[i];
    __syncthreads();
    griddep_wait();  // the previous pass has finished: its outputs are readable
    const int g = threadIdx.x >> 5, q = threadIdx.x & 31;
    const ZwLane zl = zw_lane<16>(tw, smem_addr(xo), g, q, 2);
    const int stride = gridDim.x * XWarp2::NW;
    auto load = [&](long long i, float2 *f) {
        const int b = (int)((2 * i) / NN);
        const float2 *s = reinterpret_cast<const float2 *>(rho.p[b]) + (2 * i - b * NN) * (N / 2) + q;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            f[2 * r] = __ldg(s + 32 * r);
            f[2 * r + 1] = __ldg(s + N / 2 + 32 * r);
        }
    };
    long long i = (long long)blockIdx.x * XWarp2::NW + g;
    float2 f[16];
    if (i < npairs) load(i, f);
    for (; i < npairs; i += stride) {
        CV v[16];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            v[r] = {f2(f[2 * r].x, f[2 * r + 1].x), f2(f[2 * r].y, f[2 * r + 1].y)};
            if (r & 1) v[r] = zw_sign(v[r], zl.sg);
        }
        if (i + stride < npairs) load(i + stride, f);
        zw_front<16>(v, zl, T);
        zw_exchange<16>(v, zl);
        dft<16, -1>(v);  // v[k2] = C[q + 32 k2]
        __syncwarp();
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) zw_sts(smem_addr(xo) + zw_sw128(q + 32 * k2, g), v[k2]);
        __syncwarp();
        float2 *d0 = out + (2 * i) * Px, *d1 = d0 + Px;
        const float2 h = f2(0.5f, 0.5f);
#pragma unroll
        for (int k2 = 0; k2 < 9; ++k2) {
            const int k = q + 32 * k2;
            if (k > N / 2) continue;
            const CV ck = v[k2], cn = zw_lds(smem_addr(xo) + zw_sw128((N - k) & (N - 1), g));
            const CV ev = {f2mul(h, f2add(ck.re, cn.re)), f2mul(h, f2sub(ck.im, cn.im))};
            const CV od = {f2mul(h, f2add(ck.im, cn.im)), f2mul(h, f2sub(cn.re, ck.re))};
            if (k == 0) {
                const float2 x0 = f2add(ev.re, od.re), xn = f2sub(ev.re, od.re);
                d0[0] = f2(x0.x, 0.f);
                d1[0] = f2(x0.y, 0.f);
                d0[N] = f2(xn.x, 0.f);
                d1[N] = f2(xn.y, 0.f);
            } else {
                const CV t = zw_twmul<-1>(od, T2[k]);
                const CV xk = cadd(ev, t);
                d0[k] = f2(xk.re.x, xk.im.x);
                d1[k] = f2(xk.re.y, xk.im.y);
                if (2 * k != N) {
                    const CV xn = csub(ev, t);
                    d0[N - k] = f2(xn.re.x, -xn.im.x);
                    d1[N - k] = f2(xn.re.y, -xn.im.y);
                }
            }
        }
        __syncwarp();  // the slots are read before the next pair's exchange writes them
    }
}

template <int N>
__global__ void __launch_bounds__(XWarp2::NT, 2)
k_x_warp2_inv(const float2 *__restrict__ in, const PtrArray u, const float2 *__restrict__ tw, int npairs, int Px) {
    static_assert(N == XWarp2::N, "one warp per row pair: 512 = 16 x 2 x 16");
    constexpr long long NN = (long long)N * N;
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned char *base = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    unsigned char *xo = base + XWarp2::OFF_XO;
    float2 *T = reinterpret_cast<float2 *>(base + XWarp2::OFF_T);
    float2 *T2 = reinterpret_cast<float2 *>(base + XWarp2::OFF_T2);
    for (int i = threadIdx.x; i < 512; i += XWarp2::NT) T[i] = tw[2 * (i & 31) * (i >> 5)];
    for (int i = threadIdx.x; i <= N / 2; i += XWarp2::NT) T2[i] = tw[i];
    __syncthreads();
    griddep_wait();  // the previous pass has finished: its outputs are readable
    const int g = threadIdx.x >> 5, q = threadIdx.x & 31;
    const ZwLane zl = zw_lane<16>(tw, smem_addr(xo), g, q, 2);
    const int stride = gridDim.x * XWarp2::NW;
    for (long long i = (long long)blockIdx.x * XWarp2::NW + g; i < npairs; i += stride) {
        const float2 *s0 = in + (2 * i) * Px, *s1 = s0 + Px;
        float2 yk0[9], yk1[9], yn0[9], yn1[9];
#pragma unroll
        for (int k2 = 0; k2 < 9; ++k2) {
            const int k = q + 32 * k2;
            if (k > N / 2) continue;
            yk0[k2] = __ldg(s0 + k);
            yk1[k2] = __ldg(s1 + k);
            yn0[k2] = __ldg(s0 + (N - k));
            yn1[k2] = __ldg(s1 + (N - k));
        }
        CV v[16];
#pragma unroll
        for (int k2 = 0; k2 < 9; ++k2) {
            const int k = q + 32 * k2;
            if (k > N / 2) continue;
            if (k == 0) {
                v[0] = {f2(yk0[0].x + yn0[0].x, yk1[0].x + yn1[0].x), f2(yk0[0].x - yn0[0].x, yk1[0].x - yn1[0].x)};
            } else {
                const CV yk = {f2(yk0[k2].x, yk1[k2].x), f2(yk0[k2].y, yk1[k2].y)};
                const CV yn = {f2(yn0[k2].x, yn1[k2].x), f2(yn0[k2].y, yn1[k2].y)};
                const CV ev = {f2add(yk.re, yn.re), f2sub(yk.im, yn.im)};
                const CV od = zw_twmul<1>(CV{f2sub(yk.re, yn.re), f2add(yk.im, yn.im)}, T2[k]);
                v[k2] = add_rot<1>(ev, od);
                if (2 * k != N) zw_sts(smem_addr(xo) + zw_sw128(N - k, g), add_rot<1>(cconj_cv(ev), cconj_cv(od)));
            }
        }
        __syncwarp();
#pragma unroll
        for (int k2 = 8; k2 < 16; ++k2) {
            const int k = q + 32 * k2;
            if (k != N / 2) v[k2] = zw_lds(smem_addr(xo) + zw_sw128(k, g));
        }
        __syncwarp();
        dft<16, 1>(v);
        zw_exchange_adj<16>(v, zl);
        zw_back<16>(v, zl, T);
        const int b = (int)((2 * i) / NN);
        float2 *d = reinterpret_cast<float2 *>(const_cast<void *>(u.p[b])) + (2 * i - b * NN) * (N / 2) + q;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            CV x = v[r];
            if (r & 1) x = zw_sign(x, zl.sg);
            d[32 * r] = f2(x.re.x, x.im.x);
            d[N / 2 + 32 * r] = f2(x.re.y, x.im.y);
        }
        __syncwarp();  // the slots are read before the next pair writes them
    }
}

}  // namespace gsp

namespace gsp {

// ---- K3, warp form at N = 512 (FP32) -------------------------------------------------------
// The fused z pass of k_z_warp for L = 2N = 1024, where a packed column pair would need 32
// CV values (128 registers) per lane: one warp per column, L = 32 x 32.  Lane q holds
// x[q + 32 r] of its column (r < 16 nonzero) in register r.  The steps below are those of
// the y passes (k_y_w512, on unpacked complex values CF); k_z_w512 runs the same steps on
// packed pairs of one column's values (its own description):
//   F1  A_q[k1] = sum_{r<16} x[q + 32 r] W_32^{r k1}   pruned 32-point DFT in registers
//       (two 16-point DFTs of the inputs and of the inputs times W_32^r): register j holds
//       k1 = kappa(j) = 2j (j < 16) or 2(j - 16) + 1
//   F2  B_q[k1] = A_q[k1] W_1024^{q k1}                (shared table T[k1][q])
//   F3  transpose through the warp's own 8 KB of shared memory: lane l gathers B_q[l], q < 32,
//       slot (q, k1) at byte 256 k1 + 8 (q ^ (k1 & 15)) (both directions conflict free)
//   F4  X[l + 32 k2] = sum_q B_q[l] W_32^{q k2}        32-point DFT in registers
// then the product with G(kx, |ky|, |kz|) at kz = l + 32 k2 (folded to kz <= N), and the
// adjoint of each step in reverse order, which returns z = q + 32 r to the lanes and
// registers the inputs came from; rows r < 16 are kept (Sec. 2: the convolution with the
// G-tensor on the zero-padded grid and the crop).
//
// A CTA of 8 warps owns a tile of 8 consecutive columns kx at one ky.  Shared memory:
//   B   32 KB: the input tile (512 z-rows x 64 B, two TMA boxes of 256 rows, 64-byte
//       swizzle), then the tile's symbol lines (three boxes of 256 kz x 8 kx: the octant
//       table is symmetric in (kx, ky, kz), so with kz as its innermost index each column's
//       kz values lie contiguous), then the next tile's input;
//   XO  64 KB: the warps' 8 KB exchange regions; the first 32 KB is also the output tile
//       in the TMA store's 64-byte swizzle, written after a block barrier that ends every
//       warp's exchange reads;
//   T   8 KB: W_1024^{q k1} as T[k1][q] (k_z_w512: the pairs for k1 = 2m, 2m + 1 as one float4).
struct ZW512 {
    static constexpr int N = 512, L = 1024, TC = 8, NW = 8, NT = 256;
    static constexpr int IN_BYTES = N * TC * 8;                  // two 16 KB boxes
    static constexpr int SYM_BOX = 256, SYM_NB = 3;              // kz boxes 0, 256, 512
    static constexpr int SYM_BYTES = SYM_NB * SYM_BOX * TC * 4;  // 24 KB
    static constexpr int OFF_B = 0, OFF_XO = 32768, OFF_T = OFF_XO + 65536, OFF_BAR = OFF_T + 8192;
    static constexpr int SMEM = 1024 + OFF_BAR + 64;
    static_assert(IN_BYTES == 32768 && SYM_BYTES <= 32768, "input and symbol share B");
};

// exp(-2 pi i r / 32) for r < 16.
__host__ __device__ constexpr float w32c(int r) {
    constexpr float c1 = 0.98078528040323044913f, c2 = 0.92387953251128675613f, c3 = 0.83146961230254523708f;
    constexpr float s1 = 0.19509032201612826785f, s2 = 0.38268343236508977173f, s3 = 0.55557023301960222474f;
    constexpr float c4 = 0.70710678118654752440f;
    return r == 0 ? 1.f : r == 1 ? c1 : r == 2 ? c2 : r == 3 ? c3 : r == 4 ? c4 : r == 5 ? s3 : r == 6 ? s2
         : r == 7 ? s1 : r == 8 ? 0.f : r == 9 ? -s1 : r == 10 ? -s2 : r == 11 ? -s3 : r == 12 ? -c4
         : r == 13 ? -c3 : r == 14 ? -c2 : -c1;
}
__host__ __device__ constexpr float w32s(int r) {
    constexpr float c1 = 0.98078528040323044913f, c2 = 0.92387953251128675613f, c3 = 0.83146961230254523708f;
    constexpr float s1 = 0.19509032201612826785f, s2 = 0.38268343236508977173f, s3 = 0.55557023301960222474f;
    constexpr float c4 = 0.70710678118654752440f;
    return r == 0 ? 0.f : r == 1 ? -s1 : r == 2 ? -s2 : r == 3 ? -s3 : r == 4 ? -c4 : r == 5 ? -c3 : r == 6 ? -c2
         : r == 7 ? -c1 : r == 8 ? -1.f : r == 9 ? -c1 : r == 10 ? -c2 : r == 11 ? -c3 : r == 12 ? -c4
         : r == 13 ? -s3 : r == 14 ? -s2 : -s1;
}

// 32-point DFT of v in natural order, X_k = sum_n v_n exp(D 2 pi i n k / 32).
template <int D> __device__ __forceinline__ void dft32(CF *v) {
    CF e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        e[i] = v[2 * i];
        o[i] = v[2 * i + 1];
    }
    dft<16, D>(e);
    dft<16, D>(o);
    float cs[16], sn[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) cs[k] = w32c(k), sn[k] = w32s(k);
    combine2<D, 16>(e, o, v, cs, sn);
}
// F1: v[0..15] inputs (v[16..31] ignored) -> v[m] = A[2m], v[16 + m] = A[2m + 1].
__device__ __forceinline__ void w512_f1(CF *v) {
#pragma unroll
    for (int r = 0; r < 16; ++r) v[16 + r] = r == 0 ? v[0] : r == 8 ? add_rot<-1>(czero<CF>(), v[8]) : cmulk<-1>(v[r], w32c(r), w32s(r));
    dft<16, -1>(v);
    dft<16, -1>(v + 16);
}
// Adjoint of F1, outputs r < 16 in v[0..15].
__device__ __forceinline__ void w512_f1_adj(CF *v) {
    dft<16, 1>(v);
    dft<16, 1>(v + 16);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const CF o = r == 0 ? v[16] : r == 8 ? add_rot<1>(czero<CF>(), v[24]) : cmulk<1>(v[16 + r], w32c(r), w32s(r));
        v[r] = cadd(v[r], o);
    }
}
__host__ __device__ constexpr int w512_kappa(int j) { return j < 16 ? 2 * j : 2 * (j - 16) + 1; }

// Byte offset of row z, column c (8 bytes) in a tile of 64-byte rows with the 64-byte swizzle.
__device__ __forceinline__ int sw64(int z, int c) { return z * 64 + ((((c >> 1) ^ (z >> 1)) & 3) << 4) + ((c & 1) << 3); }

__device__ __forceinline__ void sts2(uint32_t a, CF x) {
    if (!dbg_smem_ok(a, 8)) return;
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x.re), "f"(x.im) : "memory");
}
__device__ __forceinline__ CF lds2(uint32_t a) {
    if (!dbg_smem_ok(a, 8)) return czero<CF>();
    float2 f;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(f.x), "=f"(f.y) : "r"(a) : "memory");
    return {f.x, f.y};
}

// Shared 32-bit access by address.
__device__ __forceinline__ void sts1(uint32_t a, float x) {
    if (!dbg_smem_ok(a, 4)) return;
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(x) : "memory");
}
__device__ __forceinline__ float lds1(uint32_t a) {
    if (!dbg_smem_ok(a, 4)) return 0.f;
    float f;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(f) : "r"(a) : "memory");
    return f;
}
__device__ __forceinline__ void sts2f(uint32_t a, float2 x) {
    if (!dbg_smem_ok(a, 8)) return;
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x.x), "f"(x.y) : "memory");
}
__device__ __forceinline__ float2 lds2f(uint32_t a) {
    if (!dbg_smem_ok(a, 8)) return make_float2(0.f, 0.f);
    float2 f;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(f.x), "=f"(f.y) : "r"(a) : "memory");
    return f;
}
// The two halves of a CV pair as scalar complex values.
__device__ __forceinline__ CF cv_lo(CV a) { return {a.re.x, a.im.x}; }
__device__ __forceinline__ CF cv_hi(CV a) { return {a.re.y, a.im.y}; }
__device__ __forceinline__ CV cv_pair(CF a, CF b) { return {f2(a.re, b.re), f2(a.im, b.im)}; }
// exp(D 2 pi i r / 32) times x, r < 16 (compile-time r after unrolling).
template <int D> __device__ __forceinline__ CF w32mul(CF x, int r) {
    return r == 0 ? x : r == 8 ? (D < 0 ? CF{x.im, -x.re} : CF{-x.im, x.re}) : cmulk<D>(x, w32c(r), w32s(r));
}

// Tile t = (tx, ky, b): tx the 8-column block, consecutive tiles take ky and its mirror
// 2N - ky (same symbol lines), b the density.  With TAIL the forward spectrum's shell and
// total energies are added to tail[2 b], tail[2 b + 1] (as in k_z_warp).
//
// Each step runs on packed pairs of the lane's 32 values (CV u[16]), two DFT lanes of one
// column per packed instruction:
//   F1  u[r] = (x_r, x_r W_32^r), one packed 16-point DFT: u[m] = (A_q[2m], A_q[2m + 1]);
//   F2  u[m] times (W_1024^{2m q}, W_1024^{(2m + 1) q}) (table T4[m][q], float4 pairs);
//   F3  the writer stores its 32 values one float at a time into a re plane and an im
//       plane (4 KB each), slot (q, k1) at byte 128 k1 + 4 (q ^ 2 (k1 & 15)); reader lane l
//       loads the pair of slots (2i, l), (2i + 1, l), adjacent in each plane, so that
//       u[i] = (B_{2i}[l], B_{2i+1}[l]) (both directions conflict free);
//   F4  a packed 16-point DFT gives (E[k], O[k]), the DFTs of the even and odd q; then
//       u[k] = (X[l + 32 k], X[l + 32 (k + 16)]) = (E + W_32^k O, E - W_32^k O).
// The symbol product scales each pair by (G at kz = l + 32 k, G at 512 - l - 32 k), and the
// adjoint steps run in reverse order.
template <bool TAIL>
__global__ void __launch_bounds__(ZW512::NT, 2)
k_z_w512(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tsym,
         const __grid_constant__ CUtensorMap tout, const float2 *__restrict__ tw, int ntx, int ntiles,
         int ncols, int *__restrict__ status, double *__restrict__ tail) {
    using Z = ZW512;
    constexpr int L = Z::L, N = Z::N, NW = Z::NW;
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned char *base = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    unsigned char *Bb = base + Z::OFF_B;
    unsigned char *xo = base + Z::OFF_XO;
    float4 *T4 = reinterpret_cast<float4 *>(base + Z::OFF_T);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + Z::OFF_BAR);  // input, symbol, XO free
    int *cnt = reinterpret_cast<int *>(bar + 3);                       // input, symbol, output
    const int g = threadIdx.x >> 5, q = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        mbar_init(bar + 2, 1);
        cnt[0] = cnt[1] = cnt[2] = 0;
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < 512; i += Z::NT) {
        const int m = i >> 5, qq = i & 31;
        const float2 w0 = tw[2 * m * qq], w1 = tw[(2 * m + 1) * qq];
        T4[i] = make_float4(w0.x, w1.x, w0.y, w1.y);
    }
    __syncthreads();
    griddep_wait();  // the previous pass has finished: its outputs are readable

    auto ky_of = [&](int by) { return (by & 1) ? L - ((by + 1) >> 1) : (by >> 1); };
    auto issue_in = [&](int t) {
        const int tx = t % ntx, ky = ky_of((t / ntx) % L), b = t / (ntx * L);
        mbar_arrive_expect_tx(bar, Z::IN_BYTES);
        tma_load_3d(Bb, &tin, bar, tx * Z::TC, ky, b * N);
        tma_load_3d(Bb + Z::IN_BYTES / 2, &tin, bar, tx * Z::TC, ky, b * N + N / 2);
    };
    auto issue_sym = [&](int t) {
        const int tx = t % ntx, ky = ky_of((t / ntx) % L);
        const int kya = ky <= N ? ky : L - ky;
        mbar_arrive_expect_tx(bar + 1, Z::SYM_BYTES);
#pragma unroll
        for (int c = 0; c < Z::SYM_NB; ++c)
            tma_load_3d(Bb + c * Z::SYM_BOX * Z::TC * 4, &tsym, bar + 1, c * Z::SYM_BOX, kya, tx * Z::TC);
    };
    // Arrival of this warp on counter c; true on the lane-0 thread of the tile's last warp.
    auto last_arrival = [&](int c) {
        __syncwarp();
        bool last = false;
        if (q == 0) {
            __threadfence_block();
            last = atomicAdd(cnt + c, 1) % NW == NW - 1;
            if (last) {
                __threadfence_block();
                fence_proxy_async();
            }
        }
        return last;
    };
    if (threadIdx.x == 0) {
        mbar_arrive(bar + 2);  // XO starts free
        if ((int)blockIdx.x < ntiles) issue_in(blockIdx.x);
    }

    const uint32_t xw = smem_addr(xo) + 8192 * g;     // this warp's exchange region (re plane, im plane)
    const uint32_t aw = xw + 4 * q;                    // writer (lane q): slot (q, k1) at (aw ^ 8 (k1 & 15)) + 128 k1
    const uint32_t ar = xw + 128 * q + 8 * (q & 15);   // reader (lane l = q): pair i at ar ^ 8 i
    // Symbol value at kz <= N for this lane's column.
    auto sym_at = [&](int kz) {
        return sm_ld(reinterpret_cast<const float *>(Bb + (kz >> 8) * (Z::SYM_BOX * Z::TC * 4) + 1024 * g + 4 * (kz & 255)));
    };
    bool stored = false;
    uint32_t ph = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ph ^= 1) {
        const int tx = t % ntx, ky = ky_of((t / ntx) % L), bb = t / (ntx * L);
        const int kya = ky <= N ? ky : L - ky;
        const int col = tx * Z::TC + g;
        const bool valid = col < ncols;
        CV u[16];
        // A wait that gives up marks the thread; the block leaves together at its barrier
        // below (no thread may return while others still wait there).
        bool bad = !mbar_wait(bar, ph, status);
        if (valid && !bad) {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const float2 f = sm_ld(reinterpret_cast<const float2 *>(Bb + sw64(q + 32 * r, g)));
                const CF x = {f.x, f.y};
                u[r] = cv_pair(x, w32mul<-1>(x, r));
            }
        }
        if (last_arrival(0)) issue_sym(t);
        if (valid) {
            dft<16, -1>(u);  // u[m] = (A[2m], A[2m + 1])
#pragma unroll
            for (int m = 0; m < 16; ++m) u[m] = twmul<-1>(u[m], sm_ld(T4 + m * 32 + q));
        }
        if (!bad) bad = !mbar_wait(bar + 2, ph, status);  // the previous tile's store has read XO
        if (valid) {
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                const uint32_t sa = (aw ^ (8 * ((2 * m) & 15))) + 128 * (2 * m);
                const uint32_t sb = (aw ^ (8 * ((2 * m + 1) & 15))) + 128 * (2 * m + 1);
                sts1(sa, u[m].re.x);
                sts1(sa + 4096, u[m].im.x);
                sts1(sb, u[m].re.y);
                sts1(sb + 4096, u[m].im.y);
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 16; ++i) u[i] = {lds2f(ar ^ (8 * i)), lds2f((ar ^ (8 * i)) + 4096)};
            dft<16, -1>(u);  // u[k] = (E[k], O[k])
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const CF e = cv_lo(u[k]), o = w32mul<-1>(cv_hi(u[k]), k);
                u[k] = cv_pair(cadd(e, o), csub(e, o));  // (X[q + 32 k], X[q + 32 k + 512])
            }
        }
        if constexpr (TAIL) {
            constexpr int SHELL = N - N / 8;
            float eshell = 0.f, etot = 0.f;
            if (valid) {
                const float w0 = (col == 0 || col == N) ? 1.f : 2.f;
                const bool cs = kya >= SHELL || col >= SHELL;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int kz1 = q + 32 * k, kz2 = N - q - 32 * k;  // the second folded
                    const float2 en = cenergy(u[k]);
                    etot += w0 * (en.x + en.y);
                    if (cs || kz1 >= SHELL) eshell += w0 * en.x;
                    if (cs || kz2 >= SHELL) eshell += w0 * en.y;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                eshell += __shfl_xor_sync(0xffffffffu, eshell, o);
                etot += __shfl_xor_sync(0xffffffffu, etot, o);
            }
            if (valid && q == 0) {
                atomicAdd(tail + 2 * bb, (double)eshell);
                atomicAdd(tail + 2 * bb + 1, (double)etot);
            }
        }
        if (!bad) bad = !mbar_wait(bar + 1, ph, status);
        if (valid) {
#pragma unroll
            for (int k = 0; k < 16; ++k) u[k] = cscale2(u[k], f2(sym_at(q + 32 * k), sym_at(N - q - 32 * k)));
        }
        if (last_arrival(1) && t + (int)gridDim.x < ntiles) issue_in(t + gridDim.x);
        if (valid) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {  // adjoint of F4's last step: (a + b, conj(W_32^k) (a - b))
                const CF a = cv_lo(u[k]), b = cv_hi(u[k]);
                u[k] = cv_pair(cadd(a, b), w32mul<1>(csub(a, b), k));
            }
            dft<16, 1>(u);  // u[i] = (B_{2i}[q], B_{2i+1}[q]) of the adjoint
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                sts2f(ar ^ (8 * i), u[i].re);
                sts2f((ar ^ (8 * i)) + 4096, u[i].im);
            }
            __syncwarp();
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                const uint32_t sa = (aw ^ (8 * ((2 * m) & 15))) + 128 * (2 * m);
                const uint32_t sb = (aw ^ (8 * ((2 * m + 1) & 15))) + 128 * (2 * m + 1);
                u[m] = {f2(lds1(sa), lds1(sb)), f2(lds1(sa + 4096), lds1(sb + 4096))};
            }
#pragma unroll
            for (int m = 0; m < 16; ++m) u[m] = twmul<1>(u[m], sm_ld(T4 + m * 32 + q));
            dft<16, 1>(u);  // u[r] = (a_r, b_r)
        }
        // Every warp's exchange reads are done: XO takes the output tile.
        if (__syncthreads_or(bad)) break;
        if (valid) {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const CF z = cadd(cv_lo(u[r]), w32mul<1>(cv_hi(u[r]), r));  // adjoint of F1, row q + 32 r
                sm_st(reinterpret_cast<float2 *>(xo + sw64(q + 32 * r, g)), make_float2(z.re, z.im));
            }
        }
        fence_proxy_async();
        if (last_arrival(2)) {
            tma_store_3d(&tout, xo, tx * Z::TC, ky, bb * N);
            tma_store_3d(&tout, xo + Z::IN_BYTES / 2, tx * Z::TC, ky, bb * N + N / 2);
            bulk_commit();
            bulk_wait_read0();
            stored = true;
            mbar_arrive(bar + 2);
        }
    }
    if (stored) bulk_wait0();
}

}  // namespace gsp

namespace gsp {

// ---- K2 / K4, warp form at N = 512 (FP32) --------------------------------------------------
// The y passes with the transform halves of k_z_w512: the forward half (F1..F4) alone for
// the y forward (N input rows, all 2N rows kept) and the adjoint half alone for the y
// inverse (2N input rows, rows y < N kept), one warp per column, a tile of 8 columns kx of
// one plane.  Shared memory (104 KB, two CTAs per SM):
//   y forward: B holds the 512 input rows (prefetched for the next tile as soon as every
//     warp has read them); XO holds the exchange regions, then the 1024-row output tile,
//     written after a block barrier and freed for the next tile once the store has read it;
//   y inverse: the 1024 input rows arrive split, rows < 512 in B and rows >= 512 in the
//     upper half of XO; a block barrier after the input reads frees B for the next tile's
//     first half and the upper exchange regions; a second one after the exchange frees the
//     upper half of XO for the next tile's second half while the outputs (rows < 512) go to
//     the lower half.
template <bool FWD>
__global__ void __launch_bounds__(ZW512::NT, 2)
k_y_w512(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
         const float2 *__restrict__ tw, int ntx, int ntiles, int ncols, int *__restrict__ status, int z0) {
    using Z = ZW512;
    constexpr int NW = Z::NW, HALF = 16384;  // one 256-row box of 64-byte rows
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned char *base = smraw + ((1024 - (smem_addr(smraw) & 1023)) & 1023);
    unsigned char *Bb = base + Z::OFF_B;
    unsigned char *xo = base + Z::OFF_XO;
    float2 *T = reinterpret_cast<float2 *>(base + Z::OFF_T);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + Z::OFF_BAR);  // input, XO (lower half) free
    int *cnt = reinterpret_cast<int *>(bar + 2);                       // input read, outputs written
    const int g = threadIdx.x >> 5, q = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        cnt[0] = cnt[1] = 0;
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < 1024; i += Z::NT) T[i] = tw[(i & 31) * (i >> 5)];
    __syncthreads();
    griddep_wait();  // the previous pass has finished: its outputs are readable

    // Loads of tile t: forward, rows 0..511 into B; inverse, rows 0..511 into B (first)
    // and rows 512..1023 into the upper half of XO (second), on one barrier phase.
    auto issue_first = [&](int t) {
        const int tx = t % ntx, zz = z0 + t / ntx;
        mbar_arrive_expect_tx(bar, FWD ? 2 * HALF : 4 * HALF);
        tma_load_3d(Bb, &tin, bar, tx * Z::TC, 0, zz);
        tma_load_3d(Bb + HALF, &tin, bar, tx * Z::TC, 256, zz);
    };
    auto issue_second = [&](int t) {
        const int tx = t % ntx, zz = z0 + t / ntx;
        tma_load_3d(xo + 2 * HALF, &tin, bar, tx * Z::TC, 512, zz);
        tma_load_3d(xo + 3 * HALF, &tin, bar, tx * Z::TC, 768, zz);
    };
    auto last_arrival = [&](int c) {
        __syncwarp();
        bool last = false;
        if (q == 0) {
            __threadfence_block();
            last = atomicAdd(cnt + c, 1) % NW == NW - 1;
            if (last) {
                __threadfence_block();
                fence_proxy_async();
            }
        }
        return last;
    };
    if (threadIdx.x == 0) {
        mbar_arrive(bar + 1);  // XO starts free
        if ((int)blockIdx.x < ntiles) {
            issue_first(blockIdx.x);
            if (!FWD) issue_second(blockIdx.x);
        }
    }
    const uint32_t xw = smem_addr(xo) + 8192 * g;
    const uint32_t aw = xw + 8 * q;
    const uint32_t ar = xw + 256 * q + 8 * (q & 15);
    bool stored = false;
    uint32_t ph = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ph ^= 1) {
        const int tx = t % ntx, zz = z0 + t / ntx;
        const bool valid = tx * Z::TC + g < ncols;
        const bool more = t + (int)gridDim.x < ntiles;
        CF v[32];
        bool bad = !mbar_wait(bar, ph, status);
        if constexpr (FWD) {
            if (valid && !bad) {
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const float2 f = sm_ld(reinterpret_cast<const float2 *>(Bb + sw64(q + 32 * r, g)));
                    v[r] = {f.x, f.y};
                }
            }
            if (last_arrival(0) && more) issue_first(t + gridDim.x);
            if (valid) {
                w512_f1(v);
#pragma unroll
                for (int j = 1; j < 32; ++j) v[j] = twmul<-1>(v[j], T[w512_kappa(j) * 32 + q]);
            }
            if (!bad) bad = !mbar_wait(bar + 1, ph, status);  // the previous tile's store has read XO
            if (valid) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int k1 = w512_kappa(j);
                    sts2((aw ^ (8 * (k1 & 15))) + 256 * k1, v[j]);
                }
                __syncwarp();
#pragma unroll
                for (int p = 0; p < 32; ++p) v[p] = lds2(ar ^ (8 * p));
                dft32<-1>(v);  // v[k2] = X[q + 32 k2]
            }
            if (__syncthreads_or(bad)) break;  // every warp's exchange reads are done
            if (valid) {
#pragma unroll
                for (int k2 = 0; k2 < 32; ++k2)
                    *reinterpret_cast<float2 *>(xo + sw64(q + 32 * k2, g)) = make_float2(v[k2].re, v[k2].im);
            }
            fence_proxy_async();
            if (last_arrival(1)) {
#pragma unroll
                for (int c = 0; c < 4; ++c) tma_store_3d(&tout, xo + c * HALF, tx * Z::TC, 256 * c, zz);
                bulk_commit();
                bulk_wait_read0();
                stored = true;
                mbar_arrive(bar + 1);
            }
        } else {
            if (valid && !bad) {
#pragma unroll
                for (int k2 = 0; k2 < 32; ++k2) {
                    const int row = q + 32 * k2;
                    const unsigned char *src = k2 < 16 ? Bb + sw64(row, g) : xo + 2 * HALF + sw64(row - 512, g);
                    const float2 f = *reinterpret_cast<const float2 *>(src);
                    v[k2] = {f.x, f.y};
                }
            }
            if (__syncthreads_or(bad)) break;  // every warp has read its input rows
            if (threadIdx.x == 0 && more) {
                fence_proxy_async();
                issue_first(t + gridDim.x);  // B is free
            }
            if (valid) dft32<1>(v);  // v[p] = B_p[q]
            if (!bad) bad = !mbar_wait(bar + 1, ph, status);  // the previous tile's store has read XO
            if (valid) {
#pragma unroll
                for (int p = 0; p < 32; ++p) sts2(ar ^ (8 * p), v[p]);
                __syncwarp();
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int k1 = w512_kappa(j);
                    v[j] = lds2((aw ^ (8 * (k1 & 15))) + 256 * k1);
                }
#pragma unroll
                for (int j = 1; j < 32; ++j) v[j] = twmul<1>(v[j], T[w512_kappa(j) * 32 + q]);
                w512_f1_adj(v);
            }
            if (__syncthreads_or(bad)) break;  // every warp's exchange reads are done
            if (threadIdx.x == 0 && more) {
                fence_proxy_async();
                issue_second(t + gridDim.x);  // the upper half of XO is free
            }
            if (valid) {
#pragma unroll
                for (int r = 0; r < 16; ++r)
                    *reinterpret_cast<float2 *>(xo + sw64(q + 32 * r, g)) = make_float2(v[r].re, v[r].im);
            }
            fence_proxy_async();
            if (last_arrival(1)) {
                tma_store_3d(&tout, xo, tx * Z::TC, 0, zz);
                tma_store_3d(&tout, xo + HALF, tx * Z::TC, 256, zz);
                bulk_commit();
                bulk_wait_read0();
                stored = true;
                mbar_arrive(bar + 1);
            }
        }
    }
    if (stored) bulk_wait0();
}

}  // namespace gsp
