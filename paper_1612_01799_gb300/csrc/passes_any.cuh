// Runtime-length forms of the five passes: any even N with N 5-smooth (4 <= N <= 1024)
// and boxes with a different number of points per axis (Sec. 2 standardised form, n_q
// points on axis q).  Same operations as the compiled-length forms of passes.cuh (K1 x
// forward, K2 y forward, K3 z fused with the symbol, K4 y inverse, K5 x inverse), with
// the transform lengths, radix schedules and grid dimensions as kernel arguments, so one
// instantiation per arithmetic serves every shape.
//
// A tile of T transforms sits in shared memory, element (position, transform) at
// buf[pos * T + c]; each stage of radix R in {2, 3, 4, 5} (Stockham autosort, decimation in
// time, the ordering of fft_core.cuh) gathers R values per butterfly, applies the twiddles
// W_{Ns R}^{r (j mod Ns)} from the plan's table, runs the length-R DFT in registers and
// scatters into the other buffer of a ping-pong pair.  The zero half of the padded input
// is zero-filled in shared memory (never read from device memory) and only the kept half
// of an inverse is stored.
//
// Workspace layout (complex, the arithmetic's storage): w1 [b][z < nz][y < ny][kx < Px],
// w2 and w3 [b][z < nz][ky < 2 ny][kx < Px], Px = pitch of nx + 1; symbol
// [kz <= nz][ky <= ny][kx < Ps] (Ps = pitch of nx + 1), real, scaled by lambda^2 /
// (8 nx ny nz).
#pragma once

namespace gsp {

// ---- one runtime-length transform over a shared tile ---------------------------------------
// e / d by the reciprocal mul = floor(2^32 / d) + 1 (exact for 2 <= d <= 1024, e <= 16384).
__device__ __forceinline__ int rdiv(int e, unsigned mul) { return (int)__umulhi((unsigned)e, mul); }
__host__ __device__ inline unsigned recip32(int d) { return (unsigned)((1ull << 32) / (unsigned)d + 1); }

// Row r (< TR) of the tile starting at batch row r0: its density and its row in that density.
// rows_b >= TR, so a tile crosses at most one density boundary.
struct AnyRows {
    int b0;
    long long first;  // row of r0 within density b0
    long long left;   // rows of density b0 from r0 on
    __device__ AnyRows(long long r0, int rows_b) {
        b0 = (int)(r0 / rows_b);
        first = r0 - (long long)b0 * rows_b;
        left = rows_b - first;
    }
    __device__ int density(int r) const { return r < left ? b0 : b0 + 1; }
    __device__ long long row(int r) const { return r < left ? first + r : r - left; }
};
template <int D, typename C> __device__ __forceinline__ void dft_radix(C *x, int R) {
    switch (R) {
        case 2: dft2<D>(x[0], x[1]); break;
        case 3: dft3<D>(x[0], x[1], x[2]); break;
        case 4: dft4<D>(x[0], x[1], x[2], x[3]); break;
        default: dft5<D>(x[0], x[1], x[2], x[3], x[4]); break;
    }
}

// Transform of length s.L of each of the T = 2^logT columns of a (element (pos, c) at
// buf[pos * P + c], P >= T); b is scratch of the same size.  tw holds exp(-2 pi i e /
// (L twstride)), e < L twstride.  D = -1 forward, +1 inverse (unnormalised).  Returns the
// buffer that holds the result.  Starts and ends with a block barrier.  Butterfly j of a
// stage splits as j = jh Ns + k by the stage's reciprocal (no integer division).
template <int D, typename C, typename TW>
__device__ C *any_fft(C *a, C *b, int logT, int P, const AnySched &s, const TW *__restrict__ tw, int twstride) {
    const int L = s.L, T = 1 << logT;
    int Ns = 1;
    __syncthreads();
    for (int st = 0; st < s.nst; ++st) {
        const int R = s.r[st], LR = L / R, NsR = Ns * R;
        const unsigned mul = s.mul[st];
        const int tws = (L / NsR) * twstride;
        const int nw = LR << logT;
#pragma unroll 2
        for (int w = threadIdx.x; w < nw; w += blockDim.x) {
            const int c = w & (T - 1), j = w >> logT;
            const int jh = Ns == 1 ? j : (int)__umulhi((unsigned)j, mul);
            const int k = j - jh * Ns;
            C x[5];
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                if (r < R) {
                    x[r] = sm_ld(a + (j + r * LR) * P + c);
                    if (r > 0 && Ns > 1) x[r] = twmul<D>(x[r], __ldg(tw + r * k * tws));
                }
            }
            dft_radix<D>(x, R);
            const int base = jh * NsR + k;
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < R) sm_st(b + (base + r * Ns) * P + c, x[r]);
        }
        __syncthreads();
        C *t = a;
        a = b;
        b = t;
        Ns = NsR;
    }
    return a;
}

// ---- K1: x forward ----------------------------------------------------------------------------
// Rows of nx = s.L reals (row g of the batch: density g / rows_b, row g % rows_b of it),
// TR = 2^logTR per CTA, stored in shared memory at a[m * (TR + 1) + r] (the odd pitch keeps
// the row-wise loads and stores free of bank conflicts).  The padded length-2nx real DFT is
// the nx-point complex FFT of the (even, odd) sample pairs (pairs >= nx/2 zero) and the
// Hermitian split into the nx + 1 bins (twiddles W_{2nx}^k; the nx-point FFT reads the same
// table at stride 2).
template <typename Real>
__global__ void k_any_x_fwd(const PtrArray rho, Cx2<Real> *__restrict__ out, const AnyTw<Real> *__restrict__ tw,
                            AnySched s, int rows_b, int nrows, int Px, int logTR) {
    using C = typename Types<Real>::CS;
    using X2 = Ext2<Real>;
    extern __shared__ __align__(16) unsigned char smraw[];
    griddep_wait();
    const int n = s.L, h = n / 2, TR = 1 << logTR, P = TR + 1;
    C *a = reinterpret_cast<C *>(smraw), *b = a + n * P;
    const long long r0 = (long long)blockIdx.x * TR;
    const int nr = (int)min((long long)TR, (long long)nrows - r0);
    const unsigned rn = recip32(n), rh1 = recip32(h + 1);
    const AnyRows rows(r0, rows_b);
    for (int e = threadIdx.x; e < TR * n; e += blockDim.x) {
        const int r = rdiv(e, rn), m = e - r * n;
        C v = czero<C>();
        if (r < nr && m < h && dbg_index_ok(rows.row(r), rows_b)) {
            const X2 f = __ldg(reinterpret_cast<const X2 *>(rho.p[rows.density(r)]) + rows.row(r) * h + m);
            v = C{f.x, f.y};
        }
        sm_st(a + m * P + r, v);
    }
    const C *y = any_fft<-1>(a, b, logTR, P, s, tw, 2);
    // X_k = Ev_k + W_{2n}^k Od_k, X_{n-k} = conj(Ev_k - W_{2n}^k Od_k), with Ev, Od the DFTs
    // of the even and odd samples from C_k and conj C_{n-k}.
    for (int e = threadIdx.x; e < nr * (h + 1); e += blockDim.x) {
        const int r = rdiv(e, rh1), k = e - r * (h + 1);
        {
            Cx2<Real> *dst = out + (r0 + r) * Px;
            const C ck = sm_ld(y + k * P + r), cn = sm_ld(y + (k == 0 ? 0 : n - k) * P + r);
            const C ev = {(Real)0.5 * (ck.re + cn.re), (Real)0.5 * (ck.im - cn.im)};
            const C od = {(Real)0.5 * (ck.im + cn.im), (Real)0.5 * (cn.re - ck.re)};
            if (k == 0) {
                st_ws(dst, C{ev.re + od.re, (Real)0});
                st_ws(dst + n, C{ev.re - od.re, (Real)0});
            } else {
                const C wo = twmul<-1>(od, __ldg(tw + k));
                st_ws(dst + k, cadd(ev, wo));
                if (2 * k != n) {
                    const C d = csub(ev, wo);
                    st_ws(dst + n - k, C{d.re, -d.im});
                }
            }
        }
    }
}

// ---- K5: x inverse ----------------------------------------------------------------------------
// The nx + 1 Hermitian bins of each row -> C_k = Ev_k + i Od_k (Ev_k = Y_k + conj Y_{n-k},
// Od_k = (Y_k - conj Y_{n-k}) W_{2n}^{-k}), the inverse nx-point FFT gives y_{2m} + i y_{2m+1};
// pairs m < nx/2 are kept (the crop).  Shared layout as in the forward.
template <typename Real>
__global__ void k_any_x_inv(const Cx2<Real> *__restrict__ in, const PtrArray u, const AnyTw<Real> *__restrict__ tw,
                            AnySched s, int rows_b, int nrows, int Px, int logTR) {
    using C = typename Types<Real>::CS;
    using X2 = Ext2<Real>;
    extern __shared__ __align__(16) unsigned char smraw[];
    griddep_wait();
    const int n = s.L, h = n / 2, TR = 1 << logTR, P = TR + 1;
    C *a = reinterpret_cast<C *>(smraw), *b = a + n * P;
    const long long r0 = (long long)blockIdx.x * TR;
    const int nr = (int)min((long long)TR, (long long)nrows - r0);
    const unsigned rh1 = recip32(h + 1), rh = recip32(h);
    for (int e = threadIdx.x; e < TR * (h + 1); e += blockDim.x) {
        const int r = rdiv(e, rh1), k = e - r * (h + 1);
        {
            const Cx2<Real> *src = r < nr ? in + (r0 + r) * Px : nullptr;
            if (!src) {
                sm_st(a + k * P + r, czero<C>());
                if (k > 0 && 2 * k != n) sm_st(a + (n - k) * P + r, czero<C>());
                continue;
            }
            const C yk = ws_c(src[k]), yn = ws_c(src[n - k]);
            if (k == 0) {
                sm_st(a + r, C{yk.re + yn.re, yk.re - yn.re});
            } else {
                const C ev = {yk.re + yn.re, yk.im - yn.im};
                const C od = twmul<1>(C{yk.re - yn.re, yk.im + yn.im}, __ldg(tw + k));
                sm_st(a + k * P + r, add_rot<1>(ev, od));
                if (2 * k != n) sm_st(a + (n - k) * P + r, add_rot<1>(C{ev.re, -ev.im}, C{od.re, -od.im}));
            }
        }
    }
    const C *y = any_fft<1>(a, b, logTR, P, s, tw, 2);
    const AnyRows rows(r0, rows_b);
    for (int e = threadIdx.x; e < nr * h; e += blockDim.x) {
        const int r = rdiv(e, rh), m = e - r * h;
        if (!dbg_index_ok(rows.row(r), rows_b)) continue;
        X2 *dst = reinterpret_cast<X2 *>(const_cast<void *>(u.p[rows.density(r)])) + rows.row(r) * h;
        dst[m] = c_ext(sm_ld(y + m * P + r));
    }
}

// ---- K2 / K4: y passes --------------------------------------------------------------------------
// Tile (tx, plane): TC = 2^logTC columns from tx * TC of one plane.  FWD: input rows < L/2
// (the rest zero), all L rows stored; !FWD: all L input rows, rows < L/2 stored.
template <typename Real, bool FWD>
__global__ void k_any_col(const Cx2<Real> *__restrict__ in, Cx2<Real> *__restrict__ out,
                          const AnyTw<Real> *__restrict__ tw, AnySched s, int ncols, int ntx, int logTC,
                          long long in_row, long long in_outer, long long out_row, long long out_outer) {
    using C = typename Types<Real>::CS;
    extern __shared__ __align__(16) unsigned char smraw[];
    griddep_wait();
    const int L = s.L, TC = 1 << logTC;
    C *a = reinterpret_cast<C *>(smraw), *b = a + L * TC;
    const int tx = blockIdx.x % ntx;
    const long long plane = blockIdx.x / ntx;
    const int c0 = tx * TC;
    const int nin = FWD ? L / 2 : L, nout = FWD ? L : L / 2;
    const Cx2<Real> *src = in + plane * in_outer + c0;
    for (int e = threadIdx.x; e < L * TC; e += blockDim.x) {
        const int row = e >> logTC, c = e & (TC - 1);
        sm_st(a + e, row < nin && c0 + c < ncols ? ws_c(src[row * in_row + c]) : czero<C>());
    }
    const C *y = any_fft<FWD ? -1 : 1>(a, b, logTC, TC, s, tw, 1);
    Cx2<Real> *dst = out + plane * out_outer + c0;
    for (int e = threadIdx.x; e < nout * TC; e += blockDim.x) {
        const int row = e >> logTC, c = e & (TC - 1);
        if (c0 + c < ncols) st_ws(dst + row * out_row + c, sm_ld(y + e));
    }
}

// ---- K3: z fused ------------------------------------------------------------------------------------
// Tile (tx, ky, b): TC = 2^logTC columns kx of line ky of density b.  Forward length Lz = 2 nz
// (input z < nz), product with the symbol at (|kx|, |ky|, |kz|), inverse, z < nz stored.  With
// TAIL the forward spectrum's energy in the outer shell (|k_q| >= n_q - n_q / 8 on some axis)
// and its total energy go to tail[2 b], tail[2 b + 1].  The tiles cover the lines
// ky0 <= ky < ky0 + nky (all of them: ky0 = 0, nky = 2 ny; a rank's slab of lines in the slab
// decomposition of one solve).
template <typename Real, bool TAIL>
__global__ void k_any_z(const Cx2<Real> *__restrict__ in, Cx2<Real> *__restrict__ out, const Real *__restrict__ sym,
                        const AnyTw<Real> *__restrict__ tw, AnySched s, int nx, int ny, int ntx, int logTC, int Px,
                        int Ps, double *__restrict__ tail, int ky0, int nky) {
    using C = typename Types<Real>::CS;
    extern __shared__ __align__(16) unsigned char smraw[];
    griddep_wait();
    const int Lz = s.L, nz = Lz / 2, Ly = 2 * ny, ncols = nx + 1, TC = 1 << logTC;
    C *a = reinterpret_cast<C *>(smraw), *b = a + Lz * TC;
    const int tx = blockIdx.x % ntx;
    const int ky = ky0 + (blockIdx.x / ntx) % nky;
    const int bb = blockIdx.x / (ntx * nky);
    const int kya = ky <= ny ? ky : Ly - ky;
    const int c0 = tx * TC;
    const long long zs = (long long)Ly * Px;  // z stride of w2 and w3
    const long long base = ((long long)bb * nz * Ly + ky) * Px + c0;
    for (int e = threadIdx.x; e < Lz * TC; e += blockDim.x) {
        const int row = e >> logTC, c = e & (TC - 1);
        sm_st(a + e, row < nz && c0 + c < ncols ? ws_c(in[base + row * zs + c]) : czero<C>());
    }
    C *y = any_fft<-1>(a, b, logTC, TC, s, tw, 1);
    C *other = y == a ? b : a;
    float eshell = 0.f, etot = 0.f;
    const Real *srow = sym + (long long)kya * Ps + c0;
    const long long splane = (long long)(ny + 1) * Ps;
    for (int e = threadIdx.x; e < Lz * TC; e += blockDim.x) {
        const int row = e >> logTC, c = e & (TC - 1);
        const int kx = c0 + c;
        if (kx >= ncols) continue;
        const int kz = row <= nz ? row : Lz - row;
        if (!dbg_index_ok(kz, nz + 1) || !dbg_index_ok(kya, ny + 1)) continue;
        if constexpr (TAIL) {
            const float wgt = (kx == 0 || kx == nx) ? 1.f : 2.f;
            const float en = wgt * cenergy(sm_ld(y + e));
            etot += en;
            if (kx >= nx - nx / 8 || kya >= ny - ny / 8 || kz >= nz - nz / 8) eshell += en;
        }
        sm_st(y + e, cscale(sm_ld(y + e), srow[kz * splane + c]));
    }
    if constexpr (TAIL) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            eshell += __shfl_xor_sync(0xffffffffu, eshell, o);
            etot += __shfl_xor_sync(0xffffffffu, etot, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(tail + 2 * bb, (double)eshell);
            atomicAdd(tail + 2 * bb + 1, (double)etot);
        }
    }
    const C *z = any_fft<1>(y, other, logTC, TC, s, tw, 1);
    for (int e = threadIdx.x; e < nz * TC; e += blockDim.x) {
        const int row = e >> logTC, c = e & (TC - 1);
        if (c0 + c < ncols) st_ws(out + base + row * zs + c, sm_ld(z + e));
    }
}

}  // namespace gsp
