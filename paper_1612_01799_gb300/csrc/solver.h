// Internal interface between the C-ABI layer and the CUDA passes.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace gsp {

// Densities one grouped launch sequence can carry (kernel-parameter arrays of pointers).
constexpr int kMaxBatch = 64;

// Per-density pointers of a batch, passed to kernels by value.
struct PtrArray {
    const void *p[kMaxBatch];
};

// Radix schedule of a runtime-length transform (the runtime-length pass forms): length L,
// nst stages of radices r[0..nst) in {2, 3, 4, 5}, first to last; mul[st] the reciprocal
// floor(2^32 / Ns) + 1 of the product Ns of the earlier radices (0 for the first stage), so
// that j / Ns = umulhi(j, mul[st]) exactly for j < 4096.
constexpr int kAnyMaxStages = 16;
struct AnySched {
    int L;
    int nst;
    int r[kAnyMaxStages];
    unsigned mul[kAnyMaxStages];
};
// The schedule of length L (fives, threes, fours, then a two), or nst = 0 if L has a prime
// factor above 5.
AnySched any_sched(int L);
// N of the runtime-length forms: even, 4 <= N <= 1024, no prime factor above 5.
bool n_any(int N);

// Device side of a plan.  Workspace layout (complex values of the plan's dtype) for up to
// max_batch densities b stacked along z:
//   w1: [b][z < N][y < N][kx < Px]     after the x pass (and again after the y inverse)
//   w2: [b][z < N][ky < 2N][kx < Px]   after the y pass
//   w3: [b][z < N][ky < 2N][kx < Px]   after the fused z pass
// kx runs over the N+1 Hermitian frequencies 0..N of the real x transform; the pitch
// Px = N+1 rounded up to a multiple of 16 keeps every row 128-byte aligned.
// sym: symbol octant [kz <= N][ky <= N][kx < Ps] (Ps = N+1 rounded up to a multiple of
// 4, entries kx > N zero), real, already scaled by lambda^2 / (2N)^3.
// tw: W_{2N}^e = exp(-2 pi i e / (2N)), e < 2N, as (re, im) pairs of the dtype.
// twc: the same twiddles in the form the column passes read: (re, re, im, im) float4 for
// FP32 (two columns per thread), equal to tw for FP64.
struct DevicePlan {
    int N = 0;
    int max_batch = 1;
    int dtype = 0;  // POISSON_F32 / POISSON_F64
    // Arithmetic of an FP64 plan: 0 FP64 (the FP64 pipe), 1 double-float (pairs of FP32 on
    // the FP32 pipe; workspace, twiddles and symbol then hold (hi, lo) float pairs, and rho
    // and u stay FP64).  Always 0 for FP32 plans.
    int arith = 0;
    // Runtime-length forms (any = 1): the points per axis n3 = (nx, ny, nz), which may
    // differ; N = nx.  Their passes read the twiddles W_{2 n_q}^e of axis q from tw3[q]
    // (the dtype's storage: float2, double2, or double-float float4), the symbol as
    // [kz <= nz][ky <= ny][kx < Ps], and use no TMA descriptors and no form knobs.
    int any = 0;
    int n3[3] = {0, 0, 0};
    void *tw3[3] = {nullptr, nullptr, nullptr};
    int Px = 0;
    int Ps = 0;
    void *sym = nullptr;
    void *symT = nullptr;  // a box plan's symbol with kz innermost, read by the z warp forms
    void *tw = nullptr;
    void *twc = nullptr;
    void *w1 = nullptr;
    void *w2 = nullptr;
    void *w3 = nullptr;
    int *status = nullptr;  // device status word (bit 0: a bounded wait timed out)
    double *tail = nullptr; // 2 max_batch doubles: spectral-tail sums of a checked solve
    // z pass form: 0 length-2N transforms, 1 even/odd length-N split, 2 warp form (one
    // warp per column pair, FP32, N = 64 ... 256; one warp per column at N = 512)
    int zform = 0;
    // y pass form: 0 block form (a column pair spread over a block), 1 warp form (FP32,
    // N = 64 ... 256: a warp per column pair; N = 512: a warp per column)
    int yform = 0;
    // x pass form: 0 block form (a tile of rows staged in shared memory), 1 warp form (a
    // half-warp or warp per row pair, FP32, N = 64 ... 256 and 512)
    int xform = 0;
    // x-y form: 0 the x and y passes as separate launches, 1 fused (k_xy_fwd / k_yx_inv:
    // the x spectrum passes through an L2-resident ring of plane slots; FP32, N = 64 ... 256,
    // plans with a counter block)
    int xyform = 0;
    // Counter block of the fused x-y passes (kSyncInts ints, zero between launches), or null.
    int *sync = nullptr;
    // TMA descriptors of the column passes' inputs (y forward: w1, z: w2 and the symbol,
    // y inverse: w3), encoded once for these buffers; and of the warp-form z pass (w2 in,
    // symbol, w3 out; 128- and 64-byte swizzled boxes), encoded where that form exists.
    CUtensorMap tm_y_in, tm_z_in, tm_z_sym, tm_yi_in;
    CUtensorMap tm_zw_in, tm_zw_sym, tm_zw_out;
    CUtensorMap tm_yw1, tm_yw2, tm_yw3;  // warp-form y passes: boxes of N rows (256 at N = 512) of w1, w2, w3
    CUtensorMap tm_ywi1, tm_ywi3;        // warp-form y inverse (N <= 256): 8-column boxes of w1, w3
    CUtensorMap tm_rf;                   // fused forward x-y pass: N-row boxes of its ring in w3
};

constexpr int kStatusTimeoutBit = 1;  // bit of DevicePlan::status set by a timed-out wait

inline int pitch_for(int N) { return ((N + 1 + 15) / 16) * 16; }
inline int sym_pitch_for(int N) { return ((N + 1 + 3) / 4) * 4; }

bool n_supported(int N);

// Record a failed CUDA call for poisson_last_cuda_error() (per host thread).
void note_cuda_error(cudaError_t e);

// Encode the TMA descriptors of p for its buffers.  Returns cudaSuccess or an error
// (cudaErrorNotSupported when the driver has no tensor-map encoder).
cudaError_t encode_tma_maps(DevicePlan &p);

// The five passes of `count` solves (1 <= count <= p.max_batch) of the plan's geometry on
// `s`: rho[b] -> u[b].  ev: null, or 6 events recorded before pass 1, between the passes
// and after pass 5.  tail: null, or 2 count zeroed doubles that receive, per density, the
// padded spectrum's energy in the outer |k|_inf shell and its total energy.  skip: bit 0
// leaves out the forward x and y passes, bit 1 the inverse y and x passes (the caller runs
// them with launch_xy_slab); not with the fused x-y form.
cudaError_t launch_solve(const DevicePlan &p, const PtrArray &rho, const PtrArray &u, int count,
                         cudaStream_t s, cudaEvent_t *ev, double *tail = nullptr, int skip = 0);

// The x and y passes (forward: x then y; inverse: y then x) of planes z0 .. z0 + nz - 1 of
// one density, in the plan's separate forms: rho, u device pointers to the whole density.
cudaError_t launch_xy_slab(const DevicePlan &p, const void *rho, void *u, int z0, int nz, cudaStream_t s, bool fwd);

// Forms of the z pass that exist for (N, dtype, arith), as a bit mask over DevicePlan::zform:
// bit 0 always; bit 1 where the length-N schedule has fewer stages than the length-2N one
// (not in double-float arithmetic); bit 2 for FP32 at N = 64, 96, 128, 160, 192, 256 and 512.
int z_forms(int N, int dtype, int arith = 0);

// Forms of the x passes that exist for (N, dtype), as a bit mask over DevicePlan::xform:
// bit 0 always; bit 1 for FP32 at N = 64, 96, 128, 160, 192, 256 and 512.
int x_forms(int N, int dtype);

// The two x passes alone, one density on spare workspace, in the form p.xform selects.
cudaError_t launch_x_passes(const DevicePlan &p, cudaStream_t s);

// Forms of the y passes that exist for (N, dtype), as a bit mask over DevicePlan::yform:
// bit 0 always; bit 1 for FP32 at N = 64, 96, 128, 160, 192, 256 and 512.
int y_forms(int N, int dtype);

// The two y passes alone, one density, in the form p.yform selects (for timing the forms).
cudaError_t launch_y_passes(const DevicePlan &p, cudaStream_t s);

// Forms of the x-y passes that exist for (N, dtype), as a bit mask over
// DevicePlan::xyform: bit 0 always; bit 1 for FP32 at N = 64, 96, 128, 160, 192, 256.
int xy_forms(int N, int dtype);

// Ints of the counter block DevicePlan::sync.
int xy_sync_ints();

// The forward and inverse x and y passes alone, one density, in the forms p.xyform (and,
// when separate, p.xform and p.yform) select (for timing the forms).
cudaError_t launch_xy_passes(const DevicePlan &p, cudaStream_t s);

// The z pass alone, one density, in the form p.zform selects (for timing the forms).
cudaError_t launch_z_pass(const DevicePlan &p, cudaStream_t s);

// One bounded device-side wait that nothing completes, `polls` polls on p's status word
// (the test hook of poisson_selftest_wait).
cudaError_t launch_wait_selftest(const DevicePlan &p, long long polls, cudaStream_t s);

// The per-axis factors A_j(k), k = 0..N, of the S Gaussian-sum terms dtau into dA (S x (N+1),
// FP64, on the device) by the host setup's rule; dgl: the 16-point Gauss-Legendre nodes
// then weights.
cudaError_t launch_axis_table(const double *dtau, const double *dgl, int S, int N, double *dA, cudaStream_t s);

// Fill p.sym from the per-axis factors (FP64, on the device):
// sym = scale * (sum_j w_j A_j(kx) A_j(ky) A_j(kz) + C0 - C2 (pi/2)^2 |k|^2) (literal = 0),
// or with 8 (C0 - C2 (pi/2)^2 |k|^2) at all-even (kx, ky, kz) only (literal = 1: the
// correction of the unpadded N^3 transform pair).
cudaError_t launch_symbol_table(const DevicePlan &p, const double *dA, const double *dw,
                                int nterms, double C0, double C2, double scale, int literal,
                                cudaStream_t s);
// The same for a box: dA3 holds the x, y and z tables one after the other (n_q + 1 entries
// per term on axis q: p.n3 for a runtime-length plan, N on every axis otherwise), l the
// scaled half-lengths; the table is not symmetric.  p.symT, where set, also receives it with
// kz innermost.
cudaError_t launch_symbol_table_box(const DevicePlan &p, const double *dA3, const double *dw, int nterms,
                                    double C0, double C2, double scale, const double *l, int literal,
                                    cudaStream_t s);

}  // namespace gsp
