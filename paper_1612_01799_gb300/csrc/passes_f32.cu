// FP32 dispatch of the solve passes (the per-N code is in passes_f32_[abc].cu).
#include "passes.cuh"

namespace gsp {
#define GSP_EXTERN_F32(n) GSP_DECLARE_N(extern, float, n)
GSP_SUPPORTED_N(GSP_EXTERN_F32)
#undef GSP_EXTERN_F32

cudaError_t solve_f32(const DevicePlan &p, const PtrArray &rho, const PtrArray &u, int B, cudaStream_t s,
                     cudaEvent_t *ev, double *tail, int skip) {
    return solve_dispatch<float>(p, rho, u, B, s, ev, tail, skip);
}
cudaError_t xy_slab_f32(const DevicePlan &p, const void *rho, void *u, int z0, int nz, cudaStream_t s, bool fwd) {
    return xy_slab_dispatch<float>(p, rho, u, z0, nz, s, fwd);
}
cudaError_t symbol_table_f32(const DevicePlan &p, const double *dA, const double *dw, int nterms,
                             double C0, double C2, double scale, int literal, cudaStream_t s) {
    return symbol_table<float>(p, dA, dw, nterms, C0, C2, scale, literal, s);
}
cudaError_t encode_maps_f32(DevicePlan &p) { return encode_dispatch<float>(p); }
cudaError_t z_pass_f32(const DevicePlan &p, cudaStream_t s) { return z_pass_dispatch<float>(p, s); }
cudaError_t z_lines_f32(const DevicePlan &p, int ky0, int nky, cudaStream_t s) {
    return z_lines_dispatch<float>(p, ky0, nky, s);
}
cudaError_t y_passes_f32(const DevicePlan &p, cudaStream_t s) { return y_pass_dispatch<float>(p, s); }
cudaError_t x_passes_f32(const DevicePlan &p, cudaStream_t s) { return x_pass_dispatch<float>(p, s); }
cudaError_t xy_passes_f32(const DevicePlan &p, cudaStream_t s) { return xy_pass_dispatch<float>(p, s); }
int xy_sync_ints() { return kSyncInts; }
int xy_forms(int N, int dtype) { return 1 | (dtype == 0 && warp_n(N) ? 2 : 0); }
int x_forms(int N, int dtype) { return 1 | (dtype == 0 && (warp_n(N) || N == XWarp2::N) ? 2 : 0); }
int y_forms(int N, int dtype) { return 1 | (dtype == 0 && (warp_n(N) || N == ZW512::N) ? 2 : 0); }
int z_forms(int N, int dtype, int arith) {
    return 1 | (zsplit_dispatch(N) && !arith ? 2 : 0) | (dtype == 0 && zwarp_available(N) ? 4 : 0);
}
}  // namespace gsp
