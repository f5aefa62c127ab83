// Double-float dispatch of the solve passes (the per-N code is in passes_df_[abc].cu): the
// FP64 path's arithmetic on the FP32 pipe (type DF of fft_core.cuh), FP64 at the boundary.
#include "passes.cuh"

namespace gsp {
#define GSP_EXTERN_DF(n) GSP_DECLARE_N(extern, DF, n)
GSP_SUPPORTED_N(GSP_EXTERN_DF)
#undef GSP_EXTERN_DF

cudaError_t solve_df(const DevicePlan &p, const PtrArray &rho, const PtrArray &u, int B, cudaStream_t s,
                     cudaEvent_t *ev, double *tail, int skip) {
    return solve_dispatch<DF>(p, rho, u, B, s, ev, tail, skip);
}
cudaError_t xy_slab_df(const DevicePlan &p, const void *rho, void *u, int z0, int nz, cudaStream_t s, bool fwd) {
    return xy_slab_dispatch<DF>(p, rho, u, z0, nz, s, fwd);
}
cudaError_t symbol_table_df(const DevicePlan &p, const double *dA, const double *dw, int nterms,
                            double C0, double C2, double scale, int literal, cudaStream_t s) {
    return symbol_table<DF>(p, dA, dw, nterms, C0, C2, scale, literal, s);
}
cudaError_t encode_maps_df(DevicePlan &p) { return encode_dispatch<DF>(p); }
cudaError_t z_pass_df(const DevicePlan &p, cudaStream_t s) { return z_pass_dispatch<DF>(p, s); }
cudaError_t z_lines_df(const DevicePlan &p, int ky0, int nky, cudaStream_t s) {
    return z_lines_dispatch<DF>(p, ky0, nky, s);
}
cudaError_t y_passes_df(const DevicePlan &p, cudaStream_t s) { return y_pass_dispatch<DF>(p, s); }
cudaError_t x_passes_df(const DevicePlan &p, cudaStream_t s) { return x_pass_dispatch<DF>(p, s); }
cudaError_t xy_passes_df(const DevicePlan &p, cudaStream_t s) { return xy_pass_dispatch<DF>(p, s); }
}  // namespace gsp
