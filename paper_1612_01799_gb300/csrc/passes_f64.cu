// FP64 dispatch of the solve passes (the per-N code is in passes_f64_[abc].cu).
#include "passes.cuh"

namespace gsp {
#define GSP_EXTERN_F64(n) GSP_DECLARE_N(extern, double, n)
GSP_SUPPORTED_N(GSP_EXTERN_F64)
#undef GSP_EXTERN_F64

cudaError_t solve_f64(const DevicePlan &p, const PtrArray &rho, const PtrArray &u, int B, cudaStream_t s,
                     cudaEvent_t *ev, double *tail, int skip) {
    return solve_dispatch<double>(p, rho, u, B, s, ev, tail, skip);
}
cudaError_t xy_slab_f64(const DevicePlan &p, const void *rho, void *u, int z0, int nz, cudaStream_t s, bool fwd) {
    return xy_slab_dispatch<double>(p, rho, u, z0, nz, s, fwd);
}
cudaError_t symbol_table_f64(const DevicePlan &p, const double *dA, const double *dw, int nterms,
                             double C0, double C2, double scale, int literal, cudaStream_t s) {
    return symbol_table<double>(p, dA, dw, nterms, C0, C2, scale, literal, s);
}
cudaError_t encode_maps_f64(DevicePlan &p) { return encode_dispatch<double>(p); }
cudaError_t z_pass_f64(const DevicePlan &p, cudaStream_t s) { return z_pass_dispatch<double>(p, s); }
cudaError_t z_lines_f64(const DevicePlan &p, int ky0, int nky, cudaStream_t s) {
    return z_lines_dispatch<double>(p, ky0, nky, s);
}
cudaError_t y_passes_f64(const DevicePlan &p, cudaStream_t s) { return y_pass_dispatch<double>(p, s); }
cudaError_t x_passes_f64(const DevicePlan &p, cudaStream_t s) { return x_pass_dispatch<double>(p, s); }
cudaError_t xy_passes_f64(const DevicePlan &p, cudaStream_t s) { return xy_pass_dispatch<double>(p, s); }
}  // namespace gsp
