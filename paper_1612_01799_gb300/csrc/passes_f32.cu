// FP32 instantiation of the solve passes.
#include "passes.cuh"

namespace gsp {
cudaError_t solve_f32(const DevicePlan &p, const PtrArray &rho, const PtrArray &u, int B, cudaStream_t s,
                     cudaEvent_t *ev, double *tail) {
    return solve_dispatch<float>(p, rho, u, B, s, ev, tail);
}
cudaError_t symbol_table_f32(const DevicePlan &p, const double *dA, const double *dw, int nterms,
                             double C0, double C2, double scale, cudaStream_t s) {
    return symbol_table<float>(p, dA, dw, nterms, C0, C2, scale, s);
}
cudaError_t encode_maps_f32(DevicePlan &p) { return encode_dispatch<float>(p); }
}  // namespace gsp
