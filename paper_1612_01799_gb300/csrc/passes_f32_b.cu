// FP32 passes for the sizes of group B (see passes.cuh).
#include "passes.cuh"

namespace gsp {
#define GSP_INST(n) GSP_DECLARE_N(, float, n)
GSP_SIZE_GROUP_B(GSP_INST)
#undef GSP_INST
}  // namespace gsp
