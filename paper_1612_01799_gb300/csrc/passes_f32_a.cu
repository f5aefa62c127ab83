// FP32 passes for the sizes of group A (see passes.cuh).
#include "passes.cuh"

namespace gsp {
#define GSP_INST(n) GSP_DECLARE_N(, float, n)
GSP_SIZE_GROUP_A(GSP_INST)
#undef GSP_INST
}  // namespace gsp
