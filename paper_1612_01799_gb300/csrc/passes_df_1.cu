// Double-float passes for the sizes of group 1 (see passes.cuh).
#include "passes.cuh"

namespace gsp {
#define GSP_INST(n) GSP_DECLARE_N(, DF, n)
GSP_DF_GROUP_1(GSP_INST)
#undef GSP_INST
}  // namespace gsp
