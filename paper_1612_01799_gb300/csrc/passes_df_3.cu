// Double-float passes for the sizes of group 3 (see passes.cuh).
#include "passes.cuh"

namespace gsp {
#define GSP_INST(n) GSP_DECLARE_N(, DF, n)
GSP_DF_GROUP_3(GSP_INST)
#undef GSP_INST
}  // namespace gsp
