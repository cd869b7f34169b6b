// PRM roadmap and query kernels for 1..3 segments.
#include "cr_prm_impl.cuh"

namespace crk {
CR_PRM_INSTANTIATE(, 1)
CR_PRM_INSTANTIATE(, 2)
CR_PRM_INSTANTIATE(, 3)
}  // namespace crk
