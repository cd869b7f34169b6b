// PRM roadmap and query kernels for 4..6 segments.
#include "cr_prm_impl.cuh"

namespace crk {
CR_PRM_INSTANTIATE(, 4)
CR_PRM_INSTANTIATE(, 5)
CR_PRM_INSTANTIATE(, 6)
}  // namespace crk
