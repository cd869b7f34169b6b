// Persistent batch kernel for robots of 3 segment(s).
#include "cr_batch_impl.cuh"

namespace crk {
CR_BATCH_INSTANTIATE(, 3)
}  // namespace crk
