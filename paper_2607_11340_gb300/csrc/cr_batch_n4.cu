// Persistent batch kernel for robots of 4 segment(s).
#include "cr_batch_impl.cuh"

namespace crk {
CR_BATCH_INSTANTIATE(, 4)
}  // namespace crk
