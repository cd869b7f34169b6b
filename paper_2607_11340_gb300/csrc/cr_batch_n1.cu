// Persistent batch kernel for robots of 1 segment(s).
#include "cr_batch_impl.cuh"

namespace crk {
CR_BATCH_INSTANTIATE(, 1)
}  // namespace crk
