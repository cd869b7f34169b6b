// Persistent batch kernel for robots of 2 segment(s).
#include "cr_batch_impl.cuh"

namespace crk {
CR_BATCH_INSTANTIATE(, 2)
}  // namespace crk
