// Persistent batch kernel for robots of 5 segment(s).
#include "cr_batch_impl.cuh"

namespace crk {
CR_BATCH_INSTANTIATE(, 5)
}  // namespace crk
