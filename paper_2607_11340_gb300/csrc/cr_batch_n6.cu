// Persistent batch kernel for robots of 6 segment(s).
#include "cr_batch_impl.cuh"

namespace crk {
CR_BATCH_INSTANTIATE(, 6)
}  // namespace crk
