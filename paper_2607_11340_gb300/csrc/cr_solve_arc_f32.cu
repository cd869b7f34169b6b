// Arc-model (FP32-bulk) instantiation of the solver kernels, 1..4 segments.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_ARC_INSTANTIATE(, float)
}
