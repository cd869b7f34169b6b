// FP32-bulk instantiation of the solver kernels (FP64 Cholesky and acceptance inside).
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_ARC_INSTANTIATE(extern, float)
CR_SOLVE_INSTANTIATE(, float)
}
