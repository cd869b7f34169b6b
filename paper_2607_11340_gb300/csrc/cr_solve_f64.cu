// FP64 instantiation of the solver kernels.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_ARC_INSTANTIATE(extern, double)
CR_SOLVE_INSTANTIATE(, double)
}
