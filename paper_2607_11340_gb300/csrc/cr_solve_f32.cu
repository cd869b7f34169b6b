// FP32-bulk dispatch of the solver kernels (FP64 Cholesky and acceptance inside); the kernels of
// each segment count are instantiated in cr_solve_f32_n*.cu and cr_solve_arc_f32_n*.cu.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_ALL_N_EXTERN(float)
CR_SOLVE_ARC_INSTANTIATE(extern, float)
CR_SOLVE_INSTANTIATE(, float)
}
