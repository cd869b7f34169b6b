// Arc-model (FP32-bulk) dispatch of the solver kernels, 1..4 segments; the kernels are
// instantiated in cr_solve_arc_f32_n12.cu and cr_solve_arc_f32_n34.cu.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_ALL_N_EXTERN(float)
CR_SOLVE_ARC_INSTANTIATE(, float)
}
