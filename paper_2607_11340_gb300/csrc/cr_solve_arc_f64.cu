// Arc-model (FP64) dispatch of the solver kernels, 1..4 segments; the kernels are
// instantiated in cr_solve_arc_f64_n12.cu and cr_solve_arc_f64_n34.cu.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_ALL_N_EXTERN(double)
CR_SOLVE_ARC_INSTANTIATE(, double)
}
