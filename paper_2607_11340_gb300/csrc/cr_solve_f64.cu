// FP64 dispatch of the solver kernels; the kernels of each segment count are instantiated in
// cr_solve_f64_n*.cu and cr_solve_arc_f64_n*.cu.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_ALL_N_EXTERN(double)
CR_SOLVE_ARC_INSTANTIATE(extern, double)
CR_SOLVE_INSTANTIATE(, double)
}
