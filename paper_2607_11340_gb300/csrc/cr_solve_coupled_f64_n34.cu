// Coupled-routing solver kernels of 3 and 4 segments, FP64.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_N_INSTANTIATE(, double, 3, CR_MODEL_COUPLED)
CR_SOLVE_N_INSTANTIATE(, double, 4, CR_MODEL_COUPLED)
}
