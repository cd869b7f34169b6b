// Coupled-routing solver kernels of 1 and 2 segments, FP64.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_N_INSTANTIATE(, double, 1, CR_MODEL_COUPLED)
CR_SOLVE_N_INSTANTIATE(, double, 2, CR_MODEL_COUPLED)
}
