// Coupled-routing solver kernels of 3 and 4 segments, FP32 bulk.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_N_INSTANTIATE(, float, 3, CR_MODEL_COUPLED)
CR_SOLVE_N_INSTANTIATE(, float, 4, CR_MODEL_COUPLED)
}
