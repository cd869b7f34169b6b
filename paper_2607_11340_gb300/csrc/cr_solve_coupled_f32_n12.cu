// Coupled-routing solver kernels of 1 and 2 segments, FP32 bulk.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_N_INSTANTIATE(, float, 1, CR_MODEL_COUPLED)
CR_SOLVE_N_INSTANTIATE(, float, 2, CR_MODEL_COUPLED)
}
