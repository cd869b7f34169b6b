// Coupled-routing solver kernels of 5 segments, FP32 bulk.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_N_INSTANTIATE(, float, 5, CR_MODEL_COUPLED)
}
