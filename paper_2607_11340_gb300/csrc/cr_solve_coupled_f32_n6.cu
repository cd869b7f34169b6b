// Coupled-routing solver kernels of 6 segments, FP32 bulk.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_N_INSTANTIATE(, float, 6, CR_MODEL_COUPLED)
}
