// Solver kernels of the 1-segment tendon model, FP32 bulk.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_N_INSTANTIATE(, float, 1, CR_MODEL_TENDON)
}
