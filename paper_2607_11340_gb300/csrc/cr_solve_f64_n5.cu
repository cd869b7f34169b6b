// Solver kernels of the 5-segment tendon model, FP64.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_N_INSTANTIATE(, double, 5, CR_MODEL_TENDON)
}
