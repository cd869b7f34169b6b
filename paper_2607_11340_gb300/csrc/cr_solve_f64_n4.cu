// Solver kernels of the 4-segment tendon model, FP64.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_N_INSTANTIATE(, double, 4, CR_MODEL_TENDON)
}
