// Solver kernels of the 6-segment tendon model, FP64.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_N_INSTANTIATE(, double, 6, CR_MODEL_TENDON)
}
