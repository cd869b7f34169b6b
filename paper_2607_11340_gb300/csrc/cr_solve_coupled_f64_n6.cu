// Coupled-routing solver kernels of 6 segments, FP64 bulk.
#include "cr_solve_impl.cuh"
namespace crk {
CR_SOLVE_N_INSTANTIATE(, double, 6, CR_MODEL_COUPLED)
}
