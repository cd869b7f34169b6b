// Coupled-routing (float) instantiation of the kinematics / cost kernels, 1..6 segments.
#include "cr_eval_impl.cuh"
namespace crk {
CR_EVAL_COUPLED_INSTANTIATE(, float)
}
