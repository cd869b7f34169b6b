// FP32 instantiation of the kinematics / cost kernels.
#include "cr_eval_impl.cuh"
namespace crk {
CR_EVAL_ARC_INSTANTIATE(extern, float)
CR_EVAL_COUPLED_INSTANTIATE(extern, float)
CR_EVAL_INSTANTIATE(, float)
}
