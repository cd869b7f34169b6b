// Arc-model (float) instantiation of the kinematics / cost kernels, 1..4 segments.
#include "cr_eval_impl.cuh"
namespace crk {
CR_EVAL_ARC_INSTANTIATE(, float)
}
