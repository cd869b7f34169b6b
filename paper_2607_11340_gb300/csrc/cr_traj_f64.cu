// FP64 instantiation of the trajectory and calibration kernels.
#include "cr_traj_impl.cuh"
namespace crk {
CR_TRAJ_INSTANTIATE(, double)
}
