// FP32-bulk instantiation of the path-following kernels (FP64 block Cholesky inside).
#include "cr_path_impl.cuh"
namespace crk {
CR_PATH_INSTANTIATE(, float)
}
