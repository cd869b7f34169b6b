// FP64 instantiation of the path-following kernels.
#include "cr_path_impl.cuh"
namespace crk {
CR_PATH_INSTANTIATE(, double)
}
