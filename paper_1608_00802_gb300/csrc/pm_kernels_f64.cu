// fp64 instantiation of the step kernels (the plain fp64 path).
#include "pm_kernels.cuh"
#include "pm_sort.cuh"
#include "pm_instantiate.cuh"

namespace pm {

PM_INSTANTIATE(double)

}  // namespace pm
