// Patch kernels of degree k = 5 (FP32 and FP64), in a translation unit of
// their own so that the degrees compile in parallel.
#include "patch_launch.cuh"

namespace stk {
STK_PATCH_INSTANTIATE(5)
}  // namespace stk
