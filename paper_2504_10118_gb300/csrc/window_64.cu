// window_64.cu -- the window kernels (every mode, single and batched) for
// m = 64 (two-block clusters), compiled apart from the other sides.
#include "core.cuh"
#include "window_launch.cuh"

namespace magpie_impl {
MAGPIE_INSTANTIATE_WINDOW(64)
}  // namespace magpie_impl
