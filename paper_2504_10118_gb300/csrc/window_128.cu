// window_128.cu -- the window kernels (every mode, single and batched) for
// m = 128 (four-block clusters), compiled apart from the other sides.
#include "core.cuh"
#include "window_launch.cuh"

namespace magpie_impl {
MAGPIE_INSTANTIATE_WINDOW(128)
}  // namespace magpie_impl
