// window_small.cu -- the window kernels (every mode, single and batched) for
// m = 8, 16 and 32 (one block per window), compiled apart from the other sides.
#include "core.cuh"
#include "window_launch.cuh"

namespace magpie_impl {
MAGPIE_INSTANTIATE_WINDOW(8)
MAGPIE_INSTANTIATE_WINDOW(16)
MAGPIE_INSTANTIATE_WINDOW(32)
}  // namespace magpie_impl
