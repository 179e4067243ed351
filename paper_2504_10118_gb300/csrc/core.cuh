// core.cuh -- what the library's translation units share: the window
// kernel's geometry, layouts and device code (fft_lines.cuh,
// window_kernel.cuh) in namespace magpie_impl, the cluster launch helper, and
// the per-window-side launch entry points that window_launch.cuh defines and
// the window_*.cu files instantiate (the window kernels of different sides
// compile in parallel; magpie.cu holds the host side and the other kernels).
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <algorithm>
#include <utility>

namespace magpie_impl {

namespace cg = cooperative_groups;

constexpr int kMaxMinibatch = 4096;  // the update kernel keeps the minibatch's corners in smem (48 KiB)
constexpr int kMaxCluster = 8;       // largest number of blocks per window
constexpr int kMaxSlots = 16;        // partial-sum slots per window: the window kernel's blocks, or m / 16
                                     // blocks of the precision form (m <= 256)
constexpr int kApplyUnroll = 4;      // increments in flight per thread in the update kernel

#include "fft_lines.cuh"
#include "update.cuh"
#include "window_kernel.cuh"

// the window sides with a window kernel
#define MAGPIE_WINDOW_SIZES(X) X(8) X(16) X(32) X(64) X(128) X(256)

// Launch with a cluster dimension when cl > 1, and as a programmatic dependent
// launch when pdl is set (the kernel must then call grid_dep_wait before it
// touches memory that the stream's previous kernel reads or writes).
template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, int cl,
                       bool pdl, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int n = 0;
  if (cl > 1) {
    attr[n].id = cudaLaunchAttributeClusterDimension;
    attr[n].val.clusterDim.x = cl;
    attr[n].val.clusterDim.y = 1;
    attr[n].val.clusterDim.z = 1;
    ++n;
  }
  if (pdl) {  // see grid_dep_wait
    attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
  }
  cfg.attrs = attr;
  cfg.numAttrs = n;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Per window side MS (definitions in window_launch.cuh):
// the window kernel in mode `mode` (a Mode) over `windows` windows;
template <int MS>
cudaError_t window_launch(int mode, const StepArgs& a, int windows, cudaStream_t st);
// the batched minibatch-step kernel with register bound `minb` (blocks per SM);
template <int MS>
cudaError_t window_launch_batched(const StepArgs* table, const int2* map, int windows, cudaStream_t st, int minb);
// the shared-memory attribute of every window kernel of this side;
template <int MS>
cudaError_t window_prepare();
// the three register bounds the group autotuner tries (c[0] the default;
// equal entries are one candidate);
template <int MS>
void window_minb_candidates(int* c);
// the persistent step kernel on `clusters` clusters, with shared memory for
// update lists of up to max_count windows;
template <int MS>
cudaError_t window_launch_persistent(const PersistArgs& P, int clusters, int max_count, cudaStream_t st, int minb);
// the clusters of the persistent step kernel that fit on the GPU at once.
template <int MS>
int window_persistent_capacity(int max_count, int minb);

}  // namespace magpie_impl
