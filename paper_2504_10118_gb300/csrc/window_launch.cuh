// window_launch.cuh -- the per-window-side launch entry points declared in
// core.cuh; included by the window_*.cu files, each of which instantiates
// them for its window sides.
#pragma once

namespace magpie_impl {

template <int MS, int MODE>
cudaError_t launch_window(const StepArgs& a, int windows, cudaStream_t st) {
  using Gm = Geo<MS>;
  // minibatch steps overlap their launch with the previous kernel's tail
  constexpr bool pdl = MODE == kStep || MODE == kStepAtomic || MODE == kStepRecycle;
  return launch_ex(window_kernel<MS, MODE>, dim3((unsigned)windows * Gm::CL), dim3(Gm::T), Gm::SMEM, st, Gm::CL, pdl,
                   a);
}

template <int MS>
cudaError_t window_launch(int mode, const StepArgs& a, int windows, cudaStream_t st) {
  switch (mode) {
    case kStep: return launch_window<MS, kStep>(a, windows, st);
    case kEval: return launch_window<MS, kEval>(a, windows, st);
    case kSim: return launch_window<MS, kSim>(a, windows, st);
    case kStepRecycle: return launch_window<MS, kStepRecycle>(a, windows, st);
    case kStepAtomic: return launch_window<MS, kStepAtomic>(a, windows, st);
    default: return cudaErrorInvalidValue;
  }
}

// Candidate register bounds of the batched window kernel: blocks per SM.
// The default (Geo::MIN_BLOCKS), an alternative, and a third, denser one:
// three 256-thread blocks (80 registers; three of the m = 128 kernel's
// 72 KB of shared memory fit an SM), or four of 128 threads or fewer.
template <int MS>
constexpr int alt_minb() {
  return Geo<MS>::T >= 512 ? 1 : (Geo<MS>::MIN_BLOCKS == 1 ? 2 : 1);
}
template <int MS>
constexpr int third_minb() {
  return Geo<MS>::T >= 512 ? 1 : (Geo<MS>::T == 256 ? 3 : 4);
}

template <int MS>
cudaError_t window_launch_batched(const StepArgs* table, const int2* map, int windows, cudaStream_t st, int minb) {
  using Gm = Geo<MS>;
  const dim3 grid((unsigned)windows * Gm::CL);
  if (minb == third_minb<MS>() && minb != Gm::MIN_BLOCKS && minb != alt_minb<MS>())
    return launch_ex(window_kernel_batched<MS, kStep, third_minb<MS>()>, grid, dim3(Gm::T), Gm::SMEM, st, Gm::CL,
                     false, table, map);
  if (minb == alt_minb<MS>() && minb != Gm::MIN_BLOCKS)
    return launch_ex(window_kernel_batched<MS, kStep, alt_minb<MS>()>, grid, dim3(Gm::T), Gm::SMEM, st, Gm::CL,
                     false, table, map);
  return launch_ex(window_kernel_batched<MS, kStep, Gm::MIN_BLOCKS>, grid, dim3(Gm::T), Gm::SMEM, st, Gm::CL, false,
                   table, map);
}

template <int MS>
void window_minb_candidates(int* c) {
  c[0] = Geo<MS>::MIN_BLOCKS;
  c[1] = alt_minb<MS>();
  c[2] = third_minb<MS>();
}

template <int MS>
size_t persistent_smem(int max_count) {
  return std::max(Geo<MS>::SMEM, (sizeof(int2) + sizeof(int)) * (size_t)max_count);
}

template <int MS>
cudaError_t window_launch_persistent(const PersistArgs& P, int clusters, int max_count, cudaStream_t st, int minb) {
  using Gm = Geo<MS>;
  const dim3 grid((unsigned)clusters * Gm::CL);
  const size_t smem = persistent_smem<MS>(max_count);
  if (minb == alt_minb<MS>() && minb != Gm::MIN_BLOCKS)
    return launch_ex(window_kernel_persistent<MS, alt_minb<MS>()>, grid, dim3(Gm::T), smem, st, Gm::CL, false, P);
  return launch_ex(window_kernel_persistent<MS, Gm::MIN_BLOCKS>, grid, dim3(Gm::T), smem, st, Gm::CL, false, P);
}

template <int MS>
int window_persistent_capacity(int max_count, int minb) {
  using Gm = Geo<MS>;
  void (*k)(PersistArgs) = (minb == alt_minb<MS>() && minb != Gm::MIN_BLOCKS)
                               ? window_kernel_persistent<MS, alt_minb<MS>()>
                               : window_kernel_persistent<MS, Gm::MIN_BLOCKS>;
  const size_t smem = persistent_smem<MS>(max_count);
  int dev = 0, sms = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  if constexpr (Gm::CL == 1) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, Gm::T, smem) != cudaSuccess) return 0;
    return n * sms;
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(Gm::CL * sms));
    cfg.blockDim = dim3(Gm::T);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = Gm::CL;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&n, (void*)k, &cfg) != cudaSuccess) return 0;
    return n;
  }
}

template <int MS>
cudaError_t window_prepare() {
  const int bytes = (int)Geo<MS>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(window_kernel<MS, kStep>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel_batched<MS, kStep, Geo<MS>::MIN_BLOCKS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel_batched<MS, kStep, alt_minb<MS>()>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel_batched<MS, kStep, third_minb<MS>()>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)  // the densest bound needs the whole shared-memory carve-out
    e = cudaFuncSetAttribute(window_kernel_batched<MS, kStep, third_minb<MS>()>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel<MS, kStepRecycle>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel<MS, kStepAtomic>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel<MS, kEval>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel<MS, kSim>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  const int pbytes = (int)persistent_smem<MS>(kMaxMinibatch);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel_persistent<MS, Geo<MS>::MIN_BLOCKS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, pbytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel_persistent<MS, alt_minb<MS>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             pbytes);
  return e;
}

#define MAGPIE_INSTANTIATE_WINDOW(S)                                                                       \
  template cudaError_t window_launch<S>(int, const StepArgs&, int, cudaStream_t);                          \
  template cudaError_t window_launch_batched<S>(const StepArgs*, const int2*, int, cudaStream_t, int);     \
  template cudaError_t window_prepare<S>();                                                                \
  template void window_minb_candidates<S>(int*);                                                            \
  template cudaError_t window_launch_persistent<S>(const PersistArgs&, int, int, cudaStream_t, int);      \
  template int window_persistent_capacity<S>(int, int);

}  // namespace magpie_impl
