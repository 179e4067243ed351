// window_launch.cuh -- the per-window-side launch entry points declared in
// core.cuh; included by the window_*.cu files, each of which instantiates
// them for its window sides.
#pragma once

namespace magpie_impl {

template <int MS, int MODE>
cudaError_t launch_window(const StepArgs& a, int windows, cudaStream_t st) {
  using Gm = Geo<MS>;
  return launch_ex(window_kernel<MS, MODE>, dim3((unsigned)windows * Gm::CL), dim3(Gm::T), Gm::SMEM, st, Gm::CL, a);
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
template <int MS>
constexpr int alt_minb() {
  return Geo<MS>::T >= 512 ? 1 : (Geo<MS>::MIN_BLOCKS == 1 ? 2 : 1);
}

template <int MS>
cudaError_t window_launch_batched(const StepArgs* table, const int2* map, int windows, cudaStream_t st, int minb) {
  using Gm = Geo<MS>;
  const dim3 grid((unsigned)windows * Gm::CL);
  if (minb == alt_minb<MS>() && minb != Gm::MIN_BLOCKS)
    return launch_ex(window_kernel_batched<MS, kStep, alt_minb<MS>()>, grid, dim3(Gm::T), Gm::SMEM, st, Gm::CL,
                     table, map);
  return launch_ex(window_kernel_batched<MS, kStep, Gm::MIN_BLOCKS>, grid, dim3(Gm::T), Gm::SMEM, st, Gm::CL, table,
                   map);
}

template <int MS>
void window_minb_candidates(int* c) {
  c[0] = Geo<MS>::MIN_BLOCKS;
  c[1] = alt_minb<MS>();
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
    e = cudaFuncSetAttribute(window_kernel<MS, kStepRecycle>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel<MS, kStepAtomic>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel<MS, kEval>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel<MS, kSim>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

#define MAGPIE_INSTANTIATE_WINDOW(S)                                                                       \
  template cudaError_t window_launch<S>(int, const StepArgs&, int, cudaStream_t);                          \
  template cudaError_t window_launch_batched<S>(const StepArgs*, const int2*, int, cudaStream_t, int);     \
  template cudaError_t window_prepare<S>();                                                                \
  template void window_minb_candidates<S>(int*);

}  // namespace magpie_impl
