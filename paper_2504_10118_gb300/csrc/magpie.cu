// magpie.cu -- MAGPIE sweep on one GB300 (sm_103a): kernels and the C ABI.
//
// Per minibatch step, one thread block per scan window k runs, entirely in
// shared memory and registers:
//   pass A  gather z_k, exit wave Q . z_k, column FFTs          (Section 2.1)
//   pass B  row FFTs, Fourier modulus projection onto sqrt(d_k),
//           inverse row FFTs                                    (Definition REW)
//   pass C  inverse column FFTs -> R_k, then g = conj(Q)(R_k - Q z_k)
//   pass D  the MAGPS V-cycle (Algorithm MAGPS) in residual form
// and writes its increment w . Delta_k (w = u + |Q|^2) to a per-window
// buffer.  A second kernel then updates every object pixel by the ordered
// sum over the minibatch, z += sum_k w.Delta_k / sum_k w, so no atomics are
// used and results are bitwise reproducible.
//
// Residual form of Algorithm MAGPS.  With the weights of Eq. (def_weights),
// W_R . Q = (I_H^h Q_H) . W_z, so by Lemma (commutative) the coarse residual
// R_H - Q_H z_H equals I_h^H(W_R . (R - Q z)).  Writing g^l = conj(Q^l)(R^l -
// Q^l z^l) and w^l = u^l + |Q^l|^2 one level at a time gives
//   g^{l+1} = W_u^l . I_h^H g^l,            (W_u^l = |Q^{l+1}|^2 / I_h^H|Q^l|^2)
//   e^{L-1} = g^{L-1} / w^{L-1}             (coarsest proximal step)
//   e^l     = g^l / w^l + (u^l / w^l) . I_H^h e^{l+1}   (post-smoothing)
//   w^0 . Delta = g^0 + u^0 . I_H^h e^1,
// where e^l is the increment of level l.  Every per-level factor is real and
// depends on the probe only; they are computed once in float64 (Eq.
// def_weights with the division rule: a quotient whose denominator is at most
// 1e-30 is 0, and where w^l vanishes the step passes the coarse increment
// through unchanged, as the proximal factor conj(Q^l)/w^l is then 0).
//
// FFTs: an m-point line is split over G lanes of one warp holding E = m/G
// points each (m = E G, four-step Cooley-Tukey): an E-point DFT in registers,
// twiddles w_m^{g k1}, an exchange through the line's own shared-memory
// storage (XOR-swizzled so that both sides of the exchange are free of bank
// conflicts), and G-point DFTs in registers.  The inverse transform consumes
// the forward transform's output distribution directly (the four steps in
// reverse), so each 2-D transform needs one smem round trip per direction.


#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <algorithm>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "core.cuh"
#include "magpie.h"

namespace magpie_impl {

constexpr int kVersion = 10300;  // 1.3.0

#include "learned.cuh"
#include "umma.cuh"
#include "precision.cuh"

// The precision form's window hand-off counts are final once the update
// kernel that ends the step may run: block (0, 0) zeroes them for the next
// step (whose exit kernel waits for this grid to complete).
__device__ __forceinline__ void clear_handoff(const ApplyArgs& P) {
  if (P.hand && blockIdx.x == 0 && blockIdx.y == 0)
    for (int i = threadIdx.x; i < P.nhand; i += blockDim.x) P.hand[i] = 0;
}

// One problem: a 2-D grid of tiles.
// Launched as a programmatic dependent of the window kernel (its blocks, let
// in early, would slow the next window kernel: 0.328 against 0.319 ms per
// sweep, so it does not trigger its dependents).
__global__ void __launch_bounds__(256) apply_kernel(ApplyArgs P) {
  grid_dep_wait();
  clear_handoff(P);
  apply_body<kApplyTile, kApplyTile>(P, blockIdx.x, blockIdx.y);
}

// The precision form's update: the same ordered sum, each window's
// increment formed from g^0 and its coarse corrections as it is read.
__global__ void __launch_bounds__(256) apply_tail_kernel(ApplyArgs P) {
  grid_dep_wait();
  clear_handoff(P);
  apply_body<kApplyTile, kApplyTile, 256, true>(P, blockIdx.x, blockIdx.y);
}

// Several problems in one launch (1-D grid): problem i owns blocks
// table[i].block0 .. table[i + 1].block0 - 1.
template <int TW, int TH>
__global__ void __launch_bounds__(256) apply_kernel_batched(const ApplyArgs* __restrict__ table, int n) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {  // last problem whose first block is <= blockIdx.x
    const int mid = (lo + hi + 1) >> 1;
    if (table[mid].block0 <= (int)blockIdx.x)
      lo = mid;
    else
      hi = mid - 1;
  }
  const ApplyArgs& P = table[lo];
  const int t = (int)blockIdx.x - P.block0;
  apply_body<TW, TH>(P, t % P.tiles_x, t / P.tiles_x);
}

// Atomic update (deterministic = 0): the window kernel has added, pixel by
// pixel, sum_k w . Delta_k (x, y) and sum_k w (z) into object-sized
// accumulators; every pixel with a positive weight moves by their ratio, the
// same rule as the ordered update, and every touched accumulator is cleared
// for the next step.  One pixel per thread, its accumulator and object loads
// issued together (four pixels per thread, a quarter of the threads,
// measured slower: 122 against 106 us per sweep).  Block 0 also turns the
// window kernel's block partials into Phi_k and ||grad Phi_k||.
__global__ void __launch_bounds__(256) accum_apply_kernel(float2* __restrict__ z, float4* __restrict__ acc,
                                                          size_t npix, const int32_t* __restrict__ idx, int count,
                                                          int n_pos, const double* __restrict__ part, int slots,
                                                          int MS, double* phi_pos, double* gn_pos) {
  grid_dep_wait();  // launched as a programmatic dependent of the window kernel
  if (blockIdx.x == 0) {
    for (int b = threadIdx.x; b < count; b += blockDim.x) {
      const int k = idx[b];
      if ((unsigned)k >= (unsigned)n_pos) continue;
      double a = 0.0, g = 0.0;
      for (int q = 0; q < slots; ++q) {
        a += part[(size_t)(b * slots + q) * 2];
        g += part[(size_t)(b * slots + q) * 2 + 1];
      }
      phi_pos[k] = a / (2.0 * (double)MS * (double)MS);
      gn_pos[k] = sqrt(g);
    }
  }
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < npix; p += (size_t)gridDim.x * blockDim.x) {
    const float4 a = __ldcg(&acc[p]);
    const float2 zz = z[p];  // unconditional: both loads in flight together
    if (a.z > 0.f) z[p] = make_float2(zz.x + a.x / a.z, zz.y + a.y / a.z);
    if (a.x != 0.f || a.y != 0.f || a.z != 0.f) acc[p] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// FP32 FMA throughput: every thread runs kFmaChains independent chains of
// a <- a * b + c (one fused multiply-add, 2 flops, per element per
// iteration); the sums are stored so that nothing is optimised away.
constexpr int kFmaChains = 8;
__global__ void __launch_bounds__(256) fma_rate_kernel(float* out, int iters, float b, float c) {
  float a[kFmaChains];
#pragma unroll
  for (int i = 0; i < kFmaChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
#pragma unroll 4
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i) a[i] = fmaf(a[i], b, c);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kFmaChains; ++i) s += a[i];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

// dst[i] = src[i] with dst in mapped host memory (the object of a pipelined
// host sweep, written over the host link without the copy engines).
__global__ void store_host_kernel(const float2* __restrict__ src, float2* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void sqrt_kernel(const float* d, float* a, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a[i] = sqrtf(fmaxf(d[i], 0.f));
}

// Per-level probe factors in float64 (Eq. def_weights and the rPIE
// regulariser), in three launches: max |Q|^2; the levels inside 16 x 16
// tiles of the finest grid (one block per tile, levels in shared memory);
// and the levels coarser than a tile (one block).  Each element's arithmetic
// and summation order is the same in all three.
constexpr double kTiny = 1e-30;  // division rule threshold

__global__ void __launch_bounds__(256) probe_max_kernel(const float2* Q, int M, unsigned long long* mx_bits) {
  __shared__ double red[8];
  double mx = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const float2 q = Q[i];
    mx = fmax(mx, (double)q.x * q.x + (double)q.y * q.y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x / 32); ++i) mx = fmax(mx, red[i]);
    // non-negative doubles order like their bit patterns
    atomicMax(mx_bits, (unsigned long long)__double_as_longlong(mx));
  }
}

// one coarsening of a 2x2 bin: Q_H, S = mean |Q|^2, W_u, u_H and the floats
__device__ __forceinline__ void coarsen(const double2* q4, const double* u4, double2& qm, double& uh, float& wu,
                                        float& iw, float& rr) {
  qm = make_double2(0.0, 0.0);
  double sa = 0.0, um = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    qm.x += q4[i].x;
    qm.y += q4[i].y;
    sa += q4[i].x * q4[i].x + q4[i].y * q4[i].y;
    um += u4[i];
  }
  qm.x *= 0.25;
  qm.y *= 0.25;
  sa *= 0.25;
  um *= 0.25;
  const double qh2 = qm.x * qm.x + qm.y * qm.y;
  const double w_u = sa > kTiny ? qh2 / sa : 0.0;
  uh = w_u * um;
  const double wh = uh + qh2;
  wu = (float)w_u;
  iw = wh > kTiny ? (float)(1.0 / wh) : 0.f;
  rr = wh > kTiny ? (float)(uh / wh) : 1.f;
}

// One block of TS x TS threads per TS x TS tile of the finest grid
// (TS = min(16, MS)): levels 0 .. min(L-1, log2 TS).  The tile's top level is
// also written in float64 to qtop/utop when coarser levels remain.
__global__ void __launch_bounds__(256) pyramid_tile_kernel(const float2* Q, int MS, int L, float alpha,
                                                            const unsigned long long* mx_bits, double2* qtop,
                                                            double* utop, float* pyr, int unit_wu) {
  __shared__ double2 qsh[2][256];
  __shared__ double ush[2][256];
  const int TS = MS < 16 ? MS : 16;
  const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;
  const int R0 = blockIdx.y * TS, C0 = blockIdx.x * TS;
  const int M = MS * MS;
  const double mx = __longlong_as_double((long long)*mx_bits);
  {
    const int i = (R0 + ty) * MS + C0 + tx;
    const float2 q = Q[i];
    const double2 qd = make_double2(q.x, q.y);
    const double a2 = qd.x * qd.x + qd.y * qd.y;
    const double u = (double)alpha * (mx - a2);
    pyr[i] = (float)u;
    pyr[M + i] = (float)(u + a2);
    qsh[0][ty * TS + tx] = qd;
    ush[0][ty * TS + tx] = u;
  }
  __syncthreads();
  int lt = 0;
  while ((TS >> (lt + 1)) >= 1 && lt + 1 <= L - 1) {
    const int l = lt + 1, ts = TS >> l, src = lt & 1, dst = l & 1;
    if ((int)threadIdx.x < ts * ts) {
      const int r = threadIdx.x / ts, c = threadIdx.x % ts;
      double2 q4[4];
      double u4[4];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          q4[2 * a + b] = qsh[src][(2 * r + a) * (2 * ts) + 2 * c + b];
          u4[2 * a + b] = ush[src][(2 * r + a) * (2 * ts) + 2 * c + b];
        }
      double2 qm;
      double uh;
      float wu, iw, rr;
      coarsen(q4, u4, qm, uh, wu, iw, rr);
      const int s = MS >> l;
      const int o = ((R0 >> l) + r) * s + (C0 >> l) + c;
      float* base = pyr + lvl_off(MS, l);
      base[o] = unit_wu ? 1.f : wu;
      base[s * s + o] = iw;
      base[2 * s * s + o] = rr;
      qsh[dst][r * ts + c] = qm;
      ush[dst][r * ts + c] = uh;
    }
    __syncthreads();
    lt = l;
  }
  if (lt < L - 1) {
    // the tile's top level feeds the coarser levels
    const int ts = TS >> lt, s = MS >> lt;
    if ((int)threadIdx.x < ts * ts) {
      const int r = threadIdx.x / ts, c = threadIdx.x % ts;
      const int o = ((R0 >> lt) + r) * s + (C0 >> lt) + c;
      qtop[o] = qsh[lt & 1][threadIdx.x];
      utop[o] = ush[lt & 1][threadIdx.x];
    }
  }
}

// Levels coarser than a tile, from the level-`lt` float64 arrays (one block).
__global__ void __launch_bounds__(256) pyramid_top_kernel(int MS, int L, int lt, double2* qtop, double* utop,
                                                           float* pyr, int unit_wu) {
  int off = 0;  // level l's arrays at qtop + off (level lt at 0)
  for (int l = lt + 1; l < L; ++l) {
    const int sf = MS >> (l - 1), s = MS >> l;
    const int noff = off + sf * sf;
    for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
      const int r = i / s, c = i % s;
      double2 q4[4];
      double u4[4];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          q4[2 * a + b] = qtop[off + (2 * r + a) * sf + 2 * c + b];
          u4[2 * a + b] = utop[off + (2 * r + a) * sf + 2 * c + b];
        }
      double2 qm;
      double uh;
      float wu, iw, rr;
      coarsen(q4, u4, qm, uh, wu, iw, rr);
      float* base = pyr + lvl_off(MS, l);
      base[i] = unit_wu ? 1.f : wu;
      base[s * s + i] = iw;
      base[2 * s * s + i] = rr;
      qtop[noff + i] = qm;
      utop[noff + i] = uh;
    }
    off = noff;
    __syncthreads();
  }
}

// Probe step of one minibatch (simultaneous with the object step): every
// probe pixel sums, in minibatch order, the windows' conj(z_k)(R_k - Q z_k)
// and beta (max|z_k|^2 - |z_k|^2) + |z_k|^2, and moves by their ratio.
__global__ void __launch_bounds__(256) probe_apply_kernel(float2* Q, int M, const int32_t* idx, int count, int n_pos,
                                                          const float2* pnum, const float* pa2, const double* pmax,
                                                          int CL, float beta) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= M) return;
  float nx = 0.f, ny = 0.f, d = 0.f;
  for (int b = 0; b < count; ++b) {
    if ((unsigned)idx[b] >= (unsigned)n_pos) continue;
    double mb = 0.0;
    for (int q = 0; q < CL; ++q) mb = fmax(mb, pmax[b * CL + q]);
    const float2 v = pnum[(size_t)b * M + p];
    const float a2 = pa2[(size_t)b * M + p];
    nx += v.x;
    ny += v.y;
    d += beta * ((float)mb - a2) + a2;
  }
  if (d > 0.f) {
    float2 q = Q[p];
    q.x += nx / d;
    q.y += ny / d;
    Q[p] = q;
  }
}

// Objective and stopping metric of a full pass (window k in launch slot k):
// per-window values from the block partials, then their sums, all in a fixed
// order (one block).
__global__ void __launch_bounds__(1024) reduce_kernel(const double* part, int CL, int MS, int n, double* phi_pos,
                                                      double* gn_pos, double* out) {
  __shared__ double red[32];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double pk = 0.0, gk = 0.0;
    for (int q = 0; q < CL; ++q) {
      pk += part[(size_t)(k * CL + q) * 2];
      gk += part[(size_t)(k * CL + q) * 2 + 1];
    }
    pk /= 2.0 * (double)MS * (double)MS;
    gk = sqrt(gk);
    phi_pos[k] = pk;
    gn_pos[k] = gk;
    a += pk;
    b += gk;
  }
  const int T = blockDim.x, tid = threadIdx.x;
  for (int pass = 0; pass < 2; ++pass) {
    double v = pass ? b : a;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double r = 0.0;
      for (int i = 0; i < T / 32; ++i) r += red[i];
      out[pass] = r;
    }
    __syncthreads();
  }
}

__global__ void iota_kernel(int32_t* a, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

// ------------------------------------------------------------- host side
// An NVTX range over a host call (sweeps, minibatch steps, group sweeps), for
// timeline tools; header-only NVTX, inert unless a tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CUDA_TRY(expr)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? MAGPIE_ENOMEM : MAGPIE_ECUDA,           \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

bool supported_m(int m) { return m == 8 || m == 16 || m == 32 || m == 64 || m == 128 || m == 256; }

int ilog2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

// blocks per window of the window kernel for patch side m
int cluster_of(int m) {
  switch (m) {
#define MAGPIE_CASE(S) \
  case S:              \
    return Geo<S>::CL;
    MAGPIE_WINDOW_SIZES(MAGPIE_CASE)
#undef MAGPIE_CASE
    default: return 1;
  }
}

// The per-level probe factors of probe Q (float64 arithmetic) into pyr.
// mx: one 8-byte scratch word; qtop/utop: float64 scratch of 2 MS^2 entries.
// unit_wu: store W_u^l = 1 (the MG/OPT correction term: the coarse residual
// gradient becomes the plain restriction of the fine one; u^l and w^l keep the
// paper's weights).
cudaError_t enqueue_pyramid(const float2* Q, int MS, int L, float alpha, unsigned long long* mx, double2* qtop,
                            double* utop, float* pyr, cudaStream_t st, int unit_wu = 0) {
  const int M = MS * MS;
  cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int mb = (M + 255) / 256 < 64 ? (M + 255) / 256 : 64;
  probe_max_kernel<<<mb, 256, 0, st>>>(Q, M, mx);
  const int TS = MS < 16 ? MS : 16;
  pyramid_tile_kernel<<<dim3(MS / TS, MS / TS), TS * TS, 0, st>>>(Q, MS, L, alpha, mx, qtop, utop, pyr, unit_wu);
  int lt = 0;
  while ((TS >> (lt + 1)) >= 1 && lt + 1 <= L - 1) ++lt;
  if (lt < L - 1) pyramid_top_kernel<<<1, 256, 0, st>>>(MS, L, lt, qtop, utop, pyr, unit_wu);
  return cudaGetLastError();
}

ApplyArgs apply_args(float2* z, int n_rows, int n_cols, const int2* corners, const int32_t* idx, int count, int n_pos,
                     const float2* contrib, const float* w0, int MS, const double* part, double* phi_pos,
                     double* gn_pos, int slots = 0, ApplyShape shape = kApplyShapes[0]) {
  ApplyArgs P{};
  P.z = z;
  P.n_rows = n_rows;
  P.n_cols = n_cols;
  P.corners = corners;
  P.idx = idx;
  P.count = count;
  P.n_pos = n_pos;
  P.contrib = contrib;
  P.w0 = w0;
  P.MS = MS;
  P.part = part;
  P.slots = slots ? slots : cluster_of(MS);  // default: one per block of the window kernel
  P.phi_pos = phi_pos;
  P.gn_pos = gn_pos;
  P.tiles_x = (n_cols + shape.tw - 1) / shape.tw;
  P.tiles_y = (n_rows + shape.th - 1) / shape.th;
  P.block0 = 0;
  return P;
}

int apply_tiles(const ApplyArgs& P) { return P.tiles_x * P.tiles_y; }

cudaError_t launch_apply(float2* z, int n_rows, int n_cols, const int2* corners, const int32_t* idx, int count,
                         int n_pos, const float2* contrib, const float* w0, int MS, const double* part,
                         double* phi_pos, double* gn_pos, cudaStream_t st, int slots = 0) {
  const ApplyArgs P =
      apply_args(z, n_rows, n_cols, corners, idx, count, n_pos, contrib, w0, MS, part, phi_pos, gn_pos, slots);
  const dim3 tiles(P.tiles_x, (n_rows + kApplyTile - 1) / kApplyTile);
  return launch_ex(apply_kernel, tiles, dim3(256), (sizeof(int2) + sizeof(int)) * count, st, 1, true, P);
}

template <int MODE>
cudaError_t launch_window_m(int MS, const StepArgs& a, int blocks, cudaStream_t st) {
  switch (MS) {
#define MAGPIE_CASE(S) \
  case S:              \
    return window_launch<S>(MODE, a, blocks, st);
    MAGPIE_WINDOW_SIZES(MAGPIE_CASE)
#undef MAGPIE_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <int MODE>
cudaError_t launch_window_batched_m(int MS, const StepArgs* table, const int2* map, int windows, cudaStream_t st,
                                    int minb) {
  static_assert(MODE == kStep, "batched windows run minibatch steps");
  switch (MS) {
#define MAGPIE_CASE(S) \
  case S:              \
    return window_launch_batched<S>(table, map, windows, st, minb);
    MAGPIE_WINDOW_SIZES(MAGPIE_CASE)
#undef MAGPIE_CASE
    default: return cudaErrorInvalidValue;
  }
}

// The three register bounds the autotuner tries for window side MS (c[3];
// equal entries are one candidate).
void minb_candidates(int MS, int* c) {
  switch (MS) {
#define MAGPIE_CASE(S)               \
  case S:                            \
    window_minb_candidates<S>(c);    \
    return;
    MAGPIE_WINDOW_SIZES(MAGPIE_CASE)
#undef MAGPIE_CASE
    default: c[0] = c[1] = c[2] = 1;
  }
}

cudaError_t prepare_kernels(int MS) {
  cudaError_t e = cudaFuncSetAttribute(apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((sizeof(int2) + sizeof(int)) * kMaxMinibatch));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(apply_tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((sizeof(int2) + sizeof(int)) * kMaxMinibatch));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(apply_kernel_batched<16, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((sizeof(int2) + sizeof(int)) * kMaxMinibatch));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(apply_kernel_batched<32, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((sizeof(int2) + sizeof(int)) * kMaxMinibatch));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(apply_kernel_batched<32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((sizeof(int2) + sizeof(int)) * kMaxMinibatch));
  if (e == cudaSuccess && MS <= 128)
    e = cudaFuncSetAttribute(vcycle_up_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * sizeof(float2) * (size_t)up_off(128, 8)));
  if (e == cudaSuccess && MS >= 64)
    e = cudaFuncSetAttribute(vcycle_up_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float2) * (size_t)up_off(MS, ilog2(MS) + 1)));
  if (e != cudaSuccess) return e;
  switch (MS) {
#define MAGPIE_CASE(S) \
  case S:              \
    return window_prepare<S>();
    MAGPIE_WINDOW_SIZES(MAGPIE_CASE)
#undef MAGPIE_CASE
    default: return cudaErrorInvalidValue;
  }
}

int check_positions(const int32_t* host_pos, int n_pos, int n_rows, int n_cols, int m) {
  for (int k = 0; k < n_pos; ++k) {
    const int r = host_pos[2 * k], c = host_pos[2 * k + 1];
    if (r < 0 || c < 0 || r > n_rows - m || c > n_cols - m)
      return fail(MAGPIE_EINVAL, "position " + std::to_string(k) + " = (" + std::to_string(r) + ", " +
                                     std::to_string(c) + ") puts the window outside the object");
  }
  return MAGPIE_OK;
}

// ------------------------------------------------------------- context groups
struct GroupWindowLaunch {
  int ms;       // window side of this launch
  int map_off;  // first entry of its cluster map
  int windows;  // windows (clusters) in the launch
};
struct GroupApplyLaunch {
  int tab_off;    // first entry of its problem table
  int n;          // problems in the launch
  int blocks;     // total tiles
  int max_count;  // largest window count (shared memory)
};
// One launch of the persistent form: the members of one window side at one
// batched step, their windows and then their update tiles.
struct GroupPersistLaunch {
  int ms;         // window side
  int map_off;    // first window item (entries of the group's map and wmember)
  int nw;         // window items
  int tab_off;    // first entry of its update table
  int na;         // members
  int ntiles;     // update tiles
  int q_off;      // its queue counter in the counter buffer, followed by na done counters
  int max_count;  // largest window count of its members
  int clusters;   // its grid (set by plan_persistent)
};

// threads per block of the window kernels of side m
int window_threads(int m) {
  switch (m) {
#define MAGPIE_CASE(S) \
  case S:              \
    return Geo<S>::T;
    MAGPIE_WINDOW_SIZES(MAGPIE_CASE)
#undef MAGPIE_CASE
    default: return 0;
  }
}

cudaError_t launch_persistent_m(int MS, const PersistArgs& P, int clusters, int max_count, cudaStream_t st, int minb) {
  switch (MS) {
#define MAGPIE_CASE(S) \
  case S:              \
    return window_launch_persistent<S>(P, clusters, max_count, st, minb);
    MAGPIE_WINDOW_SIZES(MAGPIE_CASE)
#undef MAGPIE_CASE
    default: return cudaErrorInvalidValue;
  }
}

int persistent_capacity_m(int MS, int max_count, int minb) {
  switch (MS) {
#define MAGPIE_CASE(S) \
  case S:              \
    return window_persistent_capacity<S>(max_count, minb);
    MAGPIE_WINDOW_SIZES(MAGPIE_CASE)
#undef MAGPIE_CASE
    default: return 0;
  }
}

}  // namespace magpie_impl

using namespace magpie_impl;

struct magpie_group {
  std::vector<magpie_ctx*> members;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  StepArgs* table = nullptr;    // one entry per (batched step, member)
  int2* map = nullptr;          // cluster -> (table entry, window slot)
  ApplyArgs* atable[3] = {};    // per apply tile shape: one entry per (batched step, member)
  std::vector<std::vector<GroupWindowLaunch>> wl;  // per batched step
  std::vector<GroupApplyLaunch> al[3];             // per apply tile shape, per batched step
  std::vector<ApplyArgs> atable_host[3];           // host copies (the autotuner's scratch tables)
  cudaGraphExec_t graph = nullptr;
  // autotuner: register bound (blocks per SM) of the batched window kernel
  // per window side m = 8 << i, and the measured ms per launch of batched
  // step 0 for the two candidates (0 where not measured)
  int minb[6] = {0, 0, 0, 0, 0, 0};
  float tune_ms[6][3] = {};
  // autotuner: tile shape of the update kernel (index into kApplyShapes) and
  // the measured ms per launch of batched step 0 for each shape
  int apply_shape = 0;
  float apply_ms[3] = {};
  // persistent form: per batched step, one launch per window side (the
  // sides' launches run concurrently), windows and updates from a work queue
  std::vector<std::vector<GroupPersistLaunch>> pl;  // per batched step
  std::vector<ApplyArgs> ptable_host;                // update tables of the persistent launches
  ApplyArgs* ptable = nullptr;
  int* wmember = nullptr;     // member (within its launch) of every window item, aligned with map
  int* qbuf = nullptr;        // queue and done counters of every launch, zeroed at the start of a sweep
  size_t qbuf_n = 0;
  int* err = nullptr;         // bit 3: a dependency wait of the persistent form ran out
  cudaStream_t side[6] = {};  // streams of the concurrent per-side launches (side[0] unused)
  cudaEvent_t fork = nullptr, join[6] = {};
  int persistent = 0;         // 1: sweeps use the persistent form (chosen by the autotuner)
  float form_ms[2] = {};      // autotuner: batched step 0 as separate launches (0) and persistent (1)
  unsigned long long limit_ns = 1000000000ull;  // bound of each dependency wait
};

// The network of the learned coarse correction with its training state.
struct magpie_cnn {
  int h = 0, max_batch = 0, P = 0;
  cudaStream_t stream = nullptr;
  int off[kCnnLayers] = {};         // parameter offset of each layer (weights, then biases)
  float* theta = nullptr;           // FP32 parameters
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  bf16* wbf = nullptr;              // BF16 copy read by the forward and backward kernels
  float* grad = nullptr;            // [P]
  bf16* act[kCnnLayers] = {};       // layer inputs: act[0] the BF16 network input, act[l] layer l-1's output
  float* y = nullptr;               // [max_batch][h][h][2] output of the last forward pass
  float* dz[2] = {};                // backward buffers
  float* dy = nullptr;              // [max_batch][h][h][2]
  float* part = nullptr;            // split-K and weight-gradient partial sums
  size_t part_n = 0;
  int last_batch = 0;               // batch of the last forward pass (backward's batch)
  long step = 0;                    // Adam steps taken
  int tensor_path = 1;              // convolutions: 1 tcgen05 (where the layer fits it), 0 mma.sync
  int* err = nullptr;               // bit 2: a bounded wait of a tcgen05 convolution ran out
};

struct magpie_ctx {
  magpie_params p{};
  int M = 0;
  float2* z = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  float2* Q = nullptr;
  float2* tw = nullptr;
  float* amp = nullptr;
  float* stage = nullptr;  // host-sweep intensity staging
  int32_t* pos = nullptr;
  float* pyr = nullptr;
  double2* pyr_q = nullptr;
  double* pyr_u = nullptr;
  float2* contrib = nullptr;
  float4* acc = nullptr;      // deterministic = 0: [n_rows][n_cols] atomic accumulators (N re, N im, D, 0)
  unsigned long long* stamps = nullptr;  // magpie_stage_times: per-stage timestamps of the window kernel
  double* phi_pos = nullptr;
  double* gn_pos = nullptr;
  double* part = nullptr;     // [n_pos][kMaxSlots][2] per-block partial sums
  int2* corner = nullptr;     // [minibatch] corners of a step's windows
  unsigned long long* mx = nullptr;  // max |Q|^2 (bits of a double)
  float2* pnum = nullptr;     // probe step: [minibatch][m][m]
  float* pa2 = nullptr;       // probe step: [minibatch][m][m]
  double* pmax = nullptr;     // probe step: [minibatch][kMaxCluster]
  int32_t* iota = nullptr;
  int32_t* order = nullptr;
  double* sums = nullptr;
  int* err = nullptr;
  float* wz = nullptr;        // W_z^l tables, l = 0 .. L-2 (coarse object of the learned correction)
  // learned coarse correction (when a network is attached)
  magpie_cnn* cnn = nullptr;
  float4* lx = nullptr;       // [minibatch][h][h] network input
  float* lscale = nullptr;    // [minibatch] RMS of the plain coarse step
  int* lacc = nullptr;        // [minibatch] 1 = learned V-cycle output kept
  double* lmargin = nullptr;  // [minibatch] surrogate(plain) - surrogate(learned)
  unsigned long long* lstats = nullptr;  // proposals, acceptances
  // paper variants: bit 0 the MG/OPT correction term, bit 1 the phase rule of Eq. (specification)
  int variant = 0;
  float2* phase = nullptr;    // [n_pos][m][m] unit phases of the last visit (phase rule)
  // precision form (tensor-core DFTs)
  int precision = 0;
  float2* pbuf = nullptr;     // [minibatch][m][m] exit wave / spectrum / revised exit wave
  float2* g1buf = nullptr;    // [minibatch][m/2][m/2] level-1 residual gradient, then increment
  float2* g2buf = nullptr;    // [minibatch][m/4][m/4] level-2 residual gradient (three levels or more)
  int* hand = nullptr;        // [3][minibatch] window hand-off counts of the transform kernels
  TcTables* tabs = nullptr;
  cudaGraphExec_t graph = nullptr;
  // pipelined host sweeps (magpie_sweep_host_async): two amplitude buffers,
  // their raw-intensity staging, a sweep graph per buffer, and per buffer the
  // events "data landed" and "sweep done with it"
  float* amp2[2] = {nullptr, nullptr};
  float* stage2[2] = {nullptr, nullptr};
  int32_t* order2[2] = {nullptr, nullptr};  // the permutation of each buffer's sweep
  int amp_raw = 0;                          // set while a sweep reading raw intensities is captured
  cudaGraphExec_t graph2[2] = {nullptr, nullptr};
  cudaEvent_t landed[2][4] = {};
  cudaEvent_t used[2] = {nullptr, nullptr};
  cudaStream_t copy2[4] = {};  // four chunks in flight (several copy engines)
  int next_buf = 0;
  std::vector<cudaEvent_t> events;  // 4 per minibatch step (magpie_profile_sweep)
  // host sweeps: chunked uploads of the intensities on several copy streams
  cudaStream_t copy_streams[4] = {};
  cudaEvent_t copy_done[4] = {};
  cudaEvent_t copy_start = nullptr;
};

namespace magpie_impl {

StepArgs make_args(magpie_ctx* c, const int32_t* idx) {
  StepArgs a{};
  a.z = c->z;
  a.n_rows = c->p.n_rows;
  a.n_cols = c->p.n_cols;
  a.Q = c->Q;
  a.tw = c->tw;
  a.amp = c->amp;
  a.amp_raw = c->amp_raw;
  a.out_int = nullptr;
  a.pos = c->pos;
  a.idx = idx;
  a.n_pos = c->p.n_pos;
  a.contrib = c->contrib;
  a.pyr = c->pyr;
  a.levels = c->p.levels;
  a.part = c->part;
  a.corner = c->corner;
  a.pnum = c->pnum;
  a.pa2 = c->pa2;
  a.pmax = c->pmax;
  a.err = c->err;
  a.phase = (c->variant & 2) ? c->phase : nullptr;
  a.stamps = c->stamps;
  return a;
}

// ------------------------------------------------- learned coarse correction
int cnn_side_in(int h, int l) {
  int s = h;
  for (int j = 0; j < l; ++j) s = s * kCnn[j].up / kCnn[j].stride;
  return s;
}
int cnn_side_out(int h, int l) { return cnn_side_in(h, l) * kCnn[l].up / kCnn[l].stride; }
int cnn_param_count() {
  int P = 0;
  for (int l = 0; l < kCnnLayers; ++l) P += kCnn[l].cout * 9 * kCnn[l].cin + kCnn[l].cout;
  return P;
}

struct ConvPlan {
  int gx, gy, splits, ksplit, bm, bn;
};

ConvPlan conv_plan(const ConvFwd& a) {
  ConvPlan pl{};
  pl.bn = a.Cout <= 8 ? 8 : (a.Cout <= 32 ? 32 : 64);
  pl.bm = pl.bn == 64 ? 64 : 128;
  const int Mtot = a.B * a.Ho * a.Ho;
  pl.gx = (Mtot + pl.bm - 1) / pl.bm;
  pl.gy = (a.Cout + pl.bn - 1) / pl.bn;
  const int ksteps = (a.K + 31) / 32;
  const int blocks = pl.gx * pl.gy;
  int splits = 1;
  if (a.Cin % 32 == 0 && blocks < 2 * 152) splits = std::max(1, std::min(ksteps / 4, (2 * 152 + blocks - 1) / blocks));
  const int per = (ksteps + splits - 1) / splits;
  pl.ksplit = per * 32;
  pl.splits = (ksteps + per - 1) / per;
  return pl;
}

// Layers the tcgen05 convolution serves: whole 64-element K steps inside one
// tap (Cin a multiple of 64) and whole 64-wide N tiles.
bool conv_tc_fits(const ConvFwd& a) { return a.Cin % 64 == 0 && a.Cout % 64 == 0; }
// Thin layers the direct FP32-FMA kernels serve: the network's first (4 -> 32,
// BF16 output) and last (64 -> 2) convolutions, with the alignment their
// 16-byte (8-byte) loads and stores need.
bool conv_direct_fits(const ConvFwd& a) {
  const auto al = [](const void* p, uintptr_t n) { return ((uintptr_t)p & (n - 1)) == 0; };
  if (a.Cin == 64 && a.Cout == 2) return al(a.in, 16);
  if (a.Cin == 4 && a.Cout == 32) return !a.out_f32 && al(a.in, 8) && al(a.out, 16);
  return false;
}

// Tiles of the tcgen05 convolution: 128 output pixels x 128 (or 64) output
// channels, K split so that about two blocks per SM run, at least two K steps
// of 64 per split.  (One block per SM with at least four K steps per split
// and 256-wide N tiles measured slower: 185 against 166 us for the network's
// forward pass at batch 64, h = 32; the blocks are latency-bound.)
ConvPlan conv_plan_tc(const ConvFwd& a) {
  ConvPlan pl{};
  pl.bn = a.Cout % 128 == 0 ? 128 : 64;
  pl.bm = kTcBM;
  const int Mtot = a.B * a.Ho * a.Ho;
  pl.gx = (Mtot + kTcBM - 1) / kTcBM;
  pl.gy = a.Cout / pl.bn;
  const int ksteps = a.K / kTcBK;
  const int blocks = pl.gx * pl.gy;
  const int splits = std::max(1, std::min(ksteps / 2, (2 * 152 + blocks - 1) / blocks));
  const int per = (ksteps + splits - 1) / splits;
  pl.ksplit = per * kTcBK;
  pl.splits = (ksteps + per - 1) / per;
  return pl;
}

// Pixel chunks of the weight-gradient GEMM of layer l (enough blocks to
// fill the GPU, at least 64 pixels per chunk).
struct WgradPlan {
  int gx, gy, chunks, chunk;
};
WgradPlan wgrad_plan(int h, int l, int B) {
  const CnnLayer& L = kCnn[l];
  const int Ho = cnn_side_out(h, l), npix = B * Ho * Ho;
  WgradPlan w{};
  w.gx = (9 * L.cin + 1 + 63) / 64;
  w.gy = (L.cout + 63) / 64;
  const int want = std::max(1, (2 * 152 + w.gx * w.gy - 1) / (w.gx * w.gy));
  w.chunks = std::max(1, std::min(want, npix / 64));
  w.chunk = (npix + w.chunks - 1) / w.chunks;
  w.chunks = (npix + w.chunk - 1) / w.chunk;
  return w;
}

// Partial-sum floats needed by any batch of 1 .. max_batch windows.
size_t cnn_part_floats(int h, int max_batch) {
  size_t n = 0;
  for (int B = 1; B <= max_batch; ++B)
  for (int l = 0; l < kCnnLayers; ++l) {
    const int Ho = cnn_side_out(h, l);
    ConvFwd a{};
    a.B = B;
    a.Ho = Ho;
    a.Cin = kCnn[l].cin;
    a.Cout = kCnn[l].cout;
    a.K = 9 * a.Cin;
    const ConvPlan pl = conv_plan(a);
    if (pl.splits > 1) n = std::max(n, (size_t)pl.splits * B * Ho * Ho * a.Cout);
    if (conv_tc_fits(a)) {
      const ConvPlan pt = conv_plan_tc(a);
      if (pt.splits > 1) n = std::max(n, (size_t)pt.splits * B * Ho * Ho * a.Cout);
    }
    const int P = a.Cout * 9 * a.Cin + a.Cout;
    n = std::max(n, (size_t)wgrad_plan(h, l, B).chunks * P);
  }
  return n;
}

cudaError_t launch_conv(const ConvFwd& a0, float* part, cudaStream_t st, int tensor_path = 0, int* err = nullptr) {
  ConvFwd a = a0;
  const bool tc = tensor_path == 1 && conv_tc_fits(a) && err;
  const ConvPlan pl = tc ? conv_plan_tc(a) : conv_plan(a);
  a.ksplit = pl.ksplit;
  a.part = pl.splits > 1 ? part : nullptr;
  const dim3 grid(pl.gx, pl.gy, pl.splits);
  if (tensor_path == 1 && conv_direct_fits(a)) {
    const long long pixels = (long long)a.B * a.Ho * a.Ho;
    if (a.Cin == 64) {  // 8 lanes per pixel
      conv_thin_out_kernel<64, 2><<<(int)((pixels * 8 + 255) / 256), 256, 0, st>>>(a);
    } else {  // 4 lanes per pixel
      conv_thin_in_kernel<4, 32><<<(int)((pixels * 4 + 255) / 256), 256, 0, st>>>(a);
    }
    return cudaGetLastError();
  }
  if (tc && pl.bn == 128)
    conv_fwd_tc_kernel<128><<<grid, 128, TcConv<128>::SMEM, st>>>(a, err);
  else if (tc)
    conv_fwd_tc_kernel<64><<<grid, 128, TcConv<64>::SMEM, st>>>(a, err);
  else if (pl.bn == 8)
    conv_fwd_kernel<128, 8><<<grid, 128, 0, st>>>(a);
  else if (pl.bn == 32)
    conv_fwd_kernel<128, 32><<<grid, 128, 0, st>>>(a);
  else
    conv_fwd_kernel<64, 64><<<grid, 128, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || pl.splits == 1) return e;
  const size_t n = (size_t)a.B * a.Ho * a.Ho * a.Cout;
  conv_splitk_kernel<<<(int)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(a, pl.splits);
  return cudaGetLastError();
}

// Forward pass of `batch` inputs x [batch][h][h][4] (float) into y [batch][h][h][2].
int cnn_enqueue_forward(magpie_cnn* n, const float* x, int batch, float* y, cudaStream_t st) {
  const int h = n->h;
  const size_t nx = (size_t)batch * h * h * 4;
  to_bf16_kernel<<<(int)std::min<size_t>((nx + 255) / 256, 4096), 256, 0, st>>>(x, n->act[0], nx);
  CUDA_TRY(cudaGetLastError());
  for (int l = 0; l < kCnnLayers; ++l) {
    const CnnLayer& L = kCnn[l];
    ConvFwd a{};
    a.in = n->act[l];
    a.w = n->wbf + n->off[l];
    a.bias = n->theta + n->off[l] + (size_t)L.cout * 9 * L.cin;
    a.out = l + 1 < kCnnLayers ? (void*)n->act[l + 1] : (void*)y;
    a.B = batch;
    a.Hin = cnn_side_in(h, l);
    a.Cin = L.cin;
    a.Cout = L.cout;
    a.stride = L.stride;
    a.up = L.up;
    a.Ho = cnn_side_out(h, l);
    a.relu = L.relu;
    a.out_f32 = l + 1 == kCnnLayers;
    a.K = 9 * L.cin;
    CUDA_TRY(launch_conv(a, n->part, st, n->tensor_path, n->err));
  }
  n->last_batch = batch;
  return MAGPIE_OK;
}

// Gradient of <dy, y> over the parameters, for the inputs of the last forward pass.
int cnn_enqueue_backward(magpie_cnn* n, const float* dy, float* grad, cudaStream_t st) {
  const int h = n->h, B = n->last_batch;
  const float* dz = dy;
  int cur = 0;
  for (int l = kCnnLayers - 1; l >= 0; --l) {
    const CnnLayer& L = kCnn[l];
    const int Hin = cnn_side_in(h, l), Ho = cnn_side_out(h, l);
    const int P = L.cout * 9 * L.cin + L.cout;
    const WgradPlan wp = wgrad_plan(h, l, B);
    conv_wgrad_kernel<<<dim3(wp.gx, wp.gy, wp.chunks), 256, 0, st>>>(dz, n->act[l], n->part, B, Hin, L.cin, L.cout,
                                                                      L.stride, L.up, Ho, wp.chunk);
    CUDA_TRY(cudaGetLastError());
    chunk_sum_kernel<<<(P + 255) / 256, 256, 0, st>>>(n->part, grad + n->off[l], P, wp.chunks);
    CUDA_TRY(cudaGetLastError());
    if (l > 0) {
      const size_t nx = (size_t)B * Hin * Hin * L.cin;
      conv_bwd_data_kernel<<<(int)std::min<size_t>((nx + 255) / 256, 8192), 256, 0, st>>>(
          dz, n->wbf + n->off[l], n->act[l], n->dz[cur], B, Hin, L.cin, L.cout, L.stride, L.up, Ho);
      CUDA_TRY(cudaGetLastError());
      dz = n->dz[cur];
      cur ^= 1;
    }
  }
  return MAGPIE_OK;
}

int cnn_enqueue_params(magpie_cnn* n, cudaStream_t st) {
  to_bf16_kernel<<<(n->P + 255) / 256, 256, 0, st>>>(n->theta, n->wbf, (size_t)n->P);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(n->adam_m, 0, sizeof(float) * n->P, st));
  CUDA_TRY(cudaMemsetAsync(n->adam_v, 0, sizeof(float) * n->P, st));
  n->step = 0;
  return MAGPIE_OK;
}

int learned_supported(const magpie_ctx* c, const magpie_cnn* n) {
  const int L = c->p.levels, m = c->p.m;
  if (L < 2) return fail(MAGPIE_EINVAL, "the learned correction needs levels >= 2");
  if (m > 128) return fail(MAGPIE_EUNSUPPORTED, "the learned correction supports m <= 128");
  if (c->p.update_probe) return fail(MAGPIE_EINVAL, "the learned correction needs update_probe = 0");
  if (n && n->h != (m >> (L - 1)))
    return fail(MAGPIE_EINVAL, "network side " + std::to_string(n->h) + " != m / 2^(levels-1) = " +
                                   std::to_string(m >> (L - 1)));
  if (n && n->max_batch < c->p.minibatch) return fail(MAGPIE_EINVAL, "network max_batch < minibatch");
  return MAGPIE_OK;
}

int learned_buffers(magpie_ctx* c) {
  if (c->lx) return MAGPIE_OK;
  const int h = c->p.m >> (c->p.levels - 1), B = c->p.minibatch;
  cudaError_t e = cudaMalloc((void**)&c->lx, sizeof(float4) * (size_t)B * h * h);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->lscale, sizeof(float) * B);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->lacc, sizeof(int) * B);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->lmargin, sizeof(double) * B);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->lstats, sizeof(unsigned long long) * 2);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->lstats, 0, sizeof(unsigned long long) * 2, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->lacc, 0, sizeof(int) * B, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->lmargin, 0, sizeof(double) * B, c->stream);
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? MAGPIE_ENOMEM : MAGPIE_ECUDA,
                std::string("learned buffers: ") + cudaGetErrorString(e));
  return MAGPIE_OK;
}

CoarseArgs coarse_args(magpie_ctx* c, const int32_t* idx, float4* x, float* scale) {
  CoarseArgs a{};
  a.z = c->z;
  a.n_cols = c->p.n_cols;
  a.pos = c->pos;
  a.idx = idx;
  a.n_pos = c->p.n_pos;
  a.MS = c->p.m;
  a.L = c->p.levels;
  a.g0 = c->contrib;
  a.pyr = c->pyr;
  a.wz = c->wz;
  a.x = x;
  a.scale = scale;
  return a;
}

size_t learned_up_smem(int MS, int L) { return 2 * sizeof(float2) * (size_t)up_off(MS, L); }

LearnedUpArgs up_args(magpie_ctx* c, const int32_t* idx) {
  LearnedUpArgs u{};
  u.idx = idx;
  u.n_pos = c->p.n_pos;
  u.MS = c->p.m;
  u.L = c->p.levels;
  u.contrib = c->contrib;
  u.pyr = c->pyr;
  return u;
}

// From g^0 in the increments: the network's input and scale, its forward
// pass, then the V-cycle with the kept coarse correction writes w^0 Delta
// back to the increments.
int enqueue_learned_tail(magpie_ctx* c, const int32_t* idx, int count, cudaStream_t st) {
  coarse_state_kernel<<<count, 1024, 0, st>>>(coarse_args(c, idx, c->lx, c->lscale));
  CUDA_TRY(cudaGetLastError());
  int rc = cnn_enqueue_forward(c->cnn, reinterpret_cast<const float*>(c->lx), count, c->cnn->y, st);
  if (rc) return rc;
  LearnedUpArgs u = up_args(c, idx);
  u.scale = c->lscale;
  u.y = c->cnn->y;
  u.accepted = c->lacc;
  u.margin = c->lmargin;
  u.stats = c->lstats;
  vcycle_up_kernel<true><<<count, 1024, learned_up_smem(c->p.m, c->p.levels), st>>>(u);
  CUDA_TRY(cudaGetLastError());
  return MAGPIE_OK;
}

// ----------------------------------------------------------- precision form
void build_tc_tables(int MS, TcTables& T) {
  const int QR = MS / 16;
  const double pi = 3.14159265358979323846;
  std::memset(&T, 0, sizeof(T));
  for (int inv = 0; inv < 2; ++inv) {
    const double sg = inv ? 1.0 : -1.0;
    for (int k = 0; k < 16; ++k)
      for (int n = 0; n < 16; ++n) {
        const double ph = 2.0 * pi * (double)((k * n) % 16) / 16.0;
        const float fr = (float)std::cos(ph), fi = (float)(sg * std::sin(ph));
        T.f16[inv][k * 32 + n] = fr;
        T.f16[inv][k * 32 + 16 + n] = -fi;
        T.f16[inv][(16 + k) * 32 + n] = fi;
        T.f16[inv][(16 + k) * 32 + 16 + n] = fr;
      }
    for (int n2 = 0; n2 < QR; ++n2)
      for (int k2 = 0; k2 < QR; ++k2) {
        const double ph = 2.0 * pi * (double)((n2 * k2) % QR) / (double)QR;
        const float fr = (float)std::cos(ph), fi = (float)(sg * std::sin(ph));
        T.fq[inv][n2 * 32 + k2] = fr;
        T.fq[inv][(QR + n2) * 32 + k2] = -fi;
        T.fq[inv][n2 * 32 + QR + k2] = fi;
        T.fq[inv][(QR + n2) * 32 + QR + k2] = fr;
      }
  }
}

// Dynamic shared memory of the tcgen05 transform kernels (their operand
// buffers, on top of the lines' static 15-42 KB), set once per process.
template <int MS>
cudaError_t prepare_dft_umma() {
  static cudaError_t done = [] {
    const int b = kUmmaDftSmem;
    cudaError_t e = cudaFuncSetAttribute(dft_tc_kernel<MS, 0, 0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(dft_tc_kernel<MS, 1, 0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(dft_tc_kernel<MS, 0, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(dft_tc_kernel<MS, 1, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(exit_dft_kernel<MS, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(project_dft_kernel<MS, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(grad_dft_kernel<MS, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return e;
  }();
  return done;
}

// path 0: register-fragment (mma.sync) transforms; 1: tcgen05 transforms
// (err: bit 4 set when one of their bounded waits ran out).
template <int MS, int PATH>
cudaError_t launch_dft2_tc_p(float2* buf, int count, const TcTables* tabs, const float2* tw, int inv, cudaStream_t st,
                             int* err) {
  const dim3 grid((unsigned)count * (MS / kTcLines));
  const size_t smem = PATH ? kUmmaDftSmem : 0;
  if (inv) {
    dft_tc_kernel<MS, 1, 1, PATH><<<grid, 128, smem, st>>>(buf, tabs, tw, 1.f, err);
    dft_tc_kernel<MS, 0, 1, PATH><<<grid, 128, smem, st>>>(buf, tabs, tw, 1.f, err);
  } else {
    dft_tc_kernel<MS, 0, 0, PATH><<<grid, 128, smem, st>>>(buf, tabs, tw, 1.f, err);
    dft_tc_kernel<MS, 1, 0, PATH><<<grid, 128, smem, st>>>(buf, tabs, tw, 1.f, err);
  }
  return cudaGetLastError();
}

template <int MS>
cudaError_t launch_dft2_tc(float2* buf, int count, const TcTables* tabs, const float2* tw, int inv, cudaStream_t st,
                           int path, int* err) {
  if (path) {
    const cudaError_t e = prepare_dft_umma<MS>();
    if (e != cudaSuccess) return e;
    return launch_dft2_tc_p<MS, 1>(buf, count, tabs, tw, inv, st, err);
  }
  return launch_dft2_tc_p<MS, 0>(buf, count, tabs, tw, inv, st, err);
}

cudaError_t launch_dft2_tc_m(int MS, float2* buf, int count, const TcTables* tabs, const float2* tw, int inv,
                             cudaStream_t st, int path = 0, int* err = nullptr) {
  switch (MS) {
    case 64: return launch_dft2_tc<64>(buf, count, tabs, tw, inv, st, path, err);
    case 128: return launch_dft2_tc<128>(buf, count, tabs, tw, inv, st, path, err);
    case 256: return launch_dft2_tc<256>(buf, count, tabs, tw, inv, st, path, err);
    default: return cudaErrorInvalidValue;
  }
}

// Exit waves, tensor-core DFTs, projection, inverse DFTs and g^0 into the
// increments (with the per-tile partial sums and the windows' corners).
PrecArgs precision_args(magpie_ctx* c, const int32_t* idx, int count) {
  PrecArgs a{};
  a.z = c->z;
  a.n_cols = c->p.n_cols;
  a.Q = c->Q;
  a.amp = c->amp;
  a.pos = c->pos;
  a.idx = idx;
  a.n_pos = c->p.n_pos;
  a.MS = c->p.m;
  a.T = c->p.m / kTcLines;
  a.buf = c->pbuf;
  a.contrib = c->contrib;
  a.part = c->part;
  a.corner = c->corner;
  a.err = c->err;
  a.phase = (c->variant & 2) ? c->phase : nullptr;
  a.g1 = (c->p.levels >= 2 && !c->cnn) ? c->g1buf : nullptr;
  a.g2 = (c->p.levels >= 3 && !c->cnn) ? c->g2buf : nullptr;
  a.count = count;
  a.hand = c->hand;
  a.wait_bias = 0;
  a.wait_ns = kHandoffNs;
  a.pyr = c->pyr;
  a.L = c->p.levels;
  return a;
}

template <int MS>
cudaError_t launch_precision_g0(const PrecArgs& a, int count, const TcTables* tabs, const float2* tw,
                                cudaStream_t st, int path) {
  const dim3 grid((unsigned)count * (MS / kTcLines));
  // each a programmatic dependent of the kernel before it: the exit kernel
  // waits for the previous step to complete, the others take their windows
  // from the kernel before them one by one (PrecArgs::hand)
  if (path) {
    cudaError_t e = prepare_dft_umma<MS>();
    if (e == cudaSuccess)
      e = launch_ex(exit_dft_kernel<MS, 1>, grid, dim3(128), kUmmaDftSmem, st, 1, true, a, tabs, tw);
    if (e == cudaSuccess)
      e = launch_ex(project_dft_kernel<MS, 1>, grid, dim3(128), kUmmaDftSmem, st, 1, true, a, tabs, tw);
    if (e == cudaSuccess)
      e = launch_ex(grad_dft_kernel<MS, 1>, grid, dim3(128), kUmmaDftSmem, st, 1, true, a, tabs, tw);
    return e;
  }
  cudaError_t e = launch_ex(exit_dft_kernel<MS, 0>, grid, dim3(128), 0, st, 1, true, a, tabs, tw);
  if (e == cudaSuccess) e = launch_ex(project_dft_kernel<MS, 0>, grid, dim3(128), 0, st, 1, true, a, tabs, tw);
  if (e == cudaSuccess) e = launch_ex(grad_dft_kernel<MS, 0>, grid, dim3(128), 0, st, 1, true, a, tabs, tw);
  return e;
}

// The precision form's coarse levels (three levels or more), four blocks
// per window, a programmatic dependent of the gradient kernel.
cudaError_t launch_coarse_cycle(const PrecArgs& a, int count, int levels, cudaStream_t st) {
  int o = 0;
  for (int j = 2; j < levels; ++j) o += (a.MS >> j) * (a.MS >> j);
  const dim3 grid((unsigned)count, kCoarseSplit);
  const size_t smem = sizeof(float2) * (size_t)o;
  switch (a.MS) {
    case 64: return launch_ex(coarse_cycle_kernel<64>, grid, dim3(1024), smem, st, 1, true, a);
    case 128: return launch_ex(coarse_cycle_kernel<128>, grid, dim3(1024), smem, st, 1, true, a);
    case 256: return launch_ex(coarse_cycle_kernel<256>, grid, dim3(1024), smem, st, 1, true, a);
    default: return cudaErrorInvalidValue;
  }
}

int enqueue_precision_g0(magpie_ctx* c, const PrecArgs& a, int count, cudaStream_t st) {
  switch (a.MS) {
    case 64: CUDA_TRY(launch_precision_g0<64>(a, count, c->tabs, c->tw, st, c->precision == 2)); break;
    case 128: CUDA_TRY(launch_precision_g0<128>(a, count, c->tabs, c->tw, st, c->precision == 2)); break;
    case 256: CUDA_TRY(launch_precision_g0<256>(a, count, c->tabs, c->tw, st, c->precision == 2)); break;
    default: return fail(MAGPIE_EUNSUPPORTED, "the precision form needs m = 64, 128 or 256");
  }
  return MAGPIE_OK;
}
int enqueue_precision_g0(magpie_ctx* c, const int32_t* idx, int count, cudaStream_t st) {
  return enqueue_precision_g0(c, precision_args(c, idx, count), count, st);
}

// ev (optional): four events recorded before/after the window kernel and
// before/after the apply kernel.
int enqueue_step(magpie_ctx* c, const int32_t* idx, int count, cudaStream_t st, const cudaEvent_t* ev = nullptr) {
  NvtxRange range("magpie minibatch step");
  StepArgs a = make_args(c, idx);
  // the float-atomic update serves the FP32 window kernel without the phase
  // rule or the learned correction; every other form uses the ordered one
  const bool atom = c->acc && !c->precision && !c->cnn && !a.phase;
  if (ev) CUDA_TRY(cudaEventRecord(ev[0], st));
  int rc = MAGPIE_OK;
  if (c->precision) {
    rc = enqueue_precision_g0(c, idx, count, st);
    if (!rc && c->cnn) {
      rc = enqueue_learned_tail(c, idx, count, st);
    } else if (!rc && c->p.levels >= 2) {
      // the V-cycle above g^0 (g^1 and g^2 already restricted by the
      // gradient kernel): levels 1 .. L-1 on four blocks per window; the
      // finest level is formed by the update kernel as it sums the windows
      const PrecArgs v = precision_args(c, idx, count);
      if (c->p.levels >= 3) CUDA_TRY(launch_coarse_cycle(v, count, c->p.levels, st));
    }
  } else {
    a.grad_only = c->cnn ? 1 : 0;
    if (a.phase) {
      CUDA_TRY(launch_window_m<kStepRecycle>(c->p.m, a, count, st));
    } else if (atom) {
      a.acc = c->acc;
      CUDA_TRY(launch_window_m<kStepAtomic>(c->p.m, a, count, st));
    } else {
      CUDA_TRY(launch_window_m<kStep>(c->p.m, a, count, st));
    }
    if (c->cnn) rc = enqueue_learned_tail(c, idx, count, st);
  }
  if (rc) return rc;
  if (ev) CUDA_TRY(cudaEventRecord(ev[1], st));
  if (ev) CUDA_TRY(cudaEventRecord(ev[2], st));
  if (atom) {
    const size_t npix = (size_t)c->p.n_rows * c->p.n_cols;
    const unsigned blocks = (unsigned)std::min<size_t>((npix + 255) / 256, 152 * 8);
    CUDA_TRY(launch_ex(accum_apply_kernel, dim3(blocks), dim3(256), 0, st, 1, true, c->z, c->acc, npix, idx, count,
                       c->p.n_pos, (const double*)c->part, cluster_of(c->p.m), c->p.m, c->phi_pos, c->gn_pos));
  } else if (c->precision && !c->cnn && c->p.levels >= 2) {
    // contrib holds g^0 and g1buf e^1: the update forms w . Delta from them
    ApplyArgs P = apply_args(c->z, c->p.n_rows, c->p.n_cols, c->corner, idx, count, c->p.n_pos, c->contrib,
                             c->pyr + c->M, c->p.m, c->part, c->phi_pos, c->gn_pos, c->p.m / kTcLines);
    P.e1 = c->g1buf;
    P.u0 = c->pyr;
    P.hand = c->hand;
    P.nhand = 3 * count;
    const dim3 tiles(P.tiles_x, (c->p.n_rows + kApplyTile - 1) / kApplyTile);
    CUDA_TRY(launch_ex(apply_tail_kernel, tiles, dim3(256), (sizeof(int2) + sizeof(int)) * count, st, 1, true, P));
  } else {
    ApplyArgs P = apply_args(c->z, c->p.n_rows, c->p.n_cols, c->corner, idx, count, c->p.n_pos, c->contrib,
                             c->pyr + c->M, c->p.m, c->part, c->phi_pos, c->gn_pos,
                             c->precision ? c->p.m / kTcLines : 0);
    if (c->precision) {  // the transform kernels' hand-off counts
      P.hand = c->hand;
      P.nhand = 3 * count;
    }
    const dim3 tiles(P.tiles_x, (c->p.n_rows + kApplyTile - 1) / kApplyTile);
    CUDA_TRY(launch_ex(apply_kernel, tiles, dim3(256), (sizeof(int2) + sizeof(int)) * count, st, 1, true, P));
  }
  if (c->p.update_probe) {
    probe_apply_kernel<<<(c->M + 255) / 256, 256, 0, st>>>(c->Q, c->M, idx, count, c->p.n_pos, c->pnum, c->pa2,
                                                           c->pmax, cluster_of(c->p.m), c->p.beta);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(enqueue_pyramid(c->Q, c->p.m, c->p.levels, c->p.alpha, c->mx, c->pyr_q, c->pyr_u, c->pyr, st,
                             c->variant & 1));
  }
  if (ev) CUDA_TRY(cudaEventRecord(ev[3], st));
  return MAGPIE_OK;
}

int build_pyramid(magpie_ctx* c, const void* probe) {
  CUDA_TRY(cudaMemcpyAsync(c->Q, probe, sizeof(float2) * c->M, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(enqueue_pyramid(c->Q, c->p.m, c->p.levels, c->p.alpha, c->mx, c->pyr_q, c->pyr_u, c->pyr, c->stream,
                           c->variant & 1));
  if (c->wz) {
    wz_kernel<<<std::max(1, c->M / 256), 256, 0, c->stream>>>(c->Q, c->p.m, c->p.levels, c->wz);
    CUDA_TRY(cudaGetLastError());
  }
  return MAGPIE_OK;
}

int read_err(magpie_ctx* c) {
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (h) {
    CUDA_TRY(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    if (h & 16) return fail(MAGPIE_ETIMEOUT, "a bounded wait of a tcgen05 transform ran out");
    return fail(MAGPIE_EINDEX, "a window index passed to a step or sweep was outside [0, n_pos)");
  }
  return MAGPIE_OK;
}

int evaluate(magpie_ctx* c, double* phi, double* stop) {
  StepArgs a = make_args(c, c->iota);
  CUDA_TRY(launch_window_m<kEval>(c->p.m, a, c->p.n_pos, c->stream));
  reduce_kernel<<<1, 1024, 0, c->stream>>>(c->part, cluster_of(c->p.m), c->p.m, c->p.n_pos, c->phi_pos, c->gn_pos,
                                           c->sums);
  CUDA_TRY(cudaGetLastError());
  double h[2];
  CUDA_TRY(cudaMemcpyAsync(h, c->sums, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  int rc = read_err(c);
  if (rc) return rc;
  if (phi) *phi = h[0];
  if (stop) *stop = h[1] / ((double)c->p.n_pos * (double)c->p.m);
  return MAGPIE_OK;
}

int n_steps(const magpie_ctx* c) { return (c->p.n_pos + c->p.minibatch - 1) / c->p.minibatch; }

// Drops the captured sweep graphs (their launches bake in the context's mode).
void invalidate_graphs(magpie_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  for (int b = 0; b < 2; ++b) {
    if (c->graph2[b]) cudaGraphExecDestroy(c->graph2[b]);
    c->graph2[b] = nullptr;
  }
}

// Captures the graph of one sweep over the permutation in c->order.
int capture_sweep(magpie_ctx* c, cudaGraphExec_t* out) {
  const int N = c->p.n_pos, B = c->p.minibatch;
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = MAGPIE_OK;
  for (int s = 0; s < N && rc == MAGPIE_OK; s += B)
    rc = enqueue_step(c, c->order + s, N - s < B ? N - s : B, c->cap_stream);
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  CUDA_TRY(e);
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  CUDA_TRY(e);
  return MAGPIE_OK;
}

// Replays (capturing it on first use) the graph of one sweep over the
// permutation already in c->order.
int launch_sweep(magpie_ctx* c) {
  if (!c->graph) {
    const int rc = capture_sweep(c, &c->graph);
    if (rc) return rc;
  }
  CUDA_TRY(cudaGraphLaunch(c->graph, c->stream));
  return MAGPIE_OK;
}

int validate(const magpie_params* p) {
  if (!p) return fail(MAGPIE_EINVAL, "params is NULL");
  if (p->m < 1 || (p->m & (p->m - 1)))
    return fail(MAGPIE_EINVAL, "m = " + std::to_string(p->m) + " is not a power of two");
  if (!supported_m(p->m))
    return fail(MAGPIE_EUNSUPPORTED, "no kernel for m = " + std::to_string(p->m) + " (8..256)");
  if (p->n_rows < p->m || p->n_cols < p->m) return fail(MAGPIE_EINVAL, "object smaller than the window");
  if ((long long)p->n_rows * p->n_cols > (1LL << 30)) return fail(MAGPIE_EINVAL, "object larger than 2^30 pixels");
  if (p->n_pos < 1) return fail(MAGPIE_EINVAL, "n_pos < 1");
  if (p->levels < 1 || p->levels > ilog2(p->m) + 1)
    return fail(MAGPIE_EINVAL, "levels must lie in [1, log2(m) + 1]");
  if (p->minibatch < 1 || p->minibatch > p->n_pos || p->minibatch > kMaxMinibatch)
    return fail(MAGPIE_EINVAL, "minibatch must lie in [1, min(n_pos, 4096)]");
  if (!(p->alpha >= 0.f) || !std::isfinite(p->alpha)) return fail(MAGPIE_EINVAL, "alpha must be finite and >= 0");
  if (p->update_probe != 0 && p->update_probe != 1) return fail(MAGPIE_EINVAL, "update_probe must be 0 or 1");
  if (p->update_probe && (!(p->beta >= 0.f) || !std::isfinite(p->beta)))
    return fail(MAGPIE_EINVAL, "beta must be finite and >= 0");
  if (p->deterministic != 0 && p->deterministic != 1) return fail(MAGPIE_EINVAL, "deterministic must be 0 or 1");
  return MAGPIE_OK;
}


// ------------------------------------------------ minibatch step without allocation
// Fixed scratch for magpie_step_noalloc, shared by every call in the process
// (one copy per GPU that loads the library, held until exit).
constexpr size_t kNoAllocMaxIncrement = size_t(1) << 20;  // count * m^2 complex values
constexpr size_t kNoAllocContribBytes = kNoAllocMaxIncrement * sizeof(float2);                      // 8 MiB
constexpr size_t kNoAllocPyrBytes = sizeof(float) * 3 * 128 * 128;                                 // level factors
constexpr size_t kNoAllocPyrQBytes = sizeof(double2) * 2 * 128 * 128;                              // FP64 probe levels
constexpr size_t kNoAllocPyrUBytes = sizeof(double) * 2 * 128 * 128;                               // FP64 u levels
constexpr size_t kNoAllocTwBytes = sizeof(float2) * 128;
constexpr size_t kNoAllocIdxBytes = sizeof(int32_t) * kMaxMinibatch;
constexpr size_t kNoAllocPartBytes = sizeof(double) * 2 * kMaxCluster * kMaxMinibatch;              // 512 KiB
constexpr size_t kNoAllocBytes = kNoAllocContribBytes + kNoAllocPyrBytes + kNoAllocPyrQBytes + kNoAllocPyrUBytes +
                                 kNoAllocTwBytes + kNoAllocIdxBytes + kNoAllocPartBytes + 8 + sizeof(int2) * kMaxMinibatch + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// idx -> sanitized copy: a window whose index is outside [0, n_pos) or whose
// corner puts it outside the object becomes -1 (skipped by the step kernels)
// and sets bit 0 of *err.
__global__ void sanitize_idx_kernel(const int32_t* idx, int count, const int32_t* pos, int n_pos, int n_rows,
                                    int n_cols, int m, int32_t* out, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  int k = idx[i];
  bool ok = (unsigned)k < (unsigned)n_pos;
  if (ok) {
    const int r = pos[2 * k], c = pos[2 * k + 1];
    ok = r >= 0 && c >= 0 && r <= n_rows - m && c <= n_cols - m;
  }
  if (!ok) {
    k = -1;
    atomicOr(err, 1);
  }
  out[i] = k;
}

struct NoAllocScratch {
  float2* contrib;
  float* pyr;
  double2* pyr_q;
  double* pyr_u;
  float2* tw;
  int32_t* idx;
  double* part;
  unsigned long long* mx;
  int2* corner;
  int* err;
};

// Per-device base address of g_noalloc_scratch, looked up once per device
// with that device current (host code may not use the symbol's own address).
int noalloc_scratch(NoAllocScratch* out) {
  constexpr int kMaxDevices = 64;
  static unsigned char* base[kMaxDevices] = {};
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(MAGPIE_EUNSUPPORTED, "device ordinal beyond 63");
  if (!base[dev]) {
    void* p = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    base[dev] = (unsigned char*)p;
  }
  unsigned char* b = base[dev];
  out->contrib = (float2*)b;
  b += kNoAllocContribBytes;
  out->pyr = (float*)b;
  b += kNoAllocPyrBytes;
  out->pyr_q = (double2*)b;
  b += kNoAllocPyrQBytes;
  out->pyr_u = (double*)b;
  b += kNoAllocPyrUBytes;
  out->tw = (float2*)b;
  b += kNoAllocTwBytes;
  out->idx = (int32_t*)b;
  b += kNoAllocIdxBytes;
  out->part = (double*)b;
  b += kNoAllocPartBytes;
  out->mx = (unsigned long long*)b;
  b += 8;
  out->corner = (int2*)b;
  b += sizeof(int2) * kMaxMinibatch;
  out->err = (int*)b;
  return MAGPIE_OK;
}

}  // namespace magpie_impl


// The update of batched step t with apply tile shape v, from the device table
// `table` (default: the group's own table of that shape).
cudaError_t launch_apply_batched(magpie_group* g, int v, int t, cudaStream_t st, const ApplyArgs* table = nullptr) {
  const GroupApplyLaunch& A = g->al[v][t];
  const ApplyArgs* tab = table ? table : g->atable[v] + A.tab_off;
  const size_t smem = (sizeof(int2) + sizeof(int)) * A.max_count;
  switch (v) {
    case 0: apply_kernel_batched<16, 16><<<A.blocks, 256, smem, st>>>(tab, A.n); break;
    case 1: apply_kernel_batched<32, 8><<<A.blocks, 256, smem, st>>>(tab, A.n); break;
    case 2: apply_kernel_batched<32, 32><<<A.blocks, 256, smem, st>>>(tab, A.n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Times every apply tile shape on batched step 0 (one warm-up, then three
// launches each), with every member's object replaced by a scratch copy so
// that the members' objects are not touched, and keeps the fastest.
int group_tune_apply(magpie_group* g, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  if (g->al[0].empty()) return MAGPIE_OK;
  size_t total = 0;
  for (auto* c : g->members) total += (size_t)c->p.n_rows * c->p.n_cols;
  float2* scratch = nullptr;
  ApplyArgs* tab = nullptr;
  cudaError_t e = cudaMalloc(&scratch, sizeof(float2) * total);
  if (e == cudaSuccess) e = cudaMalloc(&tab, sizeof(ApplyArgs) * g->members.size());
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, sizeof(float2) * total, st);
  float best = 0.f;
  for (int v = 0; v < 3 && e == cudaSuccess; ++v) {
    const GroupApplyLaunch& A = g->al[v][0];
    std::vector<ApplyArgs> at(g->atable_host[v].begin() + A.tab_off, g->atable_host[v].begin() + A.tab_off + A.n);
    size_t off = 0;
    for (auto& P : at) {
      P.z = scratch + off;
      off += (size_t)P.n_rows * P.n_cols;
    }
    e = cudaMemcpyAsync(tab, at.data(), sizeof(ApplyArgs) * at.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_apply_batched(g, v, 0, st, tab);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_apply_batched(g, v, 0, st, tab);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    g->apply_ms[v] = ms / 3.f;
    if (e == cudaSuccess && (v == 0 || ms / 3.f < best)) {
      best = ms / 3.f;
      g->apply_shape = v;
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (scratch) cudaFree(scratch);
  if (tab) cudaFree(tab);
  if (e != cudaSuccess) return fail(MAGPIE_ECUDA, std::string("group autotuner (update): ") + cudaGetErrorString(e));
  return MAGPIE_OK;
}

// Grid of every launch of the persistent form: as many clusters as fit on
// the GPU at once with the side's register bound, at most one per item.
// Called outside stream capture (the occupancy queries).
int plan_persistent(magpie_group* g) {
  for (auto& Ls : g->pl)
    for (auto& L : Ls) {
      const int CL = cluster_of(L.ms);
      const int items = L.nw + (L.ntiles + CL - 1) / CL;
      const int cap = persistent_capacity_m(L.ms, L.max_count, g->minb[ilog2(L.ms) - 3]);
      if (cap < 1) return fail(MAGPIE_ECUDA, "persistent step kernel: no cluster of it fits on the GPU");
      L.clusters = std::min(cap, items);
    }
  return MAGPIE_OK;
}

// Batched step t of the persistent form on stream st: one launch per window
// side, forked onto the group's side streams and joined back so that the
// sides run concurrently.  ptab: the update table (the group's own, or the
// autotuner's scratch copy); bias: added to every dependency-wait target.
// The step's counters in qbuf must be zero.
int enqueue_persistent_step(magpie_group* g, size_t t, cudaStream_t st, const ApplyArgs* ptab, int bias) {
  const auto& Ls = g->pl[t];
  if (Ls.size() > 1) CUDA_TRY(cudaEventRecord(g->fork, st));
  for (size_t j = 0; j < Ls.size(); ++j) {
    const GroupPersistLaunch& L = Ls[j];
    cudaStream_t s = j == 0 ? st : g->side[j];
    if (j > 0) CUDA_TRY(cudaStreamWaitEvent(s, g->fork, 0));
    PersistArgs P{};
    P.table = g->table;
    P.map = g->map + L.map_off;
    P.wmember = g->wmember + L.map_off;
    P.atab = ptab + L.tab_off;
    P.nw = L.nw;
    P.na = L.na;
    P.ntiles = L.ntiles;
    P.head = g->qbuf + L.q_off;
    P.done = P.head + 1;
    P.err = g->err;
    P.limit_ns = g->limit_ns;
    P.bias = bias;
    CUDA_TRY(launch_persistent_m(L.ms, P, L.clusters, L.max_count, s, g->minb[ilog2(L.ms) - 3]));
    if (j > 0) {
      CUDA_TRY(cudaEventRecord(g->join[j], s));
      CUDA_TRY(cudaStreamWaitEvent(st, g->join[j], 0));
    }
  }
  return MAGPIE_OK;
}

// Times batched step 0 as separate launches (the batched window kernels and
// the update kernel with the tuned tile shape) and in the persistent form,
// one warm-up and three timed runs each, with the updates writing scratch
// copies of the members' objects, and keeps the faster form for the sweeps.
int group_tune_form(magpie_group* g, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  if (g->pl.empty() || g->al[0].empty() || g->wl.empty()) return MAGPIE_OK;
  int rc = plan_persistent(g);
  if (rc) return rc;
  size_t total = 0;
  for (auto* c : g->members) total += (size_t)c->p.n_rows * c->p.n_cols;
  const GroupApplyLaunch& A = g->al[g->apply_shape][0];
  int np = 0;
  for (const auto& L : g->pl[0]) np = std::max(np, L.tab_off + L.na);
  float2* scratch = nullptr;
  ApplyArgs *atab = nullptr, *ptab = nullptr;
  cudaError_t e = cudaMalloc(&scratch, sizeof(float2) * total);
  if (e == cudaSuccess) e = cudaMalloc(&atab, sizeof(ApplyArgs) * A.n);
  if (e == cudaSuccess) e = cudaMalloc(&ptab, sizeof(ApplyArgs) * np);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, sizeof(float2) * total, st);
  std::vector<ApplyArgs> at(g->atable_host[g->apply_shape].begin() + A.tab_off,
                            g->atable_host[g->apply_shape].begin() + A.tab_off + A.n);
  std::vector<ApplyArgs> pt(g->ptable_host.begin(), g->ptable_host.begin() + np);
  for (auto* v : {&at, &pt}) {
    size_t off = 0;
    for (auto& P : *v) {
      P.z = scratch + off;
      off += (size_t)P.n_rows * P.n_cols;
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(atab, at.data(), sizeof(ApplyArgs) * at.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ptab, pt.data(), sizeof(ApplyArgs) * pt.size(), cudaMemcpyHostToDevice, st);
  auto run = [&](int form) -> int {
    if (form == 0) {
      for (const auto& L : g->wl[0]) {
        cudaError_t le = launch_window_batched_m<kStep>(L.ms, g->table, g->map + L.map_off, L.windows, st,
                                                        g->minb[ilog2(L.ms) - 3]);
        if (le != cudaSuccess) return fail(MAGPIE_ECUDA, std::string("group autotuner: ") + cudaGetErrorString(le));
      }
      CUDA_TRY(launch_apply_batched(g, g->apply_shape, 0, st, atab));
      return MAGPIE_OK;
    }
    CUDA_TRY(cudaMemsetAsync(g->qbuf, 0, sizeof(int) * g->qbuf_n, st));
    return enqueue_persistent_step(g, 0, st, ptab, 0);
  };
  for (int form = 0; form < 2 && e == cudaSuccess && !rc; ++form) {
    rc = run(form);
    if (!rc) e = cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && e == cudaSuccess && !rc; ++r) rc = run(form);
    if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    g->form_ms[form] = ms / 3.f;
  }
  if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(st);
  int h = 0;
  if (!rc && e == cudaSuccess) e = cudaMemcpy(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (scratch) cudaFree(scratch);
  if (atab) cudaFree(atab);
  if (ptab) cudaFree(ptab);
  if (rc) return rc;
  if (e != cudaSuccess) return fail(MAGPIE_ECUDA, std::string("group autotuner (form): ") + cudaGetErrorString(e));
  if (h) return fail(MAGPIE_ETIMEOUT, "group autotuner: a dependency wait of the persistent form ran out");
  g->persistent = g->form_ms[1] < g->form_ms[0] ? 1 : 0;
  return MAGPIE_OK;
}

// Autotuner of a group: for every window side of batched step 0, launch the
// batched window kernel with each candidate register bound (one warm-up, then
// three timed launches on the group's stream) and keep the fastest; then the
// update's tile shape and the step's form.  The window launches only write
// the members' per-window scratch (increments, partial sums, corners), never
// an object; the members' permutations are set to the identity first so that
// every index is valid.
int group_autotune(magpie_group* g) {
  cudaStream_t st = g->stream;
  for (auto* c : g->members)
    CUDA_TRY(cudaMemcpyAsync(c->order, c->iota, sizeof(int32_t) * c->p.n_pos, cudaMemcpyDeviceToDevice, st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) {
    int cand[3];
    minb_candidates(8 << i, cand);
    g->minb[i] = cand[0];
  }
  if (!g->wl.empty())
    for (const auto& L : g->wl[0]) {
      if (e != cudaSuccess) break;
      const int i = ilog2(L.ms) - 3;
      int cand[3];
      minb_candidates(L.ms, cand);
      if (cand[0] == cand[1] && cand[0] == cand[2]) continue;
      float best = 0.f;
      for (int v = 0; v < 3 && e == cudaSuccess; ++v) {
        if ((v == 1 && cand[1] == cand[0]) || (v == 2 && (cand[2] == cand[0] || cand[2] == cand[1]))) continue;
        e = launch_window_batched_m<kStep>(L.ms, g->table, g->map + L.map_off, L.windows, st, cand[v]);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r)
          e = launch_window_batched_m<kStep>(L.ms, g->table, g->map + L.map_off, L.windows, st, cand[v]);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        g->tune_ms[i][v] = ms / 3.f;
        if (v == 0 || ms / 3.f < best) {
          best = ms / 3.f;
          g->minb[i] = cand[v];
        }
      }
    }
  int rc = MAGPIE_OK;
  if (e == cudaSuccess) rc = group_tune_apply(g, st, e0, e1);
  if (e == cudaSuccess && !rc) rc = group_tune_form(g, st, e0, e1);
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(MAGPIE_ECUDA, std::string("group autotuner: ") + cudaGetErrorString(e));
  return rc;
}

extern "C" {

int magpie_version(void) { return kVersion; }

const char* magpie_strerror(int code) {
  switch (code) {
    case MAGPIE_OK: return "success";
    case MAGPIE_EINVAL: return "invalid argument";
    case MAGPIE_ECUDA: return "CUDA error";
    case MAGPIE_ENOMEM: return "out of device memory";
    case MAGPIE_EUNSUPPORTED: return "unsupported size";
    case MAGPIE_EINDEX: return "window index out of range";
    case MAGPIE_ETIMEOUT: return "bounded device wait ran out";
    default: return "unknown error";
  }
}

const char* magpie_last_error(void) { return g_last_error.c_str(); }

void magpie_destroy(magpie_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (int b = 0; b < 2; ++b) {
    if (c->graph2[b]) cudaGraphExecDestroy(c->graph2[b]);
    for (auto e : c->landed[b])
      if (e) cudaEventDestroy(e);
    if (c->used[b]) cudaEventDestroy(c->used[b]);
    if (c->amp2[b]) cudaFree(c->amp2[b]);
    if (c->stage2[b]) cudaFree(c->stage2[b]);
    if (c->order2[b]) cudaFree(c->order2[b]);
  }
  for (auto cs : c->copy2)
    if (cs) cudaStreamDestroy(cs);
  for (int i = 0; i < 4; ++i) {
    if (c->copy_streams[i]) cudaStreamDestroy(c->copy_streams[i]);
    if (c->copy_done[i]) cudaEventDestroy(c->copy_done[i]);
  }
  if (c->copy_start) cudaEventDestroy(c->copy_start);
  for (auto e : c->events)
    if (e) cudaEventDestroy(e);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  void* bufs[] = {c->Q, c->tw, c->amp, c->stage, c->pos, c->pyr, c->pyr_q, c->pyr_u, c->contrib,
                  c->phi_pos, c->gn_pos, c->part, c->corner, c->mx, c->pnum, c->pa2, c->pmax, c->iota, c->order, c->sums, c->err,
                  c->wz, c->lx, c->lscale, c->lacc, c->lmargin, c->lstats, c->pbuf, c->tabs, c->phase, c->g1buf,
                  c->g2buf, c->hand, c->acc};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete c;
}

int magpie_create(magpie_ctx** out, const magpie_params* params, void* object, const void* probe,
                  const int32_t* positions, const float* intensities, void* stream) {
  if (!out) return fail(MAGPIE_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(params);
  if (rc) return rc;
  if (!object || !probe || !positions || !intensities) return fail(MAGPIE_EINVAL, "a data pointer is NULL");
  const magpie_params& p = *params;
  std::vector<int32_t> hpos(2 * (size_t)p.n_pos);
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(hpos.data(), positions, sizeof(int32_t) * hpos.size(), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  rc = check_positions(hpos.data(), p.n_pos, p.n_rows, p.n_cols, p.m);
  if (rc) return rc;

  magpie_ctx* c = new magpie_ctx();
  c->p = p;
  c->M = p.m * p.m;
  c->z = (float2*)object;
  c->stream = st;
  const size_t M = c->M, N = p.n_pos;
  auto alloc = [&](void** ptr, size_t bytes) -> int {
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
      magpie_destroy(c);
      return fail(e == cudaErrorMemoryAllocation ? MAGPIE_ENOMEM : MAGPIE_ECUDA,
                  std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return MAGPIE_OK;
  };
  if ((rc = alloc((void**)&c->Q, sizeof(float2) * M)) || (rc = alloc((void**)&c->tw, sizeof(float2) * p.m)) ||
      (rc = alloc((void**)&c->amp, sizeof(float) * M * N)) || (rc = alloc((void**)&c->pos, sizeof(int32_t) * 2 * N)) ||
      (rc = alloc((void**)&c->pyr, sizeof(float) * pyr_size(p.m, p.levels))) ||
      (rc = alloc((void**)&c->pyr_q, sizeof(double2) * 2 * M)) || (rc = alloc((void**)&c->pyr_u, sizeof(double) * 2 * M)) ||
      (rc = alloc((void**)&c->contrib, sizeof(float2) * M * p.minibatch)) ||
      (rc = alloc((void**)&c->phi_pos, sizeof(double) * N)) || (rc = alloc((void**)&c->gn_pos, sizeof(double) * N)) ||
      (rc = alloc((void**)&c->part, sizeof(double) * 2 * kMaxSlots * N)) ||
      (rc = alloc((void**)&c->mx, sizeof(unsigned long long))) ||
      (rc = alloc((void**)&c->corner, sizeof(int2) * p.minibatch)) ||
      (p.update_probe && (rc = alloc((void**)&c->pnum, sizeof(float2) * M * p.minibatch))) ||
      (p.update_probe && (rc = alloc((void**)&c->pa2, sizeof(float) * M * p.minibatch))) ||
      (p.update_probe && (rc = alloc((void**)&c->pmax, sizeof(double) * kMaxCluster * p.minibatch))) ||
      (rc = alloc((void**)&c->iota, sizeof(int32_t) * N)) || (rc = alloc((void**)&c->order, sizeof(int32_t) * N)) ||
      (rc = alloc((void**)&c->sums, sizeof(double) * 2)) || (rc = alloc((void**)&c->err, sizeof(int))) ||
      (p.levels >= 2 && (rc = alloc((void**)&c->wz, sizeof(float) * M * 2))) ||
      (!p.deterministic && (rc = alloc((void**)&c->acc, sizeof(float4) * (size_t)p.n_rows * p.n_cols))))
    return rc;

  auto cleanup_fail = [&](int code) {
    magpie_destroy(c);
    return code;
  };
#define CTX_TRY(expr)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return cleanup_fail(fail(MAGPIE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_))); \
  } while (0)
  CTX_TRY(prepare_kernels(p.m));
  CTX_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  std::vector<float2> htw(p.m);
  for (int t = 0; t < p.m; ++t) {
    const double ang = -2.0 * 3.14159265358979323846 * (double)t / (double)p.m;
    htw[t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  CTX_TRY(cudaMemcpyAsync(c->tw, htw.data(), sizeof(float2) * p.m, cudaMemcpyHostToDevice, st));
  CTX_TRY(cudaMemcpyAsync(c->pos, positions, sizeof(int32_t) * 2 * N, cudaMemcpyDeviceToDevice, st));
  CTX_TRY(cudaMemsetAsync(c->err, 0, sizeof(int), st));
  CTX_TRY(cudaMemsetAsync(c->phi_pos, 0, sizeof(double) * N, st));
  CTX_TRY(cudaMemsetAsync(c->gn_pos, 0, sizeof(double) * N, st));
  if (c->acc) CTX_TRY(cudaMemsetAsync(c->acc, 0, sizeof(float4) * (size_t)p.n_rows * p.n_cols, st));
  iota_kernel<<<(int)((N + 255) / 256), 256, 0, st>>>(c->iota, (int)N);
  CTX_TRY(cudaGetLastError());
  sqrt_kernel<<<1024, 256, 0, st>>>(intensities, c->amp, M * N);
  CTX_TRY(cudaGetLastError());
  rc = build_pyramid(c, probe);
  if (rc) return cleanup_fail(rc);
  CTX_TRY(cudaStreamSynchronize(st));
#undef CTX_TRY
  *out = c;
  return MAGPIE_OK;
}

int magpie_set_probe(magpie_ctx* c, const void* probe) {
  if (!c || !probe) return fail(MAGPIE_EINVAL, "NULL argument");
  return build_pyramid(c, probe);
}

int magpie_step(magpie_ctx* c, const int32_t* idx, int32_t count) {
  if (!c || !idx) return fail(MAGPIE_EINVAL, "NULL argument");
  if (count < 1 || count > c->p.minibatch) return fail(MAGPIE_EINVAL, "count must lie in [1, minibatch]");
  return enqueue_step(c, idx, count, c->stream);
}

int magpie_sweep(magpie_ctx* c, const int32_t* order) {
  NvtxRange range("magpie_sweep");
  if (!c || !order) return fail(MAGPIE_EINVAL, "NULL argument");
  CUDA_TRY(cudaMemcpyAsync(c->order, order, sizeof(int32_t) * c->p.n_pos, cudaMemcpyDeviceToDevice, c->stream));
  return launch_sweep(c);
}

int magpie_profile_sweep(magpie_ctx* c, const int32_t* order, double* window_ms, double* apply_ms,
                         int32_t* launches) {
  NvtxRange range("magpie_profile_sweep");
  if (!c || !order) return fail(MAGPIE_EINVAL, "NULL argument");
  CUDA_TRY(cudaMemcpyAsync(c->order, order, sizeof(int32_t) * c->p.n_pos, cudaMemcpyDeviceToDevice, c->stream));
  if (c->events.empty()) {
    c->events.resize(4 * (size_t)n_steps(c), nullptr);
    for (auto& e : c->events) CUDA_TRY(cudaEventCreate(&e));
  }
  const int N = c->p.n_pos, B = c->p.minibatch;
  for (int s = 0, i = 0; s < N; s += B, ++i) {
    int rc = enqueue_step(c, c->order + s, N - s < B ? N - s : B, c->stream, &c->events[4 * (size_t)i]);
    if (rc) return rc;
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  double wsum = 0.0, asum = 0.0;
  for (int i = 0; i < n_steps(c); ++i) {
    float a = 0.f, b = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&a, c->events[4 * i], c->events[4 * i + 1]));
    CUDA_TRY(cudaEventElapsedTime(&b, c->events[4 * i + 2], c->events[4 * i + 3]));
    wsum += a;
    asum += b;
  }
  if (window_ms) *window_ms = wsum;
  if (apply_ms) *apply_ms = asum;
  if (launches) *launches = n_steps(c);
  return read_err(c);
}

int magpie_get_probe(magpie_ctx* c, void* probe) {
  if (!c || !probe) return fail(MAGPIE_EINVAL, "NULL argument");
  CUDA_TRY(cudaMemcpyAsync(probe, c->Q, sizeof(float2) * c->M, cudaMemcpyDeviceToDevice, c->stream));
  return MAGPIE_OK;
}

int magpie_objective(magpie_ctx* c, double* phi) {
  if (!c || !phi) return fail(MAGPIE_EINVAL, "NULL argument");
  return evaluate(c, phi, nullptr);
}

int magpie_stop_metric(magpie_ctx* c, double* value) {
  if (!c || !value) return fail(MAGPIE_EINVAL, "NULL argument");
  return evaluate(c, nullptr, value);
}

int magpie_window_values(magpie_ctx* c, double* phi, double* gnorm) {
  if (!c) return fail(MAGPIE_EINVAL, "NULL argument");
  const size_t N = c->p.n_pos;
  if (phi) CUDA_TRY(cudaMemcpyAsync(phi, c->phi_pos, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
  if (gnorm) CUDA_TRY(cudaMemcpyAsync(gnorm, c->gn_pos, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
  return read_err(c);
}

int magpie_sweep_host(magpie_ctx* c, const int32_t* order, const float* intensities, void* object_out) {
  NvtxRange range("magpie_sweep_host");
  if (!c || !order) return fail(MAGPIE_EINVAL, "NULL argument");
  const size_t N = c->p.n_pos, M = c->M;
  if (intensities) {
    // four chunks on four copy streams (several copy engines), each chunk's
    // square roots taken on its own stream as soon as it has landed
    constexpr int kChunks = 4;
    if (!c->stage) CUDA_TRY(cudaMalloc((void**)&c->stage, sizeof(float) * N * M));
    if (!c->copy_start) {
      CUDA_TRY(cudaEventCreateWithFlags(&c->copy_start, cudaEventDisableTiming));
      for (int i = 0; i < kChunks; ++i) {
        CUDA_TRY(cudaStreamCreateWithFlags(&c->copy_streams[i], cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&c->copy_done[i], cudaEventDisableTiming));
      }
    }
    CUDA_TRY(cudaEventRecord(c->copy_start, c->stream));
    const size_t total = N * M, per = (total + kChunks - 1) / kChunks;
    for (int i = 0; i < kChunks; ++i) {
      const size_t b0 = i * per, n = b0 >= total ? 0 : (total - b0 < per ? total - b0 : per);
      cudaStream_t cs = c->copy_streams[i];
      CUDA_TRY(cudaStreamWaitEvent(cs, c->copy_start, 0));
      if (n) {
        CUDA_TRY(cudaMemcpyAsync(c->stage + b0, intensities + b0, sizeof(float) * n, cudaMemcpyHostToDevice, cs));
        sqrt_kernel<<<256, 256, 0, cs>>>(c->stage + b0, c->amp + b0, n);
        CUDA_TRY(cudaGetLastError());
      }
      CUDA_TRY(cudaEventRecord(c->copy_done[i], cs));
      CUDA_TRY(cudaStreamWaitEvent(c->stream, c->copy_done[i], 0));
    }
  }
  CUDA_TRY(cudaMemcpyAsync(c->order, order, sizeof(int32_t) * N, cudaMemcpyHostToDevice, c->stream));
  int rc = launch_sweep(c);
  if (rc) return rc;
  if (object_out)
    CUDA_TRY(cudaMemcpyAsync(object_out, c->z, sizeof(float2) * (size_t)c->p.n_rows * c->p.n_cols,
                             cudaMemcpyDeviceToHost, c->stream));
  return read_err(c);
}

int magpie_forward_intensities(const void* object, int32_t n_rows, int32_t n_cols, const void* probe, int32_t m,
                               const int32_t* positions, int32_t n_pos, float* out, void* stream) {
  magpie_params p{};
  p.n_rows = n_rows;
  p.n_cols = n_cols;
  p.m = m;
  p.n_pos = n_pos;
  p.levels = 1;
  p.minibatch = 1;
  p.alpha = 0.f;
  int rc = validate(&p);
  if (rc) return rc;
  if (!object || !probe || !positions || !out) return fail(MAGPIE_EINVAL, "a data pointer is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int32_t> hpos(2 * (size_t)n_pos);
  CUDA_TRY(cudaMemcpyAsync(hpos.data(), positions, sizeof(int32_t) * hpos.size(), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  rc = check_positions(hpos.data(), n_pos, n_rows, n_cols, m);
  if (rc) return rc;
  CUDA_TRY(prepare_kernels(m));
  float2* tw = nullptr;
  int32_t* iota = nullptr;
  CUDA_TRY(cudaMalloc((void**)&tw, sizeof(float2) * m));
  cudaError_t e = cudaMalloc((void**)&iota, sizeof(int32_t) * n_pos);
  if (e != cudaSuccess) {
    cudaFree(tw);
    CUDA_TRY(e);
  }
  std::vector<float2> htw(m);
  for (int t = 0; t < m; ++t) {
    const double ang = -2.0 * 3.14159265358979323846 * (double)t / (double)m;
    htw[t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  StepArgs a{};
  a.z = (const float2*)object;
  a.n_rows = n_rows;
  a.n_cols = n_cols;
  a.Q = (const float2*)probe;
  a.tw = tw;
  a.out_int = out;
  a.pos = positions;
  a.idx = iota;
  a.n_pos = n_pos;
  a.levels = 1;
  e = cudaMemcpyAsync(tw, htw.data(), sizeof(float2) * m, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    iota_kernel<<<(n_pos + 255) / 256, 256, 0, st>>>(iota, n_pos);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_window_m<kSim>(m, a, n_pos, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(tw);
  cudaFree(iota);
  CUDA_TRY(e);
  return MAGPIE_OK;
}


int magpie_step_noalloc(void* object, int32_t n_rows, int32_t n_cols, const void* probe, int32_t m,
                        const int32_t* positions, int32_t n_pos, const float* amplitudes, const int32_t* idx,
                        int32_t count, int32_t levels, float alpha, double* phi, double* gnorm, void* stream) {
  magpie_params p{};
  p.n_rows = n_rows;
  p.n_cols = n_cols;
  p.m = m;
  p.n_pos = n_pos;
  p.levels = levels;
  p.minibatch = count;
  p.alpha = alpha;
  int rc = validate(&p);
  if (rc) return rc;
  if (!object || !probe || !positions || !amplitudes || !idx || !phi || !gnorm)
    return fail(MAGPIE_EINVAL, "a data pointer is NULL");
  if (m > 128) return fail(MAGPIE_EUNSUPPORTED, "the fixed workspace holds probe factors for m <= 128");
  if ((size_t)count * (size_t)m * (size_t)m > kNoAllocMaxIncrement)
    return fail(MAGPIE_EINVAL, "count * m^2 = " + std::to_string((long long)count * m * m) +
                                   " exceeds the fixed scratch of 2^20 complex values");
  NoAllocScratch w{};
  rc = noalloc_scratch(&w);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(prepare_kernels(m));
  float2 htw[128];
  for (int t = 0; t < m; ++t) {
    const double ang = -2.0 * 3.14159265358979323846 * (double)t / (double)m;
    htw[t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  CUDA_TRY(cudaMemcpyAsync(w.tw, htw, sizeof(float2) * m, cudaMemcpyHostToDevice, st));
  sanitize_idx_kernel<<<(count + 255) / 256, 256, 0, st>>>(idx, count, positions, n_pos, n_rows, n_cols, m, w.idx,
                                                            w.err);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(enqueue_pyramid((const float2*)probe, m, levels, alpha, w.mx, w.pyr_q, w.pyr_u, w.pyr, st));
  StepArgs a{};
  a.z = (const float2*)object;
  a.n_rows = n_rows;
  a.n_cols = n_cols;
  a.Q = (const float2*)probe;
  a.tw = w.tw;
  a.amp = amplitudes;
  a.pos = positions;
  a.idx = w.idx;
  a.n_pos = n_pos;
  a.contrib = w.contrib;
  a.pyr = w.pyr;
  a.levels = levels;
  a.part = w.part;
  a.corner = w.corner;
  a.err = w.err;
  CUDA_TRY(launch_window_m<kStep>(m, a, count, st));
  CUDA_TRY(launch_apply((float2*)object, n_rows, n_cols, w.corner, w.idx, count, n_pos, w.contrib, w.pyr + m * m, m,
                        w.part, phi, gnorm, st));
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (h) return fail(MAGPIE_EINDEX, "a window index or its position was out of range; that window was skipped");
  return MAGPIE_OK;
}


void magpie_group_destroy(magpie_group* g) {
  if (!g) return;
  if (g->graph) cudaGraphExecDestroy(g->graph);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  if (g->table) cudaFree(g->table);
  if (g->map) cudaFree(g->map);
  for (auto* a : g->atable)
    if (a) cudaFree(a);
  void* bufs[] = {g->ptable, g->wmember, g->qbuf, g->err};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int j = 0; j < 6; ++j) {
    if (g->side[j]) cudaStreamDestroy(g->side[j]);
    if (g->join[j]) cudaEventDestroy(g->join[j]);
  }
  if (g->fork) cudaEventDestroy(g->fork);
  delete g;
}

int magpie_group_create(magpie_group** out, magpie_ctx* const* ctxs, int32_t n, void* stream) {
  if (!out || !ctxs || n < 1) return fail(MAGPIE_EINVAL, "need an output pointer and at least one context");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(MAGPIE_EINVAL, "context " + std::to_string(i) + " is NULL");
    if (ctxs[i]->p.update_probe) return fail(MAGPIE_EINVAL, "contexts with update_probe = 1 cannot be grouped");
    if (ctxs[i]->cnn || ctxs[i]->precision || (ctxs[i]->variant & 2))
      return fail(MAGPIE_EINVAL, "contexts with a network, tensor-core DFTs or the phase rule cannot be grouped");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(MAGPIE_EINVAL, "a context appears twice in the group");
  }
  magpie_group* g = new magpie_group();
  g->members.assign(ctxs, ctxs + n);
  g->stream = (cudaStream_t)stream;
  std::vector<StepArgs> table;
  std::vector<int2> map;
  std::vector<int> wmem;
  int q_total = 0, max_sides = 0;
  int steps = 0;
  for (auto* c : g->members) steps = std::max(steps, n_steps(c));
  for (int t = 0; t < steps; ++t) {
    std::vector<int> entry(n, -1);
    for (int i = 0; i < n; ++i) {
      magpie_ctx* c = g->members[i];
      if (t >= n_steps(c)) continue;
      entry[i] = (int)table.size();
      table.push_back(make_args(c, c->order + (size_t)t * c->p.minibatch));
    }
    std::vector<GroupWindowLaunch> wls;
    std::vector<GroupPersistLaunch> pls;
    for (int ms : {8, 16, 32, 64, 128, 256}) {
      GroupWindowLaunch L{ms, (int)map.size(), 0};
      GroupPersistLaunch PL{ms, (int)map.size(), 0, (int)g->ptable_host.size(), 0, 0, q_total, 0, 0};
      const int pt = window_threads(ms) >= 256 ? 32 : 16;  // the persistent kernel's update tile
      for (int i = 0; i < n; ++i) {
        magpie_ctx* c = g->members[i];
        if (entry[i] < 0 || c->p.m != ms) continue;
        const int cnt = std::min(c->p.minibatch, c->p.n_pos - t * c->p.minibatch);
        for (int w = 0; w < cnt; ++w) {
          map.push_back(make_int2(entry[i], w));
          wmem.push_back(PL.na);
        }
        L.windows += cnt;
        ApplyArgs P = apply_args(c->z, c->p.n_rows, c->p.n_cols, c->corner, c->order + (size_t)t * c->p.minibatch,
                                 cnt, c->p.n_pos, c->contrib, c->pyr + c->M, c->p.m, c->part, c->phi_pos,
                                 c->gn_pos, 0, ApplyShape{pt, pt});
        P.block0 = PL.ntiles;
        PL.ntiles += apply_tiles(P);
        PL.max_count = std::max(PL.max_count, cnt);
        ++PL.na;
        g->ptable_host.push_back(P);
      }
      if (L.windows) {
        wls.push_back(L);
        PL.nw = L.windows;
        q_total += 1 + PL.na;
        pls.push_back(PL);
      }
    }
    g->wl.push_back(wls);
    max_sides = std::max(max_sides, (int)pls.size());
    g->pl.push_back(pls);
    for (int v = 0; v < 3; ++v) {
      std::vector<ApplyArgs>& at = g->atable_host[v];
      GroupApplyLaunch A{(int)at.size(), 0, 0, 0};
      for (int i = 0; i < n; ++i) {
        magpie_ctx* c = g->members[i];
        if (entry[i] < 0) continue;
        const int cnt = std::min(c->p.minibatch, c->p.n_pos - t * c->p.minibatch);
        ApplyArgs P = apply_args(c->z, c->p.n_rows, c->p.n_cols, c->corner, c->order + (size_t)t * c->p.minibatch,
                                 cnt, c->p.n_pos, c->contrib, c->pyr + c->M, c->p.m, c->part, c->phi_pos,
                                 c->gn_pos, 0, kApplyShapes[v]);
        P.block0 = A.blocks;
        A.blocks += apply_tiles(P);
        A.max_count = std::max(A.max_count, cnt);
        ++A.n;
        at.push_back(P);
      }
      g->al[v].push_back(A);
    }
  }
  auto upload = [&](void** dst, const void* src, size_t bytes) -> int {
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      magpie_group_destroy(g);
      return fail(e == cudaErrorMemoryAllocation ? MAGPIE_ENOMEM : MAGPIE_ECUDA,
                  std::string("group tables: ") + cudaGetErrorString(e));
    }
    return MAGPIE_OK;
  };
  int rc;
  if ((rc = upload((void**)&g->table, table.data(), sizeof(StepArgs) * table.size())) ||
      (rc = upload((void**)&g->map, map.data(), sizeof(int2) * map.size())))
    return rc;
  for (int v = 0; v < 3; ++v)
    if ((rc = upload((void**)&g->atable[v], g->atable_host[v].data(), sizeof(ApplyArgs) * g->atable_host[v].size())))
      return rc;
  if ((rc = upload((void**)&g->ptable, g->ptable_host.data(), sizeof(ApplyArgs) * g->ptable_host.size())) ||
      (rc = upload((void**)&g->wmember, wmem.data(), sizeof(int) * wmem.size())))
    return rc;
  g->qbuf_n = (size_t)q_total;
  cudaError_t e = cudaMalloc(&g->qbuf, sizeof(int) * g->qbuf_n);
  if (e == cudaSuccess) e = cudaMalloc(&g->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(g->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && max_sides > 1) e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
  for (int j = 1; j < max_sides && e == cudaSuccess; ++j) {
    e = cudaStreamCreateWithFlags(&g->side[j], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->join[j], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    magpie_group_destroy(g);
    return fail(e == cudaErrorMemoryAllocation ? MAGPIE_ENOMEM : MAGPIE_ECUDA,
                std::string("group setup: ") + cudaGetErrorString(e));
  }
  rc = group_autotune(g);
  if (rc) {
    magpie_group_destroy(g);
    return rc;
  }
  *out = g;
  return MAGPIE_OK;
}

int magpie_group_sweep(magpie_group* g, const int32_t* const* orders) {
  NvtxRange range("magpie_group_sweep");
  if (!g || !orders) return fail(MAGPIE_EINVAL, "NULL argument");
  for (size_t i = 0; i < g->members.size(); ++i)
    if (!orders[i]) return fail(MAGPIE_EINVAL, "order " + std::to_string(i) + " is NULL");
  if (!g->graph) {
    if (g->persistent) {
      const int rc = plan_persistent(g);
      if (rc) return rc;
    }
    cudaGraph_t gr = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    int rc = MAGPIE_OK;
    if (g->persistent) {
      // the counters of every step's launches start at zero; one step after
      // another, its sides' launches concurrent
      e = cudaMemsetAsync(g->qbuf, 0, sizeof(int) * g->qbuf_n, g->cap_stream);
      for (size_t t = 0; t < g->pl.size() && e == cudaSuccess && !rc; ++t)
        rc = enqueue_persistent_step(g, t, g->cap_stream, g->ptable, 0);
    } else {
      for (size_t t = 0; t < g->wl.size() && e == cudaSuccess; ++t) {
        for (const auto& L : g->wl[t]) {
          e = launch_window_batched_m<kStep>(L.ms, g->table, g->map + L.map_off, L.windows, g->cap_stream,
                                             g->minb[ilog2(L.ms) - 3]);
          if (e != cudaSuccess) break;
        }
        if (e != cudaSuccess) break;
        e = launch_apply_batched(g, g->apply_shape, t, g->cap_stream);
      }
    }
    cudaError_t e2 = cudaStreamEndCapture(g->cap_stream, &gr);
    if (rc) {
      if (gr) cudaGraphDestroy(gr);
      return rc;
    }
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->graph, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    CUDA_TRY(e);
  }
  for (size_t i = 0; i < g->members.size(); ++i) {
    magpie_ctx* c = g->members[i];
    CUDA_TRY(cudaMemcpyAsync(c->order, orders[i], sizeof(int32_t) * c->p.n_pos, cudaMemcpyDeviceToDevice, g->stream));
  }
  CUDA_TRY(cudaGraphLaunch(g->graph, g->stream));
  return MAGPIE_OK;
}


// ------------------------------------------------- learned coarse correction

int32_t magpie_cnn_param_count(void) { return cnn_param_count(); }

void magpie_cnn_destroy(magpie_cnn* n) {
  if (!n) return;
  void* bufs[] = {n->theta, n->adam_m, n->adam_v, n->wbf, n->grad, n->y, n->dz[0], n->dz[1], n->dy, n->part, n->err};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (auto* a : n->act)
    if (a) cudaFree(a);
  delete n;
}

int magpie_cnn_create(magpie_cnn** out, int32_t h, int32_t max_batch, void* stream) {
  if (!out) return fail(MAGPIE_EINVAL, "out is NULL");
  *out = nullptr;
  if (h != 8 && h != 16 && h != 32 && h != 64) return fail(MAGPIE_EINVAL, "h must be 8, 16, 32 or 64");
  if (max_batch < 1 || max_batch > kMaxMinibatch) return fail(MAGPIE_EINVAL, "max_batch must lie in [1, 4096]");
  magpie_cnn* n = new magpie_cnn();
  n->h = h;
  n->max_batch = max_batch;
  n->stream = (cudaStream_t)stream;
  n->P = cnn_param_count();
  int o = 0;
  for (int l = 0; l < kCnnLayers; ++l) {
    n->off[l] = o;
    o += kCnn[l].cout * 9 * kCnn[l].cin + kCnn[l].cout;
  }
  const size_t B = max_batch, P = n->P;
  size_t dzn = 0;
  for (int l = 0; l < kCnnLayers; ++l) {
    const size_t so = cnn_side_out(h, l), si = cnn_side_in(h, l);
    dzn = std::max(dzn, B * so * so * kCnn[l].cout);
    dzn = std::max(dzn, B * si * si * kCnn[l].cin);
  }
  n->part_n = cnn_part_floats(h, max_batch);
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  al((void**)&n->theta, sizeof(float) * P);
  al((void**)&n->adam_m, sizeof(float) * P);
  al((void**)&n->adam_v, sizeof(float) * P);
  al((void**)&n->wbf, sizeof(bf16) * P);
  al((void**)&n->grad, sizeof(float) * P);
  for (int l = 0; l < kCnnLayers; ++l) {
    const size_t si = cnn_side_in(h, l);
    al((void**)&n->act[l], sizeof(bf16) * B * si * si * kCnn[l].cin);
  }
  al((void**)&n->y, sizeof(float) * B * h * h * 2);
  al((void**)&n->dy, sizeof(float) * B * h * h * 2);
  al((void**)&n->dz[0], sizeof(float) * dzn);
  al((void**)&n->dz[1], sizeof(float) * dzn);
  al((void**)&n->part, sizeof(float) * n->part_n);
  al((void**)&n->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(n->err, 0, sizeof(int), n->stream);
  for (int l = 0; l < kCnnLayers && e == cudaSuccess; ++l)
    if (n->off[l] % 8) e = cudaErrorMisalignedAddress;  // 16-byte rows of every layer's BF16 weights
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_fwd_tc_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcConv<128>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_fwd_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcConv<64>::SMEM);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->theta, 0, sizeof(float) * P, n->stream);
  if (e != cudaSuccess) {
    magpie_cnn_destroy(n);
    return fail(e == cudaErrorMemoryAllocation ? MAGPIE_ENOMEM : MAGPIE_ECUDA,
                std::string("network buffers: ") + cudaGetErrorString(e));
  }
  const int rc = cnn_enqueue_params(n, n->stream);
  if (rc) {
    magpie_cnn_destroy(n);
    return rc;
  }
  *out = n;
  return MAGPIE_OK;
}

int magpie_cnn_set_params(magpie_cnn* n, const float* theta) {
  if (!n || !theta) return fail(MAGPIE_EINVAL, "NULL argument");
  CUDA_TRY(cudaMemcpyAsync(n->theta, theta, sizeof(float) * n->P, cudaMemcpyDeviceToDevice, n->stream));
  return cnn_enqueue_params(n, n->stream);
}

int magpie_cnn_get_params(magpie_cnn* n, float* theta) {
  if (!n || !theta) return fail(MAGPIE_EINVAL, "NULL argument");
  CUDA_TRY(cudaMemcpyAsync(theta, n->theta, sizeof(float) * n->P, cudaMemcpyDeviceToDevice, n->stream));
  return MAGPIE_OK;
}

int magpie_cnn_forward(magpie_cnn* n, const float* x, int32_t batch, float* y) {
  if (!n || !x || !y) return fail(MAGPIE_EINVAL, "NULL argument");
  if (batch < 1 || batch > n->max_batch) return fail(MAGPIE_EINVAL, "batch must lie in [1, max_batch]");
  const int rc = cnn_enqueue_forward(n, x, batch, n->y, n->stream);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(y, n->y, sizeof(float) * (size_t)batch * n->h * n->h * 2, cudaMemcpyDeviceToDevice,
                           n->stream));
  return MAGPIE_OK;
}

int magpie_cnn_backward(magpie_cnn* n, const float* dy, float* grad) {
  if (!n || !dy || !grad) return fail(MAGPIE_EINVAL, "NULL argument");
  if (n->last_batch < 1) return fail(MAGPIE_EINVAL, "no forward pass to differentiate");
  return cnn_enqueue_backward(n, dy, grad, n->stream);
}

int magpie_cnn_train_step(magpie_cnn* n, const float* x0, const float* zh, const float* scale, int32_t batch,
                          float lr, double* loss) {
  if (!n || !x0 || !zh || !scale || !loss) return fail(MAGPIE_EINVAL, "NULL argument");
  if (batch < 1 || batch > n->max_batch) return fail(MAGPIE_EINVAL, "batch must lie in [1, max_batch]");
  if (!(lr > 0.f) || !std::isfinite(lr)) return fail(MAGPIE_EINVAL, "lr must be finite and > 0");
  cudaStream_t st = n->stream;
  int rc = cnn_enqueue_forward(n, x0, batch, n->y, st);
  if (rc) return rc;
  cnn_loss_kernel<<<1, 1024, 0, st>>>(n->y, reinterpret_cast<const float4*>(x0), reinterpret_cast<const float2*>(zh),
                                      scale, batch, n->h * n->h, n->dy, loss);
  CUDA_TRY(cudaGetLastError());
  rc = cnn_enqueue_backward(n, n->dy, n->grad, st);
  if (rc) return rc;
  n->step += 1;
  const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)n->step)));
  const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)n->step)));
  adam_kernel<<<(n->P + 255) / 256, 256, 0, st>>>(n->theta, n->grad, n->adam_m, n->adam_v, n->wbf, n->P, lr, c1, c2);
  CUDA_TRY(cudaGetLastError());
  return MAGPIE_OK;
}

int magpie_coarse_state(magpie_ctx* c, const int32_t* idx, int32_t count, float* x, float* scale) {
  if (!c || !idx || !x || !scale) return fail(MAGPIE_EINVAL, "NULL argument");
  if (count < 1 || count > c->p.minibatch) return fail(MAGPIE_EINVAL, "count must lie in [1, minibatch]");
  int rc = learned_supported(c, nullptr);
  if (rc) return rc;
  StepArgs a = make_args(c, idx);
  a.grad_only = 1;
  CUDA_TRY(launch_window_m<kStep>(c->p.m, a, count, c->stream));
  coarse_state_kernel<<<count, 1024, 0, c->stream>>>(coarse_args(c, idx, reinterpret_cast<float4*>(x), scale));
  CUDA_TRY(cudaGetLastError());
  return read_err(c);
}

int magpie_gather_windows(magpie_ctx* c, const int32_t* idx, int32_t count, void* patches) {
  if (!c || !idx || !patches) return fail(MAGPIE_EINVAL, "NULL argument");
  if (count < 1) return fail(MAGPIE_EINVAL, "count must be >= 1");
  gather_windows_kernel<<<count, 256, 0, c->stream>>>(c->z, c->p.n_cols, c->pos, idx, c->p.n_pos, c->p.m,
                                                      (float2*)patches);
  CUDA_TRY(cudaGetLastError());
  return MAGPIE_OK;
}

int magpie_attach_cnn(magpie_ctx* c, magpie_cnn* n) {
  if (!c) return fail(MAGPIE_EINVAL, "NULL context");
  if (n) {
    int rc = learned_supported(c, n);
    if (rc) return rc;
    rc = learned_buffers(c);
    if (rc) return rc;
  }
  invalidate_graphs(c);
  c->cnn = n;
  return MAGPIE_OK;
}

int magpie_cnn_set_tensor_path(magpie_cnn* n, int32_t path) {
  if (!n || (path != 0 && path != 1)) return fail(MAGPIE_EINVAL, "need a network and path 0 or 1");
  n->tensor_path = path;
  return MAGPIE_OK;
}

int magpie_cnn_status(magpie_cnn* n) {
  if (!n) return fail(MAGPIE_EINVAL, "NULL argument");
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
  CUDA_TRY(cudaStreamSynchronize(n->stream));
  if (h) {
    CUDA_TRY(cudaMemsetAsync(n->err, 0, sizeof(int), n->stream));
    return fail(MAGPIE_ETIMEOUT, "a tensor-core convolution stopped waiting for its MMAs (bounded wait ran out)");
  }
  return MAGPIE_OK;
}

int magpie_learned_stats(magpie_ctx* c, int64_t* proposed, int64_t* accepted) {
  if (!c || !proposed || !accepted) return fail(MAGPIE_EINVAL, "NULL argument");
  unsigned long long h[2] = {0ull, 0ull};
  if (c->lstats) {
    CUDA_TRY(cudaMemcpyAsync(h, c->lstats, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  *proposed = (int64_t)h[0];
  *accepted = (int64_t)h[1];
  return MAGPIE_OK;
}

int magpie_learned_window_values(magpie_ctx* c, int32_t count, int32_t* accepted, double* margin) {
  if (!c || !accepted || !margin) return fail(MAGPIE_EINVAL, "NULL argument");
  if (!c->lacc) return fail(MAGPIE_EINVAL, "no network has been attached to this context");
  if (count < 1 || count > c->p.minibatch) return fail(MAGPIE_EINVAL, "count must lie in [1, minibatch]");
  CUDA_TRY(cudaMemcpyAsync(accepted, c->lacc, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaMemcpyAsync(margin, c->lmargin, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MAGPIE_OK;
}


// ---------------------------------------------------------- precision form

int magpie_set_precision(magpie_ctx* c, int32_t mode) {
  if (!c) return fail(MAGPIE_EINVAL, "NULL context");
  if (mode < 0 || mode > 2)
    return fail(MAGPIE_EINVAL, "mode must be 0 (FP32 FFTs), 1 (mma.sync DFTs) or 2 (tcgen05 DFTs)");
  if (mode >= 1) {
    const int m = c->p.m;
    if (m != 64 && m != 128 && m != 256)
      return fail(MAGPIE_EUNSUPPORTED, "tensor-core DFTs need m = 64, 128 or 256");
    if (c->p.update_probe) return fail(MAGPIE_EINVAL, "tensor-core DFTs need update_probe = 0");
    if (!c->pbuf) {
      cudaError_t e = cudaMalloc((void**)&c->pbuf, sizeof(float2) * (size_t)c->M * c->p.minibatch);
      if (e == cudaSuccess) e = cudaMalloc((void**)&c->g1buf, sizeof(float2) * (size_t)(c->M / 4) * c->p.minibatch);
      if (e == cudaSuccess) e = cudaMalloc((void**)&c->g2buf, sizeof(float2) * (size_t)(c->M / 16) * c->p.minibatch);
      if (e == cudaSuccess) e = cudaMalloc((void**)&c->hand, sizeof(int) * 3 * (size_t)c->p.minibatch);
      if (e == cudaSuccess) e = cudaMemset(c->hand, 0, sizeof(int) * 3 * (size_t)c->p.minibatch);
      if (e == cudaSuccess) e = cudaMalloc((void**)&c->tabs, sizeof(TcTables));
      if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? MAGPIE_ENOMEM : MAGPIE_ECUDA,
                    std::string("precision buffers: ") + cudaGetErrorString(e));
      TcTables h;
      build_tc_tables(m, h);
      CUDA_TRY(cudaMemcpy(c->tabs, &h, sizeof(TcTables), cudaMemcpyHostToDevice));
    }
  }
  invalidate_graphs(c);
  c->precision = mode;
  return MAGPIE_OK;
}

int magpie_precision_check_waits(magpie_ctx* c, double seconds) {
  if (!c) return fail(MAGPIE_EINVAL, "NULL context");
  if (!c->precision) return fail(MAGPIE_EINVAL, "the context is not in the precision form");
  if (!(seconds >= 1e-6 && seconds <= 10.0)) return fail(MAGPIE_EINVAL, "seconds must lie in [1e-6, 10]");
  const int count = std::min(c->p.minibatch, c->p.n_pos);
  PrecArgs a = precision_args(c, c->iota, count);
  a.wait_bias = 1;  // one tile more than any window has: every hand-off wait runs out
  a.wait_ns = (unsigned long long)(seconds * 1e9);
  const int rc = enqueue_precision_g0(c, a, count, c->stream);
  if (rc) return rc;
  if (c->p.levels >= 3 && !c->cnn) CUDA_TRY(launch_coarse_cycle(a, count, c->p.levels, c->stream));
  // no update kernel runs: clear the counts here
  CUDA_TRY(cudaMemsetAsync(c->hand, 0, sizeof(int) * 3 * (size_t)count, c->stream));
  return read_err(c);
}

static int dft2_tc(const void* in, void* out, int32_t m, int32_t count, int32_t inverse, void* stream, int path);

int magpie_dft2_tc(const void* in, void* out, int32_t m, int32_t count, int32_t inverse, void* stream) {
  return dft2_tc(in, out, m, count, inverse, stream, 0);
}

int magpie_dft2_tcgen05(const void* in, void* out, int32_t m, int32_t count, int32_t inverse, void* stream) {
  return dft2_tc(in, out, m, count, inverse, stream, 1);
}

static int dft2_tc(const void* in, void* out, int32_t m, int32_t count, int32_t inverse, void* stream, int path) {
  if (!in || !out) return fail(MAGPIE_EINVAL, "NULL argument");
  if (m != 64 && m != 128 && m != 256) return fail(MAGPIE_EUNSUPPORTED, "m must be 64, 128 or 256");
  if (count < 1 || (long long)count * m * m > (1LL << 28)) return fail(MAGPIE_EINVAL, "count out of range");
  if (inverse != 0 && inverse != 1) return fail(MAGPIE_EINVAL, "inverse must be 0 or 1");
  cudaStream_t st = (cudaStream_t)stream;
  TcTables h;
  build_tc_tables(m, h);
  std::vector<float2> htw(m);
  for (int t = 0; t < m; ++t) {
    const double ang = -2.0 * 3.14159265358979323846 * (double)t / (double)m;
    htw[t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  TcTables* dt = nullptr;
  float2* dtw = nullptr;
  int* derr = nullptr;
  int herr = 0;
  cudaError_t e = cudaMalloc((void**)&dt, sizeof(TcTables));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dtw, sizeof(float2) * m);
  if (e == cudaSuccess) e = cudaMalloc((void**)&derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dt, &h, sizeof(TcTables), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dtw, htw.data(), sizeof(float2) * m, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && in != out)
    e = cudaMemcpyAsync(out, in, sizeof(float2) * (size_t)count * m * m, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = launch_dft2_tc_m(m, (float2*)out, count, dt, dtw, inverse, st, path, derr);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (dt) cudaFree(dt);
  if (dtw) cudaFree(dtw);
  if (derr) cudaFree(derr);
  if (e != cudaSuccess) return fail(MAGPIE_ECUDA, std::string("magpie_dft2_tc: ") + cudaGetErrorString(e));
  if (herr & 16) return fail(MAGPIE_ETIMEOUT, "a bounded wait of a tcgen05 transform ran out");
  return MAGPIE_OK;
}


// ---------------------------------------------------------- paper variants

__global__ void fill_unit_kernel(float2* p, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = make_float2(1.f, 0.f);
}

int magpie_set_variant(magpie_ctx* c, int32_t flags) {
  if (!c) return fail(MAGPIE_EINVAL, "NULL context");
  if (flags & ~3) return fail(MAGPIE_EINVAL, "flags: bit 0 MG/OPT correction, bit 1 phase rule");
  if ((flags & 1) && c->p.update_probe) return fail(MAGPIE_EINVAL, "the MG/OPT variant needs update_probe = 0");
  if (flags & 2) {
    const size_t n = (size_t)c->M * c->p.n_pos;
    if (!c->phase) {
      cudaError_t e = cudaMalloc((void**)&c->phase, sizeof(float2) * n);
      if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? MAGPIE_ENOMEM : MAGPIE_ECUDA,
                    std::string("phase buffer: ") + cudaGetErrorString(e));
    }
    fill_unit_kernel<<<1024, 256, 0, c->stream>>>(c->phase, n);
    CUDA_TRY(cudaGetLastError());
  }
  const int old = c->variant;
  c->variant = flags;
  if ((old ^ flags) & 1)
    CUDA_TRY(enqueue_pyramid(c->Q, c->p.m, c->p.levels, c->p.alpha, c->mx, c->pyr_q, c->pyr_u, c->pyr, c->stream,
                             flags & 1));
  invalidate_graphs(c);
  return MAGPIE_OK;
}


int magpie_group_tuning(magpie_group* g, int32_t* minb, float* ms) {
  if (!g || !minb || !ms) return fail(MAGPIE_EINVAL, "NULL argument");
  for (int i = 0; i < 6; ++i) {
    minb[i] = g->minb[i];
    for (int v = 0; v < 3; ++v) ms[3 * i + v] = g->tune_ms[i][v];
  }
  return MAGPIE_OK;
}

int magpie_group_apply_tuning(magpie_group* g, int32_t* shape, int32_t* tile_w, int32_t* tile_h, float* ms) {
  if (!g || !shape || !tile_w || !tile_h || !ms) return fail(MAGPIE_EINVAL, "NULL argument");
  *shape = g->apply_shape;
  for (int v = 0; v < 3; ++v) {
    tile_w[v] = kApplyShapes[v].tw;
    tile_h[v] = kApplyShapes[v].th;
    ms[v] = g->apply_ms[v];
  }
  return MAGPIE_OK;
}

int magpie_group_set_apply_shape(magpie_group* g, int32_t shape) {
  if (!g || shape < 0 || shape > 2) return fail(MAGPIE_EINVAL, "need a group and a shape index in [0, 2]");
  g->apply_shape = shape;
  if (g->graph) {
    cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
  }
  return MAGPIE_OK;
}

int magpie_group_form_tuning(magpie_group* g, int32_t* persistent, float* ms) {
  if (!g || !persistent || !ms) return fail(MAGPIE_EINVAL, "NULL argument");
  *persistent = g->persistent;
  ms[0] = g->form_ms[0];
  ms[1] = g->form_ms[1];
  return MAGPIE_OK;
}

int magpie_group_set_persistent(magpie_group* g, int32_t persistent) {
  if (!g || (persistent != 0 && persistent != 1)) return fail(MAGPIE_EINVAL, "need a group and 0 or 1");
  g->persistent = persistent;
  if (g->graph) {
    cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
  }
  return MAGPIE_OK;
}

int magpie_group_set_wait_limit(magpie_group* g, double seconds) {
  if (!g || !(seconds >= 1e-6 && seconds <= 60.0)) return fail(MAGPIE_EINVAL, "need a group and a limit in [1e-6, 60] s");
  g->limit_ns = (unsigned long long)(seconds * 1e9);
  if (g->graph) {
    cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
  }
  return MAGPIE_OK;
}

int magpie_group_status(magpie_group* g) {
  if (!g) return fail(MAGPIE_EINVAL, "NULL group");
  int h = 0;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  CUDA_TRY(cudaMemcpy(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    CUDA_TRY(cudaMemset(g->err, 0, sizeof(int)));
    return fail(MAGPIE_ETIMEOUT, "a dependency wait of the persistent step kernel ran out; its update tile was skipped");
  }
  return MAGPIE_OK;
}

int magpie_group_check_waits(magpie_group* g, double seconds) {
  if (!g || !(seconds >= 1e-6 && seconds <= 10.0)) return fail(MAGPIE_EINVAL, "need a group and a limit in [1e-6, 10] s");
  int rc = plan_persistent(g);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  const unsigned long long keep = g->limit_ns;
  g->limit_ns = (unsigned long long)(seconds * 1e9);
  cudaError_t e = cudaMemsetAsync(g->qbuf, 0, sizeof(int) * g->qbuf_n, g->stream);
  if (e == cudaSuccess) rc = enqueue_persistent_step(g, 0, g->stream, g->ptable, 1);
  g->limit_ns = keep;
  CUDA_TRY(e);
  if (rc) return rc;
  return magpie_group_status(g);
}

int magpie_group_set_minb(magpie_group* g, int32_t m, int32_t minb) {
  if (!g) return fail(MAGPIE_EINVAL, "NULL group");
  if (m < 8 || m > 256 || (m & (m - 1))) return fail(MAGPIE_EINVAL, "m must be a power of two in [8, 256]");
  int cand[3];
  minb_candidates(m, cand);
  if (minb != cand[0] && minb != cand[1] && minb != cand[2])
    return fail(MAGPIE_EINVAL, "not a candidate register bound for this m");
  g->minb[ilog2(m) - 3] = minb;
  if (g->graph) {
    cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
  }
  return MAGPIE_OK;
}




int magpie_sweep_host_async(magpie_ctx* c, const int32_t* order, const float* intensities, void* object_out) {
  NvtxRange range("magpie_sweep_host_async");
  if (!c || !order || !intensities) return fail(MAGPIE_EINVAL, "NULL argument");
  const size_t N = c->p.n_pos, M = c->M;
  const int b = c->next_buf;
  constexpr int kChunks = 4;
  if (!c->amp2[b]) {
    CUDA_TRY(cudaMalloc((void**)&c->amp2[b], sizeof(float) * N * M));
    CUDA_TRY(cudaMalloc((void**)&c->stage2[b], sizeof(float) * N * M));
    CUDA_TRY(cudaMalloc((void**)&c->order2[b], sizeof(int32_t) * N));
    for (int i = 0; i < kChunks; ++i) CUDA_TRY(cudaEventCreateWithFlags(&c->landed[b][i], cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&c->used[b], cudaEventDisableTiming));
    CUDA_TRY(cudaEventRecord(c->used[b], c->stream));
    for (int i = 0; i < kChunks; ++i)
      if (!c->copy2[i]) CUDA_TRY(cudaStreamCreateWithFlags(&c->copy2[i], cudaStreamNonBlocking));
  }
  // the FP32 path reads the raw intensities and takes square roots in the
  // window kernel (no separate pass); the other paths read square roots
  const bool raw = !c->precision && !c->cnn && !c->p.update_probe;
  if (!c->graph2[b]) {
    float* own = c->amp;
    int32_t* own_order = c->order;
    c->amp = raw ? c->stage2[b] : c->amp2[b];
    c->order = c->order2[b];
    c->amp_raw = raw ? 1 : 0;
    const int rc = capture_sweep(c, &c->graph2[b]);
    c->amp = own;
    c->order = own_order;
    c->amp_raw = 0;
    if (rc) return rc;
  }
  // copy streams: once the sweep before last is done with buffer b, bring in
  // this sweep's permutation and intensities in four chunks and take the
  // square roots; the main stream carries no copy engine work, so nothing of
  // the next sweep's input queues behind this sweep's result
  const size_t total = N * M, per = (total + kChunks - 1) / kChunks;
  for (int i = 0; i < kChunks; ++i) {
    const size_t b0 = i * per, n = b0 >= total ? 0 : std::min(per, total - b0);
    cudaStream_t cs = c->copy2[i];
    CUDA_TRY(cudaStreamWaitEvent(cs, c->used[b], 0));
    if (i == 0)
      CUDA_TRY(cudaMemcpyAsync(c->order2[b], order, sizeof(int32_t) * N, cudaMemcpyHostToDevice, cs));
    if (n) {
      CUDA_TRY(cudaMemcpyAsync(c->stage2[b] + b0, intensities + b0, sizeof(float) * n, cudaMemcpyHostToDevice, cs));
      if (!raw) {
        sqrt_kernel<<<256, 256, 0, cs>>>(c->stage2[b] + b0, c->amp2[b] + b0, n);
        CUDA_TRY(cudaGetLastError());
      }
    }
    CUDA_TRY(cudaEventRecord(c->landed[b][i], cs));
  }
  // main stream: the sweep on buffer b, then the object out -- written by a
  // kernel straight into mapped host memory when object_out is mapped
  // (pinned), else by a copy
  for (int i = 0; i < kChunks; ++i) CUDA_TRY(cudaStreamWaitEvent(c->stream, c->landed[b][i], 0));
  CUDA_TRY(cudaGraphLaunch(c->graph2[b], c->stream));
  CUDA_TRY(cudaEventRecord(c->used[b], c->stream));
  if (object_out) {
    const size_t nz = (size_t)c->p.n_rows * c->p.n_cols;
    cudaPointerAttributes at{};
    const bool mapped = cudaPointerGetAttributes(&at, object_out) == cudaSuccess &&
                        at.type == cudaMemoryTypeHost && at.devicePointer &&
                        ((uintptr_t)at.devicePointer % 16) == 0;
    cudaGetLastError();
    if (mapped) {
      store_host_kernel<<<(int)std::min<size_t>((nz + 255) / 256, 1024), 256, 0, c->stream>>>(
          c->z, (float2*)at.devicePointer, nz);
      CUDA_TRY(cudaGetLastError());
    } else {
      CUDA_TRY(cudaMemcpyAsync(object_out, c->z, sizeof(float2) * nz, cudaMemcpyDeviceToHost, c->stream));
    }
  }
  c->next_buf = b ^ 1;
  return MAGPIE_OK;
}

int32_t magpie_window_blocks(int32_t m) { return supported_m(m) ? cluster_of(m) : 0; }

int magpie_fp32_fma_rate(int32_t iters, double* tflops, double* ms, void* stream) {
  if (!tflops || iters < 1) return fail(MAGPIE_EINVAL, "need tflops and iters >= 1");
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8;  // 8 blocks of 256 threads per SM: 64 warps, the most an SM holds
  cudaStream_t st = (cudaStream_t)stream;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto release = [&]() {
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  cudaError_t e = cudaMalloc(&out, sizeof(float) * (size_t)blocks * 256);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up; the best of the others
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      fma_rate_kernel<<<blocks, 256, 0, st>>>(out, iters, 0.9999999f, 1e-7f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || t < best)) best = t;
  }
  release();
  CUDA_TRY(e);
  const double flops = 2.0 * kFmaChains * (double)iters * blocks * 256.0;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return MAGPIE_OK;
}

int magpie_stage_times(magpie_ctx* c, const int32_t* idx, int32_t count, uint64_t* stamps, int64_t capacity) {
#ifndef MAGPIE_STAGE_TIMES
  (void)c;
  (void)idx;
  (void)count;
  (void)stamps;
  (void)capacity;
  return fail(MAGPIE_EUNSUPPORTED, "this build has no per-stage timestamps (build with MAGPIE_STAGE_TIMES)");
#else
  if (!c || !idx || !stamps) return fail(MAGPIE_EINVAL, "NULL argument");
  if (count < 1 || count > c->p.minibatch) return fail(MAGPIE_EINVAL, "count must lie in [1, minibatch]");
  if (c->precision || c->cnn) return fail(MAGPIE_EINVAL, "per-stage timestamps time the FP32 window kernel");
  const size_t n = (size_t)count * cluster_of(c->p.m) * kStages;
  if (capacity < (int64_t)n) return fail(MAGPIE_EINVAL, "capacity below count * blocks per window * stages");
  CUDA_TRY(cudaMalloc(&c->stamps, sizeof(unsigned long long) * n));
  cudaError_t e = cudaMemsetAsync(c->stamps, 0, sizeof(unsigned long long) * n, c->stream);
  int rc = e == cudaSuccess ? enqueue_step(c, idx, count, c->stream) : MAGPIE_OK;
  if (e == cudaSuccess && rc == MAGPIE_OK)
    e = cudaMemcpyAsync(stamps, c->stamps, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(c->stamps);
  c->stamps = nullptr;
  CUDA_TRY(e);
  if (rc) return rc;
  return read_err(c);
#endif
}

int magpie_sync(magpie_ctx* c) {
  if (!c) return fail(MAGPIE_EINVAL, "NULL context");
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return read_err(c);
}

}  // extern "C"
