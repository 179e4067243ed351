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

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "magpie.h"

namespace {

namespace cg = cooperative_groups;

constexpr int kVersion = 10100;  // 1.1.0
constexpr int kMaxMinibatch = 4096;  // the update kernel keeps the minibatch's corners in smem (48 KiB)
constexpr int kMaxCluster = 8;       // largest number of blocks per window

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return f2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return f2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return f2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return f2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ float2 cmul_cj(float2 a, float2 b) {
  return f2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// a * w (forward) or a * conj(w) (inverse)
template <bool INV>
__device__ __forceinline__ float2 twmul(float2 a, float2 w) {
  return INV ? f2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y) : cmul(a, w);
}

// cos and sin of 2 pi r / 16 (exact decimal expansions of cos(pi/8),
// cos(pi/4), sin(pi/8)); indices are compile-time after unrolling.
__host__ __device__ constexpr float cos16(int r) {
  return r == 0 ? 1.0f : r == 1 ? 0.92387953251128675613f : r == 2 ? 0.70710678118654752440f
       : r == 3 ? 0.38268343236508977173f : r == 4 ? 0.0f : r == 5 ? -0.38268343236508977173f
       : r == 6 ? -0.70710678118654752440f : r == 7 ? -0.92387953251128675613f : r == 8 ? -1.0f
       : r == 9 ? -0.92387953251128675613f : r == 10 ? -0.70710678118654752440f
       : r == 11 ? -0.38268343236508977173f : r == 12 ? 0.0f : r == 13 ? 0.38268343236508977173f
       : r == 14 ? 0.70710678118654752440f : 0.92387953251128675613f;
}
__host__ __device__ constexpr float sin16(int r) { return cos16((r + 12) & 15); }

// a * exp(-2 pi i r / 16) (forward) or exp(+2 pi i r / 16) (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot16(float2 a, int r) {
  r &= 15;
  if (r == 0) return a;
  if (r == 8) return f2(-a.x, -a.y);
  if (r == 4) return INV ? f2(-a.y, a.x) : f2(a.y, -a.x);
  if (r == 12) return INV ? f2(a.y, -a.x) : f2(-a.y, a.x);
  const float c = cos16(r);
  const float s = INV ? sin16(r) : -sin16(r);
  return f2(a.x * c - a.y * s, a.x * s + a.y * c);
}

template <int N>
__host__ __device__ constexpr int bitrev(int k) {
  int r = 0;
  for (int b = 1; b < N; b <<= 1) {
    r = (r << 1) | (k & 1);
    k >>= 1;
  }
  return r;
}

// In-register N-point DFT (N <= 16): radix-2 decimation in frequency, then
// the bit-reversal permutation (register renaming only).  Unnormalised.
template <int N, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&a)[N]) {
#pragma unroll
  for (int len = N; len >= 2; len >>= 1) {
    const int half = len >> 1;
#pragma unroll
    for (int s = 0; s < N; s += len) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const float2 u = a[s + j];
        const float2 v = a[s + j + half];
        a[s + j] = cadd(u, v);
        a[s + j + half] = rot16<INV>(csub(u, v), j * (16 / len));
      }
    }
  }
  float2 b[N];
#pragma unroll
  for (int k = 0; k < N; ++k) b[k] = a[bitrev<N>(k)];
#pragma unroll
  for (int k = 0; k < N; ++k) a[k] = b[k];
}

// ------------------------------------------------------ per-size geometry
// An MS x MS window is handled by a cluster of CL thread blocks.  Block q owns
// a slab of SLAB = MS / CL lines: rows q*SLAB.. of the row-slab buffer X and
// columns q*SLAB.. of the column-slab buffer Y.  An MS-point line is split
// over G lanes of one warp holding E = MS / G points each; SLAB is a multiple
// of E and of G, so every cross-slab store below targets a compile-time rank.
template <int MS> struct Cfg;
template <> struct Cfg<8> { static constexpr int E = 4, G = 2, CL = 1; };
template <> struct Cfg<16> { static constexpr int E = 4, G = 4, CL = 1; };
template <> struct Cfg<32> { static constexpr int E = 8, G = 4, CL = 1; };
template <> struct Cfg<64> { static constexpr int E = 8, G = 8, CL = 2; };
template <> struct Cfg<128> { static constexpr int E = 16, G = 8, CL = 4; };
template <> struct Cfg<256> { static constexpr int E = 16, G = 16, CL = 8; };

template <int MS> struct Geo {
  static constexpr int E = Cfg<MS>::E, G = Cfg<MS>::G, CL = Cfg<MS>::CL;
  static_assert(E * G == MS && G <= E && G <= 32, "line split");
  static constexpr int SLAB = MS / CL;
  static_assert(CL == 1 || (SLAB % E == 0 && SLAB % G == 0 && SLAB >= 8), "slab split");
  static constexpr int M = MS * MS;
  static constexpr int LANES = SLAB * G;  // one lane group per line of the slab
  static constexpr int T = LANES < 32 ? 32 : LANES;
  static_assert(T <= 1024 && T % 32 == 0, "block size");
  static constexpr int XN = SLAB * MS;  // complex entries of each of X and Y
  static constexpr int LVL = (MS / 4) * (SLAB / 4) * 2 + 4 * CL * CL + 32;
  // resident blocks per SM the register budget is sized for (two 4-block
  // windows' worth of slabs share an SM for m = 128)
  static constexpr int MIN_BLOCKS = (T >= 256 && T < 512) ? 2 : 1;
  static constexpr size_t SMEM = sizeof(float2) * (2 * size_t(XN) + MS + LVL) + sizeof(double) * 64;
};

// XOR swizzle of the column index by the row index, within rows of width W:
// with it, 8 consecutive rows of one column, 4 consecutive rows of 8
// consecutive columns, and the transposed exchange reads all hit distinct
// bank pairs (for both warp halves of an 8-byte access).
template <int W>
__device__ __forceinline__ int swz(int r) {
  return ((((r & 1) << 3) | (((r >> 1) & 3) << 1))) & (W - 1);
}
// X: [SLAB][MS], Y: [MS][SLAB], both row-major with the swizzle.
template <int MS>
__device__ __forceinline__ int xi(int rho, int c) {
  return rho * MS + (c ^ swz<MS>(rho));
}
template <int MS>
__device__ __forceinline__ int yi(int r, int gam) {
  constexpr int S = Geo<MS>::SLAB;
  return r * S + (gam ^ swz<S>(r));
}

// Split barrier over the window's blocks: arrive (releasing this thread's
// earlier shared-memory writes, local and remote) ... independent work ...
// wait (acquiring the other blocks' writes).  With CL = 1 the wait is an
// ordinary block barrier.
template <int CL>
__device__ __forceinline__ void window_arrive() {
  if constexpr (CL > 1) asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
template <int CL>
__device__ __forceinline__ void window_wait() {
  if constexpr (CL > 1)
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  else
    __syncthreads();
}

// Barrier over the window's blocks; with CL = 1 an ordinary block barrier.
template <int CL>
__device__ __forceinline__ void window_sync() {
  if constexpr (CL > 1)
    cg::this_cluster().sync();
  else
    __syncthreads();
}
// The same shared-memory object in block `rank` of the window's cluster.
template <int CL, typename P>
__device__ __forceinline__ P* peer(P* p, int rank) {
  if constexpr (CL > 1)
    return cg::this_cluster().map_shared_rank(p, rank);
  else
    return p;
}

// Forward (INV=false) MS-point transform of one line whose lanes hold the
// input x[e] = line[g + G e].  On return x[j G + k2] = X[g + G j + E k2].
// slot(s) addresses the line's MS slots in shared memory (the exchange
// buffer); tw[t] = exp(-2 pi i t / MS).
template <int MS, bool INV, class Slot>
__device__ __forceinline__ void line_fwd(float2 (&x)[Cfg<MS>::E], int g, bool act, Slot slot, const float2* tw) {
  constexpr int E = Cfg<MS>::E, G = Cfg<MS>::G;
  dft_reg<E, INV>(x);
#pragma unroll
  for (int k1 = 1; k1 < E; ++k1) x[k1] = twmul<INV>(x[k1], tw[(g * k1) & (MS - 1)]);
  if constexpr (G > 1) {
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1)
      if (act) slot(k1 * G + (g ^ (k1 & (G - 1)))) = x[k1];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < E / G; ++j) {
      const int k1 = g + G * j;
      float2 v[G];
#pragma unroll
      for (int gp = 0; gp < G; ++gp) v[gp] = act ? slot(k1 * G + (gp ^ g)) : f2(0.f, 0.f);
      dft_reg<G, INV>(v);
#pragma unroll
      for (int k2 = 0; k2 < G; ++k2) x[j * G + k2] = v[k2];
    }
    __syncwarp();
  }
}

// Unnormalised inverse of line_fwd: input in line_fwd's output distribution,
// output x[e] = sum_k X[k] exp(+2 pi i k (g + G e) / MS).
template <int MS, class Slot>
__device__ __forceinline__ void line_inv(float2 (&x)[Cfg<MS>::E], int g, bool act, Slot slot, const float2* tw) {
  constexpr int E = Cfg<MS>::E, G = Cfg<MS>::G;
  if constexpr (G > 1) {
#pragma unroll
    for (int j = 0; j < E / G; ++j) {
      const int k1 = g + G * j;
      float2 v[G];
#pragma unroll
      for (int k2 = 0; k2 < G; ++k2) v[k2] = x[j * G + k2];
      dft_reg<G, true>(v);
#pragma unroll
      for (int gp = 0; gp < G; ++gp) {
        const float2 t = gp ? twmul<true>(v[gp], tw[(gp * k1) & (MS - 1)]) : v[0];
        if (act) slot(k1 * G + (gp ^ g)) = t;
      }
    }
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) x[k1] = act ? slot(k1 * G + (g ^ (k1 & (G - 1)))) : f2(0.f, 0.f);
    __syncwarp();
  }
  dft_reg<E, true>(x);
}

// Offset of level-l (l >= 1) factor arrays in the float pyramid buffer:
// [u^0: M][w^0: M] then per level l = 1.. : [W_u^{l-1}][1/w^l][u^l/w^l],
// each (MS >> l)^2 floats.
__host__ __device__ __forceinline__ int lvl_off(int MS, int l) {
  int off = 2 * MS * MS;
  for (int j = 1; j < l; ++j) off += 3 * (MS >> j) * (MS >> j);
  return off;
}
__host__ __device__ __forceinline__ int pyr_size(int MS, int L) { return lvl_off(MS, L); }

enum Mode { kStep = 0, kEval = 1, kSim = 2 };

struct StepArgs {
  const float2* z;    // object [n_rows][n_cols]
  int n_rows, n_cols;
  const float2* Q;    // probe [MS][MS]
  const float2* tw;   // exp(-2 pi i t / MS), t < MS
  const float* amp;   // amplitudes sqrt(d) [n_pos][MS][MS]
  float* out_int;     // forward intensities [n_pos][MS][MS] (kSim)
  const int32_t* pos; // [n_pos][2]
  const int32_t* idx; // window of each cluster
  int n_pos;
  float2* contrib;    // [windows][MS][MS] increments w . Delta
  const float* pyr;   // per-level factors
  int levels;
  double* part;       // [windows][CL][2] block partials of the window's two sums
  float2* pnum;       // probe step only: [windows][MS][MS] conj(z_k)(R_k - Q z_k)
  float* pa2;         // probe step only: [windows][MS][MS] |z_k|^2
  double* pmax;       // probe step only: [windows][CL] block maxima of |z_k|^2
  int* err;           // bit 0: window index out of range
};

__device__ __forceinline__ double block_sum(double v, double* red, int tid, int nthreads) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (tid == 0)
    for (int i = 0; i < nthreads / 32; ++i) r += red[i];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_max(double v, double* red, int tid, int nthreads) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (tid == 0)
    for (int i = 0; i < nthreads / 32; ++i) r = fmax(r, red[i]);
  __syncthreads();
  return r;
}

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return f2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// MAGPS V-cycle of one window in residual form, on this block's column slab
// Y (g^0 for MS rows x SLAB columns).  Lane gamma of a warp owns column
// gamma of a strip of 2^TT rows; the 2x2 restrictions pair columns by warp
// shuffles.  Levels coarser than TT are kept in `lvl` (local levels up to
// log2(SLAB); coarser ones span the cluster and are finished by block 0).
template <int MS, int TT>
__device__ __forceinline__ void vcycle(const float2* Y, float2* lvl, const float* pyr, int L, int q, float2* out,
                                       int tid) {
  using Gm = Geo<MS>;
  constexpr int SLAB = Gm::SLAB, T = Gm::T, CL = Gm::CL, H = 1 << TT, NS = MS / H, SPAR = T / SLAB;
  constexpr int LLOC = (SLAB >= 32) ? 5 : (SLAB == 16 ? 4 : 3);  // log2(SLAB)
  static_assert((1 << LLOC) == SLAB, "slab levels");
  const int gam = tid % SLAB, s0 = tid / SLAB;
  const int cgl = q * SLAB + gam;  // column in the window
  const bool deep = (L - 1) > TT;
  const float* u0 = pyr;
  const float* wu1 = pyr + lvl_off(MS, 1);
  const float* iw1 = wu1 + (MS / 2) * (MS / 2);
  const float* rr1 = iw1 + (MS / 2) * (MS / 2);
  // offsets of the slab's level arrays (levels TT .. LLOC) in lvl
  auto off = [](int l) {
    int o = 0;
    for (int j = TT; j < l; ++j) o += (MS >> j) * (SLAB >> j);
    return o;
  };

  // g at level TT of the 2^TT x 2^TT bin of column cgl in strip s (the same
  // value in all 2^TT lanes of the bin); g0 and g1 keep the finer levels.
  auto strip = [&](int s, bool ok, float2 (&g0)[H], float2 (&g1)[H / 2]) -> float2 {
    const int R0 = s * H;
#pragma unroll
    for (int a = 0; a < H; ++a) g0[a] = ok ? Y[yi<MS>(R0 + a, gam)] : f2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < H / 2; ++a) {
      float2 v = cadd(g0[2 * a], g0[2 * a + 1]);
      v = cadd(v, shfl_xor2(v, 1));
      const float w = ok ? __ldg(&wu1[(R0 / 2 + a) * (MS / 2) + (cgl >> 1)]) : 0.f;
      g1[a] = cscale(v, 0.25f * w);
    }
    if constexpr (TT == 1) {
      return g1[0];
    } else {
      float2 v = cadd(g1[0], g1[1]);
      v = cadd(v, shfl_xor2(v, 2));
      const float w = ok ? __ldg(&pyr[lvl_off(MS, 2) + (R0 / 4) * (MS / 4) + (cgl >> 2)]) : 0.f;
      return cscale(v, 0.25f * w);
    }
  };

  if (deep) {
    // phase 1: level-TT values of every strip bin
    for (int base = 0; base < NS; base += SPAR) {
      const int s = base + s0;
      const bool ok = s < NS;
      float2 g0[H], g1[H / 2];
      const float2 gT = strip(s, ok, g0, g1);
      if (ok && (gam & (H - 1)) == 0) lvl[off(TT) + s * (SLAB >> TT) + (gam >> TT)] = gT;
    }
    __syncthreads();
    // phase 2: restrictions inside the slab, levels TT+1 .. min(L-1, LLOC)
    const int ltop = (L - 1) < LLOC ? (L - 1) : LLOC;
    for (int l = TT; l < ltop; ++l) {
      const int rows = MS >> (l + 1), cols = SLAB >> (l + 1), fc = SLAB >> l;
      const float2* fine = lvl + off(l);
      float2* coarse = lvl + off(l + 1);
      const float* wu = pyr + lvl_off(MS, l + 1);
      for (int i = tid; i < rows * cols; i += T) {
        const int r = i / cols, c = i - (i / cols) * cols;
        const float2 sm = cadd(cadd(fine[(2 * r) * fc + 2 * c], fine[(2 * r) * fc + 2 * c + 1]),
                               cadd(fine[(2 * r + 1) * fc + 2 * c], fine[(2 * r + 1) * fc + 2 * c + 1]));
        coarse[i] = cscale(sm, 0.25f * __ldg(&wu[r * (MS >> (l + 1)) + q * cols + c]));
      }
      __syncthreads();
    }
    if (L - 1 <= LLOC) {
      // coarsest level inside the slab
      const int l = L - 1, rows = MS >> l, cols = SLAB >> l;
      float2* a = lvl + off(l);
      const float* iw = pyr + lvl_off(MS, l) + (MS >> l) * (MS >> l);
      for (int i = tid; i < rows * cols; i += T) {
        const int r = i / cols, c = i - (i / cols) * cols;
        a[i] = cscale(a[i], __ldg(&iw[r * (MS >> l) + q * cols + c]));
      }
      __syncthreads();
    } else {
      if constexpr (CL > 1) {
        // levels LLOC .. L-1 span the cluster: block 0 gathers the CL x CL
        // level-LLOC values (column qq from block qq), runs the coarse
        // levels, and sends back level-LLOC increments.
        window_sync<CL>();
        if (q == 0 && tid == 0) {
          float2* gl = lvl + off(LLOC + 1);  // global arrays of levels LLOC.. in block 0
          auto goff = [](int i) {  // offset of level LLOC + i
            int o = 0;
            for (int l = LLOC; l < LLOC + i; ++l) o += (MS >> l) * (MS >> l);
            return o;
          };
          for (int qq = 0; qq < CL; ++qq) {
            const float2* src = peer<CL>(lvl, qq) + off(LLOC);
            for (int i = 0; i < CL; ++i) gl[i * CL + qq] = src[i];
          }
          for (int l = LLOC; l < L - 1; ++l) {
            const int n = MS >> (l + 1), nf = MS >> l;
            const float2* fine = gl + goff(l - LLOC);
            float2* coarse = gl + goff(l - LLOC + 1);
            const float* wu = pyr + lvl_off(MS, l + 1);
            for (int i = 0; i < n * n; ++i) {
              const int r = i / n, c = i % n;
              const float2 sm = cadd(cadd(fine[(2 * r) * nf + 2 * c], fine[(2 * r) * nf + 2 * c + 1]),
                                     cadd(fine[(2 * r + 1) * nf + 2 * c], fine[(2 * r + 1) * nf + 2 * c + 1]));
              coarse[i] = cscale(sm, 0.25f * wu[i]);
            }
          }
          {
            const int l = L - 1, n = MS >> l;
            float2* a = gl + goff(l - LLOC);
            const float* iw = pyr + lvl_off(MS, l) + n * n;
            for (int i = 0; i < n * n; ++i) a[i] = cscale(a[i], iw[i]);
          }
          for (int l = L - 2; l >= LLOC; --l) {
            const int n = MS >> l, nc = n >> 1;
            float2* a = gl + goff(l - LLOC);
            const float2* pe = gl + goff(l - LLOC + 1);
            const float* iw = pyr + lvl_off(MS, l) + n * n;
            const float* rr = iw + n * n;
            for (int i = 0; i < n * n; ++i) {
              const int r = i / n, c = i % n;
              const float2 p = pe[(r >> 1) * nc + (c >> 1)];
              const float2 v = cscale(a[i], iw[i]);
              a[i] = f2(v.x + rr[i] * p.x, v.y + rr[i] * p.y);
            }
          }
          for (int qq = 0; qq < CL; ++qq) {
            float2* dst = peer<CL>(lvl, qq) + off(LLOC);
            for (int i = 0; i < CL; ++i) dst[i] = gl[i * CL + qq];
          }
        }
        window_sync<CL>();
      }
    }
    // up-pass inside the slab down to level TT
    const int lstart = ((L - 1) < LLOC ? (L - 1) : LLOC) - 1;
    for (int l = lstart; l >= TT; --l) {
      const int rows = MS >> l, cols = SLAB >> l, cc = cols >> 1;
      float2* a = lvl + off(l);
      const float2* pe = lvl + off(l + 1);
      const float* iw = pyr + lvl_off(MS, l) + (MS >> l) * (MS >> l);
      const float* rr = iw + (MS >> l) * (MS >> l);
      for (int i = tid; i < rows * cols; i += T) {
        const int r = i / cols, c = i - (i / cols) * cols;
        const int o = r * (MS >> l) + q * cols + c;
        const float2 p = pe[(r >> 1) * cc + (c >> 1)];
        const float2 v = cscale(a[i], __ldg(&iw[o]));
        const float w = __ldg(&rr[o]);
        a[i] = f2(v.x + w * p.x, v.y + w * p.y);
      }
      __syncthreads();
    }
  }
  // phase 3: per strip, the up-pass to level 0 and the increments w . Delta
  const float* iwT = pyr + lvl_off(MS, TT) + (MS >> TT) * (MS >> TT);
  for (int base = 0; base < NS; base += SPAR) {
    const int s = base + s0;
    const bool ok = s < NS;
    float2 g0[H], g1[H / 2];
    const float2 gT = strip(s, ok, g0, g1);
    const int R0 = s * H;
    float2 eT = f2(0.f, 0.f);
    if (ok) {
      eT = deep ? lvl[off(TT) + s * (SLAB >> TT) + (gam >> TT)]
                : cscale(gT, __ldg(&iwT[(R0 >> TT) * (MS >> TT) + (cgl >> TT)]));
    }
    float2 e1[H / 2];
    if constexpr (TT == 1) {
      e1[0] = eT;
    } else {
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int o = (R0 / 2 + a) * (MS / 2) + (cgl >> 1);
        const float2 v = cscale(g1[a], ok ? __ldg(&iw1[o]) : 0.f);
        const float w = ok ? __ldg(&rr1[o]) : 0.f;
        e1[a] = f2(v.x + w * eT.x, v.y + w * eT.y);
      }
    }
    if (ok) {
#pragma unroll
      for (int a = 0; a < H; ++a) {
        const int o = (R0 + a) * MS + cgl;
        const float u = __ldg(&u0[o]);
        out[o] = f2(g0[a].x + u * e1[a >> 1].x, g0[a].y + u * e1[a >> 1].y);
      }
    }
  }
}

// One cluster of Geo<MS>::CL blocks per window (grid = windows * CL), each
// with Geo<MS>::T threads and Geo<MS>::SMEM bytes of dynamic shared memory.
template <int MS, int MODE>
__global__ void __launch_bounds__(Geo<MS>::T, Geo<MS>::MIN_BLOCKS) window_kernel(StepArgs A) {
  using Gm = Geo<MS>;
  constexpr int E = Gm::E, G = Gm::G, CL = Gm::CL, SLAB = Gm::SLAB, T = Gm::T, M = Gm::M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* X = reinterpret_cast<float2*>(smem_raw);  // row slab
  float2* Y = X + Gm::XN;                            // column slab
  float2* tws = Y + Gm::XN;
  float2* lvl = tws + MS;
  double* red = reinterpret_cast<double*>(lvl + Gm::LVL);  // block_sum scratch

  const int tid = threadIdx.x;
  int q = 0;
  if constexpr (CL > 1) q = (int)cg::this_cluster().block_rank();
  const int win = blockIdx.x / CL;
  for (int i = tid; i < MS; i += T) tws[i] = A.tw[i];
  const int k = A.idx[win];
  if ((unsigned)k >= (unsigned)A.n_pos) {
    if (tid == 0 && q == 0) atomicOr(A.err, 1);
    return;  // uniform across the cluster
  }
  const int pr = A.pos[2 * k], pc = A.pos[2 * k + 1];
  const float2* zk = A.z + (size_t)pr * A.n_cols + pc;
  __syncthreads();

  const bool act = tid < Gm::LANES;
  const int lam = act ? tid / G : 0, g = tid % G;
  const int line = q * SLAB + lam;  // column (passes A, C) or row (pass B) of this lane group

  // slab geometry of the row-coalesced passes: lane gam of a row of the
  // block's column slab, rows r0, r0 + RSTEP, ...
  constexpr int RSTEP = T / SLAB, RPT = MS / RSTEP;
  const int gam = tid % SLAB, r0 = tid / SLAB;
  const int cgl = q * SLAB + gam;

  // ---- pass A: exit wave psi = Q z_k gathered row by row into Y, then the
  // column FFTs; results go to the row owners' X
  {
    float2 pv[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = r0 + RSTEP * i;
      pv[i] = cmul(__ldg(&A.Q[r * MS + cgl]), __ldg(&zk[(size_t)r * A.n_cols + cgl]));
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) Y[yi<MS>(r0 + RSTEP * i, gam)] = pv[i];
    __syncthreads();
    float2 x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = act ? Y[yi<MS>(g + G * e, lam)] : f2(0.f, 0.f);
    __syncwarp();
    line_fwd<MS, false>(x, g, act, [&](int sl) -> float2& { return Y[yi<MS>(sl, lam)]; }, tws);
#pragma unroll
    for (int j = 0; j < E / G; ++j)
#pragma unroll
      for (int k2 = 0; k2 < G; ++k2) {
        const int kr = g + G * j + E * k2;
        float2* dst = peer<CL>(X, (E * k2) / SLAB);
        if (act) dst[xi<MS>(kr % SLAB, line)] = x[j * G + k2];
      }
  }
  window_arrive<CL>();
  // amplitudes of this block's rows, fetched while the other blocks finish
  float av[E];
  if constexpr (MODE != kSim) {
    const float* ampr = A.amp + (size_t)k * M + line * MS;
#pragma unroll
    for (int j = 0; j < E / G; ++j)
#pragma unroll
      for (int k2 = 0; k2 < G; ++k2) av[j * G + k2] = act ? __ldg(&ampr[g + G * j + E * k2]) : 0.f;
  }
  window_wait<CL>();

  // ---- pass B: row FFTs, modulus projection, inverse row FFTs; results go
  // to the column owners' Y
  float res = 0.f;
  {
    const int kr = line;
    float2 x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = act ? X[xi<MS>(lam, g + G * e)] : f2(0.f, 0.f);
    __syncwarp();
    line_fwd<MS, false>(x, g, act, [&](int sl) -> float2& { return X[xi<MS>(lam, sl)]; }, tws);
    if constexpr (MODE == kSim) {
      float* outk = A.out_int + (size_t)k * M + kr * MS;
#pragma unroll
      for (int j = 0; j < E / G; ++j)
#pragma unroll
        for (int k2 = 0; k2 < G; ++k2) {
          const float2 P = x[j * G + k2];
          if (act) outk[g + G * j + E * k2] = P.x * P.x + P.y * P.y;
        }
      return;  // no block reads another block's memory after the barrier above
    } else {
      constexpr float inv_m = 1.0f / float(M);
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const float a = av[i];
        const float2 P = x[i];
        const float p2 = P.x * P.x + P.y * P.y;
        float mag;
        float2 Pp;
        if (p2 > 0.f) {
          const float rs = rsqrtf(p2);
          mag = p2 * rs;
          const float sc = a * rs * inv_m;
          Pp = f2(P.x * sc, P.y * sc);
        } else {
          mag = 0.f;
          Pp = f2(a * inv_m, 0.f);
        }
        const float dlt = mag - a;
        res += dlt * dlt;
        x[i] = Pp;
      }
      line_inv<MS>(x, g, act, [&](int sl) -> float2& { return X[xi<MS>(lam, sl)]; }, tws);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int c = g + G * e;
        float2* dst = peer<CL>(Y, (G * e) / SLAB);
        if (act) dst[yi<MS>(kr, c % SLAB)] = x[e];
      }
    }
  }
  if constexpr (MODE != kSim) {
    window_arrive<CL>();
    // the exit wave again, row by row, while the other blocks finish pass B;
    // it is parked in X (free once every block of the window is past pass B)
    float2 pv[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = r0 + RSTEP * i;
      pv[i] = cmul(__ldg(&A.Q[r * MS + cgl]), __ldg(&zk[(size_t)r * A.n_cols + cgl]));
    }
    window_wait<CL>();
#pragma unroll
    for (int i = 0; i < RPT; ++i) X[yi<MS>(r0 + RSTEP * i, gam)] = pv[i];

    // ---- pass C: inverse column FFTs; R_k into Y
    {
      float2 x[E];
#pragma unroll
      for (int j = 0; j < E / G; ++j)
#pragma unroll
        for (int k2 = 0; k2 < G; ++k2) x[j * G + k2] = act ? Y[yi<MS>(g + G * j + E * k2, lam)] : f2(0.f, 0.f);
      __syncwarp();
      line_inv<MS>(x, g, act, [&](int sl) -> float2& { return Y[yi<MS>(sl, lam)]; }, tws);
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (act) Y[yi<MS>(g + G * e, lam)] = x[e];
    }
    __syncthreads();

    // ---- g^0 = conj(Q)(R_k - psi) over the slab, lane = column; into Y, or
    // straight to the increments for one level
    float gn2 = 0.f, amax = 0.f;
    float2* out = A.contrib + (size_t)win * M;
    const bool direct = (MODE == kStep) && A.levels == 1;
    {
      float2 qv[RPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i) qv[i] = __ldg(&A.Q[(r0 + RSTEP * i) * MS + cgl]);
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = r0 + RSTEP * i;
        const int o = yi<MS>(r, gam);
        const float2 rho = csub(Y[o], X[o]);
        const float2 gg = cmul_cj(qv[i], rho);
        gn2 += gg.x * gg.x + gg.y * gg.y;
        if (MODE == kStep) {
          if (A.pnum) {
            // the probe step's window terms (same R_k and z_k)
            const float2 zz = __ldg(&zk[(size_t)r * A.n_cols + cgl]);
            const float a2 = zz.x * zz.x + zz.y * zz.y;
            A.pnum[(size_t)win * M + r * MS + cgl] = cmul_cj(zz, rho);
            A.pa2[(size_t)win * M + r * MS + cgl] = a2;
            amax = fmaxf(amax, a2);
          }
          if (direct)
            out[r * MS + cgl] = gg;
          else
            Y[o] = gg;
        }
      }
    }
    if (MODE == kStep && A.pnum) {
      const double bm = block_max((double)amax, red, tid, T);
      if (tid == 0) A.pmax[win * CL + q] = bm;
    }

    // block partials of the window's two sums (float64); the kernel that
    // follows combines them in block order
    const double rs = block_sum((double)res, red, tid, T);
    const double gs = block_sum((double)gn2, red, tid, T);
    if (tid == 0) {
      A.part[(size_t)(win * CL + q) * 2] = rs;
      A.part[(size_t)(win * CL + q) * 2 + 1] = gs;
    }
    if (MODE != kStep || direct) return;

    // ---- pass D: MAGPS V-cycle (levels >= 2) on the column slab
    if (A.levels == 2)
      vcycle<MS, 1>(Y, lvl, A.pyr, A.levels, q, out, tid);
    else
      vcycle<MS, 2>(Y, lvl, A.pyr, A.levels, q, out, tid);
  }
}

// z += sum_b contrib_b / sum_b w0 over the windows covering each pixel, in
// minibatch order (bitwise reproducible).  One block of 256 threads per
// 16 x 16 object tile, one pixel per thread: the block first lists, in
// minibatch order, the windows that overlap its tile (a ballot compaction by
// warp 0); each thread then walks that short list four entries at a time with
// predicated loads, so several increments are in flight per thread.
// Dynamic smem: count int2 corners + count ints.
constexpr int kApplyTile = 16;
__global__ void __launch_bounds__(256) apply_kernel(float2* z, int n_rows, int n_cols, const int32_t* pos,
                                                    const int32_t* idx, int count, int n_pos,
                                                    const float2* contrib, const float* w0, int MS,
                                                    const double* part, int CL, double* phi_pos, double* gn_pos) {
  extern __shared__ int2 corner[];
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    // the window kernel's block partials -> Phi_k and ||grad Phi_k||, in block order
    for (int b = threadIdx.x; b < count; b += blockDim.x) {
      const int k = idx[b];
      if ((unsigned)k >= (unsigned)n_pos) continue;
      double a = 0.0, g = 0.0;
      for (int q = 0; q < CL; ++q) {
        a += part[(size_t)(b * CL + q) * 2];
        g += part[(size_t)(b * CL + q) * 2 + 1];
      }
      phi_pos[k] = a / (2.0 * (double)MS * (double)MS);
      gn_pos[k] = sqrt(g);
    }
  }
  int* list = reinterpret_cast<int*>(corner + count);
  __shared__ int n_list;
  const int R0 = blockIdx.y * kApplyTile, C0 = blockIdx.x * kApplyTile;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const int k = idx[i];
    corner[i] = ((unsigned)k < (unsigned)n_pos) ? make_int2(pos[2 * k], pos[2 * k + 1])
                                                : make_int2(-(1 << 30), -(1 << 30));
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const unsigned lane = threadIdx.x;
    int base = 0;
    for (int b0 = 0; b0 < count; b0 += 32) {
      const int b = b0 + (int)lane;
      bool hit = false;
      if (b < count) {
        const int2 q = corner[b];
        hit = q.x < R0 + kApplyTile && q.x + MS > R0 && q.y < C0 + kApplyTile && q.y + MS > C0;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, hit);
      if (hit) list[base + __popc(mask & ((1u << lane) - 1u))] = b;
      base += __popc(mask);
    }
    if (lane == 0) n_list = base;
  }
  __syncthreads();
  const int nl = n_list;
  const int r = R0 + (threadIdx.x >> 4), c = C0 + (threadIdx.x & 15);
  if (r >= n_rows || c >= n_cols) return;
  const size_t M = (size_t)MS * MS;
  float nx = 0.f, ny = 0.f, d = 0.f;
  for (int j0 = 0; j0 < nl; j0 += 4) {
    float2 v[4];
    float wv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = j0 + u;
      const int b = j < nl ? list[j] : 0;
      const int2 q = corner[b];
      const int dr = r - q.x, dc = c - q.y;
      const bool in = j < nl && (unsigned)dr < (unsigned)MS && (unsigned)dc < (unsigned)MS;
      const int o = in ? dr * MS + dc : 0;
      v[u] = in ? contrib[(size_t)b * M + o] : make_float2(0.f, 0.f);
      wv[u] = in ? __ldg(&w0[o]) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      nx += v[u].x;
      ny += v[u].y;
      d += wv[u];
    }
  }
  if (d > 0.f) {
    const size_t p = (size_t)r * n_cols + c;
    float2 zz = z[p];
    zz.x += nx / d;
    zz.y += ny / d;
    z[p] = zz;
  }
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
                                                            double* utop, float* pyr) {
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
      base[o] = wu;
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
                                                           float* pyr) {
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
      base[i] = wu;
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

// Launch with a cluster dimension when cl > 1.
template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, int cl,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  int n = 0;
  if (cl > 1) {
    attr[n].id = cudaLaunchAttributeClusterDimension;
    attr[n].val.clusterDim.x = cl;
    attr[n].val.clusterDim.y = 1;
    attr[n].val.clusterDim.z = 1;
    ++n;
  }
  cfg.attrs = attr;
  cfg.numAttrs = n;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int MS, int MODE>
cudaError_t launch_window(const StepArgs& a, int windows, cudaStream_t st) {
  using Gm = Geo<MS>;
  return launch_ex(window_kernel<MS, MODE>, dim3((unsigned)windows * Gm::CL), dim3(Gm::T), Gm::SMEM, st, Gm::CL, a);
}

// blocks per window of the window kernel for patch side m
int cluster_of(int m) { return m >= 256 ? 8 : m == 128 ? 4 : m == 64 ? 2 : 1; }

// The per-level probe factors of probe Q (float64 arithmetic) into pyr.
// mx: one 8-byte scratch word; qtop/utop: float64 scratch of 2 MS^2 entries.
cudaError_t enqueue_pyramid(const float2* Q, int MS, int L, float alpha, unsigned long long* mx, double2* qtop,
                            double* utop, float* pyr, cudaStream_t st) {
  const int M = MS * MS;
  cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int mb = (M + 255) / 256 < 64 ? (M + 255) / 256 : 64;
  probe_max_kernel<<<mb, 256, 0, st>>>(Q, M, mx);
  const int TS = MS < 16 ? MS : 16;
  pyramid_tile_kernel<<<dim3(MS / TS, MS / TS), TS * TS, 0, st>>>(Q, MS, L, alpha, mx, qtop, utop, pyr);
  int lt = 0;
  while ((TS >> (lt + 1)) >= 1 && lt + 1 <= L - 1) ++lt;
  if (lt < L - 1) pyramid_top_kernel<<<1, 256, 0, st>>>(MS, L, lt, qtop, utop, pyr);
  return cudaGetLastError();
}

cudaError_t launch_apply(float2* z, int n_rows, int n_cols, const int32_t* pos, const int32_t* idx, int count,
                         int n_pos, const float2* contrib, const float* w0, int MS, const double* part,
                         double* phi_pos, double* gn_pos, cudaStream_t st) {
  const dim3 tiles((n_cols + kApplyTile - 1) / kApplyTile, (n_rows + kApplyTile - 1) / kApplyTile);
  return launch_ex(apply_kernel, tiles, dim3(256), (sizeof(int2) + sizeof(int)) * count, st, 1, z, n_rows, n_cols,
                   pos, idx, count, n_pos, contrib, w0, MS, part, cluster_of(MS), phi_pos, gn_pos);
}

template <int MODE>
cudaError_t launch_window_m(int MS, const StepArgs& a, int blocks, cudaStream_t st) {
  switch (MS) {
    case 8: return launch_window<8, MODE>(a, blocks, st);
    case 16: return launch_window<16, MODE>(a, blocks, st);
    case 32: return launch_window<32, MODE>(a, blocks, st);
    case 64: return launch_window<64, MODE>(a, blocks, st);
    case 128: return launch_window<128, MODE>(a, blocks, st);
    case 256: return launch_window<256, MODE>(a, blocks, st);
    default: return cudaErrorInvalidValue;
  }
}

// Opt the window kernels of one size into their dynamic shared memory; done
// before any launch (and so outside stream capture).
template <int MS>
cudaError_t prepare_size() {
  const int bytes = (int)Geo<MS>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(window_kernel<MS, kStep>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel<MS, kEval>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(window_kernel<MS, kSim>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

cudaError_t prepare_kernels(int MS) {
  cudaError_t e = cudaFuncSetAttribute(apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((sizeof(int2) + sizeof(int)) * kMaxMinibatch));
  if (e != cudaSuccess) return e;
  switch (MS) {
    case 8: return prepare_size<8>();
    case 16: return prepare_size<16>();
    case 32: return prepare_size<32>();
    case 64: return prepare_size<64>();
    case 128: return prepare_size<128>();
    case 256: return prepare_size<256>();
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

}  // namespace

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
  double* phi_pos = nullptr;
  double* gn_pos = nullptr;
  double* part = nullptr;     // [n_pos][kMaxCluster][2] per-block partial sums
  unsigned long long* mx = nullptr;  // max |Q|^2 (bits of a double)
  float2* pnum = nullptr;     // probe step: [minibatch][m][m]
  float* pa2 = nullptr;       // probe step: [minibatch][m][m]
  double* pmax = nullptr;     // probe step: [minibatch][kMaxCluster]
  int32_t* iota = nullptr;
  int32_t* order = nullptr;
  double* sums = nullptr;
  int* err = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<cudaEvent_t> events;  // 4 per minibatch step (magpie_profile_sweep)
  // host sweeps: chunked uploads of the intensities on several copy streams
  cudaStream_t copy_streams[4] = {};
  cudaEvent_t copy_done[4] = {};
  cudaEvent_t copy_start = nullptr;
};

namespace {

StepArgs make_args(magpie_ctx* c, const int32_t* idx) {
  StepArgs a{};
  a.z = c->z;
  a.n_rows = c->p.n_rows;
  a.n_cols = c->p.n_cols;
  a.Q = c->Q;
  a.tw = c->tw;
  a.amp = c->amp;
  a.out_int = nullptr;
  a.pos = c->pos;
  a.idx = idx;
  a.n_pos = c->p.n_pos;
  a.contrib = c->contrib;
  a.pyr = c->pyr;
  a.levels = c->p.levels;
  a.part = c->part;
  a.pnum = c->pnum;
  a.pa2 = c->pa2;
  a.pmax = c->pmax;
  a.err = c->err;
  return a;
}

// ev (optional): four events recorded before/after the window kernel and
// before/after the apply kernel.
int enqueue_step(magpie_ctx* c, const int32_t* idx, int count, cudaStream_t st, const cudaEvent_t* ev = nullptr) {
  StepArgs a = make_args(c, idx);
  if (ev) CUDA_TRY(cudaEventRecord(ev[0], st));
  CUDA_TRY(launch_window_m<kStep>(c->p.m, a, count, st));
  if (ev) CUDA_TRY(cudaEventRecord(ev[1], st));
  if (ev) CUDA_TRY(cudaEventRecord(ev[2], st));
  CUDA_TRY(launch_apply(c->z, c->p.n_rows, c->p.n_cols, c->pos, idx, count, c->p.n_pos, c->contrib, c->pyr + c->M,
                        c->p.m, c->part, c->phi_pos, c->gn_pos, st));
  if (c->p.update_probe) {
    probe_apply_kernel<<<(c->M + 255) / 256, 256, 0, st>>>(c->Q, c->M, idx, count, c->p.n_pos, c->pnum, c->pa2,
                                                           c->pmax, cluster_of(c->p.m), c->p.beta);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(enqueue_pyramid(c->Q, c->p.m, c->p.levels, c->p.alpha, c->mx, c->pyr_q, c->pyr_u, c->pyr, st));
  }
  if (ev) CUDA_TRY(cudaEventRecord(ev[3], st));
  return MAGPIE_OK;
}

int build_pyramid(magpie_ctx* c, const void* probe) {
  CUDA_TRY(cudaMemcpyAsync(c->Q, probe, sizeof(float2) * c->M, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(enqueue_pyramid(c->Q, c->p.m, c->p.levels, c->p.alpha, c->mx, c->pyr_q, c->pyr_u, c->pyr, c->stream));
  return MAGPIE_OK;
}

int read_err(magpie_ctx* c) {
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (h) {
    CUDA_TRY(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
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

// Replays (capturing it on first use) the graph of one sweep over the
// permutation already in c->order.
int launch_sweep(magpie_ctx* c) {
  const int N = c->p.n_pos, B = c->p.minibatch;
  if (!c->graph) {
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
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    CUDA_TRY(e);
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
                                 kNoAllocTwBytes + kNoAllocIdxBytes + kNoAllocPartBytes + 8 + 256;
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
  out->err = (int*)b;
  return MAGPIE_OK;
}

}  // namespace

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
    default: return "unknown error";
  }
}

const char* magpie_last_error(void) { return g_last_error.c_str(); }

void magpie_destroy(magpie_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (int i = 0; i < 4; ++i) {
    if (c->copy_streams[i]) cudaStreamDestroy(c->copy_streams[i]);
    if (c->copy_done[i]) cudaEventDestroy(c->copy_done[i]);
  }
  if (c->copy_start) cudaEventDestroy(c->copy_start);
  for (auto e : c->events)
    if (e) cudaEventDestroy(e);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  void* bufs[] = {c->Q, c->tw, c->amp, c->stage, c->pos, c->pyr, c->pyr_q, c->pyr_u, c->contrib,
                  c->phi_pos, c->gn_pos, c->part, c->mx, c->pnum, c->pa2, c->pmax, c->iota, c->order, c->sums, c->err};
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
      (rc = alloc((void**)&c->part, sizeof(double) * 2 * kMaxCluster * N)) ||
      (rc = alloc((void**)&c->mx, sizeof(unsigned long long))) ||
      (p.update_probe && (rc = alloc((void**)&c->pnum, sizeof(float2) * M * p.minibatch))) ||
      (p.update_probe && (rc = alloc((void**)&c->pa2, sizeof(float) * M * p.minibatch))) ||
      (p.update_probe && (rc = alloc((void**)&c->pmax, sizeof(double) * kMaxCluster * p.minibatch))) ||
      (rc = alloc((void**)&c->iota, sizeof(int32_t) * N)) || (rc = alloc((void**)&c->order, sizeof(int32_t) * N)) ||
      (rc = alloc((void**)&c->sums, sizeof(double) * 2)) || (rc = alloc((void**)&c->err, sizeof(int))))
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
  if (!c || !order) return fail(MAGPIE_EINVAL, "NULL argument");
  CUDA_TRY(cudaMemcpyAsync(c->order, order, sizeof(int32_t) * c->p.n_pos, cudaMemcpyDeviceToDevice, c->stream));
  return launch_sweep(c);
}

int magpie_profile_sweep(magpie_ctx* c, const int32_t* order, double* window_ms, double* apply_ms,
                         int32_t* launches) {
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
  a.err = w.err;
  CUDA_TRY(launch_window_m<kStep>(m, a, count, st));
  CUDA_TRY(launch_apply((float2*)object, n_rows, n_cols, positions, w.idx, count, n_pos, w.contrib, w.pyr + m * m, m,
                        w.part, phi, gnorm, st));
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (h) return fail(MAGPIE_EINDEX, "a window index or its position was out of range; that window was skipped");
  return MAGPIE_OK;
}

}  // extern "C"
