// fft_lines.cuh -- complex helpers, in-register DFTs, the per-size split of
// a window over a cluster, the slab layouts and the line FFTs of the MAGPIE
// window kernel.  Included by core.cuh inside namespace magpie_impl.
#pragma once

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return f2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return f2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return f2(a.x * s, a.y * s); }
// The products below spell out their rounding (the second product rounded,
// the first fused into the add): left to the compiler, either product of a
// sum of two could be the fused one, and the choice followed the kernel the
// code was compiled into (its register bound, inlining), so that window
// kernels of different register bounds gave different bits.
__device__ __forceinline__ float dot2(float a, float b, float c, float d) {  // a b + c d
  return __fmaf_rn(a, b, __fmul_rn(c, d));
}
__device__ __forceinline__ float cabs2(float2 a) { return dot2(a.x, a.x, a.y, a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return f2(dot2(a.x, b.x, -a.y, b.y), dot2(a.x, b.y, a.y, b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmul_cj(float2 a, float2 b) {
  return f2(dot2(a.x, b.x, a.y, b.y), dot2(a.x, b.y, -a.y, b.x));
}
// a * w (forward) or a * conj(w) (inverse)
template <bool INV>
__device__ __forceinline__ float2 twmul(float2 a, float2 w) {
  return INV ? f2(dot2(a.x, w.x, a.y, w.y), dot2(a.y, w.x, -a.x, w.y)) : cmul(a, w);
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
  return f2(dot2(a.x, c, -a.y, s), dot2(a.x, s, a.y, c));
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

// ---- programmatic dependent launch.  A kernel launched with the
// programmatic-serialization attribute may begin while the previous kernel in
// its stream is still running.  grid_dep_wait returns once that kernel has
// finished and its memory operations are visible (at once when the launch
// had no such attribute); grid_dep_launch lets the next such kernel begin
// launching its blocks once every block of this grid has called it or exited.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---- mbarriers (the tensor-core kernels' stage barriers)
constexpr int kMaxWaitTries = 1 << 20;  // bound of every mbarrier wait (a try returns within about a microsecond)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
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

