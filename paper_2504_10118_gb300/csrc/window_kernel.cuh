// window_kernel.cuh -- the per-window kernel of the MAGPIE sweep (gather,
// 2-D FFT, modulus projection, inverse FFT, MAGPS V-cycle), its level factor
// layout, and the persistent step kernel of context groups.  Included by
// core.cuh inside namespace magpie_impl.
#pragma once

// Offset of level-l (l >= 1) factor arrays in the float pyramid buffer:
// [u^0: M][w^0: M] then per level l = 1.. : [W_u^{l-1}][1/w^l][u^l/w^l],
// each (MS >> l)^2 floats.
__host__ __device__ __forceinline__ int lvl_off(int MS, int l) {
  int off = 2 * MS * MS;
  for (int j = 1; j < l; ++j) off += 3 * (MS >> j) * (MS >> j);
  return off;
}
__host__ __device__ __forceinline__ int pyr_size(int MS, int L) { return lvl_off(MS, L); }

// kStep: a minibatch step; kStepRecycle: the same with the phase rule of
// Eq. (specification) across visits (phases kept per window); kStepAtomic: a
// minibatch step whose increments are added straight into object-sized
// accumulators with float atomics (the non-deterministic update); kEval: the
// objective only; kSim: forward intensities.
enum Mode { kStep = 0, kEval = 1, kSim = 2, kStepRecycle = 3, kStepAtomic = 4 };

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
  int2* corner;       // step: [windows] top-left corner of each window (far away if skipped)
  float2* pnum;       // probe step only: [windows][MS][MS] conj(z_k)(R_k - Q z_k)
  float* pa2;         // probe step only: [windows][MS][MS] |z_k|^2
  double* pmax;       // probe step only: [windows][CL] block maxima of |z_k|^2
  int* err;           // bit 0: window index out of range
  int grad_only;      // step: write g^0 = conj(Q)(R_k - Q z_k) as the increments and skip the V-cycle
  float2* phase;      // kStepRecycle: [n_pos][MS][MS] unit phase of each spectrum entry at the last visit
  int amp_raw;        // amp holds the intensities d themselves: the kernel uses sqrt(max(d, 0))
  float4* acc;        // kStepAtomic: [n_rows][n_cols] accumulators (sum w.Delta re, im, sum w, unused)
  unsigned long long* stamps;  // builds with MAGPIE_STAGE_TIMES: [windows][CL][kStages] %globaltimer stamps
};

// Per-stage timestamps of the window kernel (thread 0 of every block), for
// builds with MAGPIE_STAGE_TIMES defined; compiled out otherwise.
constexpr int kStages = 10;
#ifdef MAGPIE_STAGE_TIMES
#define MAGPIE_STAMP(stage)                                                          \
  do {                                                                               \
    if (tid == 0 && A.stamps) {                                                      \
      unsigned long long t_;                                                         \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                         \
      A.stamps[((size_t)win * Geo<MS>::CL + q) * kStages + (stage)] = t_;            \
    }                                                                                \
  } while (0)
#else
#define MAGPIE_STAMP(stage) ((void)0)
#endif

// The increment w . Delta of window pixel (r, c): stored in the window's slot
// of the increment buffer (ordered update), or added with one 16-byte float
// atomic, together with the pixel's weight w^0, into the object-sized
// accumulators at the window's corner (kStepAtomic).  It reads the step's
// arguments in place (parameter space in the single-problem kernel) rather
// than caching pointers in registers: cached, they spilled 56 bytes per
// thread of the float-atomic kernel.
template <int MS, bool ATOM>
struct IncrementSink {
  const StepArgs* a;   // the step's arguments (the accumulators and the weights w^0 = u + |Q|^2)
  float2* out;         // [MS][MS] this window's increments (ordered update)
  int pr, pc;          // the window's corner (kStepAtomic)
  __device__ __forceinline__ void operator()(int r, int c, float2 v) const {
    if constexpr (ATOM)
      atomicAdd(a->acc + (size_t)(pr + r) * a->n_cols + (pc + c),
                make_float4(v.x, v.y, __ldg(&a->pyr[MS * MS + r * MS + c]), 0.f));
    else
      out[r * MS + c] = v;
  }
};

// Sum over the block (a fixed order: warp shuffles, then the warps in order);
// the total is returned in thread 0 only.
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

// Two sums over the block at once: each warp adds its lanes' FP32 partials
// with a fixed shuffle tree, thread 0 adds the warps' results in FP64 in warp
// order (totals valid in thread 0 only).  `red` holds 2 nthreads/32 doubles
// and is not reused before the block's next barrier.
__device__ __forceinline__ void block_sum2(float a, float b, double* red, int tid, int nthreads, double& sa,
                                           double& sb) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((tid & 31) == 0) {
    red[2 * (tid >> 5)] = a;
    red[2 * (tid >> 5) + 1] = b;
  }
  __syncthreads();
  sa = 0.0;
  sb = 0.0;
  if (tid == 0)
    for (int i = 0; i < nthreads / 32; ++i) {
      sa += red[2 * i];
      sb += red[2 * i + 1];
    }
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

// One up-pass entry: e = g / w + (u / w) P(e_coarse), i.e. g * iw + rr * p,
// with the rounding spelled out so that every kernel the V-cycle is compiled
// into gives the same bits (left to the compiler, either product could be
// the one fused into the add, and the choice followed the surrounding
// kernel).  The product g * iw is the fused one: against the oracle, one
// step's increment on the full-size workload measured 7.5e-6 relative this
// way and 1.16e-5 with rr * p fused.
__device__ __forceinline__ float2 prolong(float2 g, float iw, float rr, float2 p) {
  return f2(__fmaf_rn(g.x, iw, __fmul_rn(rr, p.x)), __fmaf_rn(g.y, iw, __fmul_rn(rr, p.y)));
}
// a * s with each product rounded (never fused into a later add)
__device__ __forceinline__ float2 cscale_rn(float2 a, float s) { return f2(__fmul_rn(a.x, s), __fmul_rn(a.y, s)); }

// MAGPS V-cycle of one window in residual form, on this block's column slab
// Y (g^0 for MS rows x SLAB columns).  Lane gamma of a warp owns column
// gamma of a strip of 2^TT rows; the 2x2 restrictions pair columns by warp
// shuffles.  Levels coarser than TT are kept in `lvl` (local levels up to
// log2(SLAB); coarser ones span the cluster and are finished by block 0).
template <int MS, int TT, class Sink>
__device__ __forceinline__ void vcycle(const float2* Y, float2* lvl, const float* pyr, int L, int q, const Sink& put,
                                       int tid) {
  using Gm = Geo<MS>;
  constexpr int SLAB = Gm::SLAB, T = Gm::T, CL = Gm::CL, H = 1 << TT, NS = MS / H, SPAR = T / SLAB;
  constexpr int LLOC = SLAB >= 64 ? 6 : SLAB == 32 ? 5 : (SLAB == 16 ? 4 : 3);  // log2(SLAB)
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
      g1[a] = cscale_rn(v, 0.25f * w);  // rounded products: their sum below is never fused
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
              a[i] = prolong(a[i], iw[i], rr[i], pe[(r >> 1) * nc + (c >> 1)]);
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
        a[i] = prolong(a[i], __ldg(&iw[o]), __ldg(&rr[o]), pe[(r >> 1) * cc + (c >> 1)]);
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
        e1[a] = prolong(g1[a], ok ? __ldg(&iw1[o]) : 0.f, ok ? __ldg(&rr1[o]) : 0.f, eT);
      }
    }
    if (ok) {
#pragma unroll
      for (int a = 0; a < H; ++a) {
        const float u = __ldg(&u0[(R0 + a) * MS + cgl]);
        put(R0 + a, cgl, f2(__fmaf_rn(u, e1[a >> 1].x, g0[a].x), __fmaf_rn(u, e1[a >> 1].y, g0[a].y)));
      }
    }
  }
}

// One problem: window slot = cluster index (grid = windows * CL).
template <int MS, int MODE>
__global__ void __launch_bounds__(Geo<MS>::T, Geo<MS>::MIN_BLOCKS) window_kernel(const __grid_constant__ StepArgs A) {
  const int win = blockIdx.x / Geo<MS>::CL;
#include "window_body.inc"
}

// Several problems in one launch: cluster c works on window slot map[c].y of
// the problem whose arguments are table[map[c].x].
// MINB: blocks per SM the register allocation is bounded for (the group's
// autotuner picks it per window side by timing).
template <int MS, int MODE, int MINB>
__global__ void __launch_bounds__(Geo<MS>::T, MINB)
    window_kernel_batched(const StepArgs* __restrict__ table, const int2* __restrict__ map) {
  __shared__ StepArgs args;
  const int2 ent = map[blockIdx.x / Geo<MS>::CL];
  if (threadIdx.x == 0) args = table[ent.x];
  __syncthreads();
  const StepArgs& A = args;
  const int win = ent.y;
#include "window_body.inc"
}

// ---- persistent minibatch step of a context group (the members of one
// window side): one launch takes the step's windows and then the members'
// update tiles from a device work queue.  Items are handed out in index order,
// windows first; a cluster fetches its next item while it works on the
// current one.  An update tile waits (bounded) until every block of its
// member's windows has counted itself done, so a member's update overlaps
// the other members' windows.  Every window item has been handed out to a
// running cluster, and one that holds a window never waits, before any
// cluster takes an update item: the waits always end unless the launch is
// broken, and then they run out.
struct PersistArgs {
  const StepArgs* table;         // per (batched step, member) entries
  const int2* map;               // [nw] window items: (table entry, window slot)
  const int* wmember;            // [nw] the item's member, 0 .. na - 1
  const ApplyArgs* atab;         // [na] the members' updates; block0 = first tile of each
  int nw, na, ntiles;            // window items, members, update tiles
  int* head;                     // work-queue counter, zero before the launch
  int* done;                     // [na] blocks finished on each member's windows, zero before the launch
  int* err;                      // bit 3: a dependency wait ran out (its tile is skipped)
  unsigned long long limit_ns;   // bound of each dependency wait
  int bias;                      // added to every wait target: 1 makes every wait run out (a self-test)
};

constexpr int kMaxSpins = 1 << 26;  // backstop of the time bound of a dependency wait

// Thread 0's wait until *ctr >= target (acquire), for at most limit_ns of
// %globaltimer time or kMaxSpins polls; returns 0 and sets err bit 3 when
// it runs out.
__device__ __forceinline__ int wait_count(const int* ctr, int target, unsigned long long limit_ns, int* err) {
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int i = 0; i < kMaxSpins; ++i) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
    if (v >= target) return 1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) break;
    __nanosleep(256);
  }
  atomicOr(err, 8);
  return 0;
}

// Update tile of the persistent step: 32 x 32 pixels for blocks of 256 or
// more threads, 16 x 16 below.
template <int NT>
struct PersistTile {
  static constexpr int TW = NT >= 256 ? 32 : 16, TH = TW;
};

// Update tile t of the persistent step, after its member's windows (a
// separate function, so that its registers do not add to the window path's).
template <int MS>
__device__ __noinline__ void persistent_update(const PersistArgs& P, int t) {
  constexpr int CL = Geo<MS>::CL, NT = Geo<MS>::T;
  __shared__ int ready;
  int lo = 0, hi = P.na - 1;
  while (lo < hi) {  // last member whose first tile is <= t
    const int mid = (lo + hi + 1) >> 1;
    if (P.atab[mid].block0 <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  const ApplyArgs& U = P.atab[lo];
  if (threadIdx.x == 0) ready = wait_count(&P.done[lo], U.count * CL + P.bias, P.limit_ns, P.err);
  __syncthreads();
  if (ready) {
    const int lt = t - U.block0;
    apply_body<PersistTile<NT>::TW, PersistTile<NT>::TH, NT>(U, lt % U.tiles_x, lt / U.tiles_x);
  }
}

// Window item of the persistent step (a separate function: the window
// path keeps the register allocation it has in the other window kernels).
template <int MS>
__device__ __noinline__ void persistent_window(const StepArgs& A, const int win) {
  constexpr int MODE = kStep;
#include "window_body.inc"
}

template <int MS, int MINB>
__global__ void __launch_bounds__(Geo<MS>::T, MINB) window_kernel_persistent(const PersistArgs P) {
  constexpr int CL = Geo<MS>::CL;
  __shared__ StepArgs args;
  __shared__ int next[2];
  int rank = 0;
  if constexpr (CL > 1) rank = (int)cg::this_cluster().block_rank();
  const bool leader = rank == 0 && threadIdx.x == 0;
  const int items = P.nw + (P.ntiles + CL - 1) / CL;
  if (leader) next[0] = atomicAdd(P.head, 1);
  window_sync<CL>();
  int item = *peer<CL>(&next[0], 0);
  for (int it = 0; item < items; ++it) {
    if (leader) next[(it + 1) & 1] = atomicAdd(P.head, 1);
    if (item < P.nw) {
      const int2 ent = P.map[item];
      if (threadIdx.x == 0) args = P.table[ent.x];
      __syncthreads();
      persistent_window<MS>(args, ent.y);
      // this block's increments, corner and partials, then its count
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&P.done[P.wmember[item]], 1);
      }
    } else {
      const int t = (item - P.nw) * CL + rank;
      if (t < P.ntiles) persistent_update<MS>(P, t);
    }
    window_sync<CL>();  // the cluster is done with this item; next[] holds the following one
    item = *peer<CL>(&next[(it + 1) & 1], 0);
  }
  window_sync<CL>();  // no block leaves while another may still read its next[]
}
