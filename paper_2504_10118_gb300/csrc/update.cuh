// update.cuh -- the ordered object update of a minibatch step (the tiled
// reduction of the windows' increments), shared by the update kernels and the
// persistent step kernel.  Included by core.cuh inside namespace magpie_impl.
#pragma once

// z += sum_b contrib_b / sum_b w0 over the windows covering each pixel, in
// minibatch order (bitwise reproducible).  One block of NT (256) threads per
// 16 x 16 object tile, one pixel per thread: the block first lists, in
// minibatch order, the windows that overlap its tile (corners as recorded by
// the window kernel; a ballot compaction over all warps); each thread then
// walks that short list four entries at a time with predicated loads, so
// several increments are in flight per thread.  Block (0, 0) also turns the
// window kernel's block partials into Phi_k and ||grad Phi_k||.
// Dynamic smem: count int2 corners + count ints.  The tile is TW x TH pixels
// (16 x 16 for single problems; the group autotuner also tries 32 x 8 and
// 32 x 32, four pixels per thread); every shape sums each pixel's windows in
// minibatch order, so all give bitwise equal objects.
constexpr int kApplyTile = 16;
struct ApplyShape {
  int tw, th;
};
constexpr ApplyShape kApplyShapes[3] = {{16, 16}, {32, 8}, {32, 32}};
struct ApplyArgs {
  float2* z;               // object [n_rows][n_cols]
  int n_rows, n_cols;
  const int2* corners;     // [count] window corners from the window kernel
  const int32_t* idx;      // [count] window indices
  int count, n_pos;
  const float2* contrib;   // [count][MS][MS] increments w . Delta
  const float* w0;         // [MS][MS] u + |Q|^2
  int MS;
  const double* part;      // [count][slots][2] partial sums of the window phase
  int slots;               // partial-sum slots per window
  double* phi_pos;         // per-window Phi_k
  double* gn_pos;          // per-window ||grad Phi_k||
  int tiles_x, tiles_y;    // tiles per object row and column
  int block0;              // batched launches: first block of this problem
  // The precision form's V-cycle tail (apply_body<..., true>): contrib holds
  // g^0, and each window's w . Delta = g^0 + u^0 I_H^h e^1 is formed here as
  // it is summed (the finest prolongation of Algorithm MAGPS, residual form).
  const float2* e1;        // [count][MS/2][MS/2] e^1
  const float* u0;         // [MS][MS] u^0
  int* hand;               // precision form: the step's window hand-off counts, zeroed by
  int nhand;               // block (0, 0) once the grid may run (null otherwise)
};

template <int TW, int TH, int NT = 256, bool TAIL = false>
__device__ __forceinline__ void apply_body(const ApplyArgs& P, const int tx, const int ty) {
  static_assert((TW * TH) % NT == 0 && NT % TW == 0 && NT % 32 == 0, "NT threads cover the tile in whole rows");
  constexpr int PPT = TW * TH / NT, RS = NT / TW, NW = NT / 32;  // pixels per thread, rows per pass, warps
  extern __shared__ int2 corner[];
  const int count = P.count, MS = P.MS;
  int* list = reinterpret_cast<int*>(corner + count);
  __shared__ int warp_hits[NW], n_list;
  if (tx == 0 && ty == 0) {
    // the window kernel's block partials -> Phi_k and ||grad Phi_k||, in block order
    for (int b = threadIdx.x; b < count; b += blockDim.x) {
      const int k = P.idx[b];
      if ((unsigned)k >= (unsigned)P.n_pos) continue;
      double a = 0.0, g = 0.0;
      for (int q = 0; q < P.slots; ++q) {
        a += P.part[(size_t)(b * P.slots + q) * 2];
        g += P.part[(size_t)(b * P.slots + q) * 2 + 1];
      }
      P.phi_pos[k] = a / (2.0 * (double)MS * (double)MS);
      P.gn_pos[k] = sqrt(g);
    }
  }
  const int R0 = ty * TH, C0 = tx * TW;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // windows meeting this tile, listed in minibatch order: every warp takes
  // 32 consecutive windows per round, ballots, and the rounds are stitched
  // together by per-warp counts
  int base = 0;
  for (int b0 = 0; b0 < count; b0 += NT) {
    const int b = b0 + threadIdx.x;
    bool hit = false;
    if (b < count) {
      const int2 q = P.corners[b];
      corner[b] = q;
      hit = q.x < R0 + TH && q.x + MS > R0 && q.y < C0 + TW && q.y + MS > C0;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) warp_hits[wid] = __popc(mask);
    __syncthreads();
    int off = base;
    for (int i = 0; i < wid; ++i) off += warp_hits[i];
    if (hit) list[off + __popc(mask & ((1u << lane) - 1u))] = b;
    int tot = 0;
    for (int i = 0; i < NW; ++i) tot += warp_hits[i];
    base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) n_list = base;
  __syncthreads();
  const int nl = n_list;
  const size_t M = (size_t)MS * MS;
#pragma unroll 1
  for (int pp = 0; pp < PPT; ++pp) {
    const int r = R0 + (int)(threadIdx.x / TW) + pp * RS, c = C0 + (int)(threadIdx.x % TW);
    if (r >= P.n_rows || c >= P.n_cols) continue;
    float nx = 0.f, ny = 0.f, d = 0.f;
    for (int j0 = 0; j0 < nl; j0 += kApplyUnroll) {
      float2 v[kApplyUnroll];
      float wv[kApplyUnroll];
#pragma unroll
      for (int u = 0; u < kApplyUnroll; ++u) {
        const int j = j0 + u;
        const int b = j < nl ? list[j] : 0;
        const int2 q = corner[b];
        const int dr = r - q.x, dc = c - q.y;
        const bool in = j < nl && (unsigned)dr < (unsigned)MS && (unsigned)dc < (unsigned)MS;
        const int o = in ? dr * MS + dc : 0;
        v[u] = in ? P.contrib[(size_t)b * M + o] : make_float2(0.f, 0.f);
        wv[u] = in ? __ldg(&P.w0[o]) : 0.f;
        if constexpr (TAIL) {
          // w . Delta = g^0 + u^0 e^1 at this window pixel, e^1 of its 2 x 2 bin
          const int h = MS >> 1;
          const float2 e = in ? P.e1[(size_t)b * h * h + (dr >> 1) * h + (dc >> 1)] : make_float2(0.f, 0.f);
          const float uo = in ? __ldg(&P.u0[o]) : 0.f;
          v[u] = make_float2(__fmaf_rn(uo, e.x, v[u].x), __fmaf_rn(uo, e.y, v[u].y));
        }
      }
#pragma unroll
      for (int u = 0; u < kApplyUnroll; ++u) {
        nx += v[u].x;
        ny += v[u].y;
        d += wv[u];
      }
    }
    if (d > 0.f) {
      const size_t p = (size_t)r * P.n_cols + c;
      float2 zz = P.z[p];
      zz.x += nx / d;
      zz.y += ny / d;
      P.z[p] = zz;
    }
  }
}

