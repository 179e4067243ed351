// precision.cuh -- the precision form of the sweep: the windows' 2-D DFTs as
// tensor-core GEMMs with FP16 hi+lo split operands and FP32 accumulation,
// around the same projection, V-cycle and update as the FP32 path.  Included
// by magpie.cu inside namespace magpie_impl.
//
// An m-point line DFT (m = 16 Qr, Qr in {4, 8, 16}) is done as two small
// complex matrix products (Cooley-Tukey with n = Qr n1 + n2, k = k1 + 16 k2):
//   stage 1  Y[k1][n2]  = sum_{n1} F16[k1][n1] x[Qr n1 + n2]      (16-point DFTs)
//   twiddle  Y'[k1][n2] = Y[k1][n2] w_m^{n2 k1}                     (FP32)
//   stage 2  X[k1 + 16 k2] = sum_{n2} Y'[k1][n2] F_Qr[n2][k2]       (Qr-point DFTs)
// Each complex product is one real GEMM on [re; im] blocks; every operand
// a = hi + lo with hi = fp16(a), lo = fp16(a - hi) (22 significant bits
// together), and a b is taken as hi_a hi_b + hi_a lo_b + lo_a hi_b (the lo lo
// term, below 2^-22 |a b|, is dropped), three FP16 MMAs with FP32
// accumulation.  FP16's range is kept by scaling the block's lines by a power
// of two s (max |s x| in [2^9, 2^10), so that stage 2's operands, sums of 32
// stage-1 products, stay below 2^15) and dividing the outputs by s, both
// exact.
#pragma once

constexpr int kTcLines = 16;  // lines per block

// Real-block DFT matrices, FP32, built on the host in float64:
//   f16[r][c]  (32 x 32): stage 1, rows (re k1 | im k1), columns (re n1 | im n1)
//   fq[kk][nn] (32 x 32, zero-padded): stage 2, rows (re n2 | im n2),
//              columns (re k2 | im k2), for the Qr of the window side
// One set for the forward (exp(-i ...)) and one for the inverse transform.
struct TcTables {
  float f16[2][32 * 32];
  float fq[2][32 * 32];
};

__device__ __forceinline__ uint32_t pack_f16(__half a, __half b) {
  __half2 v = __halves2half2(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

// hi and lo FP16 pairs of (a, b)
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
  hi = pack_f16(ha, hb);
  lo = pack_f16(__float2half_rn(a - __half2float(ha)), __float2half_rn(b - __half2float(hb)));
}

__device__ __forceinline__ void mma_f16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma3(float* c, const uint32_t* ah, const uint32_t* al, const uint32_t* bh,
                                     const uint32_t* bl) {
  mma_f16(c, ah, bh);
  mma_f16(c, ah, bl);
  mma_f16(c, al, bh);
}

// Shared-memory layout of a block's kTcLines lines: separate real and
// imaginary planes.  Within a line, element i sits at i + 4 (i / Qr): every
// run of Qr elements is followed by four pad words, so the fragment loads
// and stores that stride by Qr (stage-1 B columns, the twiddle scatter,
// stage-2 A rows) hit distinct banks or at most two threads per bank.  The
// line pitch LD = MS + 68 keeps lines four banks apart.
template <int MS>
struct TcSm {
  static constexpr int QR = MS / 16, NL = kTcLines, LD = MS + 68;
  // resident blocks per SM the fused kernels' registers are bounded for at
  // m = 256: four 128-thread blocks with register-fragment MMAs (128
  // registers, a few spilled words; 449 k against 422 k patterns/s with
  // three), three with tcgen05, whose 67 KB of shared memory allow no more
  // (a bound of four measured slower there: 374 k against 385 k)
  template <int PATH>
  static constexpr int min_blocks() { return MS == 256 ? (PATH ? 3 : 4) : 1; }
  static_assert(QR == 4 || QR == 8 || QR == 16, "window side 64, 128 or 256");
  __device__ static __forceinline__ int at(int l, int i) { return l * LD + i + 4 * (i / QR); }
};

// Fills the NL lines from src(l, p) (line l, position p along the line),
// eight loads in flight per thread.  AXIS 1: consecutive threads take
// consecutive positions of a line (rows of a window); AXIS 0: consecutive
// lines at one position (columns).  Returns the largest |re|, |im| this
// thread stored (for tc_lines' block scale).
template <int MS, int AXIS, typename Src>
__device__ __forceinline__ float tc_load(float* Sr, float* Si, Src src) {
  using S = TcSm<MS>;
  constexpr int NL = S::NL;
  constexpr int NB = (NL * MS) % (128 * 16) == 0 ? 16 : 8;
  static_assert((NL * MS) % (128 * NB) == 0, "load batches");
  float mx = 0.f;
  for (int i0 = threadIdx.x; i0 < NL * MS; i0 += 128 * NB) {
    float2 v[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int i = i0 + 128 * u;
      v[u] = AXIS == 1 ? src(i / MS, i % MS) : src(i % NL, i / NL);
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int i = i0 + 128 * u;
      const int l = AXIS == 1 ? i / MS : i % NL, p = AXIS == 1 ? i % MS : i / NL;
      Sr[S::at(l, p)] = v[u].x;
      Si[S::at(l, p)] = v[u].y;
      mx = fmaxf(mx, fmaxf(fabsf(v[u].x), fabsf(v[u].y)));
    }
  }
  return mx;
}

// dst(l, p, value) for every element of the NL lines, in the thread order of
// tc_load.
template <int MS, int AXIS, typename Dst>
__device__ __forceinline__ void tc_store(const float* Sr, const float* Si, Dst dst) {
  using S = TcSm<MS>;
  constexpr int NL = S::NL;
  for (int i = threadIdx.x; i < NL * MS; i += 128) {
    const int l = AXIS == 1 ? i / MS : i % NL, p = AXIS == 1 ? i % MS : i / NL;
    dst(l, p, make_float2(Sr[S::at(l, p)], Si[S::at(l, p)]));
  }
}

// The power of two s of the FP16 operands (see the top of this file): max
// |s x| over the block's lines in [2^9, 2^10); 1 for all-zero or non-finite
// lines.  Each of the 128 threads passes the largest |re|, |im| it wrote
// into the lines (so no pass over them is needed); one barrier, which also
// puts every thread's lines in place.
__device__ __forceinline__ float tc_scale(float mx) {
  __shared__ float red[4];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
  if (!(mx > 0.f) || !(mx <= 3.0e38f)) return 1.f;
  int e;
  frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1)
  return ldexpf(1.f, 10 - e);
}

// The forward (INV = 0) or conjugate (INV = 1) DFT of the block's NL lines,
// in place in shared memory, the output multiplied by `scale`; `mx` is the
// largest |re|, |im| this thread wrote into the lines.  128 threads; begins
// with a barrier (the lines must be in place) and ends with one.
template <int MS, int INV>
__device__ __forceinline__ void tc_lines(float* Sr, float* Si, const TcTables* __restrict__ tabs,
                                         const float2* __restrict__ tw, float scale, float mx) {
  using S = TcSm<MS>;
  constexpr int QR = S::QR, NL = S::NL;
  constexpr int K2T = (2 * QR + 15) / 16;  // stage-2 k-tiles
  constexpr int N2T = 2 * QR / 8;          // stage-2 n-tiles
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const float sx = tc_scale(mx), out_scale = scale / sx;  // its barrier: the lines in place

  // ---- stage-1 operands: the 16-point DFT matrix as A fragments (hi, lo)
  uint32_t ah[2][2][4], al[2][2][4];
  {
    const float* F = tabs->f16[INV];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int kt = 0; kt < 2; ++kt) {
        const int r = mt * 16 + g, c = kt * 16 + 2 * t;
        split2(F[r * 32 + c], F[r * 32 + c + 1], ah[mt][kt][0], al[mt][kt][0]);
        split2(F[(r + 8) * 32 + c], F[(r + 8) * 32 + c + 1], ah[mt][kt][1], al[mt][kt][1]);
        split2(F[r * 32 + c + 8], F[r * 32 + c + 9], ah[mt][kt][2], al[mt][kt][2]);
        split2(F[(r + 8) * 32 + c + 8], F[(r + 8) * 32 + c + 9], ah[mt][kt][3], al[mt][kt][3]);
      }
  }
  __syncthreads();

  // ---- stage 1: columns j = (line, n2), NL * QR of them, 8 per n-tile
  constexpr int NT1 = NL * QR / 8, PER1 = NT1 / 4;
  float acc[PER1][2][4];
#pragma unroll
  for (int i = 0; i < PER1; ++i)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][mt][e] = 0.f;
#pragma unroll
  for (int i = 0; i < PER1; ++i) {
    const int j = (warp * PER1 + i) * 8 + g;  // this thread's B column
    const int l = j / QR, n2 = j % QR;
    const float* xr = Sr + S::at(l, n2);
    const float* xi = Si + S::at(l, n2);
    uint32_t bh[2][2], bl[2][2];
    // k-tile 0: real parts of n1 = 2t, 2t+1, 2t+8, 2t+9; k-tile 1: imaginary parts
    constexpr int RS = QR + 4;
    split2(sx * xr[RS * (2 * t)], sx * xr[RS * (2 * t + 1)], bh[0][0], bl[0][0]);
    split2(sx * xr[RS * (2 * t + 8)], sx * xr[RS * (2 * t + 9)], bh[0][1], bl[0][1]);
    split2(sx * xi[RS * (2 * t)], sx * xi[RS * (2 * t + 1)], bh[1][0], bl[1][0]);
    split2(sx * xi[RS * (2 * t + 8)], sx * xi[RS * (2 * t + 9)], bh[1][1], bl[1][1]);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int kt = 0; kt < 2; ++kt) mma3(acc[i][mt], ah[mt][kt], al[mt][kt], bh[kt], bl[kt]);
  }
  __syncthreads();
  // twiddle w_m^{+-n2 k1}; thread holds re/im of k1 = g, g+8 for columns 2t, 2t+1
#pragma unroll
  for (int i = 0; i < PER1; ++i)
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const int j = (warp * PER1 + i) * 8 + 2 * t + cc;
      const int l = j / QR, n2 = j % QR;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int k1 = g + 8 * hh;
        const float yr = acc[i][0][2 * hh + cc], yi = acc[i][1][2 * hh + cc];
        float2 w = tw[(n2 * k1) % MS];
        if (INV) w.y = -w.y;
        Sr[S::at(l, k1 * QR + n2)] = yr * w.x - yi * w.y;
        Si[S::at(l, k1 * QR + n2)] = yr * w.y + yi * w.x;
      }
    }
  __syncthreads();

  // ---- stage 2: rows (line, k1), NL * 16 of them; the Qr-point DFT matrix as B fragments
  uint32_t bh2[K2T][N2T][2], bl2[K2T][N2T][2];
  {
    const float* F = tabs->fq[INV];
#pragma unroll
    for (int kt = 0; kt < K2T; ++kt)
#pragma unroll
      for (int nt = 0; nt < N2T; ++nt) {
        const int n = nt * 8 + g, k = kt * 16 + 2 * t;
        split2(F[k * 32 + n], F[(k + 1) * 32 + n], bh2[kt][nt][0], bl2[kt][nt][0]);
        split2(F[(k + 8) * 32 + n], F[(k + 9) * 32 + n], bh2[kt][nt][1], bl2[kt][nt][1]);
      }
  }
  constexpr int MT2 = NL * 16 / 16, PER2 = MT2 / 4;  // m-tiles of 16 rows = one line each
  float out[PER2][N2T][4];
#pragma unroll
  for (int i = 0; i < PER2; ++i) {
    const int l = warp * PER2 + i;  // m-tile = line l, rows k1 = 0..15
#pragma unroll
    for (int nt = 0; nt < N2T; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) out[i][nt][e] = 0.f;
#pragma unroll
    for (int kt = 0; kt < K2T; ++kt) {
      // A[row k1][col kk]: kk < QR real part of n2 = kk, QR <= kk < 2 QR imaginary, else 0
      uint32_t a_h[4], a_l[4];
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int row = g + ((q >> 1) & 1) * 8;
        const int kk = kt * 16 + 2 * t + (q & 1) + ((q >> 2) & 1) * 8;
        float val = 0.f;
        if (kk < QR)
          val = Sr[S::at(l, row * QR + kk)];
        else if (kk < 2 * QR)
          val = Si[S::at(l, row * QR + kk - QR)];
        v[q] = val;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) split2(v[2 * r], v[2 * r + 1], a_h[r], a_l[r]);
#pragma unroll
      for (int nt = 0; nt < N2T; ++nt) mma3(out[i][nt], a_h, a_l, bh2[kt][nt], bl2[kt][nt]);
    }
  }
  __syncthreads();
  // C: rows k1 = g, g+8; columns nn = 8 nt + 2t (+1): nn < QR real part of k2 = nn, else imaginary
#pragma unroll
  for (int i = 0; i < PER2; ++i) {
    const int l = warp * PER2 + i;
#pragma unroll
    for (int nt = 0; nt < N2T; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k1 = g + 8 * (e >> 1);
        const int nn = nt * 8 + 2 * t + (e & 1);
        const float v = out[i][nt][e] * out_scale;
        if (nn < QR)
          Sr[S::at(l, k1 + 16 * nn)] = v;
        else
          Si[S::at(l, k1 + 16 * (nn - QR))] = v;
      }
  }
  __syncthreads();

}

// ---- the same transform on the 5th-generation tensor cores (tcgen05).
// Both stages become M = 128 matrix products with the block's rows as M:
//   stage 1: D[j][r] = sum_c X[j][c] f16[r][c], j = (line, n2) (NL QR rows,
//            128 per tile), r = (re k1 | im k1), c = (re n1 | im n1), K = 32;
//   stage 2: D[(line, k1)][nn] = sum_kk Y'[(line, k1)][kk] fq[kk][nn], 256
//            rows in two tiles, K = N = 2 QR (both padded to 16 for m = 64).
// For each tile the threads write the A rows, one per thread, as hi and lo
// FP16 into a 64-byte-swizzled K-major buffer; thread 0 issues the
// tcgen05.mma (hi hi + hi lo + lo hi per 16-deep K step, FP16 operands) into 32 TMEM
// columns and commits them to an mbarrier; every thread waits (bounded),
// reads its row of the accumulator with tcgen05.ld, and does the twiddle
// (stage 1) or the scaled store (stage 2) in FP32 from registers.  The B
// operands (the DFT matrices) are written the same way at the start.
struct TcUmma {
  uint32_t a_hi, a_lo;    // A tile: 128 rows x 64 bytes each
  uint32_t b1_hi, b1_lo;  // stage-1 DFT matrix: 32 rows x 64 bytes
  uint32_t b2_hi, b2_lo;  // stage-2 DFT matrix: up to 32 rows x 64 bytes
  uint32_t bar, tmem, phase;
  int ok;                 // 0 once a bounded wait ran out
};
constexpr int kUmmaDftSmem = 2 * 8192 + 4 * 2048 + 1024;  // operand buffers + 1024-byte alignment slack

// hi and lo FP16 of 8 consecutive K elements (one 16-byte chunk), chunk c of
// row r of the two 64-byte-swizzled buffers
__device__ __forceinline__ void put_chunk(uint32_t hi_base, uint32_t lo_base, int r, int c, const float (&v)[8]) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) split2(v[2 * i], v[2 * i + 1], h[i], l[i]);
  const uint32_t o = umma::sw64_off(r, c);
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(hi_base + o), "r"(h[0]), "r"(h[1]), "r"(h[2]),
               "r"(h[3])
               : "memory");
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(lo_base + o), "r"(l[0]), "r"(l[1]), "r"(l[2]),
               "r"(l[3])
               : "memory");
}

// One tile's products: the A rows written, KS K steps of 16 against B
// (N rows), accumulator in U.tmem; returns once the products are complete
// (or the bounded wait ran out: U.ok = 0).
template <int N>
__device__ __forceinline__ void umma_tile(TcUmma& U, uint32_t b_hi, uint32_t b_lo, int KS) {
  umma::fence_proxy_async();  // this thread's operand writes, visible to the tensor core
  umma::fence_before();       // and its earlier tcgen05.ld ordered before the barrier
  __syncthreads();
  if (threadIdx.x == 0) {
    umma::fence_after();
    constexpr uint32_t ID = umma::idesc_f16(128, N);
    for (int k = 0; k < KS; ++k) {
      const uint32_t o = 32u * (uint32_t)k;
      const uint64_t ah = umma::desc_sw64(U.a_hi + o), al = umma::desc_sw64(U.a_lo + o);
      const uint64_t bh = umma::desc_sw64(b_hi + o), bl = umma::desc_sw64(b_lo + o);
      umma::mma_ss(U.tmem, ah, bh, ID, k != 0);
      umma::mma_ss(U.tmem, ah, bl, ID, 1);
      umma::mma_ss(U.tmem, al, bh, ID, 1);
    }
    umma::commit(U.bar);
  }
  if (!umma::wait(U.bar, U.phase)) U.ok = 0;
  U.phase ^= 1u;
  umma::fence_after();
}

template <int MS, int INV>
__device__ __forceinline__ void tc_lines_umma(float* Sr, float* Si, const TcTables* __restrict__ tabs,
                                              const float2* __restrict__ tw, float scale, float mx, TcUmma& U) {
  using S = TcSm<MS>;
  constexpr int QR = S::QR, NL = S::NL;
  constexpr int Q2 = 2 * QR < 16 ? 16 : 2 * QR;  // stage-2 K and N, padded to 16
  const int tid = threadIdx.x;
  const uint32_t trow = U.tmem + ((uint32_t)(tid & ~31) << 16);  // this warp's TMEM lanes
  const float sx = tc_scale(mx), out_scale = scale / sx;  // its barrier: the lines in place
  // B operands: stage 1 rows r, K c: f16[r][c]; stage 2 rows nn, K kk: fq[kk][nn] (0 in the padding)
  {
    const float* F1 = tabs->f16[INV];
    const int r = tid >> 2, c = tid & 3;
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = F1[r * 32 + 8 * c + k];
    put_chunk(U.b1_hi, U.b1_lo, r, c, v);
    const float* F2 = tabs->fq[INV];
    if (tid < Q2 * (Q2 / 8)) {
      const int r2 = tid / (Q2 / 8), c2 = tid % (Q2 / 8);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int kk = 8 * c2 + k;
        v[k] = kk < 2 * QR && r2 < 2 * QR ? F2[kk * 32 + r2] : 0.f;
      }
      put_chunk(U.b2_hi, U.b2_lo, r2, c2, v);
    }
  }
  __syncthreads();  // the lines in place

  // ---- stage 1: rows j = (line, n2)
  constexpr int J = NL * QR, T1 = (J + 127) / 128;
#pragma unroll 1
  for (int mt = 0; mt < T1; ++mt) {
    const int j = mt * 128 + tid;
    const bool live = j < J;
    const int l = live ? j / QR : 0, n2 = live ? j % QR : 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int kk = 8 * c + k, n1 = kk & 15;
        v[k] = live ? sx * (kk < 16 ? Sr : Si)[S::at(l, QR * n1 + n2)] : 0.f;
      }
      put_chunk(U.a_hi, U.a_lo, tid, c, v);
    }
    umma_tile<32>(U, U.b1_hi, U.b1_lo, 2);
    float y[32];
    umma::ld16(trow, *reinterpret_cast<float(*)[16]>(&y[0]));
    umma::ld16(trow + 16u, *reinterpret_cast<float(*)[16]>(&y[16]));
    if (live) {
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) {
        float2 w = tw[(n2 * k1) % MS];
        if (INV) w.y = -w.y;
        const float yr = y[k1], yi = y[16 + k1];
        Sr[S::at(l, k1 * QR + n2)] = yr * w.x - yi * w.y;
        Si[S::at(l, k1 * QR + n2)] = yr * w.y + yi * w.x;
      }
    }
  }
  __syncthreads();  // stage 1's rows in place before stage 2 reads them

  // ---- stage 2: rows (line, k1), two tiles of 128
#pragma unroll 1
  for (int mt = 0; mt < NL * 16 / 128; ++mt) {
    const int row = mt * 128 + tid, l = row >> 4, k1 = row & 15;
#pragma unroll
    for (int c = 0; c < Q2 / 8; ++c) {
      float v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int kk = 8 * c + k;
        v[k] = kk < QR ? Sr[S::at(l, k1 * QR + kk)] : kk < 2 * QR ? Si[S::at(l, k1 * QR + kk - QR)] : 0.f;
      }
      put_chunk(U.a_hi, U.a_lo, tid, c, v);
    }
    umma_tile<Q2>(U, U.b2_hi, U.b2_lo, Q2 / 16);
    float o[32];
    umma::ld16(trow, *reinterpret_cast<float(*)[16]>(&o[0]));
    if constexpr (Q2 > 16) umma::ld16(trow + 16u, *reinterpret_cast<float(*)[16]>(&o[16]));
#pragma unroll
    for (int nn = 0; nn < 2 * QR; ++nn) {
      const float v = o[nn] * out_scale;
      if (nn < QR)
        Sr[S::at(l, k1 + 16 * nn)] = v;
      else
        Si[S::at(l, k1 + 16 * (nn - QR))] = v;
    }
  }
  __syncthreads();
}

// Per-block state of a transform path: PATH 0 the register-fragment
// (mma.sync) transforms, nothing to set up; PATH 1 the tcgen05 transforms,
// with 32 tensor-memory columns, one mbarrier and kUmmaDftSmem bytes of
// dynamic shared memory for the operands.  end() frees the tensor memory and
// sets bit 4 of `err` if a bounded wait ran out.  Every thread of the block
// calls begin() and end().
template <int PATH>
struct TcPath {
  __device__ __forceinline__ void begin() {}
  __device__ __forceinline__ void end(int*) {}
  template <int MS, int INV>
  __device__ __forceinline__ void lines(float* Sr, float* Si, const TcTables* tabs, const float2* tw, float sc,
                                        float mx) {
    tc_lines<MS, INV>(Sr, Si, tabs, tw, sc, mx);
  }
};
template <>
struct TcPath<1> {
  TcUmma U;
  __device__ __forceinline__ void begin() {
    extern __shared__ __align__(16) unsigned char tc_dyn[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ uint32_t slot;
    const uint32_t base = (smem_addr(tc_dyn) + 1023u) & ~1023u;
    U.a_hi = base;
    U.a_lo = base + 8192;
    U.b1_hi = base + 16384;
    U.b1_lo = base + 18432;
    U.b2_hi = base + 20480;
    U.b2_lo = base + 22528;
    if (threadIdx.x < 32) umma::alloc(smem_addr(&slot), 32);
    if (threadIdx.x == 0) {
      mbar_init(smem_addr(&bar), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    U.tmem = slot;
    U.bar = smem_addr(&bar);
    U.phase = 0;
    U.ok = 1;
  }
  __device__ __forceinline__ void end(int* err) {
    umma::fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
      umma::fence_after();
      umma::dealloc(U.tmem, 32);
    }
    if (!U.ok && err) atomicOr(err, 16);
  }
  template <int MS, int INV>
  __device__ __forceinline__ void lines(float* Sr, float* Si, const TcTables* tabs, const float2* tw, float sc,
                                        float mx) {
    tc_lines_umma<MS, INV>(Sr, Si, tabs, tw, sc, mx, U);
  }
};

// One block: kTcLines lines of one window through the transform, in place in
// `data` ([windows][MS][MS]).  AXIS 0: lines are columns (element stride
// MS); AXIS 1: rows.  `scale` multiplies the output.
template <int MS, int AXIS, int INV, int PATH>
__global__ void __launch_bounds__(128) dft_tc_kernel(float2* __restrict__ data, const TcTables* __restrict__ tabs,
                                                     const float2* __restrict__ tw, float scale, int* err) {
  using S = TcSm<MS>;
  __shared__ float Sr[S::NL * S::LD];
  __shared__ float Si[S::NL * S::LD];
  TcPath<PATH> T;
  T.begin();
  const int tiles = MS / S::NL;
  const int win = blockIdx.x / tiles, l0 = (blockIdx.x % tiles) * S::NL;
  float2* base = data + (size_t)win * MS * MS;
  const float mx = tc_load<MS, AXIS>(Sr, Si, [&](int l, int p) {
    return AXIS == 1 ? base[(size_t)(l0 + l) * MS + p] : base[(size_t)p * MS + l0 + l];
  });
  T.template lines<MS, INV>(Sr, Si, tabs, tw, scale, mx);
  tc_store<MS, AXIS>(Sr, Si, [&](int l, int p, float2 v) {
    if (AXIS == 1)
      base[(size_t)(l0 + l) * MS + p] = v;
    else
      base[(size_t)p * MS + l0 + l] = v;
  });
  T.end(err);
}

struct PrecArgs {
  const float2* z;     // object [n_rows][n_cols]
  int n_cols;
  const float2* Q;     // probe [MS][MS]
  const float* amp;    // sqrt(d) [n_pos][MS][MS]
  const int32_t* pos;  // [n_pos][2]
  const int32_t* idx;  // [count]
  int n_pos, MS;
  int count;           // windows of the step
  int T;               // partial-sum slots per window: one per block of kTcLines lines
  float2* buf;         // [count][MS][MS] exit wave -> spectrum -> revised exit wave
  float2* contrib;     // [count][MS][MS] g^0 = conj(Q)(R - Q z)
  double* part;        // [count][T][2] partial sums: (|Psi| - sqrt d)^2, |g^0|^2
  int2* corner;        // [count] window corners for the update kernel
  int* err;            // bit 0: window index out of range
  float2* phase;       // phase rule: [n_pos][MS][MS] unit phases of the last visit, else null
  float2* g1;          // levels >= 2: [count][MS/2][MS/2] g^1 = W_u^0 . I(g^0), then e^1; else null
  float2* g2;          // levels >= 3: [count][MS/4][MS/4] g^2 = W_u^1 . I(g^1)
  int* hand;           // [3][count] tiles of each window finished by the exit, project and gradient
                       // kernels (zeroed by the update kernel that ends the step)
  int wait_bias;       // added to every hand-off target: 1 makes every wait run out (a self-test)
  unsigned long long wait_ns;  // bound of each hand-off wait
  const float* pyr;    // level factors (window-kernel layout)
  int L;               // levels
};

// The three window-phase kernels of a minibatch step.  Each block takes
// kTcLines lines of one window (grid: windows x MS / kTcLines) through one
// or two tensor-core transforms, with the element-wise steps around them
// fused into its loads and stores:
//   exit_dft_kernel    columns: psi = Q . z_k loaded from the object, forward DFT
//   project_dft_kernel rows:    forward DFT, modulus projection (+ the tile's
//                               sum of (|Psi| - sqrt d)^2), inverse DFT
//   grad_dft_kernel    columns: inverse DFT, g^0 = conj(Q)(R - Q z_k) into the
//                               increments (+ the tile's sum of |g^0|^2), and
//                               for two levels or more g^1 = W_u^0 . I(g^0)
// The window buffer holds psi's column transforms, then R's row transforms.

// Window hand-off between the step's kernels.  Each transform kernel lets
// the next one launch as soon as all of its own blocks are running
// (griddepcontrol.launch_dependents at block start), and the next kernel's
// blocks wait, window by window, for the count of that window's finished
// tiles instead of for the whole previous grid: the last partial wave of
// one kernel then overlaps the first windows of the next.  The producer
// block counts its tile after its last global store (block barrier, fence,
// atomic add: a release at GPU scope); the consumer's thread 0 polls with
// acquire loads, bounded by kHandoffNs of %globaltimer time (on expiry it
// sets bit 4 of the error word, MAGPIE_ETIMEOUT, and the block skips its
// tile but still counts it).  Consumers read the handed-off buffers through
// L2 (ld.global.cg).
constexpr unsigned long long kHandoffNs = 200000000ull;  // 0.2 s, the default bound
__device__ __forceinline__ void handoff_signal(int* cnt) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(cnt, 1);
  }
}
// Returns false (in every thread of the block) when the wait ran out.
__device__ __forceinline__ bool handoff_wait(const PrecArgs& A, const int* cnt, int tiles) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    const int target = tiles + A.wait_bias;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    int good = 1;
    for (int i = 0;; ++i) {
      int v;
      asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
      if (v >= target) break;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > A.wait_ns || i >= (1 << 26)) {
        atomicOr(A.err, 16);
        good = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// Window index of block b, its first line, and whether the index is valid.
struct TcBlock {
  int w, tile, l0, k;
  bool ok;
};
template <int MS>
__device__ __forceinline__ TcBlock tc_block(const PrecArgs& A) {
  constexpr int tiles = MS / kTcLines;
  TcBlock b;
  b.w = blockIdx.x / tiles;
  b.tile = blockIdx.x % tiles;
  b.l0 = b.tile * kTcLines;
  b.k = A.idx[b.w];
  b.ok = (unsigned)b.k < (unsigned)A.n_pos;
  return b;
}

template <int MS, int PATH>
__global__ void __launch_bounds__(128, TcSm<MS>::template min_blocks<PATH>()) exit_dft_kernel(const PrecArgs A, const TcTables* __restrict__ tabs,
                                                       const float2* __restrict__ tw) {
  using S = TcSm<MS>;
  __shared__ float Sr[S::NL * S::LD];
  __shared__ float Si[S::NL * S::LD];
  grid_dep_wait();  // launched as a programmatic dependent of the step's last kernel before
  grid_dep_launch();
  TcPath<PATH> T;
  T.begin();
  const TcBlock B = tc_block<MS>(A);
  if (threadIdx.x == 0 && B.tile == 0) {
    if (B.ok)
      A.corner[B.w] = make_int2(A.pos[2 * B.k], A.pos[2 * B.k + 1]);
    else {
      A.corner[B.w] = make_int2(-(1 << 30), -(1 << 30));
      atomicOr(A.err, 1);
    }
  }
  const float2* zk = A.z + (B.ok ? (size_t)A.pos[2 * B.k] * A.n_cols + A.pos[2 * B.k + 1] : 0);
  const float mx = tc_load<MS, 0>(Sr, Si, [&](int l, int p) {
    if (!B.ok) return make_float2(0.f, 0.f);
    const float2 zz = zk[(size_t)p * A.n_cols + B.l0 + l];
    const float2 qq = __ldg(&A.Q[p * MS + B.l0 + l]);
    return make_float2(qq.x * zz.x - qq.y * zz.y, qq.x * zz.y + qq.y * zz.x);
  });
  T.template lines<MS, 0>(Sr, Si, tabs, tw, 1.f, mx);
  float2* base = A.buf + (size_t)B.w * MS * MS;
  tc_store<MS, 0>(Sr, Si, [&](int l, int p, float2 v) { base[(size_t)p * MS + B.l0 + l] = v; });
  handoff_signal(&A.hand[B.w]);
  T.end(A.err);
}

template <int MS, int PATH>
__global__ void __launch_bounds__(128, TcSm<MS>::template min_blocks<PATH>()) project_dft_kernel(const PrecArgs A, const TcTables* __restrict__ tabs,
                                                          const float2* __restrict__ tw) {
  using S = TcSm<MS>;
  __shared__ float Sr[S::NL * S::LD];
  __shared__ float Si[S::NL * S::LD];
  __shared__ double red[4];
  grid_dep_launch();  // the exit kernel's windows are handed off one by one
  TcPath<PATH> T;
  T.begin();
  const TcBlock B = tc_block<MS>(A);
  float2* base = A.buf + (size_t)B.w * MS * MS;
  if (B.ok) {
    // the block's amplitude rows on their way into L2 while the forward transform runs
    const char* ab = reinterpret_cast<const char*>(A.amp + (size_t)B.k * MS * MS + (size_t)B.l0 * MS);
    for (int i = threadIdx.x; i < S::NL * MS * 4 / 128; i += 128)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(ab + 128 * i)));
  }
  if (!handoff_wait(A, &A.hand[B.w], MS / kTcLines)) {  // ran out: skip the tile
    handoff_signal(&A.hand[A.count + B.w]);
    T.end(A.err);
    return;
  }
  const float mx = tc_load<MS, 1>(Sr, Si, [&](int l, int p) { return __ldcg(&base[(size_t)(B.l0 + l) * MS + p]); });
  T.template lines<MS, 0>(Sr, Si, tabs, tw, 1.f, mx);
  // Psi <- sqrt(d) Psi / |Psi| / m^2 (sqrt(d) / m^2 where Psi = 0, or the
  // previous visit's phase under the phase rule)
  const float* am = A.amp + (size_t)(B.ok ? B.k : 0) * MS * MS;
  const float inv_m2 = 1.f / (float)(MS * MS);
  float res = 0.f, mx2 = 0.f;  // mx2: the inverse transform's block scale, from the values written
  for (int i0 = threadIdx.x; i0 < S::NL * MS; i0 += 128 * 8) {
    float av[8];  // eight amplitude loads in flight per thread
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + 128 * u;
      av[u] = B.ok ? __ldg(&am[(B.l0 + i / MS) * MS + i % MS]) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + 128 * u;
      const int l = i / MS, p = i % MS, o = (B.l0 + l) * MS + p;
      const float vx = Sr[S::at(l, p)], vy = Si[S::at(l, p)];
      const float a = av[u];
      const float n2 = vx * vx + vy * vy;
      const float mag = sqrtf(n2);
      const float d = mag - a;
      res += d * d;
      float2 ph = make_float2(1.f, 0.f);  // theta(0) = 0
      if (n2 > 0.f) {
        ph = make_float2(vx / mag, vy / mag);
        if (A.phase && B.ok) A.phase[(size_t)B.k * MS * MS + o] = ph;
      } else if (A.phase && B.ok) {
        ph = A.phase[(size_t)B.k * MS * MS + o];  // Eq. (specification): the previous visit's phase
      }
      const float px = a * inv_m2 * ph.x, py = a * inv_m2 * ph.y;
      Sr[S::at(l, p)] = px;
      Si[S::at(l, p)] = py;
      mx2 = fmaxf(mx2, fmaxf(fabsf(px), fabsf(py)));
    }
  }
  const double s = block_sum((double)res, red, threadIdx.x, 128);
  if (threadIdx.x == 0) A.part[((size_t)B.w * A.T + B.tile) * 2] = B.ok ? s : 0.0;
  T.template lines<MS, 1>(Sr, Si, tabs, tw, 1.f, mx2);
  tc_store<MS, 1>(Sr, Si, [&](int l, int p, float2 v) { base[(size_t)(B.l0 + l) * MS + p] = v; });
  handoff_signal(&A.hand[A.count + B.w]);
  T.end(A.err);
}

template <int MS, int PATH>
__global__ void __launch_bounds__(128, TcSm<MS>::template min_blocks<PATH>()) grad_dft_kernel(const PrecArgs A, const TcTables* __restrict__ tabs,
                                                       const float2* __restrict__ tw) {
  using S = TcSm<MS>;
  constexpr int NL = S::NL, h = MS / 2;
  __shared__ float Sr[NL * S::LD];
  __shared__ float Si[NL * S::LD];
  __shared__ double red[4];
  grid_dep_launch();  // the project kernel's windows are handed off one by one
  TcPath<PATH> T;
  T.begin();
  const TcBlock B = tc_block<MS>(A);
  const float2* base = A.buf + (size_t)B.w * MS * MS;
  if (!handoff_wait(A, &A.hand[A.count + B.w], MS / kTcLines)) {  // ran out: skip the tile
    handoff_signal(&A.hand[2 * A.count + B.w]);
    T.end(A.err);
    return;
  }
  const float mx = tc_load<MS, 0>(Sr, Si, [&](int l, int p) { return __ldcg(&base[(size_t)p * MS + B.l0 + l]); });
  T.template lines<MS, 1>(Sr, Si, tabs, tw, 1.f, mx);
  const float2* zk = A.z + (B.ok ? (size_t)A.pos[2 * B.k] * A.n_cols + A.pos[2 * B.k + 1] : 0);
  float2* out = A.contrib + (size_t)B.w * MS * MS;
  float gn = 0.f;
  for (int i0 = threadIdx.x; i0 < NL * MS; i0 += 128 * 8) {
    float2 zv[8], qv[8];  // eight object and probe loads in flight per thread
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + 128 * u, c = B.l0 + i % NL, p = i / NL;
      zv[u] = B.ok ? zk[(size_t)p * A.n_cols + c] : make_float2(0.f, 0.f);
      qv[u] = __ldg(&A.Q[p * MS + c]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + 128 * u, l = i % NL, p = i / NL, c = B.l0 + l;
      const float2 zz = zv[u], qq = qv[u];
      float2 g = make_float2(0.f, 0.f);
      if (B.ok) {
        const float dx = Sr[S::at(l, p)] - (qq.x * zz.x - qq.y * zz.y);
        const float dy = Si[S::at(l, p)] - (qq.x * zz.y + qq.y * zz.x);
        g = make_float2(qq.x * dx + qq.y * dy, qq.x * dy - qq.y * dx);
      }
      gn += g.x * g.x + g.y * g.y;
      out[(size_t)p * MS + c] = g;
      Sr[S::at(l, p)] = g.x;
      Si[S::at(l, p)] = g.y;
    }
  }
  const double s = block_sum((double)gn, red, threadIdx.x, 128);  // also the barrier before g^1
  if (threadIdx.x == 0) A.part[((size_t)B.w * A.T + B.tile) * 2 + 1] = B.ok ? s : 0.0;
  if (A.g1) {
    // the block's NL / 2 bin columns, every bin row; the four g^0 of a bin
    // summed row by row
    constexpr int NB = (NL / 2) * h / 128;  // bins per thread
    static_assert(NB >= 1 && (NL / 2) * h % 128 == 0, "bins per thread");
    const float* wu0 = A.pyr + lvl_off(MS, 1);
    float wv[NB];  // the bins' W_u^0, loaded together
    float2 gv[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int i = threadIdx.x + 128 * u;
      wv[u] = __ldg(&wu0[(i / (NL / 2)) * h + B.l0 / 2 + i % (NL / 2)]);
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int i = threadIdx.x + 128 * u;
      const int j = i % (NL / 2), br = i / (NL / 2), bc = B.l0 / 2 + j;
      float sx = 0.f, sy = 0.f;
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          sx += Sr[S::at(2 * j + b, 2 * br + a)];
          sy += Si[S::at(2 * j + b, 2 * br + a)];
        }
      const float f = 0.25f * wv[u];
      float2 g1 = make_float2(f * sx, f * sy);
      gv[u] = g1;
      if (A.L == 2) {  // the coarsest step e^1 = g^1 / w^1, rounded after g^1
        const float iw = __ldg(&A.pyr[lvl_off(MS, 1) + h * h + br * h + bc]);
        g1 = make_float2(__fmul_rn(g1.x, iw), __fmul_rn(g1.y, iw));
      }
      A.g1[(size_t)B.w * h * h + br * h + bc] = g1;
    }
    if (A.L >= 3) {
      // g^2 = W_u^1 . I(g^1) of the block's NL / 4 level-2 columns: bin i of
      // g^1 is (row i / (NL / 2), column i % (NL / 2)), so the four g^1 of a
      // level-2 bin sit in lanes i, i ^ 1, i ^ NL / 2, i ^ (NL / 2 + 1) of one
      // warp; summed row by row, as the coarse kernel's restrictions
      static_assert(NL / 2 == 8, "bin row of g^1 = eight lanes");
      const float* wu1 = A.pyr + lvl_off(MS, 2);
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int i = threadIdx.x + 128 * u;
        const float2 b = shfl_xor2(gv[u], 1), cc = shfl_xor2(gv[u], 8), d = shfl_xor2(gv[u], 9);
        const int j = i % (NL / 2), br = i / (NL / 2);
        if (((j | br) & 1) == 0) {
          const int o = (br / 2) * (MS / 4) + B.l0 / 4 + j / 2;
          const float f = 0.25f * __ldg(&wu1[o]);
          A.g2[(size_t)B.w * (h / 2) * (h / 2) + o] =
              make_float2(f * (gv[u].x + b.x + cc.x + d.x), f * (gv[u].y + b.y + cc.y + d.y));
        }
      }
    }
  }
  handoff_signal(&A.hand[2 * A.count + B.w]);
  T.end(A.err);
}

// Levels 1 .. L-1 of the V-cycle of one window (levels >= 3), four blocks
// per window (blockIdx.y = q): each takes g^2 from the gradient kernel into
// shared memory, restricts it to the coarser levels, takes the coarsest step
// and the way up to level 2 (the same work in all four blocks), then writes
// e^1 = g^1 / w^1 + (u^1 / w^1) I_H^h e^2 over its quarter of the rows of
// g^1, every product rounded as written.  The finest level (w . Delta =
// g^0 + u^0 I_H^h e^1) is formed pixel by pixel by the update kernel.
// Dynamic shared memory: levels 2 .. L-1 as float2.  Launched as a
// programmatic dependent of the gradient kernel; each block starts on its
// window once the gradient kernel has handed it over.
constexpr int kCoarseSplit = 4;
template <int MS>
__global__ void __launch_bounds__(1024) coarse_cycle_kernel(const PrecArgs A) {
  extern __shared__ __align__(16) unsigned char csm[];
  float2* E = reinterpret_cast<float2*>(csm);
  constexpr int nt = 1024;
  const int w = blockIdx.x, q = blockIdx.y, tid = threadIdx.x, L = A.L;
  grid_dep_launch();  // the update kernel after it waits for the whole grid
  if ((unsigned)A.idx[w] >= (unsigned)A.n_pos) return;
  if (!handoff_wait(A, &A.hand[2 * A.count + w], MS / kTcLines)) return;  // ran out: skip the window
  auto off = [&](int l) {  // level l >= 2
    int o = 0;
    for (int j = 2; j < l; ++j) o += (MS >> j) * (MS >> j);
    return o;
  };
  {
    constexpr int s2 = MS >> 2;
    const float2* g2 = A.g2 + (size_t)w * s2 * s2;
#pragma unroll
    for (int i = tid; i < s2 * s2; i += nt) E[i] = __ldcg(&g2[i]);  // off(2) = 0
    __syncthreads();
  }
  constexpr int LM = MS == 256 ? 8 : MS == 128 ? 7 : 6;  // log2(MS)
  for (int l = 3; l < L; ++l) {
    const int s = MS >> l, sf = MS >> (l - 1), ls = LM - l;
    const float2* src = E + off(l - 1);
    const float* wu = A.pyr + lvl_off(MS, l);
    for (int i = tid; i < s * s; i += nt) {
      const int r = i >> ls, c = i & (s - 1);
      const float2 a = src[(2 * r) * sf + 2 * c], b = src[(2 * r) * sf + 2 * c + 1];
      const float2 cc = src[(2 * r + 1) * sf + 2 * c], d = src[(2 * r + 1) * sf + 2 * c + 1];
      const float f = 0.25f * __ldg(&wu[i]);
      E[off(l) + i] = make_float2(f * (a.x + b.x + cc.x + d.x), f * (a.y + b.y + cc.y + d.y));
    }
    __syncthreads();
  }
  {
    const int s = MS >> (L - 1);
    const float* iw = A.pyr + lvl_off(MS, L - 1) + s * s;
    for (int i = tid; i < s * s; i += nt) {
      const float2 g = E[off(L - 1) + i];
      const float f = __ldg(&iw[i]);
      E[off(L - 1) + i] = make_float2(g.x * f, g.y * f);
    }
    __syncthreads();
  }
  for (int l = L - 2; l >= 2; --l) {
    const int s = MS >> l, sc = MS >> (l + 1), ls = LM - l;
    const float* iw = A.pyr + lvl_off(MS, l) + s * s;
    const float* rr = iw + s * s;
    float2* a = E + off(l);
    const float2* pe = E + off(l + 1);
    for (int i = tid; i < s * s; i += nt) {
      const int r = i >> ls, c = i & (s - 1);
      const float2 p = pe[(r >> 1) * sc + (c >> 1)];
      const float2 g = a[i];
      const float f = __ldg(&iw[i]), q2 = __ldg(&rr[i]);
      a[i] = make_float2(__fmaf_rn(q2, p.x, __fmul_rn(g.x, f)), __fmaf_rn(q2, p.y, __fmul_rn(g.y, f)));
    }
    __syncthreads();
  }
  {
    // level 1 over this block's quarter of the rows of g^1 (in place)
    constexpr int s = MS >> 1, sc = MS >> 2, rows = s / kCoarseSplit;
    float2* g1 = A.g1 + (size_t)w * s * s;
    const float* iw = A.pyr + lvl_off(MS, 1) + s * s;
    const float* rr = iw + s * s;
    const float2* pe = E;  // level 2
#pragma unroll
    for (int i = q * rows * s + tid; i < (q + 1) * rows * s; i += nt) {
      const int r = i >> (LM - 1), c = i & (s - 1);
      const float2 p = pe[(r >> 1) * sc + (c >> 1)];
      const float2 g = __ldcg(&g1[i]);
      const float f = __ldg(&iw[i]), qq = __ldg(&rr[i]);
      g1[i] = make_float2(__fmaf_rn(qq, p.x, __fmul_rn(g.x, f)), __fmaf_rn(qq, p.y, __fmul_rn(g.y, f)));
    }
  }
}

