// learned.cuh -- the learned coarse-level correction: the network's forward
// pass (BF16 tensor-core implicit GEMM, FP32 accumulation), its backward pass
// and Adam step (FP32), and the per-window kernels that build the network's
// input on the coarsest grid of the V-cycle and apply its proposal with the
// surrogate acceptance test.  Included by magpie.cu inside its anonymous
// namespace.
//
// The paper has no network; its MAGPS (Algorithm MAGPS) ends the recursion on
// the coarsest grid with one proximal step, e_plain = g_H / w_H.  Here a
// six-layer convolutional network sees (z_H, e_plain / s) on that grid, s the
// RMS of e_plain over the window, and proposes e_nn = e_plain + s y.  Each
// window keeps the V-cycle output built on e_nn only when the window's
// quadratic surrogate 1/2 ||Q x - R_k||^2 (Eq. quadratic_surrogate) is no
// larger there than at the output built on e_plain.
#pragma once
#include <cuda_bf16.h>

constexpr int kCnnLayers = 6;
struct CnnLayer {
  int cin, cout, stride, up, relu;
};
// 3x3 convolutions, zero padding 1, nearest-neighbour upsampling of the input
// by `up`; sides h, h, h/2, h/4, h/8, h/4, h.
constexpr CnnLayer kCnn[kCnnLayers] = {
    {4, 32, 1, 1, 1}, {32, 64, 2, 1, 1}, {64, 128, 2, 1, 1}, {128, 512, 2, 1, 1}, {512, 64, 1, 2, 1}, {64, 2, 1, 4, 0},
};

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------ forward (MMA)
struct ConvFwd {
  const bf16* in;     // [B][Hin][Hin][Cin]
  const bf16* w;      // [Cout][3][3][Cin]
  const float* bias;  // [Cout]
  void* out;          // [B][Ho][Ho][Cout]: bf16 (hidden layers) or float (last)
  float* part;        // split-K: [splits][Mtot][Cout] partial sums, else null
  int B, Hin, Cin, Cout, stride, up, Ho, relu, out_f32;
  int K;       // 9 Cin
  int ksplit;  // K elements per split (multiple of 32)
};

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Implicit GEMM: rows = output pixels (b, oy, ox), columns = output channels,
// k = (ky, kx, ci).  Four warps; BM x BN tile, BK = 32 per stage.
template <int BM, int BN>
__global__ void __launch_bounds__(128) conv_fwd_kernel(const ConvFwd a) {
  constexpr int BK = 32, LDS = BK + 8;
  constexpr int WARPS_M = BM / 32, WARPS_N = 4 / WARPS_M, WTN = BN / WARPS_N, WN = WTN / 8;
  static_assert(WARPS_M * WARPS_N == 4 && WN >= 1, "tile");
  __shared__ __align__(16) bf16 As[BM * LDS];
  __shared__ __align__(16) bf16 Bs[BN * LDS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp % WARPS_M, wn = warp / WARPS_M;
  const int g = lane >> 2, t = lane & 3;
  const int HoHo = a.Ho * a.Ho;
  const int Mtot = a.B * HoHo;
  const int bm = blockIdx.x * BM, bn = blockIdx.y * BN;
  const int kbeg = blockIdx.z * a.ksplit;
  const int kend = min(a.K, kbeg + a.ksplit);
  const int Hv = a.Hin * a.up;
  const bool vec = (a.Cin % BK) == 0;
  float acc[2][WN][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < WN; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

  // global -> registers (the next stage, while the current one is multiplied)
  constexpr int AC = (BM * 4 + 127) / 128, BC = (BN * 4 + 127) / 128;
  uint4 ra[AC], rb[BC];
  auto load_a = [&](int c, int k0) -> uint4 {
    const int row = c >> 2, qd = c & 3;
    const int p = bm + row;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (p < Mtot) {
      const int b = p / HoHo, rem = p - b * HoHo;
      const int oy = rem / a.Ho, ox = rem - oy * a.Ho;
      if (vec) {
        const int tap = k0 / a.Cin, ci0 = k0 - tap * a.Cin + 8 * qd;
        const int ky = tap / 3, kx = tap - 3 * ky;
        const int vy = oy * a.stride + ky - 1, vx = ox * a.stride + kx - 1;
        if (vy >= 0 && vy < Hv && vx >= 0 && vx < Hv) {
          const int iy = vy / a.up, ix = vx / a.up;
          v = *reinterpret_cast<const uint4*>(a.in + ((size_t)(b * a.Hin + iy) * a.Hin + ix) * a.Cin + ci0);
        }
      } else {
        bf16 e8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = k0 + 8 * qd + j;
          bf16 val = __float2bfloat16_rn(0.f);
          if (k < a.K) {
            const int tap = k / a.Cin, ci = k - tap * a.Cin;
            const int ky = tap / 3, kx = tap - 3 * ky;
            const int vy = oy * a.stride + ky - 1, vx = ox * a.stride + kx - 1;
            if (vy >= 0 && vy < Hv && vx >= 0 && vx < Hv)
              val = a.in[((size_t)(b * a.Hin + vy / a.up) * a.Hin + vx / a.up) * a.Cin + ci];
          }
          e8[j] = val;
        }
        v = *reinterpret_cast<const uint4*>(e8);
      }
    }
    return v;
  };
  auto load_b = [&](int c, int k0) -> uint4 {
    const int row = c >> 2, qd = c & 3;
    const int co = bn + row;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (co < a.Cout) {
      const bf16* src = a.w + (size_t)co * a.K + k0 + 8 * qd;
      if (vec) {
        v = *reinterpret_cast<const uint4*>(src);
      } else {
        bf16 e8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) e8[j] = (k0 + 8 * qd + j < a.K) ? src[j] : __float2bfloat16_rn(0.f);
        v = *reinterpret_cast<const uint4*>(e8);
      }
    }
    return v;
  };
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < AC; ++u) {
      const int c = tid + 128 * u;
      if (c < BM * 4) ra[u] = load_a(c, k0);
    }
#pragma unroll
    for (int u = 0; u < BC; ++u) {
      const int c = tid + 128 * u;
      if (c < BN * 4) rb[u] = load_b(c, k0);
    }
  };
  if (kbeg < kend) fetch(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int u = 0; u < AC; ++u) {
      const int c = tid + 128 * u;
      if (c < BM * 4) *reinterpret_cast<uint4*>(&As[(c >> 2) * LDS + 8 * (c & 3)]) = ra[u];
    }
#pragma unroll
    for (int u = 0; u < BC; ++u) {
      const int c = tid + 128 * u;
      if (c < BN * 4) *reinterpret_cast<uint4*>(&Bs[(c >> 2) * LDS + 8 * (c & 3)]) = rb[u];
    }
    __syncthreads();
    if (k0 + BK < kend) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[2][4], bfr[WN][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = wm * 32 + mi * 16 + g;
        af[mi][0] = *reinterpret_cast<const uint32_t*>(&As[r * LDS + kk + 2 * t]);
        af[mi][1] = *reinterpret_cast<const uint32_t*>(&As[(r + 8) * LDS + kk + 2 * t]);
        af[mi][2] = *reinterpret_cast<const uint32_t*>(&As[r * LDS + kk + 8 + 2 * t]);
        af[mi][3] = *reinterpret_cast<const uint32_t*>(&As[(r + 8) * LDS + kk + 8 + 2 * t]);
      }
#pragma unroll
      for (int j = 0; j < WN; ++j) {
        const int n = wn * WTN + j * 8 + g;
        bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[n * LDS + kk + 2 * t]);
        bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[n * LDS + kk + 8 + 2 * t]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int j = 0; j < WN; ++j) mma_bf16(acc[mi][j], af[mi], bfr[j]);
    }
    __syncthreads();
  }

  // ---- epilogue: C fragment (row g / g+8, columns 2t, 2t+1)
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int j = 0; j < WN; ++j) {
      const int co = bn + wn * WTN + j * 8 + 2 * t;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int r = bm + wm * 32 + mi * 16 + g + 8 * hh;
        if (r >= Mtot || co >= a.Cout) continue;
        float v0 = acc[mi][j][2 * hh], v1 = acc[mi][j][2 * hh + 1];
        if (a.part) {
          *reinterpret_cast<float2*>(&a.part[((size_t)blockIdx.z * Mtot + r) * a.Cout + co]) = make_float2(v0, v1);
          continue;
        }
        v0 += a.bias[co];
        v1 += a.bias[co + 1];
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (a.out_f32)
          *reinterpret_cast<float2*>(&static_cast<float*>(a.out)[(size_t)r * a.Cout + co]) = make_float2(v0, v1);
        else
          *reinterpret_cast<__nv_bfloat162*>(&static_cast<bf16*>(a.out)[(size_t)r * a.Cout + co]) =
              __floats2bfloat162_rn(v0, v1);
      }
    }
}

// Direct convolutions for the thin layers, where an implicit-GEMM tile would
// be mostly padding.  Both read the BF16 inputs and weights (exact in FP32)
// and accumulate in FP32; consecutive lanes take consecutive 16-byte pieces of
// one pixel's channels, so a warp's loads and stores are contiguous.
//
// Few outputs (the last layer, 64 -> 2): S = CIN / 8 lanes per output pixel,
// lane `part` holding input channels 8 part .. 8 part + 7 of every tap; the S
// partial sums of each output are added with butterfly shuffles.  Weights sit
// in shared memory as BF16 [tap][co][ci], so the S lanes of a pixel read one
// contiguous 16 S-byte row per (tap, co).  Needs `in` 16-byte aligned.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) conv_thin_out_kernel(const ConvFwd a) {
  constexpr int S = CIN / 8;
  static_assert(CIN % 8 == 0 && (S & (S - 1)) == 0 && S <= 32, "channel split");
  __shared__ __align__(16) bf16 wsm[9 * COUT * CIN];
  for (int i = threadIdx.x; i < 9 * COUT * CIN; i += blockDim.x) {
    const int co = i / (9 * CIN), r = i - co * 9 * CIN, tap = r / CIN, ci = r - tap * CIN;
    wsm[(tap * COUT + co) * CIN + ci] = a.w[i];
  }
  __syncthreads();
  const int HH = a.Ho * a.Ho, Mtot = a.B * HH, Hv = a.Hin * a.up;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = t < (long long)Mtot * S;  // whole pixel groups: S divides 32
  const int pix = live ? (int)(t / S) : 0, part = (int)(t % S);
  const int b = pix / HH, rem = pix - b * HH, oy = rem / a.Ho, ox = rem - oy * a.Ho;
  float acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = 0.f;
  for (int ky = 0; ky < 3; ++ky) {
    const int vy = oy * a.stride + ky - 1;
    if (!live || vy < 0 || vy >= Hv) continue;
    const bf16* rowp = a.in + (size_t)(b * a.Hin + vy / a.up) * a.Hin * CIN + part * 8;
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
      const int vx = ox * a.stride + kx - 1;
      if (vx < 0 || vx >= Hv) continue;
      const uint4 raw = __ldg(reinterpret_cast<const uint4*>(rowp + (size_t)(vx / a.up) * CIN));
      const __nv_bfloat162* xh = reinterpret_cast<const __nv_bfloat162*>(&raw);
      float x[8];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x[2 * j] = __low2float(xh[j]);
        x[2 * j + 1] = __high2float(xh[j]);
      }
#pragma unroll
      for (int co = 0; co < COUT; ++co) {
        const uint4 wr = *reinterpret_cast<const uint4*>(&wsm[((ky * 3 + kx) * COUT + co) * CIN + part * 8]);
        const __nv_bfloat162* wh = reinterpret_cast<const __nv_bfloat162*>(&wr);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[co] = fmaf(x[2 * j], __low2float(wh[j]), acc[co]);
          acc[co] = fmaf(x[2 * j + 1], __high2float(wh[j]), acc[co]);
        }
      }
    }
  }
#pragma unroll
  for (int co = 0; co < COUT; ++co)
#pragma unroll
    for (int off = S / 2; off > 0; off >>= 1) acc[co] += __shfl_xor_sync(0xffffffffu, acc[co], off);
  if (!live || part != 0) return;
#pragma unroll
  for (int co = 0; co < COUT; ++co) {
    float v = acc[co] + a.bias[co];
    if (a.relu) v = fmaxf(v, 0.f);
    if (a.out_f32)
      static_cast<float*>(a.out)[(size_t)pix * COUT + co] = v;
    else
      static_cast<bf16*>(a.out)[(size_t)pix * COUT + co] = __float2bfloat16_rn(v);
  }
}

// Few inputs (the first layer, 4 -> 32): OS = COUT / 8 lanes per output pixel,
// lane `part` computing outputs 8 part .. 8 part + 7 from the pixel's 9 x 4
// inputs (one 8-byte load per tap, shared by the OS lanes).  Weights sit in
// shared memory as FP32 [tap][ci][co]; the OS lanes of a pixel read
// consecutive 32-byte pieces of one row.  BF16 output only, stored as one
// 16-byte piece per lane; needs `in` 8-byte and `out` 16-byte aligned.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) conv_thin_in_kernel(const ConvFwd a) {
  constexpr int OS = COUT / 8;
  static_assert(CIN == 4 && COUT % 8 == 0 && (OS & (OS - 1)) == 0 && OS <= 32, "output split");
  __shared__ __align__(16) float wsm[9 * CIN * COUT];
  for (int i = threadIdx.x; i < 9 * COUT * CIN; i += blockDim.x) {
    const int co = i / (9 * CIN), r = i - co * 9 * CIN;
    wsm[r * COUT + co] = __bfloat162float(a.w[i]);
  }
  __syncthreads();
  const int HH = a.Ho * a.Ho, Mtot = a.B * HH, Hv = a.Hin * a.up;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)Mtot * OS) return;
  const int pix = (int)(t / OS), part = (int)(t % OS);
  const int b = pix / HH, rem = pix - b * HH, oy = rem / a.Ho, ox = rem - oy * a.Ho;
  float acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.f;
  for (int ky = 0; ky < 3; ++ky) {
    const int vy = oy * a.stride + ky - 1;
    if (vy < 0 || vy >= Hv) continue;
    const bf16* rowp = a.in + (size_t)(b * a.Hin + vy / a.up) * a.Hin * CIN;
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
      const int vx = ox * a.stride + kx - 1;
      if (vx < 0 || vx >= Hv) continue;
      const uint2 raw = __ldg(reinterpret_cast<const uint2*>(rowp + (size_t)(vx / a.up) * CIN));
      const __nv_bfloat162* xh = reinterpret_cast<const __nv_bfloat162*>(&raw);
      const float x[4] = {__low2float(xh[0]), __high2float(xh[0]), __low2float(xh[1]), __high2float(xh[1])};
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci) {
        const float4* wr = reinterpret_cast<const float4*>(&wsm[((ky * 3 + kx) * CIN + ci) * COUT + part * 8]);
        const float4 w0 = wr[0], w1 = wr[1];
        acc[0] = fmaf(x[ci], w0.x, acc[0]);
        acc[1] = fmaf(x[ci], w0.y, acc[1]);
        acc[2] = fmaf(x[ci], w0.z, acc[2]);
        acc[3] = fmaf(x[ci], w0.w, acc[3]);
        acc[4] = fmaf(x[ci], w1.x, acc[4]);
        acc[5] = fmaf(x[ci], w1.y, acc[5]);
        acc[6] = fmaf(x[ci], w1.z, acc[6]);
        acc[7] = fmaf(x[ci], w1.w, acc[7]);
      }
    }
  }
  uint4 o;
  __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float v0 = acc[2 * j] + a.bias[part * 8 + 2 * j], v1 = acc[2 * j + 1] + a.bias[part * 8 + 2 * j + 1];
    if (a.relu) {
      v0 = fmaxf(v0, 0.f);
      v1 = fmaxf(v1, 0.f);
    }
    oh[j] = __floats2bfloat162_rn(v0, v1);
  }
  *reinterpret_cast<uint4*>(static_cast<bf16*>(a.out) + (size_t)pix * COUT + part * 8) = o;
}

// Split-K epilogue: partial sums added in split order, then bias and ReLU.
__global__ void __launch_bounds__(256) conv_splitk_kernel(const ConvFwd a, int splits) {
  const int Mtot = a.B * a.Ho * a.Ho;
  const size_t n = (size_t)Mtot * a.Cout;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int s = 0; s < splits; ++s) v += a.part[(size_t)s * n + i];
    v += a.bias[i % a.Cout];
    if (a.relu) v = fmaxf(v, 0.f);
    if (a.out_f32)
      static_cast<float*>(a.out)[i] = v;
    else
      static_cast<bf16*>(a.out)[i] = __float2bfloat16_rn(v);
  }
}

// --------------------------------------------------------- backward (FP32)
// dx[b, iy, ix, ci] = sum over the outputs that read (iy, ix) of
// dz[b, oy, ox, co] W[co, ky, kx, ci], then the previous layer's ReLU mask.
__global__ void __launch_bounds__(256) conv_bwd_data_kernel(const float* __restrict__ dz, const bf16* __restrict__ w,
                                                            const bf16* __restrict__ a_prev, float* __restrict__ dx,
                                                            int B, int Hin, int Cin, int Cout, int stride, int up,
                                                            int Ho) {
  const size_t n = (size_t)B * Hin * Hin * Cin;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int ci = (int)(e % Cin);
    const size_t pix = e / Cin;
    const int ix = (int)(pix % Hin), iy = (int)((pix / Hin) % Hin), b = (int)(pix / ((size_t)Hin * Hin));
    float acc = 0.f;
    if (__bfloat162float(a_prev[e]) > 0.f) {
      for (int uy = 0; uy < up; ++uy)
        for (int ky = 0; ky < 3; ++ky) {
          const int ty = iy * up + uy + 1 - ky;
          if (ty < 0 || ty % stride) continue;
          const int oy = ty / stride;
          if (oy >= Ho) continue;
          for (int ux = 0; ux < up; ++ux)
            for (int kx = 0; kx < 3; ++kx) {
              const int tx = ix * up + ux + 1 - kx;
              if (tx < 0 || tx % stride) continue;
              const int ox = tx / stride;
              if (ox >= Ho) continue;
              const float* d = dz + ((size_t)(b * Ho + oy) * Ho + ox) * Cout;
              const bf16* wp = w + (size_t)(ky * 3 + kx) * Cin + ci;
              for (int co = 0; co < Cout; ++co) acc += d[co] * __bfloat162float(wp[(size_t)co * 9 * Cin]);
            }
        }
    }
    dx[e] = acc;
  }
}

// Weight and bias gradients of one layer as an FP32 GEMM over the output
// pixels p: dW[co][k] = sum_p dz[p][co] A[p][k], where A is the forward
// pass's gather (k < K = 9 Cin) and A[p][K] = 1 (the bias column).  Block:
// 64 channels x 64 k, 256 threads with 4 x 4 results each, 16 pixels per
// shared-memory stage; the pixel range is split over gridDim.z (chunks of
// `chunk` pixels) into partial sums part[z][param] (weights, then biases).
__global__ void __launch_bounds__(256) conv_wgrad_kernel(const float* __restrict__ dz, const bf16* __restrict__ a_in,
                                                         float* __restrict__ part, int B, int Hin, int Cin, int Cout,
                                                         int stride, int up, int Ho, int chunk) {
  __shared__ float Ds[16][64];
  __shared__ float As[16][64];
  const int K = 9 * Cin, Kb = K + 1, P = Cout * K + Cout;
  const int co0 = blockIdx.y * 64, k0 = blockIdx.x * 64;
  const int npix = B * Ho * Ho;
  const int p0 = blockIdx.z * chunk, p1 = min(npix, p0 + chunk);
  const int Hv = Hin * up;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int pb = p0; pb < p1; pb += 16) {
    for (int i = threadIdx.x; i < 16 * 64; i += 256) {
      const int pp = i / 64, c = i % 64;
      const int p = pb + pp, co = co0 + c, k = k0 + c;
      Ds[pp][c] = (p < p1 && co < Cout) ? dz[(size_t)p * Cout + co] : 0.f;
      float av = 0.f;
      if (p < p1 && k < Kb) {
        if (k == K) {
          av = 1.f;
        } else {
          const int tap = k / Cin, ci = k - tap * Cin;
          const int ky = tap / 3, kx = tap - 3 * ky;
          const int b = p / (Ho * Ho), r2 = p - b * Ho * Ho;
          const int oy = r2 / Ho, ox = r2 - oy * Ho;
          const int vy = oy * stride + ky - 1, vx = ox * stride + kx - 1;
          if (vy >= 0 && vy < Hv && vx >= 0 && vx < Hv)
            av = __bfloat162float(a_in[((size_t)(b * Hin + vy / up) * Hin + vx / up) * Cin + ci]);
        }
      }
      As[pp][c] = av;
    }
    __syncthreads();
#pragma unroll
    for (int pp = 0; pp < 16; ++pp) {
      float d[4], a[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        d[j] = Ds[pp][ty * 4 + j];
        a[j] = As[pp][tx * 4 + j];
      }
#pragma unroll
      for (int i2 = 0; i2 < 4; ++i2)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i2][j] += d[i2] * a[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i2 = 0; i2 < 4; ++i2)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int co = co0 + ty * 4 + i2, k = k0 + tx * 4 + j;
      if (co < Cout && k < Kb) part[(size_t)blockIdx.z * P + (k < K ? co * K + k : Cout * K + co)] = acc[i2][j];
    }
}

// grad[p] = sum over chunks of part[chunk][p], in chunk order.
__global__ void __launch_bounds__(256) chunk_sum_kernel(const float* __restrict__ part, float* __restrict__ grad, int P,
                                                        int chunks) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float s = 0.f;
  for (int c = 0; c < chunks; ++c) s += part[(size_t)c * P + p];
  grad[p] = s;
}

// --------------------------------------------------------------- training
// L = 1/2 mean((y - t)^2) with t = (z_H^T - z_H^0) / s - e_plain / s taken
// from the input x0 = (z_H^0, e_plain / s), the later z_H^T and s; dy = (y - t) / n.
// One block; the sum is reduced in a fixed order.
__global__ void __launch_bounds__(1024) cnn_loss_kernel(const float* __restrict__ y, const float4* __restrict__ x0,
                                                        const float2* __restrict__ zh, const float* __restrict__ scale,
                                                        int batch, int hh, float* __restrict__ dy,
                                                        double* __restrict__ loss) {
  __shared__ double red[32];
  const int n = batch * hh;  // pixels
  const double inv_n = 1.0 / (2.0 * (double)n);
  double s2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float s = scale[i / hh];
    const float is = s > 1e-30f ? 1.f / s : 0.f;
    const float4 x = x0[i];
    const float2 zt = zh[i];
    const float tx = (zt.x - x.x) * is - x.z, ty = (zt.y - x.y) * is - x.w;
    const float rx = y[2 * i] - tx, ry = y[2 * i + 1] - ty;
    dy[2 * i] = (float)(rx * inv_n);
    dy[2 * i + 1] = (float)(ry * inv_n);
    s2 += (double)rx * rx + (double)ry * ry;
  }
  const double tot = block_sum(s2, red, threadIdx.x, blockDim.x);
  if (threadIdx.x == 0) *loss = 0.5 * tot * inv_n;
}

// Adam (bias-corrected, c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)); writes the BF16
// copy of the weights the forward pass reads.
__global__ void __launch_bounds__(256) adam_kernel(float* __restrict__ theta, const float* __restrict__ g,
                                                   float* __restrict__ m, float* __restrict__ v, bf16* __restrict__ wbf,
                                                   int P, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float th = theta[i] - lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
  theta[i] = th;
  wbf[i] = __float2bfloat16_rn(th);
}

__global__ void __launch_bounds__(256) to_bf16_kernel(const float* __restrict__ src, bf16* __restrict__ dst, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

// ------------------------------------------------------ per-window kernels
// W_z^l = |Q^l|^2 / (I_H^h I_h^H |Q^l|^2) for l = 0 .. L-2 (Eq. def_weights),
// level l at wz + sum_{j<l} (MS>>j)^2, from block means of Q in float64.
__global__ void __launch_bounds__(256) wz_kernel(const float2* __restrict__ Q, int MS, int L, float* __restrict__ wz) {
  int off = 0;
  for (int l = 0; l + 1 < L; ++l) {
    const int s = MS >> l, f = 1 << l;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s * s; i += gridDim.x * blockDim.x) {
      const int r = i / s, c = i - r * s;
      double a2[4], self = 0.0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          const int rr = (r & ~1) + a, cc = (c & ~1) + b;
          double qx = 0.0, qy = 0.0;
          for (int y = 0; y < f; ++y)
            for (int x = 0; x < f; ++x) {
              const float2 q = Q[(rr * f + y) * MS + cc * f + x];
              qx += q.x;
              qy += q.y;
            }
          qx /= (double)(f * f);
          qy /= (double)(f * f);
          a2[2 * a + b] = qx * qx + qy * qy;
          if (rr == r && cc == c) self = a2[2 * a + b];
        }
      const double S = 0.25 * (a2[0] + a2[1] + a2[2] + a2[3]);
      wz[off + i] = S > 1e-30 ? (float)(self / S) : 0.f;
    }
    off += s * s;
  }
}

struct CoarseArgs {
  const float2* z;      // object [n_rows][n_cols]
  int n_cols;
  const int32_t* pos;   // [n_pos][2]
  const int32_t* idx;   // [count]
  int n_pos, MS, L;
  const float2* g0;     // [count][MS][MS] conj(Q)(R - Q z) from the window kernel
  const float* pyr;     // level factors (window-kernel layout)
  const float* wz;      // W_z^l tables
  float4* x;            // [count][h][h] (Re z_H, Im z_H, Re e/s, Im e/s)
  float* scale;         // [count] s
};

// One block per window: z_H and g_H on the coarsest grid as weighted sums over
// each coarse pixel's fine block, e_plain = g_H / w_H, s = RMS(e_plain).
__global__ void __launch_bounds__(1024) coarse_state_kernel(const CoarseArgs A) {
  __shared__ double red[32];
  const int w = blockIdx.x, tid = threadIdx.x;
  const int MS = A.MS, L = A.L, F = 1 << (L - 1), h = MS >> (L - 1);
  const int k = A.idx[w];
  float4* xo = A.x + (size_t)w * h * h;
  if ((unsigned)k >= (unsigned)A.n_pos) {
    for (int c = tid; c < h * h; c += blockDim.x) xo[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid == 0) A.scale[w] = 0.f;
    return;
  }
  const int pr = A.pos[2 * k], pc = A.pos[2 * k + 1];
  const float2* g0 = A.g0 + (size_t)w * MS * MS;
  const float norm = 1.f / (float)(F * F);
  const float* iwH = A.pyr + lvl_off(MS, L - 1) + h * h;
  float e2 = 0.f;
  for (int c = tid; c < h * h; c += blockDim.x) {
    const int cy = c / h, cx = c - cy * h;
    float2 gs = make_float2(0.f, 0.f), zs = make_float2(0.f, 0.f);
    for (int fy = 0; fy < F; ++fy)
      for (int fx = 0; fx < F; ++fx) {
        const int r = cy * F + fy, cc = cx * F + fx;
        float al = norm, be = norm;
        int woff = 0;
        for (int l = 0; l + 1 < L; ++l) {
          al *= __ldg(&A.pyr[lvl_off(MS, l + 1) + (r >> (l + 1)) * (MS >> (l + 1)) + (cc >> (l + 1))]);
          be *= __ldg(&A.wz[woff + (r >> l) * (MS >> l) + (cc >> l)]);
          woff += (MS >> l) * (MS >> l);
        }
        const float2 gv = g0[r * MS + cc];
        const float2 zv = __ldg(&A.z[(size_t)(pr + r) * A.n_cols + pc + cc]);
        gs.x += al * gv.x;
        gs.y += al * gv.y;
        zs.x += be * zv.x;
        zs.y += be * zv.y;
      }
    const float iw = __ldg(&iwH[c]);
    const float ex = gs.x * iw, ey = gs.y * iw;
    e2 += ex * ex + ey * ey;
    xo[c] = make_float4(zs.x, zs.y, ex, ey);
  }
  __shared__ float s_sh;
  const double tot = block_sum((double)e2, red, tid, blockDim.x);  // valid in thread 0
  if (tid == 0) s_sh = (float)sqrt(tot / (double)(h * h));
  __syncthreads();
  const float s = s_sh;
  const float is = s > 1e-30f ? 1.f / s : 0.f;
  for (int c = tid; c < h * h; c += blockDim.x) {
    float4 v = xo[c];
    v.z *= is;
    v.w *= is;
    xo[c] = v;
  }
  if (tid == 0) A.scale[w] = s;
}

struct LearnedUpArgs {
  const int32_t* idx;  // [count]
  int n_pos, MS, L;
  float2* contrib;     // in: g^0; out: w^0 Delta of the kept V-cycle output
  const float* pyr;    // level factors
  const float* scale;  // [count] s
  const float* y;      // [count][h][h][2] network output
  int* accepted;       // [count] 1 = learned output kept
  double* margin;      // [count] surrogate(plain) - surrogate(learned)
  unsigned long long* stats;  // [0] proposals, [1] acceptances (running totals)
};

// Offsets of level l >= 1 in a per-window pyramid of levels 1 .. L-1.
__host__ __device__ __forceinline__ int up_off(int MS, int l) {
  int o = 0;
  for (int j = 1; j < l; ++j) o += (MS >> j) * (MS >> j);
  return o;
}

// One block per window: the V-cycle above the finest level in residual form,
// from g^0 in the increments, in shared memory.  LEARN: two float2 pyramids of
// levels 1 .. L-1 (plain and learned coarsest correction), the surrogate test
// and the kept one written back as w^0 Delta; otherwise one pyramid (the plain
// MAGPS V-cycle, as the window kernel's pass D computes it).
template <bool LEARN>
__global__ void __launch_bounds__(1024) vcycle_up_kernel(const LearnedUpArgs A) {
  extern __shared__ __align__(16) unsigned char lsm[];
  __shared__ double red[32];
  __shared__ int keep;
  const int w = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int MS = A.MS, L = A.L, M = MS * MS;
  const int k = A.idx[w];
  if ((unsigned)k >= (unsigned)A.n_pos) {
    if (LEARN && tid == 0) {
      A.accepted[w] = 0;
      A.margin[w] = 0.0;
    }
    return;
  }
  const int tot = up_off(MS, L);
  float2* Ep = reinterpret_cast<float2*>(lsm);
  float2* En = LEARN ? Ep + tot : Ep;
  float2* g0 = A.contrib + (size_t)w * M;

  // ---- g^l, l = 1 .. L-1: g^{l+1} = W_u^l . I(g^l)
  for (int l = 1; l < L; ++l) {
    const int s = MS >> l, sf = MS >> (l - 1);
    const float* wu = A.pyr + lvl_off(MS, l);
    float2* dst = Ep + up_off(MS, l);
    const float2* src = (l == 1) ? g0 : Ep + up_off(MS, l - 1);
    for (int i = tid; i < s * s; i += nt) {
      const int r = i / s, c = i - r * s;
      const float2 a = src[(2 * r) * sf + 2 * c], b = src[(2 * r) * sf + 2 * c + 1];
      const float2 cc = src[(2 * r + 1) * sf + 2 * c], d = src[(2 * r + 1) * sf + 2 * c + 1];
      const float f = 0.25f * __ldg(&wu[i]);
      dst[i] = make_float2(f * (a.x + b.x + cc.x + d.x), f * (a.y + b.y + cc.y + d.y));
    }
    __syncthreads();
  }
  // ---- coarsest: plain step and proposal
  const float s = LEARN ? A.scale[w] : 0.f;
  const bool proposed = LEARN && s > 1e-30f;
  {
    const int h = MS >> (L - 1);
    const float* iw = A.pyr + lvl_off(MS, L - 1) + h * h;
    float2* P = Ep + up_off(MS, L - 1);
    float2* N = En + up_off(MS, L - 1);
    const float2* yy = LEARN ? reinterpret_cast<const float2*>(A.y) + (size_t)w * h * h : nullptr;
    for (int i = tid; i < h * h; i += nt) {
      const float2 g = P[i];
      const float f = __ldg(&iw[i]);
      const float2 e = make_float2(g.x * f, g.y * f);
      P[i] = e;
      if (LEARN) {
        if (proposed) {
          const float2 d = yy[i];
          N[i] = make_float2(e.x + s * d.x, e.y + s * d.y);
        } else {
          N[i] = e;
        }
      }
    }
  }
  __syncthreads();
  // ---- up: e^l = g^l / w^l + (u^l / w^l) I_H^h e^{l+1}, l = L-2 .. 1
  for (int l = L - 2; l >= 1; --l) {
    const int s2 = MS >> l, sc = MS >> (l + 1);
    const float* iw = A.pyr + lvl_off(MS, l) + s2 * s2;
    const float* rr = iw + s2 * s2;
    float2* P = Ep + up_off(MS, l);
    float2* N = En + up_off(MS, l);
    const float2* Pc = Ep + up_off(MS, l + 1);
    const float2* Nc = En + up_off(MS, l + 1);
    for (int i = tid; i < s2 * s2; i += nt) {
      const int r = i / s2, c = i - r * s2;
      const int pi = (r >> 1) * sc + (c >> 1);
      const float2 g = P[i];
      const float f = __ldg(&iw[i]), q = __ldg(&rr[i]);
      const float2 ep = Pc[pi];
      if (LEARN) {
        const float2 en = Nc[pi];
        N[i] = make_float2(g.x * f + q * en.x, g.y * f + q * en.y);
      }
      P[i] = make_float2(g.x * f + q * ep.x, g.y * f + q * ep.y);
    }
    __syncthreads();
  }
  const float* u0 = A.pyr;
  const float* w0 = A.pyr + M;
  const int s1 = MS >> 1;
  if (LEARN) {
    // ---- finest: w^0 Delta = g^0 + u^0 I_H^h e^1; surrogate difference
    // 1/2 |Q|^2 |Delta|^2 - Re(conj(Delta) g^0) summed for both candidates
    float dsum = 0.f;
    for (int i = tid; i < M; i += nt) {
      const int r = i / MS, c = i - r * MS;
      const int pi = (r >> 1) * s1 + (c >> 1);
      const float2 g = g0[i];
      const float u = __ldg(&u0[i]), wv = __ldg(&w0[i]);
      const float iwv = wv > 1e-30f ? 1.f / wv : 0.f;
      const float q2 = wv - u;
      const float2 ep = Ep[pi], en = En[pi];
      const float2 dp = make_float2((g.x + u * ep.x) * iwv, (g.y + u * ep.y) * iwv);
      const float2 dn = make_float2((g.x + u * en.x) * iwv, (g.y + u * en.y) * iwv);
      const float sp = 0.5f * q2 * (dp.x * dp.x + dp.y * dp.y) - (dp.x * g.x + dp.y * g.y);
      const float sn = 0.5f * q2 * (dn.x * dn.x + dn.y * dn.y) - (dn.x * g.x + dn.y * g.y);
      dsum += sp - sn;
    }
    const double mg = block_sum((double)dsum, red, tid, nt);
    if (tid == 0) {
      keep = (proposed && mg >= 0.0) ? 1 : 0;
      A.accepted[w] = keep;
      A.margin[w] = proposed ? mg : 0.0;
      if (proposed) atomicAdd(&A.stats[0], 1ull);
      if (keep) atomicAdd(&A.stats[1], 1ull);
    }
    __syncthreads();
  }
  const float2* E = (LEARN && keep) ? En : Ep;
  for (int i = tid; i < M; i += nt) {
    const int r = i / MS, c = i - r * MS;
    const float2 e = E[(r >> 1) * s1 + (c >> 1)];
    const float u = __ldg(&u0[i]);
    const float2 g = g0[i];
    g0[i] = make_float2(g.x + u * e.x, g.y + u * e.y);
  }
}

// patches[w] = the m x m window of the object at window idx[w] (zeros for an
// index out of range).
__global__ void __launch_bounds__(256) gather_windows_kernel(const float2* __restrict__ z, int n_cols,
                                                             const int32_t* __restrict__ pos,
                                                             const int32_t* __restrict__ idx, int n_pos, int MS,
                                                             float2* __restrict__ out) {
  const int w = blockIdx.x, k = idx[w];
  const bool ok = (unsigned)k < (unsigned)n_pos;
  const int pr = ok ? pos[2 * k] : 0, pc = ok ? pos[2 * k + 1] : 0;
  for (int i = threadIdx.x; i < MS * MS; i += blockDim.x) {
    const int r = i / MS, c = i - r * MS;
    out[(size_t)w * MS * MS + i] = ok ? z[(size_t)(pr + r) * n_cols + pc + c] : make_float2(0.f, 0.f);
  }
}
