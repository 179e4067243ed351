// umma.cuh -- the 5th-generation tensor-core (tcgen05) helpers, and the
// learned correction's convolutions on them: BF16 operands staged in shared
// memory, FP32 accumulators in tensor memory.  Included by magpie.cu inside
// namespace magpie_impl, after learned.cuh (ConvFwd, bf16) and before
// precision.cuh (whose transforms also run on them).
//
// One 128-thread block computes a 128 x BN tile of the implicit GEMM
// D[pixel][cout] = sum_k A[pixel][k] W[cout][k], k = (ky, kx, ci), over its
// share of K (split-K as the register-fragment kernel does):
//   * every K step of 64 elements, the block's threads gather the tile's
//     A rows (im2col of the NHWC activations, zero outside the image) and
//     W rows with 16-byte cp.async into one of two or three stages (up to two
//     steps in flight ahead of the tensor core), laid out K-major
//     with the 128-byte swizzle (8 rows x 128 bytes per 1024-byte atom,
//     16-byte chunk c of row r at chunk c ^ (r mod 8));
//   * thread 0 issues four tcgen05.mma (M = 128, N = BN, K = 16 each) on the
//     stage and commits them to the stage's mbarrier, which the threads wait
//     on before loading that stage again;
//   * the accumulator (128 TMEM lanes x BN fp32 columns) is read back with
//     tcgen05.ld, one row per thread, for the bias / ReLU / BF16 epilogue or
//     the split-K partial sums.
// Layers with Cin and Cout multiples of 64 take this path.
#pragma once

namespace umma {

// Shared-memory matrix descriptor of a K-major operand with the 128-byte
// swizzle: start address, leading-dimension offset (unused for this layout,
// encoded 1), stride between 8-row groups 1024 bytes, descriptor version 1,
// swizzle mode 2 (128 bytes).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// The same for the 64-byte swizzle (rows of 64 bytes, 8-row atoms of 512
// bytes, 16-byte chunk c of row r at chunk c ^ ((r >> 1) mod 4)): swizzle
// mode 4, stride between 8-row groups 512 bytes.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}
// byte offset of 16-byte chunk c of row r in a 64-byte-swizzled operand
__host__ __device__ constexpr uint32_t sw64_off(int r, int c) {
  return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((c ^ ((r >> 1) & 3)) << 4));
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor of kind::f16 with FP16 A and B (format fields 0).
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (+)= A B^T, both operands in shared memory, kind::f16 (BF16 or FP16 per
// the instruction descriptor), accumulate when acc != 0.
__device__ __forceinline__ void mma_ss(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on the mbarrier once every tcgen05 operation issued so far by this thread has completed
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 16 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// bounded wait for phase `parity` of a CTA-local mbarrier
__device__ __forceinline__ bool wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kMaxWaitTries; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace umma

constexpr int kTcBM = 128, kTcBK = 64;
// Shared-memory stages of the pipeline: three for N tiles up to 128 (two or
// three blocks per SM), two for 256 (two blocks per SM); the tensor memory
// the resident blocks allocate stays within an SM's 512 columns.
template <int BN>
struct TcConv {
  static constexpr int STAGES = BN >= 256 ? 2 : 3;  // N tiles of 64 and 128 are used
  static constexpr int A_BYTES = kTcBM * kTcBK * 2, B_BYTES = BN * kTcBK * 2, STAGE = A_BYTES + B_BYTES;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE + 1024;  // + alignment slack for 1024-byte atoms
};

// err: bit 2 is set when a bounded wait ran out (the block then skips its
// epilogue, still frees its tensor memory, and returns).
template <int BN>
__global__ void __launch_bounds__(128) conv_fwd_tc_kernel(const ConvFwd a, int* err) {
  static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256 && (BN & (BN - 1)) == 0, "N tile");
  using S = TcConv<BN>;
  constexpr int NS = S::STAGES;
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) unsigned long long bars[NS];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t raw = smem_addr(tc_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t bar0 = smem_addr(&bars[0]);

  if (warp == 0) umma::alloc(smem_addr(&tmem_slot), BN);
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(bar0 + 8 * s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = tmem_slot;

  const int HoHo = a.Ho * a.Ho, Mtot = a.B * HoHo, Hv = a.Hin * a.up;
  const int bm = blockIdx.x * kTcBM, bn = blockIdx.y * BN;
  const int kbeg = blockIdx.z * a.ksplit, kend = min(a.K, kbeg + a.ksplit);
  const int nk = (kend - kbeg) / kTcBK;  // K and the split are multiples of 64
  const int c = tid & 7, r0 = tid >> 3;  // this thread's 16-byte chunk and first row

  // the output pixels of this thread's eight A rows
  int pb[8], py[8], px[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int p = bm + r0 + 16 * i;
    if (p < Mtot) {
      const int b = p / HoHo, rem = p - b * HoHo, oy = rem / a.Ho, ox = rem - oy * a.Ho;
      pb[i] = b;
      py[i] = oy * a.stride - 1;
      px[i] = ox * a.stride - 1;
    } else {
      pb[i] = -1;
      py[i] = px[i] = 0;
    }
  }
  auto load_stage = [&](int st, int k0) {
    const uint32_t sa = base + (uint32_t)(st * S::STAGE), sb = sa + S::A_BYTES;
    const int tap = k0 / a.Cin, ci = k0 - tap * a.Cin + 8 * c;
    const int ky = tap / 3, kx = tap - 3 * ky;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = r0 + 16 * i;
      const int vy = py[i] + ky, vx = px[i] + kx;
      const bool ok = pb[i] >= 0 && vy >= 0 && vy < Hv && vx >= 0 && vx < Hv;
      const bf16* src = ok ? a.in + ((size_t)(pb[i] * a.Hin + vy / a.up) * a.Hin + vx / a.up) * a.Cin + ci : a.in;
      umma::cp_async16(sa + (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4)), src, ok ? 16 : 0);
    }
#pragma unroll
    for (int i = 0; i < BN / 16; ++i) {
      const int n = r0 + 16 * i, co = bn + n;
      const bool ok = co < a.Cout;
      const bf16* src = ok ? a.w + (size_t)co * a.K + k0 + 8 * c : a.w;
      umma::cp_async16(sb + (uint32_t)((n >> 3) * 1024 + (n & 7) * 128 + ((c ^ (n & 7)) << 4)), src, ok ? 16 : 0);
    }
    umma::cp_async_commit();
  };

  constexpr uint32_t IDESC = umma::idesc_bf16(kTcBM, BN);
  bool ok = true;
  // K step j goes to stage j mod NS, one cp.async group per step; the first
  // NS - 1 steps are in flight before the first MMA
  for (int j = 0; j < NS - 1 && j < nk; ++j) load_stage(j, kbeg + j * kTcBK);
  for (int ks = 0; ks < nk; ++ks) {
    const int st = ks % NS;
    // step ks's group is complete once at most (groups issued - ks - 1) remain
    const int pending = min(ks + NS - 1, nk) - ks - 1;
    if (pending >= 2)
      asm volatile("cp.async.wait_group 2;" ::: "memory");
    else if (pending == 1)
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    else
      umma::cp_async_wait_all();
    umma::fence_proxy_async();  // this thread's stage writes, visible to the tensor core
    __syncthreads();
    if (tid == 0) {
      umma::fence_after();
      const uint32_t sa = base + (uint32_t)(st * S::STAGE), sb = sa + S::A_BYTES;
#pragma unroll
      for (int kk = 0; kk < kTcBK / 16; ++kk)
        umma::mma_ss(tmem, umma::desc_sw128(sa + 32 * kk), umma::desc_sw128(sb + 32 * kk), IDESC,
                          (ks | kk) != 0);
      umma::commit(bar0 + 8 * st);
    }
    const int nxt = ks + NS - 1;
    if (nxt < nk) {
      // step nxt reuses the stage of step ks - 1, free once that step's MMAs completed
      if (ks >= 1 && !umma::wait(bar0 + 8 * ((ks - 1) % NS), ((ks - 1) / NS) & 1)) ok = false;
      load_stage(nxt % NS, kbeg + nxt * kTcBK);
    }
  }
  if (nk > 0 && !umma::wait(bar0 + 8 * ((nk - 1) % NS), ((nk - 1) / NS) & 1)) ok = false;
  umma::fence_after();
  if (!ok && lane == 0) atomicOr(err, 4);

  // epilogue: TMEM lane (32 warp + lane) = tile row
  const int p = bm + warp * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
  for (int cc = 0; cc < BN; cc += 16) {
    float v[16];
    if (nk > 0) {
      umma::ld16(trow + (uint32_t)cc, v);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.f;
    }
    const int co = bn + cc;
    if (!ok || p >= Mtot || co >= a.Cout) continue;
    if (a.part) {
      float4* dst = reinterpret_cast<float4*>(&a.part[((size_t)blockIdx.z * Mtot + p) * a.Cout + co]);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      continue;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      v[i] += a.bias[co + i];
      if (a.relu) v[i] = fmaxf(v[i], 0.f);
    }
    if (a.out_f32) {
      float4* dst = reinterpret_cast<float4*>(&static_cast<float*>(a.out)[(size_t)p * a.Cout + co]);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
      uint4 w[2];
      uint32_t* wp = reinterpret_cast<uint32_t*>(w);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        wp[i] = *reinterpret_cast<uint32_t*>(&h);
      }
      uint4* dst = reinterpret_cast<uint4*>(&static_cast<bf16*>(a.out)[(size_t)p * a.Cout + co]);
      dst[0] = w[0];
      dst[1] = w[1];
    }
  }
  umma::fence_before();
  __syncthreads();
  if (warp == 0) {
    umma::fence_after();
    umma::dealloc(tmem, BN);
  }
}
