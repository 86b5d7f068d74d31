// Reduced-precision sector GEMMs on the 5th-generation tensor cores, fed by TMA.
//
// arXiv:2303.11409, Sec. II: the U(1) split turns the two-site contraction into many
// small dense products of charge blocks, and the text names tensor cores for them.  In
// the TF32 and BF16x3 modes both products of an update run here: T_m = B^[s][l,m] B^[s+1][m,r]
// for every charge triple (the Theta build, gate mixed afterwards by mix_kernel) and
// B^[s][l,c] = Theta'(c)[rows of l] Y(c)[:, :k] / |S_kept| (the reassembly).
//
// Operands are first written as shadow tiles (shadow_kernel, mix_kernel): 128 rows of
// 128 bytes, TF32 floats or BF16 hi / lo pairs, with rows and K padded by zeros.  A complex
// product is one real GEMM over the interleaved K (a row of an A tile is re0 im0 re1 im1 ...)
// with the B operand stored as two rows per complex column j, conj(b_j) and i conj(b_j),
// so that the accumulator holds Re and Im of C(i, j) in adjacent columns; the multiply count
// is that of the complex product.  All tiles of a launch are slots of one buffer described
// by one 2-D tensor map (128-byte rows, 128-byte swizzle), so every stage is loaded by
// cp.async.bulk.tensor into the canonical SW128 K-major layout the MMA descriptors expect.
//
// tma_zgemm_kernel is persistent and warp specialised, one CTA per SM:
//   warp 0   one thread issues the TMA loads of a 6-stage (TF32) / 3-stage (BF16x3) ring;
//   warp 1   allocates 256 TMEM columns (two 128 x 128 FP32 accumulators) and one thread
//            issues tcgen05.mma (K = 8 TF32 or 16 BF16 per instruction, BF16x3 as
//            lo.hi + hi.lo + hi.hi), committing each stage back to the producer and each
//            finished tile to the epilogue;
//   warps 2-5 read the accumulator with tcgen05.ld (warp w owns TMEM lanes 32 (w % 4) ..),
//            convert and store the tile while the next tile accumulates in the other buffer.
// Every mbarrier wait is bounded (about 2 s; 50 ms with stall injection, which issues no
// copy and no MMA): on expiry the CTA stops issuing, waits (bounded) for the MMAs it
// committed, records an error and frees its tensor memory.  A real expiry is reported but
// its clean-up is proven safe only when the last wait succeeds; the tests drive the path
// through stall injection.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <vector>

#include "mps_internal.h"

namespace mps {

std::atomic<bool> g_tc_stall{false};   // mps_tc_inject_stall

namespace {

constexpr int kTmThreads = 192;
constexpr int kStagesTF32 = 6, kStagesBF16 = 3;
constexpr int kAccCols = 2 * kShTileN;            // FP32 accumulator columns of one output tile
constexpr uint32_t kTmemCols = 2 * kAccCols;      // double-buffered accumulator
constexpr int kRingBytes = 6 * 2 * (int)kShTileBytes;   // 192 KB for both precisions
constexpr long long kWaitCycles = 4000000000LL;
constexpr long long kStallWaitCycles = 100000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long bound) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 >= bound) return false;
  }
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// one 128-row tile (slot) of the shadow buffer into shared memory, completing on bar
__device__ __forceinline__ void tma_tile(void* dst, const CUtensorMap* tm, int64_t slot, uint64_t* bar) {
  const int y = (int)(slot * kShRows);
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle layout: rows of
// 128 bytes, 8-row groups 1024 bytes apart (SBO); the leading offset is unused for this layout.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                  // LBO = 16 bytes (ignored)
  d |= (uint64_t)(1024 >> 4) << 32;        // SBO
  d |= (uint64_t)1 << 46;                  // descriptor version of this architecture
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}
// Instruction descriptor: D = F32, A and B K-major, format 2 = TF32, 1 = BF16.
__host__ __device__ constexpr uint32_t idesc_f32acc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma(bool tf32, uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  if (tf32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// FP64 -> FP32, round to nearest even, in integer operations only (this part runs FP64 and
// the FP64 <-> FP32 conversions at 2 operations per clock per SM; the integer pipe is 32x
// faster).  From the IEEE-754 binary64 and binary32 layouts: rebias the exponent, keep the top
// 23 of the 52 fraction bits, round on the 29 dropped bits (a carry into the exponent is the
// correct result).  Magnitudes below 2^-126 (FP32 subnormals) become signed zero, overflow
// becomes infinity, NaN stays NaN.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const int fe = e - 1023 + 127;
  if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
  const uint32_t fm = (uint32_t)(m >> 29);
  const uint32_t rem = (uint32_t)(m & 0x1FFFFFFFu);
  uint32_t r = ((uint32_t)fe << 23) | fm;
  if (rem > 0x10000000u || (rem == 0x10000000u && (fm & 1u))) ++r;
  if (r > 0x7F800000u) r = 0x7F800000u;
  return __uint_as_float(sign | r);
}
// FP32 -> FP64 exactly, in integer operations (same layouts; subnormals normalised).
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  unsigned long long r;
  if (e == 0xFFu) {
    r = sgn | 0x7FF0000000000000ull | ((unsigned long long)m << 29);
  } else if (e != 0u) {
    r = sgn | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  } else if (m == 0u) {
    r = sgn;
  } else {
    const int p = 31 - __clz(m);                          // leading bit of the subnormal fraction
    r = sgn | ((unsigned long long)(p + 874) << 52) | (((unsigned long long)m << (52 - p)) & 0xFFFFFFFFFFFFFull);
  }
  return __longlong_as_double((long long)r);
}
__device__ __forceinline__ float to_tf32(float x) {   // round to nearest (ties away) in TF32
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// x = hi + lo to about 2^-17 relative: hi = bf16(x), lo = bf16(x - hi) (x - hi exact in FP32)
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// ---------------------------------------------------------------------------------------
// Shadow tiles.  One CTA per tile; a work item is one 16-byte chunk of a tile row (TF32: 2
// complex; BF16: 4 complex, written to the hi and the lo tile) of one operand row unit u
// (an A row, or a B column giving tile rows 2u and 2u + 1).
// ---------------------------------------------------------------------------------------
template <bool TF32>
__device__ __forceinline__ void put_chunk(char* slot, int row, int chunk, const float* re, const float* im) {
  if constexpr (TF32) {
    float4 v = make_float4(to_tf32(re[0]), to_tf32(im[0]), to_tf32(re[1]), to_tf32(im[1]));
    *reinterpret_cast<float4*>(slot + row * kShRowBytes + chunk * 16) = v;
  } else {
    __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      split_bf16(re[e], h[2 * e], l[2 * e]);
      split_bf16(im[e], h[2 * e + 1], l[2 * e + 1]);
    }
    *reinterpret_cast<uint4*>(slot + row * kShRowBytes + chunk * 16) = *reinterpret_cast<const uint4*>(h);
    *reinterpret_cast<uint4*>(slot + kShTileBytes + row * kShRowBytes + chunk * 16) =
        *reinterpret_cast<const uint4*>(l);
  }
}

template <bool TF32>
__global__ void __launch_bounds__(256) shadow_kernel(const ShadowTask* __restrict__ tasks,
                                                     const ShadowTile* __restrict__ tiles, char* __restrict__ slots) {
  constexpr int CPC = TF32 ? 2 : 4;                 // complex per 16-byte chunk
  constexpr int KC = 8 * CPC;                       // complex K per tile row
  constexpr int TPK = TF32 ? 1 : 2;
  const ShadowTile t = tiles[blockIdx.x];
  const ShadowTask T = tasks[t.task];
  char* slot = slots + (T.tile0 + ((int64_t)t.it * T.kt_n + t.kt) * TPK) * kShTileBytes;
  const int units = T.is_b ? kShTileN : kShRows;
  const int i0 = t.it * units, k0 = t.kt * KC;
  const bool kfast = T.s_k == 1;
  for (int w = threadIdx.x; w < units * 8; w += blockDim.x) {
    const int u = kfast ? (w >> 3) : (w % units);
    const int c = kfast ? (w & 7) : (w / units);
    const int i = i0 + u;
    float re[CPC], im[CPC];
#pragma unroll
    for (int e = 0; e < CPC; ++e) {
      const int k = k0 + c * CPC + e;
      double2 v = make_double2(0.0, 0.0);
      if (i < T.n_i && k < T.K) v = T.src[(int64_t)i * T.s_i + (int64_t)k * T.s_k];
      re[e] = d2f_rn(v.x);
      im[e] = d2f_rn(v.y);
    }
    if (!T.is_b) {
      put_chunk<TF32>(slot, u, c, re, im);
    } else {
      float nim[CPC];
#pragma unroll
      for (int e = 0; e < CPC; ++e) nim[e] = -im[e];
      put_chunk<TF32>(slot, 2 * u, c, re, nim);      // conj(b):   (re, -im)
      put_chunk<TF32>(slot, 2 * u + 1, c, im, re);   // i conj(b): (im, re)
    }
  }
}

// ---------------------------------------------------------------------------------------
// The GEMM.
// ---------------------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kTmThreads, 1)
    tma_zgemm_kernel(const __grid_constant__ CUtensorMap tm, const TmaJob* __restrict__ jobs, int n_jobs,
                     int* __restrict__ error_flag, int stall) {
  constexpr bool kTF = (P == MPS_TF32);
  constexpr int S = kTF ? kStagesTF32 : kStagesBF16;
  constexpr int TPK = kTF ? 1 : 2;                       // slots per K tile of one operand
  constexpr uint32_t kStageBytes = 2 * TPK * (uint32_t)kShTileBytes;
  constexpr uint32_t idesc = idesc_f32acc(kTF ? 2 : 1, kShRows, kAccCols);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* ring = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[S], empty[S], tfull[2], tempty[2], fin;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long bound = stall ? kStallWaitCycles : kWaitCycles;
  volatile int* abort_flag = &s_abort;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 128);
    }
    mbar_init(&fin, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tm)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---- producer: the K tiles of this CTA's jobs, in order, through the ring ----
    if (lane == 0 && !stall) {
      int it = 0;
      for (int j = blockIdx.x; j < n_jobs && !*abort_flag; j += gridDim.x) {
        const TmaJob J = jobs[j];
        for (int kt = 0; kt < J.kt_n; ++kt, ++it) {
          const int s = it % S;
          if (!mbar_wait(&empty[s], (uint32_t)(((it / S) & 1) ^ 1), bound) || *abort_flag) {
            *abort_flag = 1;
            break;
          }
          mbar_expect_tx(&full[s], kStageBytes);
          unsigned char* st = ring + s * kStageBytes;
          const int64_t a = J.a0 + (int64_t)kt * TPK, b = J.b0 + (int64_t)kt * TPK;
          tma_tile(st, &tm, a, &full[s]);
          if constexpr (kTF) {
            tma_tile(st + kShTileBytes, &tm, b, &full[s]);
          } else {
            tma_tile(st + kShTileBytes, &tm, a + 1, &full[s]);
            tma_tile(st + 2 * kShTileBytes, &tm, b, &full[s]);
            tma_tile(st + 3 * kShTileBytes, &tm, b + 1, &full[s]);
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      int it = 0, jt = 0;
      bool issued = false;
      for (int j = blockIdx.x; j < n_jobs && !*abort_flag; j += gridDim.x, ++jt) {
        const TmaJob J = jobs[j];
        const int buf = jt & 1;
        if (!mbar_wait(&tempty[buf], (uint32_t)(((jt >> 1) & 1) ^ 1), bound) || *abort_flag) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * kAccCols);
        bool ok = true;
        for (int kt = 0; kt < J.kt_n; ++kt, ++it) {
          const int s = it % S;
          if (!mbar_wait(&full[s], (uint32_t)((it / S) & 1), bound) || *abort_flag) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(ring + s * kStageBytes);
#pragma unroll
          for (int q = 0; q < 4; ++q) {          // 32 bytes of K per instruction
            if constexpr (kTF) {
              mma(true, d, desc_sw128(st + 32 * q), desc_sw128(st + kShTileBytes + 32 * q), idesc,
                  (kt > 0 || q > 0) ? 1u : 0u);
            } else {
              const uint32_t ah = st, al = st + kShTileBytes, bh = st + 2 * kShTileBytes, bl = st + 3 * kShTileBytes;
              mma(false, d, desc_sw128(al + 32 * q), desc_sw128(bh + 32 * q), idesc, (kt > 0 || q > 0) ? 1u : 0u);
              mma(false, d, desc_sw128(ah + 32 * q), desc_sw128(bl + 32 * q), idesc, 1u);
              mma(false, d, desc_sw128(ah + 32 * q), desc_sw128(bh + 32 * q), idesc, 1u);
            }
          }
          issued = true;
          tc_commit(&empty[s]);                  // the stage is free once these MMAs are done
        }
        if (!ok) {
          *abort_flag = 1;
          break;
        }
        tc_commit(&tfull[buf]);                  // the tile is complete in TMEM
      }
      // nothing may be in flight when the tensor memory is freed
      if (issued) {
        tc_commit(&fin);
        if (!mbar_wait(&fin, 0u, bound)) *abort_flag = 1;
      }
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 ----
    const int q = warp & 3;
    const int row = 32 * q + lane;
    int jt = 0;
    for (int j = blockIdx.x; j < n_jobs; j += gridDim.x, ++jt) {
      const TmaJob J = jobs[j];
      const int buf = jt & 1;
      const bool ok = mbar_wait(&tfull[buf], (uint32_t)((jt >> 1) & 1), bound);
      if (!__all_sync(0xffffffffu, ok) || *abort_flag) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * kAccCols);
      for (int c0 = 0; c0 < kAccCols; c0 += 16) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (J.kt_n == 0) {
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = 0u;
        }
        const int col = c0 / 2;                  // first complex column of the chunk
        if (row < J.M) {
          if (J.mode == 0) {
            float2* dst = reinterpret_cast<float2*>(J.C) + (int64_t)row * J.ldc + col;
            if (col + 8 <= J.N) {
#pragma unroll
              for (int e = 0; e < 4; ++e)
                reinterpret_cast<float4*>(dst)[e] = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                                                                __uint_as_float(v[4 * e + 2]),
                                                                __uint_as_float(v[4 * e + 3]));
            } else {
              for (int e = 0; e < 8 && col + e < J.N; ++e)
                dst[e] = make_float2(__uint_as_float(v[2 * e]), __uint_as_float(v[2 * e + 1]));
            }
          } else {
            double2* dst = reinterpret_cast<double2*>(J.C) + (int64_t)row * J.ldc + col;
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (col + e < J.N)
                dst[e] = make_double2(f2d(J.alpha * __uint_as_float(v[2 * e])),
                                      f2d(J.alpha * __uint_as_float(v[2 * e + 1])));
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && s_abort) atomicExch(error_flag, 1);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
  }
}

// ---------------------------------------------------------------------------------------
// The gate mix of the Theta build (one CTA per (l, r) pair).
// ---------------------------------------------------------------------------------------
template <bool TF32>
__global__ void __launch_bounds__(256) mix_kernel(const MixTask* __restrict__ tasks, char* __restrict__ slots) {
  constexpr int KC = TF32 ? 16 : 32;
  constexpr int TPK = TF32 ? 1 : 2;
  __shared__ float2 g[MPS_MAX_D][MPS_MAX_D];       // g[o][i] = G_n[go_o, gi_i]
  const MixTask& T = tasks[blockIdx.x];
  const int nm = T.nm, nc = T.nc;
  if (threadIdx.x < nm * nc) {
    const int o = threadIdx.x / nm, i = threadIdx.x % nm;
    const double2 v = T.gate[T.go[o] * T.sn + T.gi[i]];
    g[o][i] = make_float2(d2f_rn(v.x), d2f_rn(v.y));
  }
  __syncthreads();
  const int64_t n = (int64_t)T.Dl * T.Dr;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const int row = (int)(e / T.Dr), col = (int)(e % T.Dr);
    float2 t[MPS_MAX_D];
#pragma unroll
    for (int i = 0; i < MPS_MAX_D; ++i)
      if (i < nm) t[i] = T.T[i][(int64_t)row * T.ldt + col];
    for (int o = 0; o < nc; ++o) {
      float ar = 0.f, ai = 0.f;
#pragma unroll
      for (int i = 0; i < MPS_MAX_D; ++i)
        if (i < nm) {
          ar = fmaf(g[o][i].x, t[i].x, fmaf(-g[o][i].y, t[i].y, ar));
          ai = fmaf(g[o][i].x, t[i].y, fmaf(g[o][i].y, t[i].x, ai));
        }
      T.out[o][(int64_t)row * T.ldo[o] + col] = make_double2(f2d(ar), f2d(ai));
      // the same value in the reassembly's A tiles of block (l, c_o)
      const int k = T.coff[o] + col;
      char* slot = slots + (T.sh0[o] + ((int64_t)(row / kShRows) * T.sh_ktn[o] + k / KC) * TPK) * kShTileBytes;
      const int r = row % kShRows, kk = k % KC;
      if constexpr (TF32) {
        *reinterpret_cast<float2*>(slot + r * kShRowBytes + kk * 8) = make_float2(to_tf32(ar), to_tf32(ai));
      } else {
        __nv_bfloat16 h[2], l[2];
        split_bf16(ar, h[0], l[0]);
        split_bf16(ai, h[1], l[1]);
        *reinterpret_cast<__nv_bfloat162*>(slot + r * kShRowBytes + kk * 4) = __halves2bfloat162(h[0], h[1]);
        *reinterpret_cast<__nv_bfloat162*>(slot + kShTileBytes + r * kShRowBytes + kk * 4) =
            __halves2bfloat162(l[0], l[1]);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

cudaError_t encoder(PFN_cuTensorMapEncodeTiled_v12000* out) {
  std::lock_guard<std::mutex> lk(g_encode_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  *out = g_encode;
  return cudaSuccess;
}

// The whole shadow buffer as a 2-D tensor of 128-byte rows; a box is one 128-row slot.
cudaError_t make_map(int precision, const char* d_slots, int64_t n_slots, CUtensorMap* tm) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  cudaError_t e = encoder(&enc);
  if (e != cudaSuccess) return e;
  if (((uintptr_t)d_slots & 1023) != 0 || n_slots <= 0 || n_slots * kShRows > 0x7FFFFFFFLL)
    return cudaErrorInvalidValue;
  const bool tf = precision == MPS_TF32;
  const cuuint64_t dims[2] = {(cuuint64_t)(tf ? 32 : 64), (cuuint64_t)(n_slots * kShRows)};
  const cuuint64_t strides[1] = {(cuuint64_t)kShRowBytes};
  const cuuint32_t box[2] = {(cuuint32_t)(tf ? 32 : 64), (cuuint32_t)kShRows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(tm, tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                         const_cast<char*>(d_slots), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int g_num_sms = 0;

template <int P>
cudaError_t launch_gemm_p(const TmaJob* d_jobs, int n_jobs, const char* d_slots, int64_t n_slots, int* d_err,
                          cudaStream_t st) {
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  constexpr int smem = kRingBytes + 1024;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(tma_zgemm_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
  if (attr_err != cudaSuccess) return attr_err;
  CUtensorMap tm;
  cudaError_t e = make_map(P, d_slots, n_slots, &tm);
  if (e != cudaSuccess) return e;
  if (g_num_sms <= 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || g_num_sms <= 0)
      g_num_sms = 148;
  }
  const int grid = std::min(n_jobs, g_num_sms);
  count_launch();
  tma_zgemm_kernel<P><<<grid, kTmThreads, smem, st>>>(tm, d_jobs, n_jobs, d_err, g_tc_stall.load() ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_shadow(int precision, const ShadowTask* d_tasks, const ShadowTile* d_tiles, int n_tiles,
                          char* d_slots, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  count_launch();
  if (precision == MPS_TF32)
    shadow_kernel<true><<<n_tiles, 256, 0, st>>>(d_tasks, d_tiles, d_slots);
  else if (precision == MPS_BF16X3)
    shadow_kernel<false><<<n_tiles, 256, 0, st>>>(d_tasks, d_tiles, d_slots);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_tma_zgemm(int precision, const TmaJob* d_jobs, int n_jobs, const char* d_slots, int64_t n_slots,
                             int* d_err, cudaStream_t st) {
  if (n_jobs <= 0) return cudaSuccess;
  if (precision == MPS_TF32) return launch_gemm_p<MPS_TF32>(d_jobs, n_jobs, d_slots, n_slots, d_err, st);
  if (precision == MPS_BF16X3) return launch_gemm_p<MPS_BF16X3>(d_jobs, n_jobs, d_slots, n_slots, d_err, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_mix(int precision, const MixTask* d_tasks, int n_tasks, char* d_slots, cudaStream_t st) {
  if (n_tasks <= 0) return cudaSuccess;
  count_launch();
  if (precision == MPS_TF32)
    mix_kernel<true><<<n_tasks, 256, 0, st>>>(d_tasks, d_slots);
  else if (precision == MPS_BF16X3)
    mix_kernel<false><<<n_tasks, 256, 0, st>>>(d_tasks, d_slots);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace mps
