// Complex GEMMs on the 5th-generation tensor cores (tcgen05) for the
// reduced-precision sector GEMMs: TF32 inputs, or BF16x3 split precision, with
// FP32 accumulation in tensor memory.
//
// A complex product C = A B (A: M x K, B: K x N, complex128 in global memory) is
// lowered to one real GEMM (M x 2K) . (2K x 2N) with the same multiply count.  The
// real K index is interleaved, so that every complex input lands in two adjacent
// K elements and is read from memory once:
//     A'(i, 2k) = Re A(i, k)            A'(i, 2k + 1) = Im A(i, k)
//     B'(2k, j) = Re B(k, j)            B'(2k + 1, j) = -Im B(k, j)       (column j: Re C)
//     B'(2k, 64 + j) = Im B(k, j)       B'(2k + 1, 64 + j) = Re B(k, j)   (column 64 + j: Im C)
// Each CTA computes a 128 x 64 complex output tile: a 128 x 128 real FP32
// accumulator in TMEM (128 columns), fed from shared memory in the canonical
// no-swizzle K-major layout (core matrices of 8 rows x 16 bytes; LBO = next core
// matrix along K, SBO = next 8-row group).  The operands are converted from FP64
// (A multiplied by a complex scalar per K segment, which is how the gate
// coefficient of the Theta build and the 1/|S_kept| of the reassembly enter)
// while being staged: TF32 rounds to nearest; BF16x3 splits x = hi + lo with
// hi = bf16(x), lo = bf16(x - hi) and accumulates lo.hi + hi.lo + hi.hi, dropping
// lo.lo (about 2^-16 relative).  The global loads of the next K step are issued
// before the MMAs of the current one complete; one thread issues tcgen05.mma and
// commits to an mbarrier that releases the stage.  Every wait on an mbarrier is
// bounded: on expiry the CTA records an error and still frees its tensor memory.
// The epilogue stages the accumulator through shared memory so that the FP64
// stores of each output row are contiguous.
#include <cuda_bf16.h>
#include <atomic>
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "mps_internal.h"

namespace mps {
namespace {

constexpr int kTcM = 128;          // rows of the output tile (TMEM lanes)
constexpr int kTcNc = 64;          // complex columns of the output tile
constexpr int kTcN = 2 * kTcNc;    // real accumulator columns
constexpr int kTcKc = 16;          // complex K staged per step (32 real K elements)
constexpr int kTcThreads = 128;
constexpr int kTcStages = 2;
constexpr uint32_t kStageBytes = 32 * 1024;          // TF32: A, B (16 KB each); BF16x3: A hi, A lo, B hi, B lo
constexpr long long kWaitCycles = 4000000000LL;      // bound of every mbarrier wait (~2 s)
constexpr long long kStallWaitCycles = 100000000LL;  // the bound in stall-injection mode (~50 ms)
constexpr int kEpiLd = 17;                           // padded row stride (double2) of the epilogue staging

static_assert(kTcM == kTcTileM && kTcNc == kTcTileN, "tile shape");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: no swizzle, K-major.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;                  // descriptor version for this architecture
  return d;                                // base offset 0, relative LBO, no swizzle
}

// Instruction descriptors: D = F32, A and B K-major; operand format 2 = TF32, 1 = BF16.
__host__ __device__ constexpr uint32_t idesc_f32acc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the phase with the given parity; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long bound) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (clock64() - t0 < bound) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

// FP64 -> FP32, round to nearest even, in integer operations only.  GB300 runs FP64 (and the
// FP64-to-FP32 conversion) at 2 operations per clock per SM, and staging two operand tiles per
// K step converts 48 values per thread: with hardware conversions and the coefficient applied
// in FP64 the kernel was bound by the FP64 pipe (87% busy, tensor pipe 3%).  From the IEEE-754
// binary64 and binary32 layouts: rebias the exponent, keep the top 23 of the 52 fraction bits,
// round on the 29 dropped bits (a carry into the exponent is the correct result).  Magnitudes
// below 2^-126 (FP32 subnormals) become signed zero, overflow becomes infinity, NaN stays NaN.
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

__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc,
                                          bool tf32) {
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

// Staged layout of one K step (32 real K elements) as K-major core matrices of
// 8 rows x 16 bytes: byte offset of (row, real k) =
//   TF32 (4 B):  (row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4
//   BF16 (2 B):  (row >> 3) * 512  + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2
// The complex element kc of a row fills real k = 2 kc (real part) and 2 kc + 1.
// Thread -> (row & 7, kc) is chosen so that a warp writes whole core matrices
// (conflict-free) and reads 8 rows x 4 consecutive complex elements of global memory.
template <bool TF32>
struct Lanes {
  static __device__ __forceinline__ int r7(int tid) { return TF32 ? (tid >> 1) & 7 : (tid >> 2) & 7; }
  static __device__ __forceinline__ int kc(int tid) {
    return TF32 ? (((tid >> 4) << 1) | (tid & 1)) : (((tid >> 5) << 2) | (tid & 3));
  }
  // offset of (row = 8 g + r7, real k = 2 kc) inside an operand tile
  static __device__ __forceinline__ uint32_t off(int g, int r7, int kc) {
    return TF32 ? (uint32_t)(g * 1024 + (kc >> 1) * 128 + r7 * 16 + (kc & 1) * 8)
                : (uint32_t)(g * 512 + (kc >> 2) * 128 + r7 * 16 + (kc & 3) * 4);
  }
};

template <int P>
__global__ void __launch_bounds__(kTcThreads) tc_zgemm_kernel(const TcTile* __restrict__ tiles,
                                                              const TcSegment* __restrict__ segs,
                                                              int* __restrict__ error_flag, int stall) {
  constexpr bool kTF32 = (P == MPS_TF32);
  using Ln = Lanes<kTF32>;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar_mma[kTcStages];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TcTile T = tiles[blockIdx.x];
  const int r7 = Ln::r7(tid), kc = Ln::kc(tid);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"((uint32_t)kTcN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) mbar_init(&bar_mma[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_f32acc(kTF32 ? 2 : 1, kTcM, kTcN);
  // stall injection (tests of the bounded-wait path): no MMA and no commit is issued, so no
  // mbarrier phase completes and every wait runs out after the short bound; nothing is in
  // flight when the tensor memory is freed
  const long long wait_bound = stall ? kStallWaitCycles : kWaitCycles;

  int nsteps = 0;
  for (int sg = 0; sg < T.nseg; ++sg) nsteps += (max(segs[T.seg0 + sg].Kc, 0) + kTcKc - 1) / kTcKc;

  // registers of one step: A rows 8 g + r7 (g < 16), B columns 8 g + r7 (g < 8), element kc
  double2 ra[kTcM / 8], rb[kTcNc / 8];
  double2 ralpha = make_double2(0.0, 0.0);
  int cur_sg = 0, cur_k0 = 0;
  auto load_step = [&]() {
    while (segs[T.seg0 + cur_sg].Kc <= cur_k0) { ++cur_sg; cur_k0 = 0; }   // skips empty segments
    const TcSegment S = segs[T.seg0 + cur_sg];
    const int k = cur_k0 + kc;
    const bool kin = k < S.Kc;
#pragma unroll
    for (int g = 0; g < kTcM / 8; ++g) {
      const int row = T.row0 + 8 * g + r7;
      ra[g] = (kin && row < T.M) ? S.A[(int64_t)row * S.sar + (int64_t)k * S.sac] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int g = 0; g < kTcNc / 8; ++g) {
      const int col = T.col0 + 8 * g + r7;
      rb[g] = (kin && col < T.N) ? S.B[(int64_t)k * S.sbr + (int64_t)col * S.sbc] : make_double2(0.0, 0.0);
    }
    ralpha = S.alpha;
    cur_k0 += kTcKc;
  };
  // operands are converted to FP32 first (d2f_rn) and scaled by the segment's complex
  // coefficient in FP32: the FP32 rounding (2^-24) is far below the TF32 / BF16x3 one
  auto store_step = [&](unsigned char* stage) {
    const float alr = d2f_rn(ralpha.x), ali = d2f_rn(ralpha.y);
    if constexpr (kTF32) {
      unsigned char* a_s = stage;
      unsigned char* b_s = stage + 16 * 1024;
#pragma unroll
      for (int g = 0; g < kTcM / 8; ++g) {
        const float xr = d2f_rn(ra[g].x), xi = d2f_rn(ra[g].y);
        const float vr = fmaf(alr, xr, -ali * xi), vi = fmaf(alr, xi, ali * xr);
        *reinterpret_cast<float2*>(a_s + Ln::off(g, r7, kc)) = make_float2(to_tf32(vr), to_tf32(vi));
      }
#pragma unroll
      for (int g = 0; g < kTcNc / 8; ++g) {
        const float yr = to_tf32(d2f_rn(rb[g].x)), yi = to_tf32(d2f_rn(rb[g].y));
        *reinterpret_cast<float2*>(b_s + Ln::off(g, r7, kc)) = make_float2(yr, -yi);
        *reinterpret_cast<float2*>(b_s + Ln::off(g + kTcNc / 8, r7, kc)) = make_float2(yi, yr);
      }
    } else {
      unsigned char* ah = stage;
      unsigned char* al = stage + 8 * 1024;
      unsigned char* bh = stage + 16 * 1024;
      unsigned char* bl = stage + 24 * 1024;
      __nv_bfloat16 h0, l0, h1, l1;
#pragma unroll
      for (int g = 0; g < kTcM / 8; ++g) {
        const float xr = d2f_rn(ra[g].x), xi = d2f_rn(ra[g].y);
        split_bf16(fmaf(alr, xr, -ali * xi), h0, l0);
        split_bf16(fmaf(alr, xi, ali * xr), h1, l1);
        const uint32_t o = Ln::off(g, r7, kc);
        *reinterpret_cast<__nv_bfloat162*>(ah + o) = __halves2bfloat162(h0, h1);
        *reinterpret_cast<__nv_bfloat162*>(al + o) = __halves2bfloat162(l0, l1);
      }
#pragma unroll
      for (int g = 0; g < kTcNc / 8; ++g) {
        const float2 y = make_float2(d2f_rn(rb[g].x), d2f_rn(rb[g].y));
        const uint32_t o_re = Ln::off(g, r7, kc), o_im = Ln::off(g + kTcNc / 8, r7, kc);
        split_bf16(y.x, h0, l0);
        split_bf16(-y.y, h1, l1);
        *reinterpret_cast<__nv_bfloat162*>(bh + o_re) = __halves2bfloat162(h0, h1);   // [Br; -Bi]
        *reinterpret_cast<__nv_bfloat162*>(bl + o_re) = __halves2bfloat162(l0, l1);
        split_bf16(y.y, h0, l0);
        split_bf16(y.x, h1, l1);
        *reinterpret_cast<__nv_bfloat162*>(bh + o_im) = __halves2bfloat162(h0, h1);   // [Bi; Br]
        *reinterpret_cast<__nv_bfloat162*>(bl + o_im) = __halves2bfloat162(l0, l1);
      }
    }
  };

  bool ok = true;
  int step = 0;                   // K steps issued so far (stage = step % 2)
  if (nsteps > 0) load_step();
  for (; step < nsteps;) {
    const int st = step % kTcStages;
    if (step >= kTcStages) {      // the MMAs that last read this stage must have completed
      const bool w = mbar_wait(&bar_mma[st], (uint32_t)((step / kTcStages - 1) & 1), wait_bound);
      ok = __syncthreads_and(w);  // every thread takes the same branch
      if (!ok) break;
    }
    unsigned char* stage = smem + st * kStageBytes;
    store_step(stage);
    // make the staged tiles visible to the tensor core (async proxy), then issue
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && !stall) {
      const uint32_t s0 = smem_u32(stage);
      if constexpr (kTF32) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {             // K = 8 per MMA: two core matrices along K
          const uint64_t ad = make_desc(s0 + q * 256, 128, 1024);
          const uint64_t bd = make_desc(s0 + 16 * 1024 + q * 256, 128, 1024);
          mma_issue(tmem, ad, bd, idesc, (step > 0 || q > 0) ? 1u : 0u, true);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 2; ++q) {             // K = 16 per MMA; hi.hi + hi.lo + lo.hi
          const uint64_t ah = make_desc(s0 + q * 256, 128, 512);
          const uint64_t al = make_desc(s0 + 8 * 1024 + q * 256, 128, 512);
          const uint64_t bh = make_desc(s0 + 16 * 1024 + q * 256, 128, 512);
          const uint64_t bl = make_desc(s0 + 24 * 1024 + q * 256, 128, 512);
          mma_issue(tmem, al, bh, idesc, (step > 0 || q > 0) ? 1u : 0u, false);
          mma_issue(tmem, ah, bl, idesc, 1u, false);
          mma_issue(tmem, ah, bh, idesc, 1u, false);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(&bar_mma[st])));
    }
    ++step;
    if (step < nsteps) load_step();   // global loads of the next step overlap the MMAs
  }
  // wait for the last MMAs (also on the error path, so that none is in flight when the
  // tensor memory is freed); a commit completes after every earlier MMA of the thread
  if (step > 0) {
    const int last = (step - 1) % kTcStages;
    const bool w = mbar_wait(&bar_mma[last], (uint32_t)(((step - 1) / kTcStages) & 1), wait_bound);
    ok = __syncthreads_and(ok && w);
  }
  tc_fence_after();
  __syncthreads();
  if (ok) {
    // warp w owns TMEM lanes (rows) 32 w .. 32 w + 31; staged through shared memory
    // (free now) so that the FP64 stores of a row segment are contiguous
    double2* stg = reinterpret_cast<double2*>(smem) + warp * 32 * kEpiLd;
    const int rr = lane >> 4, cc = lane & 15;
    for (int c0 = 0; c0 < kTcNc; c0 += 16) {
      uint32_t re[16], im[16];
      if (nsteps > 0) {
        const uint32_t taddr_re = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        const uint32_t taddr_im = taddr_re + kTcNc;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]), "=r"(re[6]),
              "=r"(re[7]), "=r"(re[8]), "=r"(re[9]), "=r"(re[10]), "=r"(re[11]), "=r"(re[12]), "=r"(re[13]),
              "=r"(re[14]), "=r"(re[15])
            : "r"(taddr_re));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]), "=r"(im[6]),
              "=r"(im[7]), "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]), "=r"(im[12]), "=r"(im[13]),
              "=r"(im[14]), "=r"(im[15])
            : "r"(taddr_im));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) re[j] = im[j] = 0u;   // no K at all: the product is zero
      }
#pragma unroll
      for (int j = 0; j < 16; ++j)
        stg[lane * kEpiLd + j] = make_double2((double)__uint_as_float(re[j]), (double)__uint_as_float(im[j]));
      __syncwarp();
      const int col = T.col0 + c0 + cc;
#pragma unroll 4
      for (int r2 = 0; r2 < 16; ++r2) {
        const int rl = 2 * r2 + rr, row = T.row0 + warp * 32 + rl;
        if (row < T.M && col < T.N) T.C[(int64_t)row * T.ldc + col] = stg[rl * kEpiLd + cc];
      }
      __syncwarp();
    }
  } else if (tid == 0) {
    atomicExch(error_flag, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)kTcN));
}

std::atomic<bool> g_tc_stall{false};   // mps_tc_inject_stall

template <int P>
cudaError_t launch_tc(const TcTile* d_tiles, int n_tiles, const TcSegment* d_segs, int* d_err, cudaStream_t st) {
  static bool attr = false;
  constexpr int smem = kTcStages * (int)kStageBytes;
  static_assert(4 * 32 * kEpiLd * 16 <= smem, "epilogue staging fits in the operand stages");
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_zgemm_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  count_launch();
  tc_zgemm_kernel<P><<<n_tiles, kTcThreads, smem, st>>>(d_tiles, d_segs, d_err, g_tc_stall.load() ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_zgemm(int precision, const TcTile* d_tiles, int n_tiles, const TcSegment* d_segs, int* d_err,
                            cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  if (precision == MPS_TF32) return launch_tc<MPS_TF32>(d_tiles, n_tiles, d_segs, d_err, st);
  if (precision == MPS_BF16X3) return launch_tc<MPS_BF16X3>(d_tiles, n_tiles, d_segs, d_err, st);
  return cudaErrorInvalidValue;
}

}  // namespace mps

using namespace mps;

extern "C" int mps_tc_inject_stall(int on) {
  g_tc_stall.store(on != 0);
  return MPS_OK;
}

// Standalone entry point: C = A B on the tensor cores (see the header).
extern "C" int mps_zgemm_tc(int precision, int M, int N, int K, const double* d_A, int lda, const double* d_B,
                            int ldb, double* d_C, int ldc, void* d_work, int64_t work_bytes, void* cuda_stream) {
  if (precision != MPS_TF32 && precision != MPS_BF16X3) return MPS_EINVAL;
  if (M < 1 || N < 1 || K < 1 || lda < K || ldb < N || ldc < N || !d_A || !d_B || !d_C || !d_work) return MPS_EINVAL;
  const int tm = (M + kTcTileM - 1) / kTcTileM, tn = (N + kTcTileN - 1) / kTcTileN;
  static_assert(16 + sizeof(TcSegment) <= 256 && sizeof(TcTile) <= 64, "scratch layout");
  const int64_t need = 256 + (int64_t)sizeof(TcTile) * tm * tn;   // flag, segment, then the tiles
  if (work_bytes < need) return MPS_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  char* base = (char*)d_work;
  int* d_err = reinterpret_cast<int*>(base);
  TcSegment* d_seg = reinterpret_cast<TcSegment*>(base + 16);
  TcTile* d_tiles = reinterpret_cast<TcTile*>(base + 256);
  TcSegment seg;
  seg.A = reinterpret_cast<const double2*>(d_A);
  seg.B = reinterpret_cast<const double2*>(d_B);
  seg.Kc = K;
  seg.sar = lda; seg.sac = 1;
  seg.sbr = ldb; seg.sbc = 1;
  seg.alpha = make_double2(1.0, 0.0);
  std::vector<TcTile> tiles;
  for (int i = 0; i < tm; ++i)
    for (int j = 0; j < tn; ++j) {
      TcTile t;
      t.C = reinterpret_cast<double2*>(d_C);
      t.ldc = ldc; t.M = M; t.N = N;
      t.row0 = i * kTcTileM; t.col0 = j * kTcTileN;
      t.seg0 = 0; t.nseg = 1;
      tiles.push_back(t);
    }
  if (cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) return MPS_ECUDA;
  if (cudaMemcpyAsync(d_seg, &seg, sizeof(seg), cudaMemcpyHostToDevice, st) != cudaSuccess) return MPS_ECUDA;
  if (cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(TcTile) * tiles.size(), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return MPS_ECUDA;
  if (launch_tc_zgemm(precision, d_tiles, (int)tiles.size(), d_seg, d_err, st) != cudaSuccess) return MPS_ECUDA;
  int err = 0;
  if (cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MPS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MPS_ECUDA;
  return err ? MPS_ETIMEOUT : MPS_OK;
}
