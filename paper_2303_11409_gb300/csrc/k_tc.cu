// Complex GEMMs on the 5th-generation tensor cores (tcgen05), TF32 inputs with
// FP32 accumulation in tensor memory, for the reduced-precision sector GEMMs.
//
// A complex product C = A B (A: M x K, B: K x N, complex128 in global memory) is
// lowered to one real GEMM with the same multiply count:
//     [Cr | Ci] = [Ar | Ai] . [[Br, Bi], [-Bi, Br]]        (M x 2K) . (2K x 2N).
// Each CTA computes a 128 x 64 complex output tile: a 128 x 128 real FP32
// accumulator in TMEM (128 columns), fed from shared memory in the canonical
// no-swizzle K-major layout (core matrices of 8 rows x 16 bytes; LBO = next core
// matrix along K, SBO = next 8-row group).  The operand tiles are converted from
// FP64 (and optionally multiplied by a complex scalar per K segment, which is how
// the gate coefficient of the Theta build enters) while being staged, so the FP64
// master copies in HBM are read exactly once; one elected thread issues
// tcgen05.mma for each K step and commits to an mbarrier that releases the stage.
// Every wait on an mbarrier is bounded: on expiry the CTA records an error and
// still frees its tensor memory before returning.
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "mps_internal.h"

namespace mps {
namespace {

constexpr int kTcM = 128;          // rows of the output tile (TMEM lanes)
constexpr int kTcNc = 64;          // complex columns of the output tile
constexpr int kTcN = 2 * kTcNc;    // real accumulator columns
constexpr int kTcK = 32;           // real K elements staged per step (4 MMAs of K = 8)
constexpr int kTcThreads = 128;
constexpr int kTcStages = 2;
constexpr uint32_t kTileABytes = kTcM * kTcK * 4;   // 16 KB
constexpr uint32_t kTileBBytes = kTcN * kTcK * 4;   // 16 KB
constexpr long long kWaitCycles = 4000000000LL;      // bound of every mbarrier wait (~2 s)

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

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) inside a staged K-major tile with 8-row core groups
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)((row >> 3) * (kTcK / 4) * 128 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the phase with the given parity; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (clock64() - t0 < kWaitCycles) {
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

struct TcSegment {            // one K segment: C += (alpha * A_seg) . B_seg
  const double2* A;           // M x Kc complex, row stride lda
  const double2* B;           // Kc x N complex, row stride ldb
  int Kc, lda, ldb;
  double2 alpha;
};

// The work of one CTA: a 128 x 64 complex tile of one output matrix over a list of segments.
struct TcTile {
  double2* C;                 // output, row stride ldc; written (not accumulated)
  int ldc, M, N;              // full output extent (rows, complex columns)
  int row0, col0;
  int seg0, nseg;             // segments [seg0, seg0 + nseg) of the segment array
};

__global__ void __launch_bounds__(kTcThreads, 1) tc_zgemm_kernel(const TcTile* __restrict__ tiles,
                                                                  const TcSegment* __restrict__ segs,
                                                                  int* __restrict__ error_flag) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar_mma[kTcStages];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TcTile T = tiles[blockIdx.x];
  unsigned char* tileA[kTcStages] = {smem, smem + kTileABytes + kTileBBytes};
  unsigned char* tileB[kTcStages] = {smem + kTileABytes, smem + 2 * kTileABytes + kTileBBytes};

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
  constexpr uint32_t idesc = idesc_tf32(kTcM, kTcN);

  bool ok = true;
  int step = 0;                   // global K step counter (for stage and parity)
  for (int sg = 0; sg < T.nseg && ok; ++sg) {
    const TcSegment S = segs[T.seg0 + sg];
    const int K2 = 2 * S.Kc;      // real K of this segment
    for (int k0 = 0; k0 < K2; k0 += kTcK) {
      const int st = step % kTcStages;
      if (step >= kTcStages) {    // the MMAs that last read this stage must have completed
        const bool w = mbar_wait(&bar_mma[st], (uint32_t)((step / kTcStages - 1) & 1));
        ok = __syncthreads_and(w);   // every thread takes the same branch
        if (!ok) break;
      }
      // stage A: rows row0.., real K index kk in [k0, k0+32): kk < Kc -> Re, else Im (times alpha)
      unsigned char* a_s = tileA[st];
      for (int e = tid; e < kTcM * kTcK; e += kTcThreads) {
        const int r = e / kTcK, kk = e % kTcK;
        const int gk = k0 + kk, row = T.row0 + r;
        float v = 0.f;
        if (row < T.M && gk < K2) {
          const int kc = gk < S.Kc ? gk : gk - S.Kc;
          const double2 x = S.A[(int64_t)row * S.lda + kc];
          const double xr = S.alpha.x * x.x - S.alpha.y * x.y;
          const double xi = S.alpha.x * x.y + S.alpha.y * x.x;
          v = (float)(gk < S.Kc ? xr : xi);
        }
        *reinterpret_cast<float*>(a_s + core_off(r, kk)) = v;
      }
      // stage B^T (K-major): real column n of [[Br, Bi], [-Bi, Br]] for the tile's 64 complex columns
      unsigned char* b_s = tileB[st];
      for (int e = tid; e < kTcN * kTcK; e += kTcThreads) {
        const int n = e / kTcK, kk = e % kTcK;
        const int gk = k0 + kk;
        const int j = T.col0 + (n < kTcNc ? n : n - kTcNc);
        float v = 0.f;
        if (j < T.N && gk < K2) {
          const bool upper = gk < S.Kc;
          const int kc = upper ? gk : gk - S.Kc;
          const double2 y = S.B[(int64_t)kc * S.ldb + j];
          if (n < kTcNc) v = (float)(upper ? y.x : -y.y);   // real output column: [Br; -Bi]
          else v = (float)(upper ? y.y : y.x);              // imaginary output column: [Bi; Br]
        }
        *reinterpret_cast<float*>(b_s + core_off(n, kk)) = v;
      }
      // make the staged tiles visible to the tensor core (async proxy), then issue
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0) {
        const uint32_t a0 = smem_u32(a_s), b0 = smem_u32(b_s);
#pragma unroll
        for (int q = 0; q < kTcK / 8; ++q) {         // K = 8 per MMA: two core matrices along K
          const uint64_t ad = make_desc(a0 + q * 256, 128, (kTcK / 4) * 128);
          const uint64_t bd = make_desc(b0 + q * 256, 128, (kTcK / 4) * 128);
          const uint32_t acc = (step > 0 || q > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(&bar_mma[st])));
      }
      ++step;
    }
  }
  // wait for the last MMAs (also on the error path, so that none is in flight when the
  // tensor memory is freed), then read the accumulator: warp w owns TMEM lanes 32w..32w+31
  if (step > 0) {
    const int last = (step - 1) % kTcStages;
    const bool w = mbar_wait(&bar_mma[last], (uint32_t)(((step - 1) / kTcStages) & 1));
    ok = __syncthreads_and(ok && w);
  }
  tc_fence_after();
  __syncthreads();
  if (ok) {
    const int row = T.row0 + warp * 32 + lane;
    for (int c0 = 0; c0 < kTcNc; c0 += 16) {
      uint32_t re[16], im[16];
      const uint32_t taddr_re = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      const uint32_t taddr_im = taddr_re + kTcNc;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]), "=r"(re[6]), "=r"(re[7]),
            "=r"(re[8]), "=r"(re[9]), "=r"(re[10]), "=r"(re[11]), "=r"(re[12]), "=r"(re[13]), "=r"(re[14]),
            "=r"(re[15])
          : "r"(taddr_re));
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]), "=r"(im[6]), "=r"(im[7]),
            "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]), "=r"(im[12]), "=r"(im[13]), "=r"(im[14]),
            "=r"(im[15])
          : "r"(taddr_im));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (row < T.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = T.col0 + c0 + j;
          if (col < T.N)
            T.C[(int64_t)row * T.ldc + col] = make_double2((double)__uint_as_float(re[j]), (double)__uint_as_float(im[j]));
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(error_flag, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)kTcN));
}

bool g_tc_attr = false;

}  // namespace

constexpr int kTcSmem = kTcStages * (kTileABytes + kTileBBytes);

cudaError_t launch_tc_zgemm(const TcTile* d_tiles, int n_tiles, const TcSegment* d_segs, int* d_err, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  if (!g_tc_attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_zgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    g_tc_attr = true;
  }
  count_launch();
  tc_zgemm_kernel<<<n_tiles, kTcThreads, kTcSmem, st>>>(d_tiles, d_segs, d_err);
  return cudaGetLastError();
}

}  // namespace mps

using namespace mps;

// Standalone entry point: C = A B on the tensor cores (see the header).
extern "C" int mps_zgemm_tc(int precision, int M, int N, int K, const double* d_A, int lda, const double* d_B,
                            int ldb, double* d_C, int ldc, void* d_work, int64_t work_bytes, void* cuda_stream) {
  if (precision != MPS_TF32) return MPS_EINVAL;
  if (M < 1 || N < 1 || K < 1 || lda < K || ldb < N || ldc < N || !d_A || !d_B || !d_C || !d_work) return MPS_EINVAL;
  const int tm = (M + kTcM - 1) / kTcM, tn = (N + kTcNc - 1) / kTcNc;
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
  seg.Kc = K; seg.lda = lda; seg.ldb = ldb;
  seg.alpha = make_double2(1.0, 0.0);
  std::vector<TcTile> tiles;
  for (int i = 0; i < tm; ++i)
    for (int j = 0; j < tn; ++j) {
      TcTile t;
      t.C = reinterpret_cast<double2*>(d_C);
      t.ldc = ldc; t.M = M; t.N = N;
      t.row0 = i * kTcM; t.col0 = j * kTcNc;
      t.seg0 = 0; t.nseg = 1;
      tiles.push_back(t);
    }
  if (cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) return MPS_ECUDA;
  if (cudaMemcpyAsync(d_seg, &seg, sizeof(seg), cudaMemcpyHostToDevice, st) != cudaSuccess) return MPS_ECUDA;
  if (cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(TcTile) * tiles.size(), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return MPS_ECUDA;
  if (launch_tc_zgemm(d_tiles, (int)tiles.size(), d_seg, d_err, st) != cudaSuccess) return MPS_ECUDA;
  int err = 0;
  if (cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MPS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MPS_ECUDA;
  return err ? MPS_ETIMEOUT : MPS_OK;
}
