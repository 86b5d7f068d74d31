// Standalone entry points of the tensor-core complex GEMM (the kernels are in k_tma.cu):
// C = A B for one pair of FP64 complex matrices, through the same shadow tiles, TMA loads
// and tcgen05 MMAs as the sector GEMMs of the TF32 / BF16x3 update modes.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <vector>

#include "mps_internal.h"

namespace mps {
extern std::atomic<bool> g_tc_stall;
namespace {

inline int64_t up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline int cdv(int a, int b) { return (a + b - 1) / b; }

struct ZgemmLayout {
  int64_t tasks, tiles, jobs, slots, n_tiles, n_jobs, n_slots, total;
};

// flag | two shadow tasks | shadow tiles | jobs | slots (1 KB slack for their alignment)
ZgemmLayout zgemm_layout(int precision, int M, int N, int K) {
  const int KC = sh_kc(precision), TPK = sh_tiles_per_k(precision), kt = cdv(K, KC);
  ZgemmLayout L;
  L.n_tiles = (int64_t)cdv(M, kShRows) * kt + (int64_t)cdv(N, kShTileN) * kt;
  L.n_jobs = (int64_t)cdv(M, kShRows) * cdv(N, kShTileN);
  L.n_slots = L.n_tiles * TPK;
  L.tasks = 256;
  L.tiles = L.tasks + 256;
  L.jobs = up(L.tiles + (int64_t)sizeof(ShadowTile) * L.n_tiles, 256);
  L.slots = up(L.jobs + (int64_t)sizeof(TmaJob) * L.n_jobs, 256);
  L.total = L.slots + L.n_slots * kShTileBytes + 1024;
  return L;
}

}  // namespace
}  // namespace mps

using namespace mps;

extern "C" int mps_tc_inject_stall(int on) {
  g_tc_stall.store(on != 0);
  return MPS_OK;
}

extern "C" int64_t mps_zgemm_tc_work_bytes(int precision, int M, int N, int K) {
  if ((precision != MPS_TF32 && precision != MPS_BF16X3) || M < 1 || N < 1 || K < 1) return -1;
  return zgemm_layout(precision, M, N, K).total;
}

extern "C" int mps_zgemm_tc(int precision, int M, int N, int K, const double* d_A, int lda, const double* d_B,
                            int ldb, double* d_C, int ldc, void* d_work, int64_t work_bytes, void* cuda_stream) {
  if (precision != MPS_TF32 && precision != MPS_BF16X3) return MPS_EINVAL;
  if (M < 1 || N < 1 || K < 1 || lda < K || ldb < N || ldc < N || !d_A || !d_B || !d_C || !d_work) return MPS_EINVAL;
  const ZgemmLayout L = zgemm_layout(precision, M, N, K);
  if (work_bytes < L.total) return MPS_EINVAL;
  const int KC = sh_kc(precision), TPK = sh_tiles_per_k(precision), ktn = cdv(K, KC);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  char* base = (char*)d_work;
  int* d_err = reinterpret_cast<int*>(base);
  char* slots = reinterpret_cast<char*>(((uintptr_t)(base + L.slots) + 1023) & ~(uintptr_t)1023);
  // A: rows of A over K; B: columns of B over K (element (k, j) at B[k * ldb + j])
  const int64_t b0 = (int64_t)cdv(M, kShRows) * ktn * TPK;
  ShadowTask tasks[2] = {
      {reinterpret_cast<const double2*>(d_A), lda, 1, M, K, 0, ktn, 0},
      {reinterpret_cast<const double2*>(d_B), 1, ldb, N, K, b0, ktn, 1},
  };
  std::vector<ShadowTile> tiles;
  for (int it = 0; it < cdv(M, kShRows); ++it)
    for (int kt = 0; kt < ktn; ++kt) tiles.push_back(ShadowTile{0, it, kt});
  for (int it = 0; it < cdv(N, kShTileN); ++it)
    for (int kt = 0; kt < ktn; ++kt) tiles.push_back(ShadowTile{1, it, kt});
  std::vector<TmaJob> jobs;
  for (int rt = 0; rt < cdv(M, kShRows); ++rt)
    for (int ct = 0; ct < cdv(N, kShTileN); ++ct) {
      TmaJob J;
      J.a0 = (int64_t)rt * ktn * TPK;
      J.b0 = b0 + (int64_t)ct * ktn * TPK;
      J.kt_n = ktn;
      J.M = std::min(kShRows, M - rt * kShRows);
      J.N = std::min(kShTileN, N - ct * kShTileN);
      J.mode = 1;
      J.alpha = 1.0f;
      J.C = reinterpret_cast<double2*>(d_C) + (int64_t)rt * kShRows * ldc + (int64_t)ct * kShTileN;
      J.ldc = ldc;
      jobs.push_back(J);
    }
  if (cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) return MPS_ECUDA;
  if (cudaMemsetAsync(slots, 0, (size_t)(L.n_slots * kShTileBytes), st) != cudaSuccess) return MPS_ECUDA;
  if (cudaMemcpyAsync(base + L.tasks, tasks, sizeof(tasks), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(base + L.tiles, tiles.data(), sizeof(ShadowTile) * tiles.size(), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(base + L.jobs, jobs.data(), sizeof(TmaJob) * jobs.size(), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return MPS_ECUDA;
  if (launch_shadow(precision, reinterpret_cast<const ShadowTask*>(base + L.tasks),
                    reinterpret_cast<const ShadowTile*>(base + L.tiles), (int)tiles.size(), slots, st) != cudaSuccess)
    return MPS_ECUDA;
  if (launch_tma_zgemm(precision, reinterpret_cast<const TmaJob*>(base + L.jobs), (int)jobs.size(), slots, L.n_slots,
                       d_err, st) != cudaSuccess)
    return MPS_ECUDA;
  int err = 0;
  if (cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MPS_ECUDA;
  // the descriptors came from pageable host memory: finish before returning
  if (cudaStreamSynchronize(st) != cudaSuccess) return MPS_ECUDA;
  return err ? MPS_ETIMEOUT : MPS_OK;
}
