// Sector GEMMs of the two-site update, FP64 complex on the CUDA cores.
//
// K1 (theta_kernel): for every (l, r) pair of one update,
//     Theta'(c)[l, r] += G_n[l - c, l - m] * (B^[s][l, m] . B^[s+1][m, r])
// summed over the middle charges m, for every new middle charge c of the pair
// (n = l - r).  This is the block-sparse construction of Theta of Sec. II: each
// product B[l,m] B[m,r] is formed once and mixed into all output charges c in
// the epilogue, so the GEMM work is that of the (l, m, r) triples alone.
//
// K4 (gemm_kernel, scatter_kernel, lambda_kernel): reassembly after truncation,
//     B^[s][l, c]   = Theta'(c)[rows of l] . Y(c)[:, kept] / |S_kept|
//     B^[s+1][c, r] = Y(c)[cols of r, kept]^dag
//     lambda^[s+1]  = S_kept / |S_kept|
// Sites are written in charge-sorted block order with coalesced row-major stores.
//
// GB300 note: FP64 runs at 1.2 TFLOP/s on this part (measured), so these kernels
// are FP64-pipe bound; tiles skip whole 16-row/16-column groups that fall
// outside a ragged block instead of spending FP64 issue slots on padding.
#include "mps_internal.h"

namespace mps {
namespace {

constexpr int kK = 16;             // K chunk staged in shared memory
constexpr int kThreads = 256;      // 16 x 16 threads, 4 x 4 complex outputs each

struct TileSmem {
  double2 A[kTile][kK + 1];        // +1: rows of A read by two lanes do not share banks
  double2 B[kK][kTile];
};

__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// acc += A[row0:row0+64, :] . B[:, col0:col0+64] with general strides.
// Thread (tx, ty) owns rows row0 + ty + 16 i and columns col0 + tx + 16 j.
__device__ void tile_mma(const double2* __restrict__ A, int sar, int sac,
                         const double2* __restrict__ B, int sbr, int sbc,
                         int M, int N, int K, int row0, int col0,
                         double2 (&acc)[4][4], TileSmem& sm) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int warp_ty = (tid >> 5) * 2;               // smallest ty in this warp
  int ni = 0, nj = 0;                               // warp-uniform live row / column groups
#pragma unroll
  for (int i = 0; i < 4; ++i) ni += (row0 + warp_ty + 16 * i < M);
#pragma unroll
  for (int j = 0; j < 4; ++j) nj += (col0 + 16 * j < N);
  for (int k0 = 0; k0 < K; k0 += kK) {
    const int kc = min(kK, K - k0);
    // stage A: 64 x 16 (k fastest for row-major A)
    for (int e = tid; e < kTile * kK; e += kThreads) {
      int r, k;
      if (sac == 1) { r = e / kK; k = e % kK; } else { k = e / kTile; r = e % kTile; }
      double2 v = make_double2(0.0, 0.0);
      if (row0 + r < M && k < kc) v = A[(int64_t)(row0 + r) * sar + (int64_t)(k0 + k) * sac];
      sm.A[r][k] = v;
    }
    // stage B: 16 x 64 (j fastest for row-major B, k fastest for column-major B)
    for (int e = tid; e < kTile * kK; e += kThreads) {
      int k, c;
      if (sbc == 1) { k = e / kTile; c = e % kTile; } else { c = e / kK; k = e % kK; }
      double2 v = make_double2(0.0, 0.0);
      if (col0 + c < N && k < kc) v = B[(int64_t)(k0 + k) * sbr + (int64_t)(col0 + c) * sbc];
      sm.B[k][c] = v;
    }
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sm.A[ty + 16 * i][kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sm.B[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (i < ni) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (j < nj) cfma(acc[i][j], a[i], b[j]);
        }
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) theta_kernel(const ThetaTask* __restrict__ tasks,
                                                         const TileRef* __restrict__ tiles) {
  __shared__ TileSmem sm;
  const TileRef tr = tiles[blockIdx.x];
  const ThetaTask& T = tasks[tr.task];
  const int row0 = tr.ti * kTile, col0 = tr.tj * kTile;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int Dl = T.Dl, Dr = T.Dr, nc = T.nc, sn = T.sn;
  for (int mi = 0; mi < T.nm; ++mi) {
    double2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
    tile_mma(T.A[mi], T.Dm[mi], 1, T.B[mi], Dr, 1, Dl, Dr, T.Dm[mi], row0, col0, acc, sm);
    // epilogue: mix this product into every output charge of the (l, r) pair
    for (int k = 0; k < nc; ++k) {
      const double2 g = T.gate[T.go[k] * sn + T.gi[mi]];
      double2* __restrict__ out = T.out[k];
      const int ldo = T.ldo[k];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = row0 + ty + 16 * i;
        if (r >= Dl) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = col0 + tx + 16 * j;
          if (c >= Dr) continue;
          double2 v = out[(int64_t)r * ldo + c];
          cfma(v, g, acc[i][j]);
          out[(int64_t)r * ldo + c] = v;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) gemm_kernel(const GemmTask* __restrict__ tasks,
                                                        const TileRef* __restrict__ tiles) {
  __shared__ TileSmem sm;
  const TileRef tr = tiles[blockIdx.x];
  const GemmTask& T = tasks[tr.task];
  const int row0 = tr.ti * kTile, col0 = tr.tj * kTile;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
  tile_mma(T.A, T.sar, T.sac, T.B, T.sbr, T.sbc, T.M, T.N, T.K, row0, col0, acc, sm);
  const double alpha = T.alpha;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= T.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx + 16 * j;
      if (c >= T.N) continue;
      T.C[(int64_t)r * T.ldc + c] = make_double2(alpha * acc[i][j].x, alpha * acc[i][j].y);
    }
  }
}

// One flat element per thread; tasks are sorted by their first element index.
__global__ void scatter_kernel(const ScatterTask* __restrict__ tasks, int n_tasks, int64_t n_elems) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_elems;
       e += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_tasks - 1;
    while (lo < hi) {                       // last task with first <= e
      int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].first <= e) lo = mid; else hi = mid - 1;
    }
    const ScatterTask& T = tasks[lo];
    const int64_t idx = e - T.first;
    const int j = (int)(idx / T.Dr), b = (int)(idx % T.Dr);
    const double2 y = T.Y[(int64_t)(T.coff + b) + (int64_t)j * T.n];
    T.out[idx] = make_double2(y.x, -y.y);
  }
}

__global__ void lambda_kernel(const LambdaTask* __restrict__ tasks) {
  const LambdaTask& T = tasks[blockIdx.x];
  for (int j = threadIdx.x; j < T.k; j += blockDim.x) T.lambda[j] = T.sigma[j] * T.scale;
}

}  // namespace

cudaError_t launch_theta(const ThetaTask* d_tasks, const TileRef* d_tiles, int n_tiles, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  count_launch();
  theta_kernel<<<n_tiles, kThreads, 0, st>>>(d_tasks, d_tiles);
  return cudaGetLastError();
}

cudaError_t launch_gemm(const GemmTask* d_tasks, const TileRef* d_tiles, int n_tiles, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  count_launch();
  gemm_kernel<<<n_tiles, kThreads, 0, st>>>(d_tasks, d_tiles);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const ScatterTask* d_tasks, int n_tasks, int64_t n_elems, cudaStream_t st) {
  if (n_tasks <= 0 || n_elems <= 0) return cudaSuccess;
  int64_t blocks = (n_elems + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  count_launch();
  scatter_kernel<<<(int)blocks, 256, 0, st>>>(d_tasks, n_tasks, n_elems);
  return cudaGetLastError();
}

cudaError_t launch_lambda(const LambdaTask* d_tasks, int n_tasks, cudaStream_t st) {
  if (n_tasks <= 0) return cudaSuccess;
  count_launch();
  lambda_kernel<<<n_tasks, 128, 0, st>>>(d_tasks);
  return cudaGetLastError();
}

}  // namespace mps
