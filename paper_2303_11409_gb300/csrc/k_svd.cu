// Batched per-sector SVD of the two-site update (K2), FP64 one-sided Jacobi.
//
// arXiv:2303.11409, Sec. II: after the U(1) split a local update needs only
// block-sparse SVDs of the submatrices Theta(c), each at most chi x chi.  One CTA
// decomposes one sector M = diag(lambda) Theta'(c) (m x n).  It works on the
// columns of A = M^dag (n x m): Hestenes rotations orthogonalise the m columns of
// A; at convergence A V = [sigma_1 y_1, ..., sigma_m y_m], so the column norms are
// the singular values and the normalised columns are the right singular vectors Y
// of M = X S Y^dag that the right-canonical reassembly needs (X is never formed).
//
// Pairs follow the round-robin (circle) ordering, so each round's pairs are
// disjoint and are spread over the CTA's warps; every dot product and rotation is
// one warp with a shuffle reduction.  A sector whose working set fits in shared
// memory is staged there; larger ones work in global memory (L2 resident).
// Convergence: a whole sweep without a rotation, where a pair is rotated when
// |a_p^dag a_q| > tol |a_p| |a_q|, tol = eps * max(n, 32), and both columns are
// above the noise floor 32 eps |A|_F.  Singular values at or below that floor are
// reported as exactly 0 (their vectors are not determined by the data).  A sector that is not
// converged after the sweep limit reports -1 (MPS_ENOCONV at the API).
#include <algorithm>
#include <vector>

#include "mps_internal.h"

namespace mps {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Round-robin pairing of mp (even) slots, round r in [0, mp-1), pair k in [0, mp/2).
__device__ __forceinline__ void rr_pair(int k, int r, int mp, int& p, int& q) {
  const int ring = mp - 1;
  if (k == 0) {
    p = 0;
    q = r % ring + 1;
  } else {
    p = (k + r) % ring + 1;
    q = (ring - k + r) % ring + 1;
  }
}

__global__ void __launch_bounds__(kSvdThreads) jacobi_svd_kernel(const SvdSector* __restrict__ secs,
                                                                 int max_sweeps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_rot;
  __shared__ double s_fro2;
  const SvdSector S = secs[blockIdx.x];
  const int m = S.m, n = S.n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  double2* A;
  double* nrm;
  int* ord;
  if (S.smem) {
    A = reinterpret_cast<double2*>(smem_raw);
    nrm = reinterpret_cast<double*>(A + (int64_t)m * n);
    ord = reinterpret_cast<int*>(nrm + m);
  } else {
    A = S.work;
    nrm = S.norms;
    ord = S.order;
  }
  // A[:, j] = conj(rowscale_j * Theta'[j, :])  (column j of A is row j of M, conjugated)
  const int64_t mn = (int64_t)m * n;
  for (int64_t e = tid; e < mn; e += blockDim.x) {
    const int j = (int)(e / n);
    const double s = S.rowscale ? S.rowscale[j] : 1.0;
    const double2 v = S.theta[e];
    A[e] = make_double2(s * v.x, -s * v.y);
  }
  __syncthreads();
  for (int j = warp; j < m; j += nwarps) {
    const double2* a = A + (int64_t)j * n;
    double acc = 0.0;
    for (int i = lane; i < n; i += 32) acc = fma(a[i].x, a[i].x, fma(a[i].y, a[i].y, acc));
    acc = warp_sum(acc);
    if (lane == 0) nrm[j] = acc;
  }
  __syncthreads();
  if (warp == 0) {   // |A|_F^2 is invariant under the rotations
    double f = 0.0;
    for (int j = lane; j < m; j += 32) f += nrm[j];
    f = warp_sum(f);
    if (lane == 0) s_fro2 = f;
  }
  __syncthreads();
  const double tol = 2.220446049250313e-16 * (double)max(n, 32);
  // a column whose norm is below 32 eps |A|_F is rounding noise: rotating it against
  // another column cannot make the pair more orthogonal (two noise columns of a
  // rank-deficient sector stay parallel), so such pairs are left alone
  const double floor2 = (32.0 * 2.220446049250313e-16) * (32.0 * 2.220446049250313e-16) * s_fro2;
  const int mp = m + (m & 1);
  int sweep = 0;
  bool converged = (m < 2);
  for (; !converged && sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < mp - 1; ++r) {
      for (int k = warp; k < mp / 2; k += nwarps) {
        int p, q;
        rr_pair(k, r, mp, p, q);
        if (p >= m || q >= m) continue;
        if (p > q) { int t = p; p = q; q = t; }
        double2* ap = A + (int64_t)p * n;
        double2* aq = A + (int64_t)q * n;
        double gr = 0.0, gi = 0.0;
        for (int i = lane; i < n; i += 32) {
          const double2 x = ap[i], y = aq[i];
          gr = fma(x.x, y.x, fma(x.y, y.y, gr));      // Re conj(x) y
          gi = fma(x.x, y.y, fma(-x.y, y.x, gi));     // Im conj(x) y
        }
        gr = warp_sum(gr);
        gi = warp_sum(gi);
        const double alpha = nrm[p], beta = nrm[q];
        const double g = hypot(gr, gi);
        if (!(g > 0.0) || !(g > tol * sqrt(alpha) * sqrt(beta)) || fmin(alpha, beta) <= floor2) continue;
        // 2x2 Hermitian Gram [[alpha, gamma], [conj(gamma), beta]] -> diagonal
        const double zeta = (beta - alpha) / (2.0 * g);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double s = c * t;
        const double er = gr / g, ei = gi / g;          // gamma / |gamma|
        double np = 0.0, nq = 0.0;
        for (int i = lane; i < n; i += 32) {
          const double2 x = ap[i], y = aq[i];
          double2 xn, yn;
          // x' = c x - s conj(e) y ;  y' = s e x + c y
          xn.x = c * x.x - s * (er * y.x + ei * y.y);
          xn.y = c * x.y - s * (er * y.y - ei * y.x);
          yn.x = c * y.x + s * (er * x.x - ei * x.y);
          yn.y = c * y.y + s * (er * x.y + ei * x.x);
          ap[i] = xn;
          aq[i] = yn;
          np = fma(xn.x, xn.x, fma(xn.y, xn.y, np));
          nq = fma(yn.x, yn.x, fma(yn.y, yn.y, nq));
        }
        np = warp_sum(np);
        nq = warp_sum(nq);
        if (lane == 0) {
          nrm[p] = np;
          nrm[q] = nq;
          s_rot = 1;
        }
      }
      __syncthreads();
    }
    converged = (s_rot == 0);
    __syncthreads();
  }
  // singular values: fresh column norms, sorted descending (ties by column index)
  for (int j = warp; j < m; j += nwarps) {
    const double2* a = A + (int64_t)j * n;
    double acc = 0.0;
    for (int i = lane; i < n; i += 32) acc = fma(a[i].x, a[i].x, fma(a[i].y, a[i].y, acc));
    acc = warp_sum(acc);
    // at or below the noise floor a column is rounding noise: its singular value is 0
    if (lane == 0) nrm[j] = acc <= floor2 ? 0.0 : sqrt(acc);
  }
  __syncthreads();
  // NaN (from non-finite input) ranks last, so the ranks always form a permutation
  for (int j = tid; j < m; j += blockDim.x) {
    const double v = isnan(nrm[j]) ? -1.0 : nrm[j];
    int rank = 0;
    for (int k = 0; k < m; ++k) {
      const double w = isnan(nrm[k]) ? -1.0 : nrm[k];
      rank += (w > v) || (w == v && k < j);
    }
    ord[rank] = j;
  }
  __syncthreads();
  const int kmin = min(m, n);
  for (int r = tid; r < kmin; r += blockDim.x) S.sigma[r] = nrm[ord[r]];
  const int64_t ny = (int64_t)n * kmin;
  for (int64_t e = tid; e < ny; e += blockDim.x) {
    const int r = (int)(e / n), i = (int)(e % n);
    const int j = ord[r];
    const double sv = nrm[j];
    double2 y = make_double2(0.0, 0.0);
    if (sv > 0.0) {
      const double2 a = A[(int64_t)j * n + i];
      y = make_double2(a.x / sv, a.y / sv);
    }
    S.Y[e] = y;
  }
  if (tid == 0) *S.status = converged ? sweep : -1;
}

bool g_svd_attr_set = false;

}  // namespace

cudaError_t launch_svd(const SvdSector* d_secs, int n_secs, int smem_bytes, int max_sweeps, cudaStream_t st) {
  if (n_secs <= 0) return cudaSuccess;
  if (!g_svd_attr_set) {
    cudaError_t e = cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSvdSmemMax);
    if (e != cudaSuccess) return e;
    g_svd_attr_set = true;
  }
  count_launch();
  jacobi_svd_kernel<<<n_secs, kSvdThreads, smem_bytes, st>>>(d_secs, max_sweeps);
  return cudaGetLastError();
}

// Layout of the scratch of the standalone entry point: descriptors, then per
// sector the Jacobi matrix (when not staged), norms and order.
struct SvdScratchLayout {
  int64_t desc_bytes = 0;
  std::vector<int64_t> work_off, norm_off, ord_off;
  int64_t total = 0;
};

static int64_t align256(int64_t x) { return (x + 255) & ~int64_t(255); }

static bool svd_layout(int ns, const int* m, const int* n, SvdScratchLayout& L) {
  L.work_off.assign(ns, -1);
  L.norm_off.assign(ns, 0);
  L.ord_off.assign(ns, 0);
  int64_t off = align256((int64_t)sizeof(SvdSector) * ns);
  L.desc_bytes = off;
  for (int k = 0; k < ns; ++k) {
    if (m[k] < 1 || n[k] < 1) return false;
    if (svd_smem_need(m[k], n[k]) > kSvdSmemMax) {
      L.work_off[k] = off;
      off = align256(off + 16LL * m[k] * n[k]);
      L.norm_off[k] = off;
      off = align256(off + 8LL * m[k]);
      L.ord_off[k] = off;
      off = align256(off + 4LL * m[k]);
    }
  }
  L.total = off;
  return true;
}

}  // namespace mps

using namespace mps;

extern "C" int64_t mps_svd_work_bytes(int n_sectors, const int* m, const int* n) {
  if (n_sectors < 0 || (n_sectors > 0 && (!m || !n))) return -1;
  SvdScratchLayout L;
  if (!svd_layout(n_sectors, m, n, L)) return -1;
  return L.total;
}

extern "C" int mps_svd_sectors(int n_sectors, const int* m, const int* n,
                               const double* d_mats, const int64_t* mat_off,
                               const double* d_rowscale, const int64_t* row_off,
                               double* d_sigma, const int64_t* sig_off,
                               double* d_y, const int64_t* y_off,
                               int* d_status, void* d_work, int64_t work_bytes, void* cuda_stream) {
  if (n_sectors == 0) return MPS_OK;
  if (n_sectors < 0 || !m || !n || !d_mats || !mat_off || !d_sigma || !sig_off || !d_y || !y_off ||
      !d_status || !d_work)
    return MPS_EINVAL;
  if (d_rowscale && !row_off) return MPS_EINVAL;
  SvdScratchLayout L;
  if (!svd_layout(n_sectors, m, n, L) || work_bytes < L.total) return MPS_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::vector<SvdSector> secs(n_sectors);
  char* base = (char*)d_work;
  int smem = 0;
  for (int k = 0; k < n_sectors; ++k) {
    SvdSector& S = secs[k];
    S.theta = reinterpret_cast<const double2*>(d_mats) + mat_off[k];
    S.rowscale = d_rowscale ? d_rowscale + row_off[k] : nullptr;
    S.m = m[k];
    S.n = n[k];
    S.smem = L.work_off[k] < 0;
    S.work = S.smem ? nullptr : reinterpret_cast<double2*>(base + L.work_off[k]);
    S.norms = S.smem ? nullptr : reinterpret_cast<double*>(base + L.norm_off[k]);
    S.order = S.smem ? nullptr : reinterpret_cast<int*>(base + L.ord_off[k]);
    S.sigma = d_sigma + sig_off[k];
    S.Y = reinterpret_cast<double2*>(d_y) + y_off[k];
    S.status = d_status + k;
    if (S.smem) smem = std::max<int>(smem, (int)svd_smem_need(m[k], n[k]));
  }
  if (cudaMemcpyAsync(d_work, secs.data(), sizeof(SvdSector) * n_sectors, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return MPS_ECUDA;
  if (launch_svd(reinterpret_cast<const SvdSector*>(d_work), n_sectors, smem, kJacobiMaxSweeps, st) !=
      cudaSuccess)
    return MPS_ECUDA;
  // the descriptors live in pageable host memory: finish the copy before returning
  if (cudaStreamSynchronize(st) != cudaSuccess) return MPS_ECUDA;
  return MPS_OK;
}
