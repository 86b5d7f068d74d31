// Two-site DMRG and two-site TDVP on the U(1) block-sparse MPS (the variational methods
// Sec. I of arXiv:2303.11409 names beside TEBD; the block structure is that of Sec. II).
//
// The two-site wave function of sites (s, s+1) is the set of matrices Psi(c) over the
// middle charge c, in the layout of the TEBD update's Theta(c): rows are the left-bond
// sectors l = c .. c+d-1 (physical index i = l - c), columns the right-bond sectors
// r = c-d+1 .. c (j = c - r).  One local step
//   Psi = B^[s] B^[s+1]  ->  Lanczos on H_eff (DMRG: the ground state; TDVP: exp(-i tau H_eff))
//   -> per-sector SVD  ->  global top-chi  ->  new sites (left- or right-canonical)
//   -> environment of the new bond  (TDVP: the centre site evolved back by its one-site H_eff)
// runs in these kernels, with one host round trip per Lanczos restart and one for the
// kept counts:
//   sumprod_kernel   every block contraction (H_eff Psi, environment updates, the centre
//                    tensor, the new sites): an output tile accumulates a list of terms
//                    coef * op(A) op(B) (or coef * op(A)) in FP64, written once;
//   dots_kernel / dots_reduce_kernel / subtract_kernel / scale_kernel / combine_kernel
//                    the Krylov vector work (classical Gram-Schmidt applied twice, so the
//                    basis stays orthonormal to rounding), deterministic two-pass sums;
//   tridiag_kernel   the lowest Ritz pair of the Lanczos tridiagonal (Sturm bisection,
//                    then inverse iteration with a shift just below it);
//   expm_tridiag_kernel / combine_c_kernel   TDVP's Krylov exponential exp(-i tau T) e_1
//                    (the tridiagonal's eigenpairs by cyclic Jacobi rotations in one warp)
//                    and the complex Ritz combination;
//   the SVD, selection and lambda kernels of the TEBD update (k_svd.cu, k_select.cu).
// H = sum_k h_{k,k+1}: each bond term (given by its charge blocks in the gate layout) is
// split on the host into operator pairs sum_t O_t (x) P_t with O_t raising the left site's
// occupation by delta_t (a pivoted Gram-Schmidt of the matrix elements grouped by delta).
// Left environments at bond b hold <a|H_left|a'> (per sector, D_l x D_l) and <a|O_t|a'>
// of the last left site (D_l x D_{l+delta}); right environments hold <b|H_right|b'> and
// <b|P_t|b'> of the first right site stored transposed ([b', b]).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include "mps_internal.h"

using namespace mps;

namespace {

using cplx = std::complex<double>;

// ---------------------------------------------------------------------------
// Generic block sum-of-products kernel
// ---------------------------------------------------------------------------
constexpr int kT = 64, kKc = 16, kThr = 256;
enum : int { kAX = 1, kBX = 2, kConjA = 4, kConjB = 8, kNoB = 16 };
enum : int { kCY = 1, kAccum = 2 };

struct SPTerm {
  int64_t a, b;       // absolute addresses, or element offsets from the X vector (kAX / kBX)
  int sar, sac, sbr, sbc;
  int K;
  int flags;
  double2 coef;
};
struct SPTask {
  int64_t c;          // absolute address, or element offset from the Y vector (kCY)
  int ldc, M, N;
  int t0, t1;
  int flags;
  int pad;
};
struct SPTile { int task, ti, tj; };

struct SPSmem {
  double2 A[kT][kKc + 1];
  double2 B[kKc][kT];
};

__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// A block of at most 1024 outputs (one tile): its outputs are dealt to the threads in order,
// up to four per thread, so that every warp's lanes hold real outputs (the 16 x 16 thread grid
// of the general path would spend most FP64 issue slots of a block of 17-30 rows and columns
// on padding; this part issues 2 FP64 FMA per clock per SM, so only dense warps pay).
__device__ __forceinline__ void small_block(const SPTask& T, const SPTerm* __restrict__ terms,
                                            const double2* __restrict__ X, double2* __restrict__ Y, SPSmem& sm) {
  const int tid = threadIdx.x;
  const int MN = T.M * T.N, nq = (MN + kThr - 1) / kThr;
  int rr[4], cc[4];
  bool ok[4];
  double2 acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int o = tid + kThr * q;
    ok[q] = o < MN;
    rr[q] = ok[q] ? o / T.N : 0;
    cc[q] = ok[q] ? o % T.N : 0;
    acc[q] = make_double2(0.0, 0.0);
  }
  for (int t = T.t0; t < T.t1; ++t) {
    const SPTerm P = terms[t];
    const double2* A = (P.flags & kAX) ? X + P.a : reinterpret_cast<const double2*>(P.a);
    const bool ca = (P.flags & kConjA) != 0;
    if (P.flags & kNoB) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (q < nq && ok[q]) {
          double2 v = A[(int64_t)rr[q] * P.sar + (int64_t)cc[q] * P.sac];
          if (ca) v.y = -v.y;
          cfma(acc[q], P.coef, v);
        }
      }
      continue;
    }
    const double2* B = (P.flags & kBX) ? X + P.b : reinterpret_cast<const double2*>(P.b);
    const bool cb = (P.flags & kConjB) != 0;
    for (int k0 = 0; k0 < P.K; k0 += kKc) {
      const int kc = min(kKc, P.K - k0);
      for (int e = tid; e < T.M * kc; e += kThr) {
        int r, k;
        if (P.sac == 1) { r = e / kc; k = e % kc; } else { k = e / T.M; r = e % T.M; }
        double2 v = A[(int64_t)r * P.sar + (int64_t)(k0 + k) * P.sac];
        if (ca) v.y = -v.y;
        sm.A[r][k] = cmul(P.coef, v);
      }
      for (int e = tid; e < T.N * kc; e += kThr) {
        int k, c;
        if (P.sbc == 1) { k = e / T.N; c = e % T.N; } else { c = e / kc; k = e % kc; }
        double2 v = B[(int64_t)(k0 + k) * P.sbr + (int64_t)c * P.sbc];
        if (cb) v.y = -v.y;
        sm.B[k][c] = v;
      }
      __syncthreads();
      for (int kk = 0; kk < kc; ++kk) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nq) cfma(acc[q], sm.A[rr[q]][kk], sm.B[kk][cc[q]]);
      }
      __syncthreads();
    }
  }
  double2* C = (T.flags & kCY) ? Y + T.c : reinterpret_cast<double2*>(T.c);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < nq && ok[q]) {
      double2& o = C[(int64_t)rr[q] * T.ldc + cc[q]];
      if (T.flags & kAccum) {
        double2 v = o;
        v.x += acc[q].x;
        v.y += acc[q].y;
        o = v;
      } else {
        o = acc[q];
      }
    }
  }
}

__global__ void __launch_bounds__(kThr, 2) sumprod_kernel(const SPTask* __restrict__ tasks,
                                                       const SPTerm* __restrict__ terms,
                                                       const SPTile* __restrict__ tiles,
                                                       const double2* __restrict__ X, double2* __restrict__ Y) {
  __shared__ SPSmem sm;
  const SPTile tr = tiles[blockIdx.x];
  const SPTask T = tasks[tr.task];
  if (T.M <= kT && T.N <= kT && T.M * T.N <= 4 * kThr) {
    small_block(T, terms, X, Y, sm);
    return;
  }
  const int row0 = tr.ti * kT, col0 = tr.tj * kT;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int q = T.t0; q < T.t1; ++q) {
    const SPTerm P = terms[q];
    const double2* A = (P.flags & kAX) ? X + P.a : reinterpret_cast<const double2*>(P.a);
    const bool ca = (P.flags & kConjA) != 0;
    if (P.flags & kNoB) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = row0 + ty + 16 * i;
        if (r >= T.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = col0 + tx + 16 * j;
          if (c >= T.N) continue;
          double2 v = A[(int64_t)r * P.sar + (int64_t)c * P.sac];
          if (ca) v.y = -v.y;
          cfma(acc[i][j], P.coef, v);
        }
      }
      continue;
    }
    const double2* B = (P.flags & kBX) ? X + P.b : reinterpret_cast<const double2*>(P.b);
    const bool cb = (P.flags & kConjB) != 0;
    // warp-uniform counts of the 16-row / 16-column groups that hold valid outputs: a
    // block smaller than the tile spends no FP64 issue slots on its padding
    const int warp_ty = (tid >> 5) * 2;
    int ni = 0, nj = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) ni += (row0 + warp_ty + 16 * i < T.M);
#pragma unroll
    for (int j = 0; j < 4; ++j) nj += (col0 + 16 * j < T.N);
    // only the block's own rows / columns are staged and read: the accumulators of padding rows
    // and columns see stale shared memory and are never stored
    const int mr = min(kT, T.M - row0), ncl = min(kT, T.N - col0);
    for (int k0 = 0; k0 < P.K; k0 += kKc) {
      const int kc = min(kKc, P.K - k0);
      for (int e = tid; e < mr * kc; e += kThr) {
        int r, k;
        if (P.sac == 1) { r = e / kc; k = e % kc; } else { k = e / mr; r = e % mr; }
        double2 v = A[(int64_t)(row0 + r) * P.sar + (int64_t)(k0 + k) * P.sac];
        if (ca) v.y = -v.y;
        sm.A[r][k] = cmul(P.coef, v);
      }
      for (int e = tid; e < ncl * kc; e += kThr) {
        int k, c;
        if (P.sbc == 1) { k = e / ncl; c = e % ncl; } else { c = e / kc; k = e % kc; }
        double2 v = B[(int64_t)(k0 + k) * P.sbr + (int64_t)(col0 + c) * P.sbc];
        if (cb) v.y = -v.y;
        sm.B[k][c] = v;
      }
      __syncthreads();
      for (int kk = 0; kk < kc; ++kk) {
        double2 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i < ni) a[i] = sm.A[ty + 16 * i][kk];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (j < nj) b[j] = sm.B[kk][tx + 16 * j];
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
  double2* C = (T.flags & kCY) ? Y + T.c : reinterpret_cast<double2*>(T.c);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= T.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx + 16 * j;
      if (c >= T.N) continue;
      double2& o = C[(int64_t)r * T.ldc + c];
      if (T.flags & kAccum) {
        double2 v = o;
        v.x += acc[i][j].x;
        v.y += acc[i][j].y;
        o = v;
      } else {
        o = acc[i][j];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Krylov vector kernels (deterministic: fixed grid, two-pass sums)
// ---------------------------------------------------------------------------
constexpr int kVecThreads = 256;
constexpr int kDotBlocks = 304;   // 2 x 152 SMs

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// partial[k * gridDim.x + blockIdx.x] = sum over this block's elements of conj(V_k[e]) w[e], k = blockIdx.y
__global__ void __launch_bounds__(kVecThreads) dots_kernel(const double2* __restrict__ V, int64_t ldv,
                                                           const double2* __restrict__ w, int64_t n,
                                                           double2* __restrict__ partial) {
  __shared__ double2 red[kVecThreads / 32];
  const int k = blockIdx.y;
  const double2* v = V + (int64_t)k * ldv;
  double2 s = make_double2(0.0, 0.0);
  for (int64_t e = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kVecThreads) {
    const double2 a = v[e], b = w[e];
    s.x = fma(a.x, b.x, fma(a.y, b.y, s.x));
    s.y = fma(a.x, b.y, fma(-a.y, b.x, s.y));
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double2 t = threadIdx.x < kVecThreads / 32 ? red[threadIdx.x] : make_double2(0.0, 0.0);
    t = warp_sum(t);
    if (threadIdx.x == 0) partial[(int64_t)k * gridDim.x + blockIdx.x] = t;
  }
}

// out[k] = sum_x partial[k * nb + x]; one block per k
__global__ void __launch_bounds__(kVecThreads) dots_reduce_kernel(const double2* __restrict__ partial, int nb,
                                                                  double2* __restrict__ out) {
  __shared__ double2 red[kVecThreads / 32];
  const int k = blockIdx.x;
  double2 s = make_double2(0.0, 0.0);
  for (int x = threadIdx.x; x < nb; x += kVecThreads) {
    const double2 p = partial[(int64_t)k * nb + x];
    s.x += p.x;
    s.y += p.y;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double2 t = threadIdx.x < kVecThreads / 32 ? red[threadIdx.x] : make_double2(0.0, 0.0);
    t = warp_sum(t);
    if (threadIdx.x == 0) out[k] = t;
  }
}

// w[e] -= sum_k coef[k] V_k[e]
__global__ void __launch_bounds__(kVecThreads) subtract_kernel(double2* __restrict__ w, const double2* __restrict__ V,
                                                               int64_t ldv, int nk, const double2* __restrict__ coef,
                                                               int64_t n) {
  __shared__ double2 cs[64];
  for (int k = threadIdx.x; k < nk; k += kVecThreads) cs[k] = coef[k];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kVecThreads) {
    double2 acc = w[e];
    for (int k = 0; k < nk; ++k) {
      const double2 v = V[(int64_t)k * ldv + e], c = cs[k];
      acc.x -= c.x * v.x - c.y * v.y;
      acc.y -= c.x * v.y + c.y * v.x;
    }
    w[e] = acc;
  }
}

// Lanczos scalars of iteration j: alpha_j = Re(h_j + g_j) (the two Gram-Schmidt passes),
// beta_j = |w|, and the factor that normalises w into the next basis vector.
__global__ void lanczos_scalars_kernel(int j, const double2* __restrict__ h, const double2* __restrict__ g,
                                       const double2* __restrict__ nrm2, double* __restrict__ alpha,
                                       double* __restrict__ beta, double* __restrict__ inv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  alpha[j] = h[j].x + g[j].x;
  const double b = sqrt(fmax(nrm2[0].x, 0.0));
  beta[j] = b;
  inv[0] = b > 1e-300 ? 1.0 / b : 0.0;
}

__global__ void inv_norm_kernel(const double2* __restrict__ nrm2, double* __restrict__ inv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double b = sqrt(fmax(nrm2[0].x, 0.0));
  inv[0] = b > 1e-300 ? 1.0 / b : 0.0;
}

__global__ void __launch_bounds__(kVecThreads) scale_kernel(double2* __restrict__ dst, const double2* __restrict__ src,
                                                            const double* __restrict__ f, int64_t n) {
  const double a = f[0];
  for (int64_t e = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kVecThreads) {
    const double2 v = src[e];
    dst[e] = make_double2(a * v.x, a * v.y);
  }
}

// out[e] = sum_k y[k] V_k[e] (y real)
__global__ void __launch_bounds__(kVecThreads) combine_kernel(double2* __restrict__ out, const double2* __restrict__ V,
                                                              int64_t ldv, int nk, const double* __restrict__ y,
                                                              int64_t n) {
  __shared__ double ys[64];
  for (int k = threadIdx.x; k < nk; k += kVecThreads) ys[k] = y[k];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kVecThreads) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < nk; ++k) {
      const double2 v = V[(int64_t)k * ldv + e];
      acc.x = fma(ys[k], v.x, acc.x);
      acc.y = fma(ys[k], v.y, acc.y);
    }
    out[e] = acc;
  }
}

// Lowest eigenpair of the symmetric tridiagonal T (alpha_0..n-1 on the diagonal, beta_0..n-2
// off it).  The basis ends at the first beta_j below 1e-13 of the matrix scale (an invariant
// subspace: later vectors carry only rounding).  The eigenvalue is bracketed by Sturm-sequence
// bisection; the eigenvector comes from inverse iteration with the shift just below it, where
// T - shift is positive definite and its LDL^T factorisation is stable.
// res[0] = eigenvalue, res[1] = residual estimate beta_{n-1} |y_{n-1}|, res[2] = basis size used.
__global__ void tridiag_kernel(const double* __restrict__ alpha, const double* __restrict__ beta, int n,
                               double* __restrict__ y, double* __restrict__ res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double scale = 0.0;
  for (int k = 0; k < n; ++k) scale = fmax(scale, fabs(alpha[k]) + (k + 1 < n ? fabs(beta[k]) : 0.0));
  scale = fmax(scale, 1e-300);
  int m = n;
  for (int k = 0; k + 1 < n; ++k)
    if (beta[k] <= 1e-13 * scale) { m = k + 1; break; }
  double lo = 1e300, hi = -1e300;
  for (int k = 0; k < m; ++k) {
    const double r = (k > 0 ? fabs(beta[k - 1]) : 0.0) + (k + 1 < m ? fabs(beta[k]) : 0.0);
    lo = fmin(lo, alpha[k] - r);
    hi = fmax(hi, alpha[k] + r);
  }
  for (int it = 0; it < 400 && hi - lo > 2e-16 * fmax(fabs(lo), fabs(hi)) + 1e-300; ++it) {
    const double x = 0.5 * (lo + hi);
    int below = 0;
    double q = 1.0;
    for (int k = 0; k < m; ++k) {
      const double b2 = k > 0 ? beta[k - 1] * beta[k - 1] : 0.0;
      q = alpha[k] - x - (k > 0 ? b2 / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) ++below;
    }
    if (below >= 1) hi = x; else lo = x;
  }
  const double lam = 0.5 * (lo + hi);
  const double shift = lam - 1e-13 * scale;
  double dd[64], ll[64], x[64];
  dd[0] = alpha[0] - shift;
  for (int k = 1; k < m; ++k) {
    dd[k - 1] = fmax(dd[k - 1], 1e-300);
    ll[k] = beta[k - 1] / dd[k - 1];
    dd[k] = alpha[k] - shift - ll[k] * beta[k - 1];
  }
  dd[m - 1] = fmax(dd[m - 1], 1e-300);
  for (int k = 0; k < m; ++k) x[k] = 1.0;
  for (int it = 0; it < 4; ++it) {
    for (int k = 1; k < m; ++k) x[k] -= ll[k] * x[k - 1];
    for (int k = 0; k < m; ++k) x[k] /= dd[k];
    for (int k = m - 2; k >= 0; --k) x[k] -= ll[k + 1] * x[k + 1];
    double s = 0.0;
    for (int k = 0; k < m; ++k) s += x[k] * x[k];
    s = 1.0 / sqrt(s);
    for (int k = 0; k < m; ++k) x[k] *= s;
  }
  if (x[0] < 0.0)
    for (int k = 0; k < m; ++k) x[k] = -x[k];
  for (int k = 0; k < n; ++k) y[k] = k < m ? x[k] : 0.0;
  res[0] = lam;
  res[1] = m < n ? 0.0 : fabs(beta[m - 1] * x[m - 1]);
  res[2] = (double)m;
}

// exp(-i tau T) e_1 for the Lanczos tridiagonal T (alpha on the diagonal, beta next to it),
// one warp: T's eigenpairs by cyclic Jacobi rotations (the symmetric Schur decomposition, each
// rotation zeroing one off-diagonal pair, sweeps until the off-diagonal part is below 1e-15 of
// the matrix), then y_j = sum_k Z[j][k] exp(-i tau lambda_k) Z[0][k].  The basis ends at the
// first beta below 1e-13 of the matrix scale, as for the ground state.  res[0] = alpha_0
// (<v0|H|v0>), res[1] = |beta_{m-1} y_{m-1}| (the estimate of the Krylov error), res[2] = m.
constexpr int kExpMax = 40;
__global__ void expm_tridiag_kernel(const double* __restrict__ alpha, const double* __restrict__ beta, int n,
                                    double tau, double2* __restrict__ y, double* __restrict__ res) {
  __shared__ double A[kExpMax][kExpMax + 1];
  __shared__ double Z[kExpMax][kExpMax + 1];
  const int lane = threadIdx.x;
  if (blockIdx.x != 0 || lane >= 32) return;
  double scale = 0.0;
  for (int k = 0; k < n; ++k) scale = fmax(scale, fabs(alpha[k]) + (k + 1 < n ? fabs(beta[k]) : 0.0));
  scale = fmax(scale, 1e-300);
  int m = n;
  for (int k = 0; k + 1 < n; ++k)
    if (beta[k] <= 1e-13 * scale) { m = k + 1; break; }
  for (int k = lane; k < m; k += 32)
    for (int j = 0; j < m; ++j) {
      A[k][j] = (j == k) ? alpha[k] : (j == k + 1 ? beta[k] : (j + 1 == k ? beta[j] : 0.0));
      Z[k][j] = (j == k) ? 1.0 : 0.0;
    }
  __syncwarp();
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, fro = 0.0;
    for (int k = 0; k < m; ++k)
      for (int j = 0; j < m; ++j) {
        const double v = A[k][j] * A[k][j];
        fro += v;
        if (j != k) off += v;
      }
    if (off <= 1e-30 * fro) break;
    for (int p = 0; p + 1 < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[p][q];
        if (fabs(apq) < 1e-300) continue;
        const double t0 = (A[q][q] - A[p][p]) / (2.0 * apq);
        const double t = t0 >= 0.0 ? 1.0 / (t0 + sqrt(1.0 + t0 * t0)) : -1.0 / (-t0 + sqrt(1.0 + t0 * t0));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
        __syncwarp();
        for (int k = lane; k < m; k += 32) {      // A <- A J
          const double ap = A[k][p], aq = A[k][q];
          A[k][p] = c * ap - sn * aq;
          A[k][q] = sn * ap + c * aq;
        }
        __syncwarp();
        for (int k = lane; k < m; k += 32) {      // A <- J^T A, Z <- Z J
          const double ap = A[p][k], aq = A[q][k];
          A[p][k] = c * ap - sn * aq;
          A[q][k] = sn * ap + c * aq;
          const double zp = Z[k][p], zq = Z[k][q];
          Z[k][p] = c * zp - sn * zq;
          Z[k][q] = sn * zp + c * zq;
        }
        __syncwarp();
      }
  }
  for (int j = lane; j < n; j += 32) {
    double2 acc = make_double2(0.0, 0.0);
    if (j < m)
      for (int k = 0; k < m; ++k) {
        double sv, cv;
        sincos(-tau * A[k][k], &sv, &cv);
        const double w = Z[j][k] * Z[0][k];
        acc.x = fma(w, cv, acc.x);
        acc.y = fma(w, sv, acc.y);
      }
    y[j] = acc;
  }
  __syncwarp();
  if (lane == 0) {
    res[0] = alpha[0];
    const double2 yl = y[m - 1];
    res[1] = m < n ? 0.0 : fabs(beta[m - 1]) * sqrt(yl.x * yl.x + yl.y * yl.y);
    res[2] = (double)m;
  }
}

// out[e] = f[0] * sum_k y[k] V_k[e] (y complex)
__global__ void __launch_bounds__(kVecThreads) combine_c_kernel(double2* __restrict__ out, const double2* __restrict__ V,
                                                                int64_t ldv, int nk, const double2* __restrict__ y,
                                                                const double* __restrict__ f, int64_t n) {
  __shared__ double2 ys[kExpMax];
  for (int k = threadIdx.x; k < nk; k += kVecThreads) ys[k] = y[k];
  __syncthreads();
  const double a = f[0];
  for (int64_t e = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kVecThreads) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < nk; ++k) {
      const double2 v = V[(int64_t)k * ldv + e], c = ys[k];
      acc.x = fma(c.x, v.x, fma(-c.y, v.y, acc.x));
      acc.y = fma(c.x, v.y, fma(c.y, v.x, acc.y));
    }
    out[e] = make_double2(a * acc.x, a * acc.y);
  }
}

// out[0] = |x| from out-of-place dot <x, x>
__global__ void fill_kernel(double* __restrict__ p, double v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) p[0] = v;
}

__global__ void norm_kernel(const double2* __restrict__ nrm2, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = sqrt(fmax(nrm2[0].x, 0.0));
}

int vec_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(kDotBlocks * 2, (n + kVecThreads - 1) / kVecThreads)); }

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct OpPair {        // one term O (x) P of a bond term, d x d row-major each
  int delta;
  std::vector<cplx> O, P;
};

// h = sum_t O_t (x) P_t by a pivoted Gram-Schmidt of h's matrix elements grouped by delta:
// for fixed delta the elements <i' j'|h|i j> with i' - i = delta form a matrix X over the
// pairs (i', i) x (j', j); repeatedly the residual row of largest norm is normalised into
// q_t and every row's component along it is moved into the coefficient column c_t, so
// X = sum_t c_t q_t^T.  O_t holds c_t on (i', i) and P_t holds q_t on (j', j).
std::vector<OpPair> split_bond(const double* hb, const ChargeRule& rule) {
  const int d = rule.d;
  auto elem = [&](int i2, int j2, int i, int j) -> cplx {
    const int n = i + j;
    if (i2 + j2 != n || n > 2 * (d - 1)) return 0.0;
    const int base = rule.base(n), sn = rule.sn(n);
    const int a = i2 - base, b = i - base;
    if (a < 0 || a >= sn || b < 0 || b >= sn) return 0.0;
    const double* p = hb + 2 * (rule.block_off(n) + (int64_t)a * sn + b);
    return cplx(p[0], p[1]);
  };
  double hmax = 0.0;
  for (int i2 = 0; i2 < d; ++i2)
    for (int j2 = 0; j2 < d; ++j2)
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) hmax = std::max(hmax, std::abs(elem(i2, j2, i, j)));
  std::vector<OpPair> out;
  for (int delta = -(d - 1); delta <= d - 1; ++delta) {
    std::vector<std::pair<int, int>> rows, cols;
    for (int i = 0; i < d; ++i)
      if (i + delta >= 0 && i + delta < d) rows.push_back({i + delta, i});
    for (int j = 0; j < d; ++j)
      if (j - delta >= 0 && j - delta < d) cols.push_back({j - delta, j});
    const int nr = (int)rows.size(), nc = (int)cols.size();
    std::vector<cplx> R(nr * nc);
    for (int a = 0; a < nr; ++a)
      for (int b = 0; b < nc; ++b) R[a * nc + b] = elem(rows[a].first, cols[b].first, rows[a].second, cols[b].second);
    for (int t = 0; t < nr; ++t) {
      int best = -1;
      double bn = 0.0;
      for (int a = 0; a < nr; ++a) {
        double s = 0.0;
        for (int b = 0; b < nc; ++b) s += std::norm(R[a * nc + b]);
        if (s > bn) { bn = s; best = a; }
      }
      if (best < 0 || std::sqrt(bn) <= 1e-14 * std::max(hmax, 1e-300)) break;
      std::vector<cplx> q(nc);
      const double inv = 1.0 / std::sqrt(bn);
      for (int b = 0; b < nc; ++b) q[b] = R[best * nc + b] * inv;
      OpPair op;
      op.delta = delta;
      op.O.assign(d * d, 0.0);
      op.P.assign(d * d, 0.0);
      for (int a = 0; a < nr; ++a) {
        cplx c = 0.0;
        for (int b = 0; b < nc; ++b) c += std::conj(q[b]) * R[a * nc + b];
        for (int b = 0; b < nc; ++b) R[a * nc + b] -= c * q[b];
        op.O[rows[a].first * d + rows[a].second] = c;
      }
      for (int b = 0; b < nc; ++b) op.P[cols[b].first * d + cols[b].second] = q[b];
      out.push_back(std::move(op));
    }
  }
  return out;
}

inline int64_t a256(int64_t x) { return (x + 255) & ~int64_t(255); }
inline int cdiv(int a, int b) { return (a + b - 1) / b; }
inline double2 d2(cplx z) { return make_double2(z.real(), z.imag()); }

struct SPBuild {
  std::vector<SPTask> tasks;
  std::vector<SPTerm> terms;
  std::vector<SPTile> tiles;
  double flops = 0.0, bytes = 0.0;
  // a new output block; the following terms accumulate into it
  void out(int64_t c, int ldc, int M, int N, int flags) {
    SPTask t{c, ldc, M, N, (int)terms.size(), (int)terms.size(), flags, 0};
    const int id = (int)tasks.size();
    tasks.push_back(t);
    for (int ti = 0; ti < cdiv(M, kT); ++ti)
      for (int tj = 0; tj < cdiv(N, kT); ++tj) tiles.push_back(SPTile{id, ti, tj});
    bytes += 16.0 * M * N;
  }
  void gemm(int64_t a, int sar, int sac, int64_t b, int sbr, int sbc, int K, cplx coef, int flags) {
    if (K <= 0 || coef == 0.0) return;
    SPTask& t = tasks.back();
    terms.push_back(SPTerm{a, b, sar, sac, sbr, sbc, K, flags, d2(coef)});
    t.t1 = (int)terms.size();
    flops += 8.0 * t.M * t.N * K;
    bytes += 16.0 * ((double)t.M * K + (double)K * t.N);
  }
  void copy(int64_t a, int sar, int sac, cplx coef, int flags) {
    if (coef == 0.0) return;
    SPTask& t = tasks.back();
    terms.push_back(SPTerm{a, 0, sar, sac, 0, 0, 0, flags | kNoB, d2(coef)});
    t.t1 = (int)terms.size();
    flops += 8.0 * t.M * t.N;
    bytes += 16.0 * t.M * t.N;
  }
};
inline int64_t addr(const void* p) { return (int64_t)(uintptr_t)p; }

// Environment of one bond: blocks per operator slot k (0: the block Hamiltonian, t + 1: the
// t-th crossing operator) and per sector of the bond (-1: the partner sector is absent).
struct Env {
  DevBuf buf;
  std::vector<std::vector<int64_t>> off;   // element offsets into buf
  std::vector<int> partner_delta;          // delta of slot k (0 for k = 0)
  bool valid = false;
  double2* at(int k, int si) const {
    const int64_t o = off[k][si];
    return o < 0 ? nullptr : reinterpret_cast<double2*>(buf.p) + o;
  }
};

struct Timing { int kind; cudaEvent_t a, b; };

struct Dmrg {
  mps_s* h = nullptr;
  cudaStream_t st = nullptr;
  int L = 0, d = 0;
  std::vector<std::vector<OpPair>> ops;     // per bond term k (sites k, k+1)
  std::vector<const double*> hb;
  std::vector<Env> envL, envR;
  DevBuf lz, sv, et, dd;                    // Lanczos vectors, SVD + reassembly, environment temps, descriptors
  PinnedBuf hp, rb;                         // descriptor staging, read-back
  int kdim = 24, max_restarts = 64;
  double tol = 1e-12;
  std::vector<Timing> pend;
  std::vector<cudaEvent_t> evpool;
  double ms[5] = {0, 0, 0, 0, 0}, flops[5] = {0, 0, 0, 0, 0};   // heff, env, lanczos, svd, other
  int64_t launches[5] = {0, 0, 0, 0, 0};
  int64_t matvecs = 0, restarts = 0;
  bool profiling = false;
  std::string err;

  ~Dmrg() {
    for (auto& t : pend) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    for (auto e : evpool) cudaEventDestroy(e);
    for (auto& e : envL) e.buf.release();
    for (auto& e : envR) e.buf.release();
    lz.release(); sv.release(); et.release(); dd.release();
    hp.release(); rb.release();
  }

  int fail(int code, const std::string& m) { err = m; h->err = m; return code; }

  cudaEvent_t ev() {
    if (!evpool.empty()) { cudaEvent_t e = evpool.back(); evpool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  template <typename F> cudaError_t timed(int kind, double fl, F&& f) {
    flops[kind] += fl;
    launches[kind]++;
    if (!profiling) return f();
    Timing t{kind, ev(), ev()};
    cudaEventRecord(t.a, st);
    cudaError_t e = f();
    cudaEventRecord(t.b, st);
    pend.push_back(t);
    return e;
  }
  void resolve() {
    for (auto& t : pend) {
      float x = 0.f;
      if (cudaEventElapsedTime(&x, t.a, t.b) == cudaSuccess) ms[t.kind] += x;
      evpool.push_back(t.a);
      evpool.push_back(t.b);
    }
    pend.clear();
  }

  // descriptors: staged in pinned memory, one copy, valid until the next sync point
  struct Up { int64_t tasks, terms, tiles; int n_tiles; };
  cudaError_t upload(const SPBuild& B, int64_t& cursor, Up& u) {
    const int64_t need = cursor + a256(sizeof(SPTask) * B.tasks.size()) + a256(sizeof(SPTerm) * B.terms.size()) +
                         a256(sizeof(SPTile) * B.tiles.size()) + 256;
    if ((int64_t)dd.bytes < need || (int64_t)hp.bytes < need) return cudaErrorMemoryAllocation;   // reserved before
    char* hbase = (char*)hp.p;
    const int64_t c0 = cursor;
    u.tasks = cursor;
    std::memcpy(hbase + cursor, B.tasks.data(), sizeof(SPTask) * B.tasks.size());
    cursor = a256(cursor + sizeof(SPTask) * B.tasks.size());
    u.terms = cursor;
    std::memcpy(hbase + cursor, B.terms.data(), sizeof(SPTerm) * B.terms.size());
    cursor = a256(cursor + sizeof(SPTerm) * B.terms.size());
    u.tiles = cursor;
    std::memcpy(hbase + cursor, B.tiles.data(), sizeof(SPTile) * B.tiles.size());
    cursor = a256(cursor + sizeof(SPTile) * B.tiles.size());
    u.n_tiles = (int)B.tiles.size();
    if (cursor == c0) return cudaSuccess;
    return cudaMemcpyAsync((char*)dd.p + c0, hbase + c0, cursor - c0, cudaMemcpyHostToDevice, st);
  }
  static int64_t desc_bytes(const SPBuild& B) {
    return a256(sizeof(SPTask) * B.tasks.size()) + a256(sizeof(SPTerm) * B.terms.size()) +
           a256(sizeof(SPTile) * B.tiles.size()) + 256;
  }
  cudaError_t reserve_desc(int64_t bytes) {
    cudaError_t e = dd.reserve((size_t)bytes);
    if (e == cudaSuccess) e = hp.reserve((size_t)bytes);
    return e;
  }
  cudaError_t launch(const Up& u, const double2* X, double2* Y) {
    if (u.n_tiles <= 0) return cudaSuccess;
    count_launch();
    char* base = (char*)dd.p;
    sumprod_kernel<<<u.n_tiles, kThr, 0, st>>>(reinterpret_cast<const SPTask*>(base + u.tasks),
                                               reinterpret_cast<const SPTerm*>(base + u.terms),
                                               reinterpret_cast<const SPTile*>(base + u.tiles), X, Y);
    return cudaGetLastError();
  }

  // ---- environments ------------------------------------------------------------------
  // Lays out env E for bond b with the crossing operators `cross` (deltas), zero-filled.
  cudaError_t layout_env(Env& E, const BondTable& bt, const std::vector<OpPair>* cross) {
    const int nk = 1 + (cross ? (int)cross->size() : 0);
    E.off.assign(nk, std::vector<int64_t>(bt.size(), -1));
    E.partner_delta.assign(nk, 0);
    int64_t tot = 0;
    for (int k = 0; k < nk; ++k) {
      const int delta = k ? (*cross)[k - 1].delta : 0;
      E.partner_delta[k] = delta;
      for (int si = 0; si < bt.size(); ++si) {
        const int pj = bt.find(bt.charge[si] + delta);
        if (pj < 0) continue;
        E.off[k][si] = tot;
        tot += (int64_t)bt.dim[si] * bt.dim[pj];
      }
    }
    cudaError_t e = E.buf.reserve((size_t)std::max<int64_t>(tot, 1) * 16);
    if (e == cudaSuccess && tot > 0) e = cudaMemsetAsync(E.buf.p, 0, (size_t)tot * 16, st);
    E.valid = e == cudaSuccess;
    return e;
  }

  const std::vector<OpPair>* bond_ops(int k) const { return (k >= 0 && k <= L - 2) ? &ops[k] : nullptr; }

  // Left environment at bond s+1 from the one at bond s and the left-canonical site s
  // (stored in slot cur[s]).  Stage 1: X = EH(l) A(l,m), Z_t = ET_t(l) A(l+delta, m);
  // stage 2: EH'(m) = sum A^dag X + P-weighted A^dag Z_t, ET'_t(m) = sum O-weighted A(l,m)^dag A(l,m+delta).
  int build_left(int s) {
    const BondTable &Lb = h->bonds[s], &Mb = h->bonds[s + 1];
    const SiteTable& S = h->sites[s];
    const double2* slot = h->slot_ptr(s, h->cur[s]);
    Env &E0 = envL[s], &E1 = envL[s + 1];
    const std::vector<OpPair>* cross = bond_ops(s - 1);    // terms between site s-1 and site s
    const std::vector<OpPair>* next = bond_ops(s);         // terms between site s and site s+1
    if (layout_env(E1, Mb, next) != cudaSuccess) return fail(MPS_ENOMEM, "DMRG environment");
    // temps
    struct Tmp { int blk, t; int64_t off; };
    std::vector<Tmp> tmp;
    int64_t tot = 0;
    const int nc = cross ? (int)cross->size() : 0;
    for (int bi = 0; bi < (int)S.blocks.size(); ++bi) {
      const SiteBlock& b = S.blocks[bi];
      tmp.push_back({bi, -1, tot});
      tot += (int64_t)b.Dl * b.Dm;
      for (int t = 0; t < nc; ++t) {
        const int l2 = b.l + (*cross)[t].delta;
        const int i = b.l - b.m, i2 = l2 - b.m;
        if (i2 < 0 || i2 >= d || S.find(l2, b.m) < 0 || E0.at(t + 1, b.il) == nullptr) continue;
        if ((*cross)[t].P[i * d + i2] == 0.0) continue;
        tmp.push_back({bi, t, tot});
        tot += (int64_t)b.Dl * b.Dm;
      }
    }
    if (et.reserve((size_t)std::max<int64_t>(tot, 1) * 16) != cudaSuccess) return fail(MPS_ENOMEM, "DMRG temps");
    double2* T0 = reinterpret_cast<double2*>(et.p);
    SPBuild s1, s2;
    for (const Tmp& x : tmp) {
      const SiteBlock& b = S.blocks[x.blk];
      s1.out(addr(T0 + x.off), b.Dm, b.Dl, b.Dm, 0);
      if (x.t < 0) {
        s1.gemm(addr(E0.at(0, b.il)), b.Dl, 1, addr(slot + b.off), b.Dm, 1, b.Dl, 1.0, 0);
      } else {
        const int l2 = b.l + (*cross)[x.t].delta;
        const SiteBlock& b2 = S.blocks[S.find(l2, b.m)];
        s1.gemm(addr(E0.at(x.t + 1, b.il)), b2.Dl, 1, addr(slot + b2.off), b2.Dm, 1, b2.Dl, 1.0, 0);
      }
    }
    for (int mi = 0; mi < Mb.size(); ++mi) {
      const int m = Mb.charge[mi], Dm = Mb.dim[mi];
      s2.out(addr(E1.at(0, mi)), Dm, Dm, Dm, 0);
      for (const Tmp& x : tmp) {
        const SiteBlock& b = S.blocks[x.blk];
        if (b.m != m) continue;
        cplx coef = 1.0;
        if (x.t >= 0) {
          const int i = b.l - b.m, i2 = b.l + (*cross)[x.t].delta - b.m;
          coef = (*cross)[x.t].P[i * d + i2];
        }
        s2.gemm(addr(slot + b.off), 1, b.Dm, addr(T0 + x.off), b.Dm, 1, b.Dl, coef, kConjA);
      }
      if (!next) continue;
      for (int t = 0; t < (int)next->size(); ++t) {
        const int delta = (*next)[t].delta;
        double2* dst = E1.at(t + 1, mi);
        if (!dst) continue;
        const int mj = Mb.find(m + delta);
        s2.out(addr(dst), Mb.dim[mj], Dm, Mb.dim[mj], 0);
        for (const SiteBlock& b : S.blocks) {
          if (b.m != m) continue;
          const int bj = S.find(b.l, m + delta);
          if (bj < 0) continue;
          const int i = b.l - m, i2 = b.l - m - delta;
          const cplx o = (*next)[t].O[i * d + i2];
          s2.gemm(addr(slot + b.off), 1, b.Dm, addr(slot + S.blocks[bj].off), S.blocks[bj].Dm, 1, b.Dl, o, kConjA);
        }
      }
    }
    return run_two(s1, s2, 1);
  }

  // Right environment at bond s from the one at bond s+1 and the right-canonical site s.
  // Stage 1: X = RH(r) B(m,r)^dag, Z_t = RT_t(r) B(m,r)^dag; stage 2: RH'(m) = sum B X +
  // O-weighted B(m, r+delta) Z_t, RT'_t(m) = sum P-weighted B(m+delta, r) B(m, r)^dag.
  int build_right(int s) {
    const BondTable &Lb = h->bonds[s], &Rb = h->bonds[s + 1];
    (void)Rb;
    const SiteTable& S = h->sites[s];
    const double2* slot = h->slot_ptr(s, h->cur[s]);
    Env &E1 = envR[s + 1], &E0 = envR[s];
    const std::vector<OpPair>* cross = bond_ops(s);        // terms between site s and site s+1
    const std::vector<OpPair>* next = bond_ops(s - 1);     // terms between site s-1 and site s
    if (layout_env(E0, Lb, next) != cudaSuccess) return fail(MPS_ENOMEM, "DMRG environment");
    struct Tmp { int blk, t; int64_t off; int rows; };
    std::vector<Tmp> tmp;
    int64_t tot = 0;
    const int nc = cross ? (int)cross->size() : 0;
    for (int bi = 0; bi < (int)S.blocks.size(); ++bi) {
      const SiteBlock& b = S.blocks[bi];
      tmp.push_back({bi, -1, tot, b.Dm});
      tot += (int64_t)b.Dm * b.Dl;
      for (int t = 0; t < nc; ++t) {
        const int r2 = b.m + (*cross)[t].delta;
        const int j = b.l - b.m, j2 = b.l - r2;
        if (j2 < 0 || j2 >= d || S.find(b.l, r2) < 0 || E1.at(t + 1, b.im) == nullptr) continue;
        if ((*cross)[t].O[j * d + j2] == 0.0) continue;
        const int Dr2 = S.blocks[S.find(b.l, r2)].Dm;
        tmp.push_back({bi, t, tot, Dr2});
        tot += (int64_t)Dr2 * b.Dl;
      }
    }
    if (et.reserve((size_t)std::max<int64_t>(tot, 1) * 16) != cudaSuccess) return fail(MPS_ENOMEM, "DMRG temps");
    double2* T0 = reinterpret_cast<double2*>(et.p);
    SPBuild s1, s2;
    for (const Tmp& x : tmp) {
      const SiteBlock& b = S.blocks[x.blk];    // (m = b.l, r = b.m), D_m = b.Dl, D_r = b.Dm
      s1.out(addr(T0 + x.off), b.Dl, x.rows, b.Dl, 0);
      const double2* R = x.t < 0 ? E1.at(0, b.im) : E1.at(x.t + 1, b.im);
      s1.gemm(addr(R), b.Dm, 1, addr(slot + b.off), 1, b.Dm, b.Dm, 1.0, kConjB);
    }
    for (int mi = 0; mi < Lb.size(); ++mi) {
      const int m = Lb.charge[mi], Dm = Lb.dim[mi];
      s2.out(addr(E0.at(0, mi)), Dm, Dm, Dm, 0);
      for (const Tmp& x : tmp) {
        const SiteBlock& b = S.blocks[x.blk];
        if (b.l != m) continue;
        if (x.t < 0) {
          s2.gemm(addr(slot + b.off), b.Dm, 1, addr(T0 + x.off), b.Dl, 1, b.Dm, 1.0, 0);
        } else {
          const int r2 = b.m + (*cross)[x.t].delta;
          const SiteBlock& b2 = S.blocks[S.find(m, r2)];
          const int j = m - b.m, j2 = m - r2;
          s2.gemm(addr(slot + b2.off), b2.Dm, 1, addr(T0 + x.off), b.Dl, 1, b2.Dm, (*cross)[x.t].O[j * d + j2], 0);
        }
      }
      if (!next) continue;
      for (int t = 0; t < (int)next->size(); ++t) {
        const int delta = (*next)[t].delta;
        double2* dst = E0.at(t + 1, mi);
        if (!dst) continue;
        const int mj = Lb.find(m + delta);
        s2.out(addr(dst), Dm, Lb.dim[mj], Dm, 0);
        for (const SiteBlock& b : S.blocks) {
          if (b.l != m + delta) continue;
          const int bj = S.find(m, b.m);
          if (bj < 0) continue;
          const int j = m - b.m, j2 = m + delta - b.m;
          const cplx p = (*next)[t].P[j * d + j2];
          const SiteBlock& bm = S.blocks[bj];
          s2.gemm(addr(slot + b.off), b.Dm, 1, addr(slot + bm.off), 1, bm.Dm, b.Dm, p, kConjB);
        }
      }
    }
    return run_two(s1, s2, 1);
  }

  int run_two(const SPBuild& s1, const SPBuild& s2, int kind) {
    if (reserve_desc(desc_bytes(s1) + desc_bytes(s2)) != cudaSuccess) return fail(MPS_ENOMEM, "DMRG descriptors");
    int64_t cur = 0;
    Up u1, u2;
    cudaError_t e = upload(s1, cur, u1);
    if (e == cudaSuccess) e = upload(s2, cur, u2);
    if (e == cudaSuccess) e = timed(kind, s1.flops, [&] { return launch(u1, nullptr, nullptr); });
    if (e == cudaSuccess) e = timed(kind, s2.flops, [&] { return launch(u2, nullptr, nullptr); });
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    resolve();
    if (e != cudaSuccess) return fail(MPS_ECUDA, std::string("DMRG: ") + cudaGetErrorString(e));
    return MPS_OK;
  }

  // ---- Krylov work (Lanczos ground state, or the exponential of TDVP) on one vector ----------
  struct KBuf {
    int64_t dim = 0, ldv = 0;
    int K = 0, nb = 1, vb = 1;
    double2 *V = nullptr, *w = nullptr, *tv = nullptr, *part = nullptr, *hdots = nullptr, *gdots = nullptr,
            *nrm = nullptr, *yc = nullptr;
    double *alpha = nullptr, *beta = nullptr, *inv = nullptr, *yv = nullptr, *res = nullptr, *scl = nullptr,
           *one = nullptr;
  };
  // Lays out the basis (K + 1 vectors), the product w, a scratch vector tv (the caller's start
  // vector), the dot partials and the scalars in lz, zeroed.
  int kbuf(int64_t dim, int kmax, KBuf& b) {
    b.dim = dim;
    b.K = (int)std::min<int64_t>(kmax, dim);
    b.ldv = (dim + 31) / 32 * 32;
    b.nb = std::max(1, std::min(kDotBlocks, (int)((dim + kVecThreads - 1) / kVecThreads)));
    b.vb = vec_blocks(dim);
    const int64_t o_w = (int64_t)(b.K + 1) * b.ldv, o_t = o_w + b.ldv, o_part = o_t + b.ldv;
    const int64_t o_sc = o_part + (int64_t)(b.K + 1) * b.nb;
    const int64_t nsc = 4 * 72 + 64 + 64;
    if (lz.reserve((size_t)(o_sc + nsc) * 16) != cudaSuccess) return fail(MPS_ENOMEM, "DMRG Krylov vectors");
    b.V = reinterpret_cast<double2*>(lz.p);
    b.w = b.V + o_w;
    b.tv = b.V + o_t;
    b.part = b.V + o_part;
    b.hdots = b.V + o_sc;            // 72
    b.gdots = b.hdots + 72;          // 72
    b.nrm = b.gdots + 72;            // 4
    b.yc = b.nrm + 4;                // 64 complex
    b.alpha = reinterpret_cast<double*>(b.yc + 64);   // 64
    b.beta = b.alpha + 64;           // 64
    b.inv = b.beta + 64;             // 8
    b.yv = b.inv + 8;                // 64
    b.res = b.yv + 64;               // 4
    b.scl = b.res + 4;               // 2
    b.one = b.scl + 2;               // 2
    if (cudaMemsetAsync(b.V, 0, (size_t)(o_sc + nsc) * 16, st) != cudaSuccess) return fail(MPS_ECUDA, "DMRG memset");
    return MPS_OK;
  }

  // mode 0: the lowest eigenpair of H by Lanczos with full reorthogonalisation, restarted from
  //         the Ritz vector until |H v - E v| <= tol max(1, |E|): V[0] = the normalised vector,
  //         *value = E.
  // mode 1: exp(-i tau H) of the start vector: Krylov substeps of tau / n (n doubling until every
  //         error estimate is <= tol), V[0] = the result with the start vector's norm,
  //         *value = <v|H|v> of the normalised start vector.
  // The start vector is in b.tv; mv(x, y) enqueues y = H x (mv_flops of work).
  template <class MV>
  int krylov(KBuf& b, MV&& mv, double mv_flops, int mode, double tau, double* value, bool* converged) {
    const int K = b.K;
    const int64_t dim = b.dim, ldv = b.ldv;
    double2* V = b.V;
    auto dots = [&](const double2* Vb, int nk, const double2* x, double2* out) -> cudaError_t {
      count_launch();
      dots_kernel<<<dim3(b.nb, nk), kVecThreads, 0, st>>>(Vb, ldv, x, dim, b.part);
      cudaError_t e2 = cudaGetLastError();
      if (e2 != cudaSuccess) return e2;
      count_launch();
      dots_reduce_kernel<<<nk, kVecThreads, 0, st>>>(b.part, b.nb, out);
      return cudaGetLastError();
    };
    auto normalise_into = [&](double2* dst, const double2* src) -> cudaError_t {
      cudaError_t e2 = dots(src, 1, src, b.nrm);
      if (e2 != cudaSuccess) return e2;
      count_launch();
      inv_norm_kernel<<<1, 32, 0, st>>>(b.nrm, b.inv);
      e2 = cudaGetLastError();
      if (e2 != cudaSuccess) return e2;
      count_launch();
      scale_kernel<<<b.vb, kVecThreads, 0, st>>>(dst, src, b.inv, dim);
      return cudaGetLastError();
    };
    auto lanczos = [&]() -> cudaError_t {       // K iterations from V[0]
      cudaError_t e = cudaSuccess;
      for (int j = 0; j < K && e == cudaSuccess; ++j) {
        double2* vj = V + (int64_t)j * ldv;
        e = timed(0, mv_flops, [&] { return mv(vj, b.w); });
        matvecs++;
        if (e != cudaSuccess) break;
        e = timed(2, 16.0 * dim * (j + 1) * 4, [&] {
          cudaError_t e2 = dots(V, j + 1, b.w, b.hdots);
          if (e2 == cudaSuccess) {
            count_launch();
            subtract_kernel<<<b.vb, kVecThreads, 0, st>>>(b.w, V, ldv, j + 1, b.hdots, dim);
            e2 = cudaGetLastError();
          }
          if (e2 == cudaSuccess) e2 = dots(V, j + 1, b.w, b.gdots);
          if (e2 == cudaSuccess) {
            count_launch();
            subtract_kernel<<<b.vb, kVecThreads, 0, st>>>(b.w, V, ldv, j + 1, b.gdots, dim);
            e2 = cudaGetLastError();
          }
          if (e2 == cudaSuccess) e2 = dots(b.w, 1, b.w, b.nrm);
          if (e2 == cudaSuccess) {
            count_launch();
            lanczos_scalars_kernel<<<1, 32, 0, st>>>(j, b.hdots, b.gdots, b.nrm, b.alpha, b.beta, b.inv);
            e2 = cudaGetLastError();
          }
          if (e2 == cudaSuccess) {
            count_launch();
            scale_kernel<<<b.vb, kVecThreads, 0, st>>>(V + (int64_t)(j + 1) * ldv, b.w, b.inv, dim);
            e2 = cudaGetLastError();
          }
          return e2;
        });
      }
      return e;
    };
    auto readback = [&](double* r) -> cudaError_t {
      cudaError_t e = cudaMemcpyAsync(rb.p, b.res, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      resolve();
      restarts++;
      if (e == cudaSuccess) std::memcpy(r, rb.p, 4 * sizeof(double));
      return e;
    };
    cudaError_t e = cudaSuccess;
    *converged = false;
    if (mode == 0) {
      e = timed(2, 0.0, [&] { return normalise_into(V, b.tv); });
      double E0 = 0.0, resid = 1e300;
      for (int it = 0; e == cudaSuccess && it < max_restarts; ++it) {
        e = lanczos();
        if (e != cudaSuccess) break;
        e = timed(2, 8.0 * dim * K, [&] {
          count_launch();
          tridiag_kernel<<<1, 32, 0, st>>>(b.alpha, b.beta, K, b.yv, b.res);
          cudaError_t e2 = cudaGetLastError();
          if (e2 == cudaSuccess) {
            count_launch();
            combine_kernel<<<b.vb, kVecThreads, 0, st>>>(b.tv, V, ldv, K, b.yv, dim);
            e2 = cudaGetLastError();
          }
          if (e2 == cudaSuccess) e2 = normalise_into(V, b.tv);
          return e2;
        });
        double r[4];
        if (e == cudaSuccess) e = readback(r);
        if (e != cudaSuccess) break;
        E0 = r[0];
        resid = r[1];
        if (!(resid == resid)) return fail(MPS_ECUDA, "DMRG: Lanczos produced NaN");
        if (resid <= tol * std::max(1.0, std::fabs(E0))) break;
      }
      if (e != cudaSuccess) return fail(MPS_ECUDA, std::string("DMRG Lanczos: ") + cudaGetErrorString(e));
      *value = E0;
      *converged = resid <= tol * std::max(1.0, std::fabs(E0));
      return MPS_OK;
    }
    // mode 1: the exponential; the start vector stays in tv until every substep passed
    e = timed(2, 0.0, [&] {
      cudaError_t e2 = dots(b.tv, 1, b.tv, b.nrm);
      if (e2 == cudaSuccess) {
        count_launch();
        norm_kernel<<<1, 32, 0, st>>>(b.nrm, b.scl);
        e2 = cudaGetLastError();
      }
      if (e2 == cudaSuccess) {
        count_launch();
        fill_kernel<<<1, 32, 0, st>>>(b.one, 1.0);
        e2 = cudaGetLastError();
      }
      return e2;
    });
    bool first_value = true;
    for (int nsub = 1; e == cudaSuccess && nsub <= 64; nsub *= 2) {
      bool ok = true;
      e = timed(2, 0.0, [&] { return normalise_into(V, b.tv); });
      for (int sub = 0; e == cudaSuccess && sub < nsub; ++sub) {
        e = lanczos();
        if (e != cudaSuccess) break;
        e = timed(2, 8.0 * dim * K, [&] {
          count_launch();
          expm_tridiag_kernel<<<1, 32, 0, st>>>(b.alpha, b.beta, K, tau / nsub, b.yc, b.res);
          cudaError_t e2 = cudaGetLastError();
          if (e2 == cudaSuccess) {
            count_launch();
            combine_c_kernel<<<b.vb, kVecThreads, 0, st>>>(b.w, V, ldv, K, b.yc, b.one, dim);
            e2 = cudaGetLastError();
          }
          if (e2 == cudaSuccess && sub + 1 < nsub) e2 = normalise_into(V, b.w);
          if (e2 == cudaSuccess && sub + 1 == nsub) {
            count_launch();
            scale_kernel<<<b.vb, kVecThreads, 0, st>>>(V, b.w, b.scl, dim);
            e2 = cudaGetLastError();
          }
          return e2;
        });
        double r[4];
        if (e == cudaSuccess) e = readback(r);
        if (e != cudaSuccess) break;
        if (first_value) { *value = r[0]; first_value = false; }
        if (!(r[1] == r[1])) return fail(MPS_ECUDA, "TDVP: Krylov exponential produced NaN");
        if (r[1] > tol) { ok = false; break; }
      }
      if (e != cudaSuccess) break;
      if (ok) { *converged = true; break; }
    }
    if (e != cudaSuccess) return fail(MPS_ECUDA, std::string("TDVP Krylov: ") + cudaGetErrorString(e));
    return MPS_OK;
  }

  // ---- one local step ------------------------------------------------------------------
  // mode 0: DMRG (the local ground state); mode 1: TDVP (the pair evolved by exp(-i tau H_eff))
  int step(int s, int chi, double cutoff, bool right_moving, double* energy, int mode = 0, double tau = 0.0) {
    const BondTable &Lb = h->bonds[s], &Mb = h->bonds[s + 1], &Rb = h->bonds[s + 2];
    const SiteTable &SL = h->sites[s], &SR = h->sites[s + 1];
    const double2* slotL = h->slot_ptr(s, h->cur[s]);
    const double2* slotR = h->slot_ptr(s + 1, h->cur[s + 1]);
    UpdatePlan P;
    plan_update(Lb, Mb, Rb, h->rule, P);
    const int ns = (int)P.sectors.size();
    if (ns == 0) return fail(MPS_EINVAL, "DMRG step without charge sectors");
    std::vector<int64_t> poff(ns + 1, 0);
    for (int k = 0; k < ns; ++k) poff[k + 1] = poff[k] + (int64_t)P.sectors[k].rows * P.sectors[k].cols;
    const int64_t dim = poff[ns];
    auto sector_of = [&](int c) -> int {
      for (int k = 0; k < ns; ++k)
        if (P.sectors[k].c == c) return k;
      return -1;
    };
    KBuf kb;
    if (int rc0 = kbuf(dim, mode ? std::min(kdim, kExpMax) : kdim, kb)) return rc0;
    double2* tv = kb.tv;

    // ---- H_eff descriptors (X = the vector being multiplied, Y = the product) and Theta ----
    SPBuild mv, th;
    const Env &EL = envL[s], &ER = envR[s + 2];
    const std::vector<OpPair>* lc = bond_ops(s - 1);
    const std::vector<OpPair>* rc = bond_ops(s + 1);
    const double* hc = hb[s];
    const ChargeRule& rule = h->rule;
    for (int k = 0; k < ns; ++k) {
      const SectorPlanEntry& E = P.sectors[k];
      const int c = E.c;
      for (int li = E.l0; li < E.l1; ++li) {
        const int l = Lb.charge[li], Dl = Lb.dim[li], roff = Lb.off[li] - Lb.off[E.l0];
        const int i = l - c;
        for (int ri = E.r0; ri < E.r1; ++ri) {
          const int r = Rb.charge[ri], Dr = Rb.dim[ri], coff = Rb.off[ri] - Rb.off[E.r0];
          const int j = c - r;
          const int64_t xo = poff[k] + (int64_t)roff * E.cols + coff;
          // Theta: B^[s][l, c] B^[s+1][c, r]
          th.out(xo, E.cols, Dl, Dr, kCY);
          const int bl = SL.find(l, c), br = SR.find(c, r);
          if (bl >= 0 && br >= 0)
            th.gemm(addr(slotL + SL.blocks[bl].off), SL.blocks[bl].Dm, 1, addr(slotR + SR.blocks[br].off), Dr, 1,
                    SL.blocks[bl].Dm, 1.0, 0);
          // H_eff Psi for block (c, l, r)
          mv.out(xo, E.cols, Dl, Dr, kCY);
          mv.gemm(addr(EL.at(0, li)), Dl, 1, xo, E.cols, 1, Dl, 1.0, kBX);
          mv.gemm(xo, E.cols, 1, addr(ER.at(0, ri)), Dr, 1, Dr, 1.0, kAX);
          if (lc)
            for (int t = 0; t < (int)lc->size(); ++t) {
              const int delta = (*lc)[t].delta, l2 = l + delta, i2 = i + delta;
              if (i2 < 0 || i2 >= d) continue;
              const int lj = Lb.find(l2);
              if (lj < E.l0 || lj >= E.l1) continue;
              const cplx p = (*lc)[t].P[i * d + i2];
              const double2* env = EL.at(t + 1, li);
              if (p == 0.0 || !env) continue;
              const int64_t xo2 = poff[k] + (int64_t)(Lb.off[lj] - Lb.off[E.l0]) * E.cols + coff;
              mv.gemm(addr(env), Lb.dim[lj], 1, xo2, E.cols, 1, Lb.dim[lj], p, kBX);
            }
          if (rc)
            for (int t = 0; t < (int)rc->size(); ++t) {
              const int delta = (*rc)[t].delta, r2 = r + delta, j2 = j - delta;
              if (j2 < 0 || j2 >= d) continue;
              const int rj = Rb.find(r2);
              if (rj < E.r0 || rj >= E.r1) continue;
              const cplx o = (*rc)[t].O[j * d + j2];
              const double2* env = ER.at(t + 1, ri);
              if (o == 0.0 || !env) continue;
              const int64_t xo2 = poff[k] + (int64_t)roff * E.cols + (Rb.off[rj] - Rb.off[E.r0]);
              mv.gemm(xo2, E.cols, 1, addr(env), Dr, 1, Rb.dim[rj], o, kAX);
            }
          // the centre bond term mixes the middle charges c2 of the pair (l, r)
          const int n = l - r;
          const int base = rule.base(n), sn = rule.sn(n);
          for (int c2 = rule.cmin(l, r); c2 <= rule.cmax(l, r); ++c2) {
            const int k2 = sector_of(c2);
            if (k2 < 0) continue;
            const SectorPlanEntry& E2 = P.sectors[k2];
            const int i2 = l - c2;
            const double* g = hc + 2 * (rule.block_off(n) + (int64_t)(i - base) * sn + (i2 - base));
            const cplx coef(g[0], g[1]);
            const int64_t xo2 = poff[k2] + (int64_t)(Lb.off[li] - Lb.off[E2.l0]) * E2.cols + (Rb.off[ri] - Rb.off[E2.r0]);
            mv.copy(xo2, E2.cols, 1, coef, kAX);
          }
        }
      }
    }
    if (reserve_desc(desc_bytes(mv) + desc_bytes(th)) != cudaSuccess) return fail(MPS_ENOMEM, "DMRG descriptors");
    int64_t cur = 0;
    Up umv, uth;
    cudaError_t e = upload(mv, cur, umv);
    if (e == cudaSuccess) e = upload(th, cur, uth);
    // the start vector Theta, then the local ground state or the forward exponential
    if (e == cudaSuccess) e = timed(4, th.flops, [&] { return launch(uth, nullptr, tv); });
    if (e != cudaSuccess) return fail(MPS_ECUDA, std::string("DMRG: ") + cudaGetErrorString(e));
    bool converged = false;
    double E0 = 0.0;
    const int rck = krylov(kb, [&](const double2* x, double2* y) { return launch(umv, x, y); }, mv.flops, mode, tau,
                           &E0, &converged);
    if (rck != MPS_OK) return rck;
    *energy = E0;
    double2* V = kb.V;
    const double2* psi = V;        // the normalised ground state, Theta layout

    // ---- per-sector SVD (of Psi(c)^dag when moving right: its right vectors are U) ----
    std::vector<int> sm(ns), sn(ns);
    for (int k = 0; k < ns; ++k) {
      const SectorPlanEntry& E = P.sectors[k];
      sm[k] = right_moving ? E.cols : E.rows;
      sn[k] = right_moving ? E.rows : E.cols;
    }
    // a step has few sectors: when one CTA each would leave most SMs idle, the sectors from
    // min(m, n) >= 48 run on 8-CTA clusters instead
    const bool spread = ns * 8 <= 152;
    SvdScratchLayout JL;
    if (!svd_layout(ns, sm.data(), sn.data(), JL, spread ? 48 : -1)) return fail(MPS_EINVAL, "DMRG SVD layout");
    int64_t so = 0;
    std::vector<int64_t> o_mat(ns), o_y(ns), o_sig(ns);
    for (int k = 0; k < ns; ++k) {
      o_mat[k] = so; so = a256(so + 16LL * sm[k] * sn[k]);
    }
    for (int k = 0; k < ns; ++k) {
      const int kk = std::min(sm[k], sn[k]);
      o_y[k] = so; so = a256(so + 16LL * sn[k] * kk);
      o_sig[k] = so; so = a256(so + 8LL * kk);
    }
    const int64_t o_jac = so; so = a256(so + JL.total);
    const int64_t o_status = so; so = a256(so + 4LL * ns);
    const int64_t o_kept = so; so = a256(so + 4LL * ns);
    const int64_t o_res = so; so = a256(so + (int64_t)sizeof(SelectResult));
    if (sv.reserve((size_t)so) != cudaSuccess) return fail(MPS_ENOMEM, "DMRG SVD workspace");
    char* sb = (char*)sv.p;
    SPBuild tr;
    if (right_moving)
      for (int k = 0; k < ns; ++k) {
        const SectorPlanEntry& E = P.sectors[k];
        tr.out(addr(sb + o_mat[k]), E.rows, E.cols, E.rows, 0);
        tr.copy(addr(psi + poff[k]), 1, E.cols, 1.0, kConjA);
      }
    std::vector<SvdSector> secs(ns);
    std::vector<SelectSector> sel(ns);
    double svd_flops = 0.0;
    for (int k = 0; k < ns; ++k) {
      SvdSector S = {};
      S.theta = right_moving ? reinterpret_cast<const double2*>(sb + o_mat[k]) : psi + poff[k];
      S.rowscale = nullptr;
      S.m = sm[k];
      S.n = sn[k];
      S.floor_rel = kDeflateRel * cutoff;
      S.floor_abs = 0.0;
      svd_fill_scratch(S, JL, k, sb + o_jac);
      S.sigma = reinterpret_cast<double*>(sb + o_sig[k]);
      S.Y = reinterpret_cast<double2*>(sb + o_y[k]);
      S.status = reinterpret_cast<int*>(sb + o_status) + k;
      secs[k] = S;
      sel[k] = SelectSector{S.sigma, std::min(S.m, S.n)};
      const double a = std::max(S.m, S.n), b = std::min(S.m, S.n);
      svd_flops += 4.0 * (6.0 * a * b * b + 20.0 * b * b * b);
    }
    std::vector<SvdGroup> groups;
    SvdTune tune;
    if (spread) tune.cl_min = 8;
    svd_forced_tune(tune);
    e = svd_group(secs, groups, tune);
    if (e != cudaSuccess) return fail(MPS_ECUDA, "DMRG SVD grouping");
    SelectTask task{0, ns, chi, cutoff};
    // descriptors of the SVD and the selection, then the transposes
    const int64_t sel_bytes = a256(sizeof(SvdSector) * ns) + a256(sizeof(SelectSector) * ns) + 256;
    if (reserve_desc(sel_bytes + desc_bytes(tr)) != cudaSuccess) return fail(MPS_ENOMEM, "DMRG descriptors");
    {
      char* hbase = (char*)hp.p;
      int64_t c0 = 0;
      std::memcpy(hbase, secs.data(), sizeof(SvdSector) * ns);
      const int64_t o_sel = a256(sizeof(SvdSector) * ns);
      std::memcpy(hbase + o_sel, sel.data(), sizeof(SelectSector) * ns);
      const int64_t o_task = o_sel + a256(sizeof(SelectSector) * ns);
      std::memcpy(hbase + o_task, &task, sizeof(task));
      c0 = o_task + 256;
      e = cudaMemcpyAsync(dd.p, hbase, c0, cudaMemcpyHostToDevice, st);
      Up utr;
      if (e == cudaSuccess) e = upload(tr, c0, utr);
      if (e == cudaSuccess) e = timed(4, 0.0, [&] { return launch(utr, nullptr, nullptr); });
      const SvdSector* d_secs = reinterpret_cast<const SvdSector*>(dd.p);
      if (e == cudaSuccess)
        e = timed(3, svd_flops, [&] {
          return launch_svd_groups(d_secs, groups, st, h->side, kSvdSideStreams, h->fork, h->join, h->sweep_limit);
        });
      if (e == cudaSuccess)
        e = launch_select(reinterpret_cast<const SelectSector*>((char*)dd.p + o_sel),
                          reinterpret_cast<const SelectTask*>((char*)dd.p + o_task), 1,
                          reinterpret_cast<int*>(sb + o_kept), reinterpret_cast<SelectResult*>(sb + o_res), st);
    }
    const int64_t rb_need = a256(4LL * ns) * 2 + (int64_t)sizeof(SelectResult) + 64;
    if (e == cudaSuccess && rb.reserve((size_t)rb_need) != cudaSuccess) e = cudaErrorMemoryAllocation;
    int* kept_h = (int*)rb.p;
    int* stat_h = (int*)((char*)rb.p + a256(4LL * ns));
    SelectResult* res_h = (SelectResult*)((char*)rb.p + 2 * a256(4LL * ns));
    if (e == cudaSuccess) e = cudaMemcpyAsync(kept_h, sb + o_kept, 4LL * ns, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stat_h, sb + o_status, 4LL * ns, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(res_h, sb + o_res, sizeof(SelectResult), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    resolve();
    if (e != cudaSuccess) return fail(MPS_ECUDA, std::string("DMRG SVD: ") + cudaGetErrorString(e));
    if (res_h->status != 0) return fail(MPS_EINVAL, "DMRG: all singular values vanish");
    bool noconv = false;
    for (int k = 0; k < ns; ++k) noconv = noconv || stat_h[k] < 0;

    // ---- the new bond, the new sites, lambda, and the environment of the new bond ----
    BondTable M;
    for (int k = 0; k < ns; ++k)
      if (kept_h[k] > 0) { M.charge.push_back(P.sectors[k].c); M.dim.push_back(kept_h[k]); }
    M.rebuild_offsets();
    if (M.size() == 0) return fail(MPS_EINVAL, "DMRG: the cutoff discards every singular value");
    if (M.total() > h->bond_cap[s + 1]) return fail(MPS_ENOMEM, "DMRG: new bond exceeds its capacity");
    SiteTable nL, nR;
    layout_site(Lb, M, h->rule, nL);
    layout_site(M, Rb, h->rule, nR);
    if (nL.nnz > h->site_cap[s] || nR.nnz > h->site_cap[s + 1])
      return fail(MPS_ENOMEM, "DMRG: new site tensor exceeds its capacity");
    double2* dstL = h->slot_ptr(s, h->cur[s] ^ 1);
    double2* dstR = h->slot_ptr(s + 1, h->cur[s + 1] ^ 1);
    const double scale = 1.0 / res_h->norm_kept;
    SPBuild ra;
    std::vector<LambdaTask> lam;
    int mi = 0;
    for (int k = 0; k < ns; ++k) {
      const int kk = kept_h[k];
      if (kk == 0) continue;
      const SectorPlanEntry& E = P.sectors[k];
      const double2* Y = reinterpret_cast<const double2*>(sb + o_y[k]);
      lam.push_back(LambdaTask{reinterpret_cast<const double*>(sb + o_sig[k]), h->lambda_ptr(s + 1) + M.off[mi], kk,
                               scale});
      for (int li = E.l0; li < E.l1; ++li) {
        const int b = nL.find(Lb.charge[li], E.c);
        const int roff = Lb.off[li] - Lb.off[E.l0], Dl = Lb.dim[li];
        ra.out(addr(dstL + nL.blocks[b].off), kk, Dl, kk, 0);
        if (right_moving)    // U[rows of l, :k] (Y of Psi^dag: rows x K column-major)
          ra.copy(addr(Y + roff), 1, E.rows, 1.0, 0);
        else                 // Psi(c)[rows of l] V[:, :k] / |S_kept|
          ra.gemm(addr(psi + poff[k] + (int64_t)roff * E.cols), E.cols, 1, addr(Y), 1, E.cols, E.cols, scale, 0);
      }
      for (int ri = E.r0; ri < E.r1; ++ri) {
        const int b = nR.find(E.c, Rb.charge[ri]);
        const int coff = Rb.off[ri] - Rb.off[E.r0], Dr = Rb.dim[ri];
        ra.out(addr(dstR + nR.blocks[b].off), Dr, kk, Dr, 0);
        if (right_moving)    // U[:, :k]^dag Psi(c)[:, cols of r] / |S_kept|
          ra.gemm(addr(Y), E.rows, 1, addr(psi + poff[k] + coff), E.cols, 1, E.rows, scale, kConjA);
        else                 // V[cols of r, :k]^dag
          ra.copy(addr(Y + coff), E.cols, 1, 1.0, kConjA);
      }
      ++mi;
    }
    if (reserve_desc(desc_bytes(ra) + a256(sizeof(LambdaTask) * lam.size()) + 256) != cudaSuccess)
      return fail(MPS_ENOMEM, "DMRG descriptors");
    {
      int64_t c0 = 0;
      Up ura;
      e = upload(ra, c0, ura);
      const int64_t o_lam = c0;
      std::memcpy((char*)hp.p + o_lam, lam.data(), sizeof(LambdaTask) * lam.size());
      if (e == cudaSuccess)
        e = cudaMemcpyAsync((char*)dd.p + o_lam, (char*)hp.p + o_lam, sizeof(LambdaTask) * lam.size(),
                            cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = timed(4, ra.flops, [&] { return launch(ura, nullptr, nullptr); });
      if (e == cudaSuccess)
        e = launch_lambda(reinterpret_cast<const LambdaTask*>((char*)dd.p + o_lam), (int)lam.size(), st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      resolve();
      if (e != cudaSuccess) return fail(MPS_ECUDA, std::string("DMRG reassembly: ") + cudaGetErrorString(e));
    }
    h->bonds[s + 1] = M;
    h->sites[s] = nL;
    h->sites[s + 1] = nR;
    h->cur[s] ^= 1;
    h->cur[s + 1] ^= 1;
    int rc2 = right_moving ? build_left(s) : build_right(s + 1);
    if (rc2 != MPS_OK) return rc2;
    if (!converged) {
      h->err = mode ? "TDVP Krylov exponential did not reach its tolerance"
                    : "Lanczos did not reach its tolerance; state updated with the last Ritz vector";
      return MPS_ENOCONV;
    }
    if (noconv) { h->err = "Jacobi SVD hit its sweep limit; state updated with the last iterate"; return MPS_ENOCONV; }
    return MPS_OK;
  }

  // ---- TDVP: the centre site j evolved backward, site j <- exp(+i tau H_eff^(1)) site j -------
  // One-site H_eff on the blocks C(l, m) of site j (left environment at bond j, right at j+1):
  //   EH(l) C(l, m) + C(l, m) RH(m) + sum_t P_t[i, i+delta] ET_t(l) C(l+delta, m)
  //   + sum_t O_t[i, i-delta] C(l, m+delta) RT_t(m),   i = l - m.
  // The site's slot is the vector (its blocks in (l, m) order); the result goes back in place.
  int backward(int j, double tau, double* energy) {
    const SiteTable& S = h->sites[j];
    double2* slot = h->slot_ptr(j, h->cur[j]);
    const Env &EL = envL[j], &ER = envR[j + 1];
    const std::vector<OpPair>* lcr = bond_ops(j - 1);
    const std::vector<OpPair>* rcr = bond_ops(j);
    SPBuild m1;
    for (const SiteBlock& b : S.blocks) {
      const int i = b.l - b.m;
      m1.out(b.off, b.Dm, b.Dl, b.Dm, kCY);
      m1.gemm(addr(EL.at(0, b.il)), b.Dl, 1, b.off, b.Dm, 1, b.Dl, 1.0, kBX);
      m1.gemm(b.off, b.Dm, 1, addr(ER.at(0, b.im)), b.Dm, 1, b.Dm, 1.0, kAX);
      if (lcr)
        for (int t = 0; t < (int)lcr->size(); ++t) {
          const int delta = (*lcr)[t].delta, i2 = i + delta;
          if (i2 < 0 || i2 >= d) continue;
          const int b2 = S.find(b.l + delta, b.m);
          const double2* env = EL.at(t + 1, b.il);
          const cplx p = (*lcr)[t].P[i * d + i2];
          if (b2 < 0 || !env || p == 0.0) continue;
          const SiteBlock& B2 = S.blocks[b2];
          m1.gemm(addr(env), B2.Dl, 1, B2.off, B2.Dm, 1, B2.Dl, p, kBX);
        }
      if (rcr)
        for (int t = 0; t < (int)rcr->size(); ++t) {
          const int delta = (*rcr)[t].delta, i3 = i - delta;
          if (i3 < 0 || i3 >= d) continue;
          const int b3 = S.find(b.l, b.m + delta);
          const double2* env = ER.at(t + 1, b.im);
          const cplx o = (*rcr)[t].O[i * d + i3];
          if (b3 < 0 || !env || o == 0.0) continue;
          const SiteBlock& B3 = S.blocks[b3];
          m1.gemm(B3.off, B3.Dm, 1, addr(env), b.Dm, 1, B3.Dm, o, kAX);
        }
    }
    const int64_t dim = S.nnz;
    KBuf kb;
    if (int rc0 = kbuf(dim, std::min(kdim, kExpMax), kb)) return rc0;
    if (reserve_desc(desc_bytes(m1)) != cudaSuccess) return fail(MPS_ENOMEM, "TDVP descriptors");
    int64_t cur = 0;
    Up u;
    cudaError_t e = upload(m1, cur, u);
    if (e == cudaSuccess) e = cudaMemcpyAsync(kb.tv, slot, sizeof(double2) * dim, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(MPS_ECUDA, "TDVP backward step");
    bool converged = false;
    const int rck = krylov(kb, [&](const double2* x, double2* y) { return launch(u, x, y); }, m1.flops, 1, -tau,
                           energy, &converged);
    if (rck != MPS_OK) return rck;
    e = cudaMemcpyAsync(slot, kb.V, sizeof(double2) * dim, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(MPS_ECUDA, "TDVP backward step");
    if (!converged) { h->err = "TDVP Krylov exponential did not reach its tolerance"; return MPS_ENOCONV; }
    return MPS_OK;
  }

  // ---- back to right-canonical B with Schmidt lambdas (inverse-free left-to-right pass) ----
  // B'(l, m) = W(l) B(l, m) with W = the previous site's V^dag; M(m) = diag(lambda_l) B'(., m)
  // stacked over l; M = U S V^dag; lambda(m) = S / |S|, B(l, m) <- B'(l, m) V; W(m) = V^dag.
  int canonicalize() {
    DevBuf ybuf[2];
    std::vector<int64_t> yoff_prev;            // per sector of bond s (new table): Y of the previous SVD
    std::vector<int> yn_prev;                  // its row count (the old sector dimension)
    int yb = 0;
    int rc = MPS_OK;
    const double one = 1.0;
    cudaError_t e = cudaMemcpyAsync(h->lambda_ptr(0), &one, sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(MPS_ECUDA, "DMRG canonical form");
    for (int s = 0; s < L && rc == MPS_OK; ++s) {
      const BondTable &Lb = h->bonds[s], &Mb = h->bonds[s + 1];
      // blocks of site s in the current slot: (l, m) with l a sector of the (new) bond s
      struct Blk { int li, mi, Dl_old, Dm; int64_t off; };
      std::vector<Blk> blks;
      for (const SiteBlock& b : h->sites[s].blocks) {
        const int li = Lb.find(b.l);
        if (li < 0) continue;                  // its left sector was dropped
        blks.push_back(Blk{li, b.im, b.Dl, b.Dm, b.off});
      }
      const double2* slot = h->slot_ptr(s, h->cur[s]);
      const bool last = s == L - 1;
      std::vector<int> l0_m(Mb.size(), -1), l1_m(Mb.size(), -1);
      for (const Blk& b : blks) {
        if (l0_m[b.mi] < 0 || b.li < l0_m[b.mi]) l0_m[b.mi] = b.li;
        l1_m[b.mi] = std::max(l1_m[b.mi], b.li + 1);
      }
      std::vector<int64_t> o_mat(Mb.size(), -1);
      std::vector<int> rows_m(Mb.size(), 0);
      int64_t so = 0;
      std::vector<int> sm, snn, which;
      for (int mi = 0; mi < Mb.size(); ++mi) {
        if (l0_m[mi] < 0) continue;
        rows_m[mi] = Lb.off[l1_m[mi]] - Lb.off[l0_m[mi]];
        o_mat[mi] = so;
        so = a256(so + 16LL * rows_m[mi] * Mb.dim[mi]);
        sm.push_back(rows_m[mi]);
        snn.push_back(Mb.dim[mi]);
        which.push_back(mi);
      }
      const int ns = (int)which.size();
      SvdScratchLayout JL;
      const bool spread = ns * 8 <= 152;
      if (!last && !svd_layout(ns, sm.data(), snn.data(), JL, spread ? 48 : -1))
        return fail(MPS_EINVAL, "DMRG SVD layout");
      std::vector<int64_t> o_y(ns), o_sig(ns);
      int64_t ysz = 0;
      for (int k = 0; k < ns && !last; ++k) {
        const int kk = std::min(sm[k], snn[k]);
        o_y[k] = ysz; ysz = a256(ysz + 16LL * snn[k] * kk);
        o_sig[k] = ysz; ysz = a256(ysz + 8LL * kk);
      }
      const int64_t o_jac = so; so = a256(so + (last ? 0 : JL.total));
      const int64_t o_status = so; so = a256(so + 4LL * std::max(ns, 1));
      const int64_t o_kept = so; so = a256(so + 4LL * std::max(ns, 1));
      const int64_t o_res = so; so = a256(so + (int64_t)sizeof(SelectResult));
      if (sv.reserve((size_t)so) != cudaSuccess || ybuf[yb].reserve((size_t)std::max<int64_t>(ysz, 16)) != cudaSuccess)
        return fail(MPS_ENOMEM, "DMRG canonical-form workspace");
      char* sb = (char*)sv.p;
      char* yb_p = (char*)ybuf[yb].p;
      const char* yprev = (const char*)ybuf[yb ^ 1].p;
      SiteTable nlast;
      double2* dst = h->slot_ptr(s, h->cur[s] ^ 1);
      if (last) layout_site(Lb, Mb, h->rule, nlast);
      // B' = W B: into the stacked SVD inputs M(m), or straight into the last site
      SPBuild bp;
      for (const Blk& b : blks) {
        const int Dl_new = Lb.dim[b.li];
        int64_t out;
        if (last) {
          const int nb = nlast.find(Lb.charge[b.li], Mb.charge[b.mi]);
          out = addr(dst + nlast.blocks[nb].off);
        } else {
          out = addr(sb + o_mat[b.mi] + 16LL * (int64_t)(Lb.off[b.li] - Lb.off[l0_m[b.mi]]) * b.Dm);
        }
        bp.out(out, b.Dm, Dl_new, b.Dm, 0);
        if (s == 0) {
          bp.copy(addr(slot + b.off), b.Dm, 1, 1.0, 0);
        } else {      // W(l) = V(l)[:, :K]^dag, V column-major with yn_prev rows
          const double2* Yp = reinterpret_cast<const double2*>(yprev + yoff_prev[b.li]);
          bp.gemm(addr(Yp), yn_prev[b.li], 1, addr(slot + b.off), b.Dm, 1, b.Dl_old, 1.0, kConjA);
        }
      }
      if (last) {
        if (reserve_desc(desc_bytes(bp)) != cudaSuccess) return fail(MPS_ENOMEM, "DMRG descriptors");
        int64_t c0 = 0;
        Up u;
        e = upload(bp, c0, u);
        if (e == cudaSuccess) e = timed(4, bp.flops, [&] { return launch(u, nullptr, nullptr); });
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        resolve();
        if (e != cudaSuccess) return fail(MPS_ECUDA, "DMRG canonical form");
        h->sites[s] = nlast;
        h->cur[s] ^= 1;
        break;
      }
      std::vector<SvdSector> secs(ns);
      std::vector<SelectSector> sel(ns);
      double svd_flops = 0.0;
      for (int k = 0; k < ns; ++k) {
        const int mi = which[k];
        SvdSector Sx = {};
        Sx.theta = reinterpret_cast<const double2*>(sb + o_mat[mi]);
        Sx.rowscale = h->lambda_ptr(s) + Lb.off[l0_m[mi]];
        Sx.m = sm[k];
        Sx.n = snn[k];
        Sx.floor_rel = 0.0;
        svd_fill_scratch(Sx, JL, k, sb + o_jac);
        Sx.sigma = reinterpret_cast<double*>(yb_p + o_sig[k]);
        Sx.Y = reinterpret_cast<double2*>(yb_p + o_y[k]);
        Sx.status = reinterpret_cast<int*>(sb + o_status) + k;
        secs[k] = Sx;
        sel[k] = SelectSector{Sx.sigma, std::min(Sx.m, Sx.n)};
        const double a = std::max(Sx.m, Sx.n), bb = std::min(Sx.m, Sx.n);
        svd_flops += 4.0 * (6.0 * a * bb * bb + 20.0 * bb * bb * bb);
      }
      std::vector<SvdGroup> groups;
      SvdTune tune;
      if (spread) tune.cl_min = 8;
      svd_forced_tune(tune);
      if (svd_group(secs, groups, tune) != cudaSuccess) return fail(MPS_ECUDA, "DMRG SVD grouping");
      SelectTask task{0, ns, 1 << 30, 0.0};
      const int64_t sel_bytes = a256(sizeof(SvdSector) * ns) + a256(sizeof(SelectSector) * ns) + 256;
      if (reserve_desc(sel_bytes + desc_bytes(bp)) != cudaSuccess) return fail(MPS_ENOMEM, "DMRG descriptors");
      char* hbase = (char*)hp.p;
      std::memcpy(hbase, secs.data(), sizeof(SvdSector) * ns);
      const int64_t o_sel = a256(sizeof(SvdSector) * ns);
      std::memcpy(hbase + o_sel, sel.data(), sizeof(SelectSector) * ns);
      const int64_t o_task = o_sel + a256(sizeof(SelectSector) * ns);
      std::memcpy(hbase + o_task, &task, sizeof(task));
      int64_t c0 = o_task + 256;
      e = cudaMemcpyAsync(dd.p, hbase, c0, cudaMemcpyHostToDevice, st);
      Up u;
      if (e == cudaSuccess) e = upload(bp, c0, u);
      if (e == cudaSuccess) e = timed(4, bp.flops, [&] { return launch(u, nullptr, nullptr); });
      const SvdSector* d_secs = reinterpret_cast<const SvdSector*>(dd.p);
      if (e == cudaSuccess)
        e = timed(3, svd_flops, [&] {
          return launch_svd_groups(d_secs, groups, st, h->side, kSvdSideStreams, h->fork, h->join, h->sweep_limit);
        });
      if (e == cudaSuccess)
        e = launch_select(reinterpret_cast<const SelectSector*>((char*)dd.p + o_sel),
                          reinterpret_cast<const SelectTask*>((char*)dd.p + o_task), 1,
                          reinterpret_cast<int*>(sb + o_kept), reinterpret_cast<SelectResult*>(sb + o_res), st);
      const int64_t rb_need = 2 * a256(4LL * ns) + (int64_t)sizeof(SelectResult) + 64;
      if (e == cudaSuccess && rb.reserve((size_t)rb_need) != cudaSuccess) e = cudaErrorMemoryAllocation;
      int* kept_h = (int*)rb.p;
      int* stat_h = (int*)((char*)rb.p + a256(4LL * ns));
      SelectResult* res_h = (SelectResult*)((char*)rb.p + 2 * a256(4LL * ns));
      if (e == cudaSuccess) e = cudaMemcpyAsync(kept_h, sb + o_kept, 4LL * ns, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(stat_h, sb + o_status, 4LL * ns, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(res_h, sb + o_res, sizeof(SelectResult), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      resolve();
      if (e != cudaSuccess) return fail(MPS_ECUDA, std::string("DMRG canonical form: ") + cudaGetErrorString(e));
      if (res_h->status != 0) return fail(MPS_EINVAL, "DMRG canonical form: all singular values vanish");
      for (int k = 0; k < ns; ++k)
        if (stat_h[k] < 0) rc = MPS_ENOCONV;
      // the new bond s+1, site s = B' V[:, :k], lambda = S / |S|
      BondTable nb;
      for (int k = 0; k < ns; ++k)
        if (kept_h[k] > 0) { nb.charge.push_back(Mb.charge[which[k]]); nb.dim.push_back(kept_h[k]); }
      nb.rebuild_offsets();
      if (nb.size() == 0) return fail(MPS_EINVAL, "DMRG canonical form: empty bond");
      SiteTable ntab;
      layout_site(Lb, nb, h->rule, ntab);
      SPBuild nw;
      std::vector<LambdaTask> lam;
      const double scale = 1.0 / res_h->norm_kept;
      std::vector<int64_t> ynext(nb.size(), -1);
      std::vector<int> ynext_n(nb.size(), 0);
      for (int k = 0; k < ns; ++k) {
        const int mi = which[k], kk = kept_h[k];
        if (kk == 0) continue;
        const int nbi = nb.find(Mb.charge[mi]);
        ynext[nbi] = o_y[k];
        ynext_n[nbi] = snn[k];
        lam.push_back(LambdaTask{reinterpret_cast<const double*>(yb_p + o_sig[k]), h->lambda_ptr(s + 1) + nb.off[nbi],
                                 kk, scale});
        for (int li = l0_m[mi]; li < l1_m[mi]; ++li) {
          const int b = ntab.find(Lb.charge[li], Mb.charge[mi]);
          const int Dl = Lb.dim[li];
          nw.out(addr(dst + ntab.blocks[b].off), kk, Dl, kk, 0);
          nw.gemm(addr(sb + o_mat[mi] + 16LL * (int64_t)(Lb.off[li] - Lb.off[l0_m[mi]]) * Mb.dim[mi]), Mb.dim[mi], 1,
                  addr(yb_p + o_y[k]), 1, Mb.dim[mi], Mb.dim[mi], 1.0, 0);
        }
      }
      if (reserve_desc(desc_bytes(nw) + a256(sizeof(LambdaTask) * lam.size()) + 256) != cudaSuccess)
        return fail(MPS_ENOMEM, "DMRG descriptors");
      c0 = 0;
      e = upload(nw, c0, u);
      std::memcpy((char*)hp.p + c0, lam.data(), sizeof(LambdaTask) * lam.size());
      if (e == cudaSuccess)
        e = cudaMemcpyAsync((char*)dd.p + c0, (char*)hp.p + c0, sizeof(LambdaTask) * lam.size(), cudaMemcpyHostToDevice,
                            st);
      if (e == cudaSuccess) e = timed(4, nw.flops, [&] { return launch(u, nullptr, nullptr); });
      if (e == cudaSuccess) e = launch_lambda(reinterpret_cast<const LambdaTask*>((char*)dd.p + c0), (int)lam.size(), st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      resolve();
      if (e != cudaSuccess) return fail(MPS_ECUDA, "DMRG canonical form");
      yoff_prev = ynext;
      yn_prev = ynext_n;
      h->bonds[s + 1] = nb;
      h->sites[s] = ntab;
      h->cur[s] ^= 1;
      yb ^= 1;
    }
    ybuf[0].release();
    ybuf[1].release();
    return rc;
  }
};

}  // namespace

extern "C" {

int mps_dmrg(mps_t h, const double* const* bond_terms, int n_sweeps, int chi, double cutoff, int lanczos_dim,
             double tol, double* energies, int energies_cap, int* n_energies) {
  if (!h || !bond_terms || n_sweeps < 0 || chi < 1 || !(cutoff >= 0.0) || !n_energies) return MPS_EINVAL;
  *n_energies = 0;
  if (h->precision != MPS_FP64) { h->err = "DMRG runs on FP64 handles"; return MPS_EINVAL; }
  if (h->rule.zn || h->rule.multi) { h->err = "DMRG is built for single U(1) charges"; return MPS_EINVAL; }
  if (lanczos_dim < 2 || lanczos_dim > 63 || !(tol > 0.0)) return MPS_EINVAL;
  const int L = h->L;
  if (L < 2) return MPS_EINVAL;
  for (int k = 0; k < L - 1; ++k)
    if (!bond_terms[k]) return MPS_EINVAL;
  for (int s = 0; s < L; ++s)
    if (h->dirty[s]) { h->err = "site " + std::to_string(s) + " needs mps_set_site"; return MPS_EINVAL; }
  const int64_t need = (int64_t)n_sweeps * 2 * (L - 1);
  if (energies && energies_cap < need) return MPS_EINVAL;
  Dmrg D;
  D.h = h;
  D.st = h->stream;
  D.L = L;
  D.d = h->d;
  D.kdim = lanczos_dim;
  D.tol = tol;
  D.profiling = h->profiling;
  D.hb.assign(bond_terms, bond_terms + (L - 1));
  for (int k = 0; k < L - 1; ++k) D.ops.push_back(split_bond(bond_terms[k], h->rule));
  D.envL.resize(L + 1);
  D.envR.resize(L + 1);
  if (D.rb.reserve(4096) != cudaSuccess) return MPS_ENOMEM;
  if (cudaStreamSynchronize(D.st) != cudaSuccess) return MPS_ECUDA;
  // boundary environments: zero block Hamiltonians on the one-dimensional end bonds
  if (D.layout_env(D.envL[0], h->bonds[0], nullptr) != cudaSuccess) return MPS_ENOMEM;
  if (D.layout_env(D.envR[L], h->bonds[L], nullptr) != cudaSuccess) return MPS_ENOMEM;
  for (int s = L - 1; s >= 2; --s) {
    const int rc = D.build_right(s);
    if (rc != MPS_OK) return rc;
  }
  int status = MPS_OK;
  int64_t ne = 0;
  for (int sw = 0; sw < n_sweeps; ++sw) {
    for (int pass = 0; pass < 2; ++pass) {
      const bool right = pass == 0;
      for (int k = 0; k < L - 1; ++k) {
        const int s = right ? k : L - 2 - k;
        double E = 0.0;
        const int rc = D.step(s, chi, cutoff, right, &E);
        if (rc != MPS_OK && rc != MPS_ENOCONV) return rc;
        if (rc == MPS_ENOCONV) status = MPS_ENOCONV;
        if (energies) energies[ne] = E;
        ++ne;
      }
    }
  }
  *n_energies = (int)ne;
  const int rc = D.canonicalize();
  if (rc != MPS_OK && rc != MPS_ENOCONV) return rc;
  if (rc == MPS_ENOCONV) status = MPS_ENOCONV;
  for (auto& c : h->cut_est) c = 0.0;
  // per-kind device time and work of this call, read by mps_dmrg_stats
  h->dmrg_last.matvecs = D.matvecs;
  h->dmrg_last.restarts = D.restarts;
  for (int k = 0; k < 5; ++k) {
    h->dmrg_last.ms[k] = D.ms[k];
    h->dmrg_last.flops[k] = D.flops[k];
    h->dmrg_last.launches[k] = D.launches[k];
  }
  return status;
}

int mps_tdvp(mps_t h, const double* const* bond_terms, int n_steps, double dt, int chi, double cutoff,
             int krylov_dim, double tol, double* energies, int energies_cap, int* n_energies) {
  if (!h || !bond_terms || n_steps < 0 || chi < 1 || !(cutoff >= 0.0) || !n_energies || !(dt == dt)) return MPS_EINVAL;
  *n_energies = 0;
  if (h->precision != MPS_FP64) { h->err = "TDVP runs on FP64 handles"; return MPS_EINVAL; }
  if (h->rule.zn || h->rule.multi) { h->err = "TDVP is built for single U(1) charges"; return MPS_EINVAL; }
  if (krylov_dim < 2 || krylov_dim > kExpMax || !(tol > 0.0)) return MPS_EINVAL;
  const int L = h->L;
  for (int k = 0; k < L - 1; ++k)
    if (!bond_terms[k]) return MPS_EINVAL;
  for (int s = 0; s < L; ++s)
    if (h->dirty[s]) { h->err = "site " + std::to_string(s) + " needs mps_set_site"; return MPS_EINVAL; }
  const int64_t need = (int64_t)n_steps * 2 * (L - 1);
  if (energies && energies_cap < need) return MPS_EINVAL;
  Dmrg D;
  D.h = h;
  D.st = h->stream;
  D.L = L;
  D.d = h->d;
  D.kdim = krylov_dim;
  D.tol = tol;
  D.profiling = h->profiling;
  D.hb.assign(bond_terms, bond_terms + (L - 1));
  for (int k = 0; k < L - 1; ++k) D.ops.push_back(split_bond(bond_terms[k], h->rule));
  D.envL.resize(L + 1);
  D.envR.resize(L + 1);
  if (D.rb.reserve(4096) != cudaSuccess) return MPS_ENOMEM;
  if (cudaStreamSynchronize(D.st) != cudaSuccess) return MPS_ECUDA;
  if (D.layout_env(D.envL[0], h->bonds[0], nullptr) != cudaSuccess) return MPS_ENOMEM;
  if (D.layout_env(D.envR[L], h->bonds[L], nullptr) != cudaSuccess) return MPS_ENOMEM;
  for (int s = L - 1; s >= 2; --s) {
    const int rc = D.build_right(s);
    if (rc != MPS_OK) return rc;
  }
  const double half = 0.5 * dt;
  int status = MPS_OK;
  int64_t ne = 0;
  auto note = [&](int rc) { if (rc == MPS_ENOCONV) status = MPS_ENOCONV; return rc == MPS_OK || rc == MPS_ENOCONV; };
  for (int step = 0; step < n_steps; ++step) {
    for (int s = 0; s < L - 1; ++s) {             // right-moving pass, dt/2
      double E = 0.0, Eb = 0.0;
      int rc = D.step(s, chi, cutoff, true, &E, 1, half);
      if (!note(rc)) return rc;
      if (energies) energies[ne] = E;
      ++ne;
      if (s < L - 2) {
        rc = D.backward(s + 1, half, &Eb);
        if (!note(rc)) return rc;
      }
    }
    for (int s = L - 2; s >= 0; --s) {            // left-moving pass, dt/2
      double E = 0.0, Eb = 0.0;
      int rc = D.step(s, chi, cutoff, false, &E, 1, half);
      if (!note(rc)) return rc;
      if (energies) energies[ne] = E;
      ++ne;
      if (s > 0) {
        rc = D.backward(s, half, &Eb);
        if (!note(rc)) return rc;
      }
    }
  }
  *n_energies = (int)ne;
  const int rc = D.canonicalize();
  if (!note(rc)) return rc;
  for (auto& c : h->cut_est) c = 0.0;
  h->dmrg_last.matvecs = D.matvecs;
  h->dmrg_last.restarts = D.restarts;
  for (int k = 0; k < 5; ++k) {
    h->dmrg_last.ms[k] = D.ms[k];
    h->dmrg_last.flops[k] = D.flops[k];
    h->dmrg_last.launches[k] = D.launches[k];
  }
  return status;
}

int mps_dmrg_stats(mps_t h, int kind, int64_t* launches, double* ms, double* flops) {
  if (!h || kind < 0 || kind >= 5) return MPS_EINVAL;
  if (launches) *launches = h->dmrg_last.launches[kind];
  if (ms) *ms = h->dmrg_last.ms[kind];
  if (flops) *flops = h->dmrg_last.flops[kind];
  return MPS_OK;
}

int mps_dmrg_counts(mps_t h, int64_t* matvecs, int64_t* restarts) {
  if (!h) return MPS_EINVAL;
  if (matvecs) *matvecs = h->dmrg_last.matvecs;
  if (restarts) *restarts = h->dmrg_last.restarts;
  return MPS_OK;
}

}  // extern "C"
