// Batched per-sector SVD of the two-site update (K2), FP64, QR-preconditioned
// one-sided Jacobi.
//
// arXiv:2303.11409, Sec. II: after the U(1) split a local update needs only
// block-sparse SVDs of the submatrices Theta(c), each at most chi x chi.  Each
// sector M = diag(lambda) Theta'(c) (m x n, K = min(m, n)) is decomposed as
//   1. Householder QR with column pivoting  M P = Q R  (R: K x n, upper trapezoidal);
//   2. one-sided (Hestenes) Jacobi on the columns of R^dag (n x K):
//      R^dag U = [s_1 v_1, ..., s_K v_K], so the column norms are the singular
//      values and the normalised columns are the right singular vectors of R;
//   3. Y = P [v_1 ... v_K], the right singular vectors of M = X S Y^dag.
// Neither Q nor the rotations are accumulated: the right-canonical reassembly
// needs only S and Y.  Pivoted QR is the Drmac-Veselic preconditioner: the
// lambda-graded sectors of an MPS (singular values over 10-15 decades) need
// 20-35 plain Jacobi sweeps but 6-8 after it.
//
// Wide sectors (cluster kernels, n >= 1.25 m): R^dag has m columns of length n; an
// unpivoted Householder QR R^dag = Q2 [R2; 0] lets the sweeps rotate the columns of the
// m x m factor R2 instead (the same rotations orthogonalise both), and
// Y = P Q2 [normalised columns; 0] is formed at the end, one warp per column.
//
// Storage: M is kept row-major with an odd leading dimension ld >= n, so the QR
// rank-1 updates are coalesced (32 consecutive columns per warp) and, once R's
// rows are conjugated in place, they are the contiguous columns of R^dag.
// GB300 runs FP64 at 2 FMA/clk/SM, so one SM per large sector would leave a
// layer waiting on its largest sectors.  Three kernels share the work:
//   jacobi_cta_kernel:           one CTA per sector, all of it in shared memory,
//                                round-robin pair ordering;
//   jacobi_cluster_block_kernel: a thread-block cluster of 2, 4, 8 (or 16) CTAs per
//                                large sector, data in L2 (ld.global.cg /
//                                st.global.cg, no stale L1 lines across SMs), block
//                                Jacobi with the block pairs of a round staged in
//                                shared memory, CTA barriers between the steps of a
//                                round and the hardware cluster barrier between rounds;
//   jacobi_cluster_kernel:       the same data placement with round-robin pairs and
//                                register-cached columns, for sectors whose blocks do
//                                not fit in shared memory.
// Column pairs of a step are shared by groups of 8, 16 or 32 lanes (an FP64 warp
// instruction costs the same at any lane count on this part, so a warp does several
// pairs at once).  A pair is rotated when |a_p^dag a_q|^2 > tol^2 |a_p|^2 |a_q|^2,
// tol = eps * max(n, 32), and both columns are above the floor: the noise level
// 32 eps |M|_F, or a higher deflation level the caller sets (SvdSector::floor_rel,
// a fraction of the truncation cutoff, and SvdSector::floor_abs, a fraction of the
// bond's previous cut); singular values at or below the floor are reported as
// exactly 0.
// Convergence is a sweep without a rotation; a sector that does not converge
// within the sweep limit reports -1.  FP64 costs a warp 64 cycles per
// instruction here, so per-pair scalar work is kept small (no square root in the
// test; at most two rsqrt, one sqrt and one division per rotation; column norms tracked through the
// exact 2x2 relations within a sweep).
#include <algorithm>
#include <type_traits>
#include <atomic>
#include <mutex>
#include <vector>

#include "mps_internal.h"

namespace mps {
namespace {

constexpr double kEps = 2.220446049250313e-16;
constexpr int kMaxCached = 16;          // rows cached in registers per lane (n <= 512)
constexpr int kMaxCluster = 16;
constexpr int kMaxWarps = 16;
constexpr int kBlockThreads = 192;      // block-Jacobi cluster kernel: 6 warps per CTA, 2 CTAs per SM
constexpr int kMaxStaged = 16;          // block pairs staged at once by one block-Jacobi CTA

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

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

// Memory access policy: plain (shared memory) or L2-only (cluster, global memory).
struct PlainMem {
  static constexpr bool kCache = false;
  template <typename T> static __device__ __forceinline__ T ld(const T* p) { return *p; }
  template <typename T> static __device__ __forceinline__ void st(T* p, T v) { *p = v; }
};
struct L2Mem {
  static constexpr bool kCache = true;    // load each column pair once per round
  static __device__ __forceinline__ double2 ld(const double2* p) { return __ldcg(p); }
  static __device__ __forceinline__ double ld(const double* p) { return __ldcg(p); }
  static __device__ __forceinline__ int ld(const int* p) { return __ldcg(p); }
  static __device__ __forceinline__ void st(double2* p, double2 v) { __stcg(p, v); }
  static __device__ __forceinline__ void st(double* p, double v) { __stcg(p, v); }
  static __device__ __forceinline__ void st(int* p, int v) { __stcg(p, v); }
};

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}

struct Rot { double c, u, v; };   // c = cos, (u + i v) = sin * gamma / |gamma|

__device__ __forceinline__ void rotate_pair(double2& x, double2& y, const Rot& R) {
  // x' = c x - s conj(e) y ;  y' = s e x + c y   with s e = u + i v
  const double2 xo = x, yo = y;
  x.x = fma(R.c, xo.x, -fma(R.u, yo.x, R.v * yo.y));
  x.y = fma(R.c, xo.y, -fma(R.u, yo.y, -R.v * yo.x));
  y.x = fma(R.c, yo.x, fma(R.u, xo.x, -R.v * xo.y));
  y.y = fma(R.c, yo.y, fma(R.u, xo.y, R.v * xo.x));
}

// One warp: orthogonalise columns p, q (length R, stride ld) of the Jacobi matrix.
// nrm holds squared column norms, updated by alpha' = alpha - t|g|, beta' = beta + t|g|.
template <class Mem>
__device__ bool jacobi_pair(double2* A, int R, int ld, double* nrm, int p, int q, double tol2, double floor2) {
  const int lane = threadIdx.x & 31;
  const double alpha = Mem::ld(nrm + p), beta = Mem::ld(nrm + q);
  if (fmin(alpha, beta) <= floor2) return false;      // a noise column: nothing to orthogonalise
  double2* ap = A + (int64_t)p * ld;
  double2* aq = A + (int64_t)q * ld;
  const bool cached = Mem::kCache && R <= 32 * kMaxCached;
  double2 xs[kMaxCached], ys[kMaxCached];
  double gr = 0.0, gi = 0.0;
  if (cached) {
#pragma unroll
    for (int t = 0; t < kMaxCached; ++t) {
      const int i = lane + 32 * t;
      xs[t] = make_double2(0.0, 0.0);
      ys[t] = make_double2(0.0, 0.0);
      if (i < R) {
        xs[t] = Mem::ld(ap + i);
        ys[t] = Mem::ld(aq + i);
      }
    }
#pragma unroll
    for (int t = 0; t < kMaxCached; ++t) {
      if (32 * t < R) {
        gr = fma(xs[t].x, ys[t].x, fma(xs[t].y, ys[t].y, gr));
        gi = fma(xs[t].x, ys[t].y, fma(-xs[t].y, ys[t].x, gi));
      }
    }
  } else {
    for (int i = lane; i < R; i += 32) {
      const double2 x = Mem::ld(ap + i), y = Mem::ld(aq + i);
      gr = fma(x.x, y.x, fma(x.y, y.y, gr));
      gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
    }
  }
  gr = warp_sum(gr);
  gi = warp_sum(gi);
  const double g2 = fma(gr, gr, gi * gi);
  if (!(g2 > tol2 * alpha * beta)) return false;       // orthogonal to tolerance
  // 2x2 Hermitian Gram [[alpha, gamma], [conj(gamma), beta]] -> diagonal
  const double inv_g = rsqrt(g2);
  const double g = g2 * inv_g;
  const double zeta = (beta - alpha) * (0.5 * inv_g);
  const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
  Rot Rt;
  Rt.c = rsqrt(fma(t, t, 1.0));
  const double s_over_g = Rt.c * t * inv_g;
  Rt.u = s_over_g * gr;
  Rt.v = s_over_g * gi;
  if (cached) {
#pragma unroll
    for (int k = 0; k < kMaxCached; ++k) {
      const int i = lane + 32 * k;
      if (32 * k < R) {
        rotate_pair(xs[k], ys[k], Rt);
        if (i < R) {
          Mem::st(ap + i, xs[k]);
          Mem::st(aq + i, ys[k]);
        }
      }
    }
  } else {
    for (int i = lane; i < R; i += 32) {
      double2 x = Mem::ld(ap + i), y = Mem::ld(aq + i);
      rotate_pair(x, y, Rt);
      Mem::st(ap + i, x);
      Mem::st(aq + i, y);
    }
  }
  if (lane == 0) {
    const double tg = t * g;
    Mem::st(nrm + p, fmax(alpha - tg, 0.0));
    Mem::st(nrm + q, beta + tg);
  }
  return true;
}

// G lanes (G = 8, 16 or 32; groups aligned within the warp) orthogonalise columns p, q
// (length R, column c at A + c * ld) of a shared-memory matrix, so that one warp works
// on 32 / G pairs at once.  On this part every FP64 warp instruction costs the same
// whatever its lane count, so the group-wide reduction and the scalar rotation
// parameters, which all lanes of a group compute redundantly, are shared by the
// 32 / G pairs of a warp instead of being paid per pair.  Lanes of an invalid slot only
// take part in the shuffles.  The rotation follows from the 2x2 Gram matrix
// [[alpha, g], [conj g, beta]] with tau = tan(theta) / |g| = 2 sign(D) / (|D| + sqrt(D^2 + 4|g|^2)),
// D = beta - alpha, which avoids a separate 1 / |g|; norms update by -/+ tau |g|^2.
__device__ bool jacobi_pair_grp(double2* A, int R, int ld, double* nrm, int p, int q, bool valid, int G,
                                double tol2, double floor2) {
  const int gl = threadIdx.x & (G - 1);
  double alpha = 0.0, beta = 0.0;
  if (valid) {
    alpha = nrm[p];
    beta = nrm[q];
  }
  bool act = valid && fmin(alpha, beta) > floor2;   // noise columns are left alone
  double2* ap = A + (int64_t)(act ? p : 0) * ld;
  double2* aq = A + (int64_t)(act ? q : 0) * ld;
  // two independent partial sums per component halve the FP64 dependency chains (the
  // FP64 pipe's latency, not its issue rate, bounds a lone chain)
  double gr = 0.0, gi = 0.0;
  if (act) {
    double gr1 = 0.0, gi1 = 0.0;
    int i = gl;
    for (; i + G < R; i += 2 * G) {
      const double2 x = ap[i], y = aq[i], x1 = ap[i + G], y1 = aq[i + G];
      gr = fma(x.x, y.x, fma(x.y, y.y, gr));
      gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
      gr1 = fma(x1.x, y1.x, fma(x1.y, y1.y, gr1));
      gi1 = fma(x1.x, y1.y, fma(-x1.y, y1.x, gi1));
    }
    if (i < R) {
      const double2 x = ap[i], y = aq[i];
      gr = fma(x.x, y.x, fma(x.y, y.y, gr));
      gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
    }
    gr += gr1;
    gi += gi1;
  }
  for (int o = G >> 1; o; o >>= 1) {
    gr += __shfl_xor_sync(0xffffffffu, gr, o);
    gi += __shfl_xor_sync(0xffffffffu, gi, o);
  }
  const double g2 = fma(gr, gr, gi * gi);
  act = act && (g2 > tol2 * alpha * beta);           // orthogonal to tolerance otherwise
  if (act) {
    const double delta = beta - alpha;
    const double tau = copysign(2.0, delta) / (fabs(delta) + sqrt(fma(delta, delta, 4.0 * g2)));
    Rot Rt;
    Rt.c = rsqrt(fma(tau * tau, g2, 1.0));
    const double ct = Rt.c * tau;
    Rt.u = ct * gr;
    Rt.v = ct * gi;
#pragma unroll 2
    for (int i = gl; i < R; i += G) {
      double2 x = ap[i], y = aq[i];
      rotate_pair(x, y, Rt);
      ap[i] = x;
      aq[i] = y;
    }
    if (gl == 0) {
      const double tg = tau * g2;
      nrm[p] = fmax(alpha - tg, 0.0);
      nrm[q] = beta + tg;
    }
  }
  return act;
}

// Group width for P disjoint pairs of columns of length R spread over nwarps warps:
// the width with the fewest FP64 warp instructions per warp, counting the passes
// needed (ceil(P / slots)) times the instructions of one pass (about 16 per column
// element a lane holds, plus about 50 for the reduction and the rotation parameters).
__device__ __forceinline__ int group_width(int P, int R, int nwarps) {
  int best = 32;
  long long best_cost = -1;
  for (int G = 32; G >= 8; G >>= 1) {
    const int slots = nwarps * (32 / G);
    const long long cost = (long long)((P + slots - 1) / slots) * (16 * ((R + G - 1) / G) + 50);
    if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = G; }
  }
  return best;
}

// The same for a group of G = 32 wg lanes (wg > 1 whole warps, groups aligned to wg warps)
// per pair, for steps with fewer disjoint pairs than warps (the large sectors, whose column
// blocks hold only 3-5 columns): each warp reduces its part of the dot product with shuffles
// and the group sums the warp partials through shared memory behind a named barrier (id
// bar_id, one per group).  red holds two buffers of 2 doubles per warp, used alternately
// (phase), so a warp that runs ahead into the next pair never overwrites partials still read.
__device__ bool jacobi_pair_mw(double2* A, int R, int ld, double* nrm, int p, int q, bool valid, int G,
                               double tol2, double floor2, double* red, int& phase, int bar_id) {
  const int wg = G >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w0 = warp - warp % wg, gl = (warp - w0) * 32 + lane;
  double* rb = red + phase * 2 * kMaxWarps;
  phase ^= 1;
  double alpha = 0.0, beta = 0.0;
  if (valid) {
    alpha = nrm[p];
    beta = nrm[q];
  }
  bool act = valid && fmin(alpha, beta) > floor2;
  double2* ap = A + (int64_t)(act ? p : 0) * ld;
  double2* aq = A + (int64_t)(act ? q : 0) * ld;
  double gr = 0.0, gi = 0.0;
  if (act) {
    double gr1 = 0.0, gi1 = 0.0;
    int i = gl;
    for (; i + G < R; i += 2 * G) {
      const double2 x = ap[i], y = aq[i], x1 = ap[i + G], y1 = aq[i + G];
      gr = fma(x.x, y.x, fma(x.y, y.y, gr));
      gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
      gr1 = fma(x1.x, y1.x, fma(x1.y, y1.y, gr1));
      gi1 = fma(x1.x, y1.y, fma(-x1.y, y1.x, gi1));
    }
    if (i < R) {
      const double2 x = ap[i], y = aq[i];
      gr = fma(x.x, y.x, fma(x.y, y.y, gr));
      gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
    }
    gr += gr1;
    gi += gi1;
  }
  gr = warp_sum(gr);
  gi = warp_sum(gi);
  if (lane == 0) {
    rb[2 * warp] = gr;
    rb[2 * warp + 1] = gi;
  }
  asm volatile("bar.sync %0, %1;\n" ::"r"(bar_id), "r"(G) : "memory");
  gr = 0.0;
  gi = 0.0;
  for (int x = 0; x < wg; ++x) {        // the same order in every warp of the group
    gr += rb[2 * (w0 + x)];
    gi += rb[2 * (w0 + x) + 1];
  }
  const double g2 = fma(gr, gr, gi * gi);
  act = act && (g2 > tol2 * alpha * beta);
  if (act) {
    const double delta = beta - alpha;
    const double tau = copysign(2.0, delta) / (fabs(delta) + sqrt(fma(delta, delta, 4.0 * g2)));
    Rot Rt;
    Rt.c = rsqrt(fma(tau * tau, g2, 1.0));
    const double ct = Rt.c * tau;
    Rt.u = ct * gr;
    Rt.v = ct * gi;
#pragma unroll 2
    for (int i = gl; i < R; i += G) {
      double2 x = ap[i], y = aq[i];
      rotate_pair(x, y, Rt);
      ap[i] = x;
      aq[i] = y;
    }
    if (gl == 0) {
      const double tg = tau * g2;
      nrm[p] = fmax(alpha - tg, 0.0);
      nrm[q] = beta + tg;
    }
  }
  return act;
}

// Group width for P disjoint pairs of length R over nwarps warps, multi-warp groups
// included (wg warps per pair, wg dividing nwarps; about 40 more instructions per pass for
// the shared-memory reduction).  Returns G; slots() gives the pairs one pass covers.
__device__ __forceinline__ int group_width_mw(int P, int R, int nwarps) {
  int best = 32;
  long long best_cost = -1;
  for (int G = 8; G <= 32 * nwarps; G = (G < 32) ? 2 * G : G + 32) {
    if (G > 32 && nwarps % (G >> 5) != 0) continue;
    const int slots = G <= 32 ? nwarps * (32 / G) : nwarps / (G >> 5);
    const long long cost =
        (long long)((P + slots - 1) / slots) * (16 * ((R + G - 1) / G) + 50 + (G > 32 ? 40 : 0));
    if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = G; }
  }
  return best;
}
__device__ __forceinline__ int group_slots(int G, int nwarps) { return G <= 32 ? nwarps * (32 / G) : nwarps / (G >> 5); }
__device__ __forceinline__ int group_slot(int G) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  return G <= 32 ? warp * (32 / G) + lane / G : warp / (G >> 5);
}

// Bulk copies (the TMA engine, no tensor map) of whole staged columns: a column of the Jacobi
// matrix is contiguous in global memory and in the staging area, 16-byte aligned, a multiple of
// 16 bytes long.  One thread issues them; the CTA waits on an mbarrier (loads) or the issuing
// thread on the bulk group (stores).  Global data crosses between the generic and the async
// proxy only behind fence.proxy.async and the cluster barrier.
__device__ __forceinline__ uint32_t sh_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void stage_bar_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sh_addr(b)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void stage_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sh_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   sh_addr(dst)),
               "l"(src), "r"(bytes), "r"(sh_addr(b))
               : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(sh_addr(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_store_drain() {
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
  asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
  asm volatile("fence.proxy.async.global;\n" ::: "memory");
}
__device__ __forceinline__ void fence_to_async() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }
// Bounded wait (about 2 s) for the staging barrier's phase; false when it expired.
__device__ __forceinline__ bool stage_wait(uint64_t* b, uint32_t parity) {
  const uint32_t a = sh_addr(b);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 4000000000LL) return false;
  }
}

// Per-sector working set (shared memory or global scratch).
struct Work {
  double2* W;     // m x ld, row-major: M, then R (rows 0..K-1), then R^dag's columns
  double2* u;     // m: Householder vector of the current step
  double* nu;     // n: partial squared column norms for pivoting
  double* nu0;    // n: their reference values (recompute when cancellation sets in)
  int* perm;      // n: column permutation P
  double* nrm;    // K: Jacobi column norms / singular values
  int* ord;       // K: descending order of the singular values
  int* flags;     // max_sweeps + 1: rotation seen in sweep s
  double* pv;     // per-CTA pivot candidates (value)
  int* pi;        // per-CTA pivot candidates (index)
  double* scal;   // [0] = 2 / u^dag u, [1] = |M|_F^2
};

__host__ __device__ inline int odd_ld(int n) { return n | 1; }

// Round-robin Jacobi sweeps: every round's disjoint pairs spread over all warps that
// share the sector, one barrier per round.
template <class Mem>
struct JacobiRoundRobin {
  template <class Sync>
  __device__ int operator()(double2* W, int n, int ld, int K, const Work& w, int rank, int nctas, Sync sync,
                            double tol2, double floor2, int max_sweeps, bool& converged) const {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int worker = rank * nwarps + warp, workers = nctas * nwarps;
    const int mp = K + (K & 1);
    int sweep = 0;
    converged = K < 2;
    for (; !converged && sweep < max_sweeps; ++sweep) {
      if (sweep > 0) {          // fresh squared norms at the start of every sweep
        for (int j = worker; j < K; j += workers) {
          const double2* a = W + (int64_t)j * ld;
          double acc = 0.0;
          for (int i = lane; i < n; i += 32) {
            const double2 x = Mem::ld(a + i);
            acc = fma(x.x, x.x, fma(x.y, x.y, acc));
          }
          acc = warp_sum(acc);
          if (lane == 0) Mem::st(w.nrm + j, acc);
        }
        sync();
      }
      for (int r = 0; r < mp - 1; ++r) {
        bool rot = false;
        if constexpr (!Mem::kCache) {   // shared memory: several pairs per warp
          const int G = group_width(mp / 2, n, workers), per = 32 / G, slot = worker * per + lane / G;
          for (int base = 0; base < mp / 2; base += workers * per) {
            const int kk = base + slot;
            int p = 0, q = 0;
            if (kk < mp / 2) rr_pair(kk, r, mp, p, q);
            const bool valid = kk < mp / 2 && p < K && q < K;
            rot |= jacobi_pair_grp(W, n, ld, w.nrm, min(p, q), max(p, q), valid, G, tol2, floor2);
          }
          if (rot) Mem::st(w.flags + sweep, 1);
        } else {
          for (int kk = worker; kk < mp / 2; kk += workers) {
            int p, q;
            rr_pair(kk, r, mp, p, q);
            if (p >= K || q >= K) continue;
            if (p > q) { const int t = p; p = q; q = t; }
            rot |= jacobi_pair<Mem>(W, n, ld, w.nrm, p, q, tol2, floor2);
          }
          if (rot && lane == 0) Mem::st(w.flags + sweep, 1);
        }
        sync();
      }
      converged = Mem::ld(w.flags + sweep) == 0;
    }
    return sweep;
  }
};

// Block-Jacobi sweeps for a cluster sector (data in L2).  The K columns form
// nb = 2 * nctas * g contiguous blocks; in block round r the blocks are paired by the
// round-robin ordering and CTA `rank` takes the pairs rank, rank + nctas, ... (g of
// them), staging gs of them at a time (both blocks and their norms) in shared memory.
// For the staged pairs it orthogonalises, in round 0, every pair inside each block
// (round-robin inside the block) and then every cross pair (cyclic shifts of the
// larger block against the smaller), all staged block pairs advancing together so
// that each step has about gs * K / nb disjoint pairs for the warp groups; steps are
// separated by CTA barriers, the round by one cluster barrier.  Every pair is visited
// once per sweep.
struct JacobiBlocks {
  double2* sm;   // 2 * gs * bsmax columns of n complex (shared memory)
  double* smn;   // 2 * gs * bsmax norms (shared memory)
  int bsmax;
  int g;         // block pairs per CTA and round
  int gs;        // block pairs staged at once
  template <class Sync>
  __device__ int operator()(double2* W, int n, int ld, int K, const Work& w, int rank, int nctas, Sync sync,
                            double tol2, double floor2, int max_sweeps, bool& converged) const {
    __shared__ int s_rot;
    __shared__ double s_red[2 * 2 * kMaxWarps];   // multi-warp pair partials, two buffers
    __shared__ __align__(8) uint64_t s_bar;       // staging loads
    int mw_phase = 0;
    uint32_t stage_parity = 0;
    if (threadIdx.x == 0) stage_bar_init(&s_bar);
    __syncthreads();
    __shared__ int s_col[2 * kMaxStaged];   // first column of each staged block
    __shared__ int s_len[2 * kMaxStaged];   // its width (0: slot unused)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int worker = rank * nwarps + warp, workers = nctas * nwarps;
    const int nb = 2 * nctas * g;
    int sweep = 0;
    converged = K < 2;
    for (; !converged && sweep < max_sweeps; ++sweep) {
      if (sweep > 0) {
        for (int j = worker; j < K; j += workers) {
          const double2* a = W + (int64_t)j * ld;
          double acc = 0.0;
          for (int i = lane; i < n; i += 32) {
            const double2 x = __ldcg(a + i);
            acc = fma(x.x, x.x, fma(x.y, x.y, acc));
          }
          acc = warp_sum(acc);
          if (lane == 0) __stcg(w.nrm + j, acc);
        }
        sync();
      }
      if (tid == 0) s_rot = 0;
      bool rot = false;
      for (int r = 0; r < nb - 1; ++r) {
        for (int c0 = 0; c0 < g; c0 += gs) {        // chunks of gs block pairs of this CTA
          const int ns = min(gs, g - c0);
          if (tid < 2 * gs) {
            const int j = tid >> 1;
            int col = 0, len = 0;
            if (j < ns) {
              int bp, bq;
              rr_pair(rank + (c0 + j) * nctas, r, nb, bp, bq);
              const int b = (tid & 1) ? bq : bp;
              col = (int)((int64_t)K * b / nb);
              len = (int)((int64_t)K * (b + 1) / nb) - col;
            }
            s_col[tid] = col;
            s_len[tid] = len;
          }
          __syncthreads();
          // stage: block slot j occupies columns [j * bsmax, j * bsmax + len) of sm, one bulk
          // copy per column
          if (tid == 0) {
            uint32_t bytes = 0;
            for (int j = 0; j < 2 * ns; ++j) bytes += (uint32_t)s_len[j] * (uint32_t)n * 16u;
            fence_to_async();
            stage_expect(&s_bar, bytes);
            for (int j = 0; j < 2 * ns; ++j)
              for (int c = 0; c < s_len[j]; ++c)
                bulk_load(sm + ((int64_t)j * bsmax + c) * n, W + (int64_t)(s_col[j] + c) * ld, (uint32_t)n * 16u,
                          &s_bar);
          }
          for (int j = 0; j < 2 * ns; ++j)
            for (int c = tid; c < s_len[j]; c += blockDim.x) smn[j * bsmax + c] = __ldcg(w.nrm + s_col[j] + c);
          stage_wait(&s_bar, stage_parity);
          stage_parity ^= 1u;
          __syncthreads();
          if (r == 0) {   // pairs inside each staged block, round-robin within the block
            const int mpb = bsmax + (bsmax & 1);
            const int P = 2 * ns * (mpb / 2);
            const int G = group_width_mw(P, n, nwarps), slots = group_slots(G, nwarps), slot = group_slot(G);
            for (int rr = 0; rr < mpb - 1; ++rr) {
              for (int base = 0; base < P; base += slots) {
                const int k = base + slot, j = k / (mpb / 2);
                int a = 0, b = 0;
                bool valid = k < P;
                if (valid) {
                  rr_pair(k % (mpb / 2), rr, mpb, a, b);
                  valid = a < s_len[j] && b < s_len[j];
                }
                if (G <= 32)
                  rot |= jacobi_pair_grp(sm, n, n, smn, j * bsmax + min(a, b), j * bsmax + max(a, b), valid, G,
                                         tol2, floor2);
                else
                  rot |= jacobi_pair_mw(sm, n, n, smn, j * bsmax + min(a, b), j * bsmax + max(a, b), valid, G,
                                        tol2, floor2, s_red, mw_phase, 1 + slot);
              }
              __syncthreads();
            }
          }
          {   // cross pairs: block slots 2j and 2j + 1, the smaller block shifted against the larger
            const int P = ns * bsmax;
            const int G = group_width_mw(P, n, nwarps), slots = group_slots(G, nwarps), slot = group_slot(G);
            for (int t = 0; t < bsmax; ++t) {
              for (int base = 0; base < P; base += slots) {
                const int k = base + slot, j = k / bsmax, i = k % bsmax;
                int p = 0, q = 0;
                bool valid = false;
                if (k < P) {
                  const int la = s_len[2 * j], lb = s_len[2 * j + 1];
                  const bool swap = la > lb;
                  const int sa = swap ? lb : la, sb = swap ? la : lb;
                  valid = i < sa && t < sb;
                  if (valid) {
                    const int pa = (2 * j + (swap ? 1 : 0)) * bsmax + i;
                    const int pb = (2 * j + (swap ? 0 : 1)) * bsmax + (i + t) % sb;
                    p = min(pa, pb);
                    q = max(pa, pb);
                  }
                }
                if (G <= 32)
                  rot |= jacobi_pair_grp(sm, n, n, smn, p, q, valid, G, tol2, floor2);
                else
                  rot |= jacobi_pair_mw(sm, n, n, smn, p, q, valid, G, tol2, floor2, s_red, mw_phase, 1 + slot);
              }
              __syncthreads();
            }
          }
          if (tid == 0) {   // write the staged columns back, one bulk copy each
            for (int j = 0; j < 2 * ns; ++j)
              for (int c = 0; c < s_len[j]; ++c)
                bulk_store(W + (int64_t)(s_col[j] + c) * ld, sm + ((int64_t)j * bsmax + c) * n, (uint32_t)n * 16u);
            bulk_store_drain();
          }
          for (int j = 0; j < 2 * ns; ++j)
            for (int c = tid; c < s_len[j]; c += blockDim.x) __stcg(w.nrm + s_col[j] + c, smn[j * bsmax + c]);
          __syncthreads();   // the next chunk reuses the staging buffers and block tables
        }
        sync();
      }
      if (rot) s_rot = 1;
      __syncthreads();
      if (tid == 0 && s_rot) __stcg(w.flags + sweep, 1);
      sync();
      converged = __ldcg(w.flags + sweep) == 0;
    }
    return sweep;
  }
};

// ---------------------------------------------------------------------------------------
// Mixed-precision preconditioning of a cluster sector (after Gao, Ma and Shao, "A mixed
// precision Jacobi SVD algorithm", 2022).  The Jacobi matrix J (jlen x K, FP64) is rounded to
// FP32 and stacked on the identity, F = [fl32(J); I]; FP32 one-sided Jacobi sweeps rotate the
// columns of both (the dot products run over the J rows only), so that the lower block
// accumulates the rotations V.  One-sided Jacobi is column-wise relatively accurate, so J V has
// relatively orthogonal columns to about FP32 precision even for columns 10-15 decades below
// the largest.  The columns whose FP32 norm is above a tenth of the deflation floor are kept,
// V is made unitary in FP64 by one Cholesky QR (V^dag V = U^dag U, V <- V U^-1; V is unitary to
// about 1e-5, so one pass leaves it unitary to rounding), and A1 = J V (FP64) starts the FP64
// sweeps, which then converge in 2-3 sweeps instead of 7-12.  The singular values of A1 are
// those of J (V unitary), and the FP64 sweeps make them and the vectors FP64-accurate; columns
// left out lie below the floor anyway.  FP32 runs at 64x the FP64 rate on this part.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// G lanes (8, 16 or 32) orthogonalise columns p, q of an FP32 matrix: the dot product over the
// first R rows, the rotation over the first Rr rows.  Tests and parameters avoid squaring the
// (possibly tiny) inner product: |g| against tol sqrt(alpha beta), t = tan(theta) from
// zeta = (beta - alpha) / (2 |g|).
__device__ bool jacobi_pair32(float2* A, int R, int Rr, int ld, float* nrm, int p, int q, bool valid, int G,
                              float tol, float floor2) {
  const int gl = threadIdx.x & (G - 1);
  float alpha = 0.f, beta = 0.f;
  if (valid) {
    alpha = nrm[p];
    beta = nrm[q];
  }
  bool act = valid && fminf(alpha, beta) > floor2;
  float2* ap = A + (int64_t)(act ? p : 0) * ld;
  float2* aq = A + (int64_t)(act ? q : 0) * ld;
  float gr = 0.f, gi = 0.f;
  if (act)
    for (int i = gl; i < R; i += G) {
      const float2 x = ap[i], y = aq[i];
      gr = fmaf(x.x, y.x, fmaf(x.y, y.y, gr));
      gi = fmaf(x.x, y.y, fmaf(-x.y, y.x, gi));
    }
  for (int o = G >> 1; o; o >>= 1) {
    gr += __shfl_xor_sync(0xffffffffu, gr, o);
    gi += __shfl_xor_sync(0xffffffffu, gi, o);
  }
  const float ag = hypotf(gr, gi);
  act = act && (ag > tol * sqrtf(alpha) * sqrtf(beta));
  if (act) {
    const float zeta = (beta - alpha) / (2.f * ag), az = fabsf(zeta);
    const float t = copysignf(1.f, zeta) / (az + (az < 1e18f ? sqrtf(fmaf(zeta, zeta, 1.f)) : az));
    const float c = rsqrtf(fmaf(t, t, 1.f));
    const float ct = c * t / ag;
    const float u = ct * gr, v = ct * gi;
    for (int i = gl; i < Rr; i += G) {
      const float2 x = ap[i], y = aq[i];
      ap[i] = make_float2(fmaf(c, x.x, -fmaf(u, y.x, v * y.y)), fmaf(c, x.y, -fmaf(u, y.y, -v * y.x)));
      aq[i] = make_float2(fmaf(c, y.x, fmaf(u, x.x, -v * x.y)), fmaf(c, y.y, fmaf(u, x.y, v * x.x)));
    }
    if (gl == 0) {
      const float tg = t * ag;
      nrm[p] = fmaxf(alpha - tg, 0.f);
      nrm[q] = beta + tg;
    }
  }
  return act;
}

__device__ __forceinline__ int group_width32(int P, int R, int nwarps) {
  int best = 32;
  long long best_cost = -1;
  for (int G = 32; G >= 8; G >>= 1) {
    const int slots = nwarps * (32 / G);
    const long long cost = (long long)((P + slots - 1) / slots) * (2 * ((R + G - 1) / G) + 30);
    if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = G; }
  }
  return best;
}

// FP32 block-Jacobi sweeps over the K columns of F (column c at F + c * ld): the same block
// ordering as JacobiBlocks, columns of Rr FP32 complex staged whole in shared memory (the
// FP64 kernel's staging area holds them: 8 (jlen + K) <= 16 jlen bytes per column), dot
// products over the first R rows.  Returns the sweeps used (converged: a sweep without a
// rotation).  flags: max_sweeps + 1 ints, zero on entry.
struct JacobiBlocks32 {
  float2* sm;
  float* smn;
  int bsmax, g, gs;
  template <class Sync>
  __device__ int operator()(float2* F, int R, int Rr, int ld, int K, float* nrm, int* flags, int rank, int nctas,
                            Sync sync, float tol, float floor2, int max_sweeps, bool& converged) const {
    __shared__ int s_rot32;
    __shared__ int s_col32[2 * kMaxStaged];
    __shared__ int s_len32[2 * kMaxStaged];
    __shared__ __align__(8) uint64_t s_bar32;
    uint32_t stage_parity = 0;
    if (threadIdx.x == 0) stage_bar_init(&s_bar32);
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int worker = rank * nwarps + warp, workers = nctas * nwarps;
    const int nb = 2 * nctas * g;
    int sweep = 0;
    converged = K < 2;
    for (; !converged && sweep < max_sweeps; ++sweep) {
      for (int j = worker; j < K; j += workers) {   // fresh squared norms over the J rows
        const float2* a = F + (int64_t)j * ld;
        float acc = 0.f;
        for (int i = lane; i < R; i += 32) {
          const float2 x = __ldcg(a + i);
          acc = fmaf(x.x, x.x, fmaf(x.y, x.y, acc));
        }
        acc = warp_sum_f(acc);
        if (lane == 0) __stcg(nrm + j, acc);
      }
      sync();
      if (tid == 0) s_rot32 = 0;
      bool rot = false;
      for (int r = 0; r < nb - 1; ++r) {
        for (int c0 = 0; c0 < g; c0 += gs) {
          const int ns = min(gs, g - c0);
          if (tid < 2 * gs) {
            const int j = tid >> 1;
            int col = 0, len = 0;
            if (j < ns) {
              int bp, bq;
              rr_pair(rank + (c0 + j) * nctas, r, nb, bp, bq);
              const int b = (tid & 1) ? bq : bp;
              col = (int)((int64_t)K * b / nb);
              len = (int)((int64_t)K * (b + 1) / nb) - col;
            }
            s_col32[tid] = col;
            s_len32[tid] = len;
          }
          __syncthreads();
          // one bulk copy per column (ld is even: every column starts 16-byte aligned and is
          // ld FP32 complex long, a multiple of 16 bytes; the staging stride is ld too)
          if (tid == 0) {
            uint32_t bytes = 0;
            for (int j = 0; j < 2 * ns; ++j) bytes += (uint32_t)s_len32[j] * (uint32_t)ld * 8u;
            fence_to_async();
            stage_expect(&s_bar32, bytes);
            for (int j = 0; j < 2 * ns; ++j)
              for (int c = 0; c < s_len32[j]; ++c)
                bulk_load(sm + ((int64_t)j * bsmax + c) * ld, F + (int64_t)(s_col32[j] + c) * ld, (uint32_t)ld * 8u,
                          &s_bar32);
          }
          for (int j = 0; j < 2 * ns; ++j)
            for (int c = tid; c < s_len32[j]; c += blockDim.x) smn[j * bsmax + c] = __ldcg(nrm + s_col32[j] + c);
          stage_wait(&s_bar32, stage_parity);
          stage_parity ^= 1u;
          __syncthreads();
          if (r == 0) {
            const int mpb = bsmax + (bsmax & 1);
            const int P = 2 * ns * (mpb / 2);
            const int G = group_width32(P, R, nwarps), per = 32 / G, slot = warp * per + lane / G;
            for (int rr = 0; rr < mpb - 1; ++rr) {
              for (int base = 0; base < P; base += nwarps * per) {
                const int k = base + slot, j = k / (mpb / 2);
                int a = 0, b = 0;
                bool valid = k < P;
                if (valid) {
                  rr_pair(k % (mpb / 2), rr, mpb, a, b);
                  valid = a < s_len32[j] && b < s_len32[j];
                }
                rot |= jacobi_pair32(sm, R, Rr, ld, smn, j * bsmax + min(a, b), j * bsmax + max(a, b), valid, G,
                                     tol, floor2);
              }
              __syncthreads();
            }
          }
          {
            const int P = ns * bsmax;
            const int G = group_width32(P, R, nwarps), per = 32 / G, slot = warp * per + lane / G;
            for (int t = 0; t < bsmax; ++t) {
              for (int base = 0; base < P; base += nwarps * per) {
                const int k = base + slot, j = k / bsmax, i = k % bsmax;
                int p = 0, q = 0;
                bool valid = false;
                if (k < P) {
                  const int la = s_len32[2 * j], lb = s_len32[2 * j + 1];
                  const bool swap = la > lb;
                  const int sa = swap ? lb : la, sb = swap ? la : lb;
                  valid = i < sa && t < sb;
                  if (valid) {
                    const int pa = (2 * j + (swap ? 1 : 0)) * bsmax + i;
                    const int pb = (2 * j + (swap ? 0 : 1)) * bsmax + (i + t) % sb;
                    p = min(pa, pb);
                    q = max(pa, pb);
                  }
                }
                rot |= jacobi_pair32(sm, R, Rr, ld, smn, p, q, valid, G, tol, floor2);
              }
              __syncthreads();
            }
          }
          if (tid == 0) {
            for (int j = 0; j < 2 * ns; ++j)
              for (int c = 0; c < s_len32[j]; ++c)
                bulk_store(F + (int64_t)(s_col32[j] + c) * ld, sm + ((int64_t)j * bsmax + c) * ld, (uint32_t)ld * 8u);
            bulk_store_drain();
          }
          for (int j = 0; j < 2 * ns; ++j)
            for (int c = tid; c < s_len32[j]; c += blockDim.x) __stcg(nrm + s_col32[j] + c, smn[j * bsmax + c]);
          __syncthreads();
        }
        sync();
      }
      if (rot) s_rot32 = 1;
      __syncthreads();
      if (tid == 0 && s_rot32) __stcg(flags + sweep, 1);
      sync();
      converged = __ldcg(flags + sweep) == 0;
    }
    return sweep;
  }
};
struct NoJacobi32 {};

// The mixed-precision start of a cluster sector's sweeps (see above).  J: jlen x K, column c at
// J + c * jld (FP64, L2).  On return the FP64 Jacobi matrix is S.a1 (same jld), its first
// *nsel_out columns J V and the rest zero.  Every CTA of the cluster calls it.
template <class Sync>
__device__ void mixed_precondition(const SvdSector& S, const Work& w, const double2* J, int jlen, int jld, int K,
                                   int rank, int nctas, Sync sync, double floor2, int max_sweeps,
                                   const JacobiBlocks32& j32, int* nsel_out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int tid_all = rank * blockDim.x + tid, threads_all = nctas * blockDim.x;
  const int worker = rank * nwarps + warp, workers = nctas * nwarps;
  const int Rr = jlen + K, fld = (Rr + 1) & ~1;   // even: columns 16-byte aligned for bulk copies
  float2* F = S.f32;
  // scale so that the largest column has norm 1 (keeps the FP32 squares far from underflow)
  double cmax = 0.0;
  for (int j = 0; j < K; ++j) cmax = fmax(cmax, L2Mem::ld(w.nrm + j));
  const double sc = cmax > 0.0 ? 1.0 / sqrt(cmax) : 1.0;
  for (int64_t e = tid_all; e < (int64_t)K * Rr; e += threads_all) {
    const int c = (int)(e / Rr), i = (int)(e % Rr);
    float2 v = make_float2(0.f, 0.f);
    if (i < jlen) {
      const double2 x = L2Mem::ld(J + (int64_t)c * jld + i);
      v = make_float2((float)(x.x * sc), (float)(x.y * sc));
    } else if (i - jlen == c) {
      v.x = 1.f;
    }
    __stcg(F + (int64_t)c * fld + i, v);
  }
  for (int s = tid_all; s <= max_sweeps; s += threads_all) L2Mem::st(w.flags + s, 0);
  sync();
  // FP32 sweeps to FP32 convergence; the floor is a tenth of the FP64 one (in the scaled units)
  const float tol32 = 1.1920929e-07f * (float)max(jlen, 32);
  const float fl32 = (float)(0.01 * floor2 * sc * sc);
  bool conv32 = false;
  j32(F, jlen, Rr, fld, K, S.nrm32, w.flags, rank, nctas, sync, tol32, fl32, min(max_sweeps, S.fp32_sweeps),
      conv32);
  for (int j = worker; j < K; j += workers) {   // final FP32 norms
    const float2* a = F + (int64_t)j * fld;
    float acc = 0.f;
    for (int i = lane; i < jlen; i += 32) {
      const float2 x = __ldcg(a + i);
      acc = fmaf(x.x, x.x, fmaf(x.y, x.y, acc));
    }
    acc = warp_sum_f(acc);
    if (lane == 0) __stcg(S.nrm32 + j, acc);
  }
  sync();
  if (tid_all == 0) {   // the kept columns, in column order
    int ns = 0;
    for (int c = 0; c < K; ++c)
      if (__ldcg(S.nrm32 + c) > fl32) __stcg(S.sel + ns++, c);
    __stcg(S.sel + K, ns);
  }
  sync();
  const int ns = __ldcg(S.sel + K);
  double2* Vd = S.vd;     // K x ns, column-major (ld K)
  double2* G = S.gm;      // ns x ns, column-major
  for (int64_t e = tid_all; e < (int64_t)K * ns; e += threads_all) {
    const int t = (int)(e / K), k = (int)(e % K);
    const float2 v = __ldcg(F + (int64_t)__ldcg(S.sel + t) * fld + jlen + k);
    L2Mem::st(Vd + e, make_double2((double)v.x, (double)v.y));
  }
  sync();
  // Gram matrix G = Vd^dag Vd (upper triangle; a warp per entry)
  for (int64_t e = worker; e < (int64_t)ns * ns; e += workers) {
    const int a = (int)(e % ns), b = (int)(e / ns);
    if (a > b) continue;
    const double2* va = Vd + (int64_t)a * K;
    const double2* vb = Vd + (int64_t)b * K;
    double gr = 0.0, gi = 0.0;
    for (int k = lane; k < K; k += 32) {
      const double2 x = L2Mem::ld(va + k), y = L2Mem::ld(vb + k);
      gr = fma(x.x, y.x, fma(x.y, y.y, gr));      // conj(x) y
      gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
    }
    gr = warp_sum(gr);
    gi = warp_sum(gi);
    if (lane == 0) L2Mem::st(G + (int64_t)b * ns + a, make_double2(gr, gi));
  }
  sync();
  // Cholesky G = U^dag U in place (upper triangle), column by column
  for (int j = 0; j < ns; ++j) {
    if (tid_all == 0) {
      const double2 gjj = L2Mem::ld(G + (int64_t)j * ns + j);
      L2Mem::st(G + (int64_t)j * ns + j, make_double2(sqrt(fmax(gjj.x, 1e-300)), 0.0));
    }
    sync();
    const double d = L2Mem::ld(G + (int64_t)j * ns + j).x, id = 1.0 / d;
    for (int c = j + 1 + tid_all; c < ns; c += threads_all) {   // row j of U
      const double2 x = L2Mem::ld(G + (int64_t)c * ns + j);
      L2Mem::st(G + (int64_t)c * ns + j, make_double2(x.x * id, x.y * id));
    }
    sync();
    // trailing update G[a, c] -= conj(U[j, a]) U[j, c], j < a <= c
    const int tr = ns - j - 1;
    for (int64_t e = tid_all; e < (int64_t)tr * tr; e += threads_all) {
      const int a = j + 1 + (int)(e % tr), c = j + 1 + (int)(e / tr);
      if (a > c) continue;
      const double2 ua = L2Mem::ld(G + (int64_t)a * ns + j), uc = L2Mem::ld(G + (int64_t)c * ns + j);
      double2 x = L2Mem::ld(G + (int64_t)c * ns + a);
      x.x -= ua.x * uc.x + ua.y * uc.y;
      x.y -= ua.x * uc.y - ua.y * uc.x;
      L2Mem::st(G + (int64_t)c * ns + a, x);
    }
    sync();
  }
  // V <- Vd U^-1, row by row (x U = v by forward substitution; a warp per row)
  for (int k = worker; k < K; k += workers) {
    for (int c = 0; c < ns; ++c) {
      double sr = 0.0, si = 0.0;
      for (int a = lane; a < c; a += 32) {
        const double2 x = L2Mem::ld(Vd + (int64_t)a * K + k), u = L2Mem::ld(G + (int64_t)c * ns + a);
        sr = fma(x.x, u.x, fma(-x.y, u.y, sr));
        si = fma(x.x, u.y, fma(x.y, u.x, si));
      }
      sr = warp_sum(sr);
      si = warp_sum(si);
      if (lane == 0) {
        const double2 v = L2Mem::ld(Vd + (int64_t)c * K + k);
        const double id = 1.0 / L2Mem::ld(G + (int64_t)c * ns + c).x;
        L2Mem::st(Vd + (int64_t)c * K + k, make_double2((v.x - sr) * id, (v.y - si) * id));
      }
      __syncwarp();
    }
  }
  sync();
  // A1 = J V (jlen x ns), the remaining columns zero
  double2* A1 = S.a1;
  for (int64_t e = tid_all; e < (int64_t)K * jlen; e += threads_all) {
    const int t = (int)(e / jlen), i = (int)(e % jlen);
    double ar = 0.0, ai = 0.0;
    if (t < ns) {
      const double2* vt = Vd + (int64_t)t * K;
      for (int k = 0; k < K; ++k) {
        const double2 x = L2Mem::ld(J + (int64_t)k * jld + i), v = L2Mem::ld(vt + k);
        ar = fma(x.x, v.x, fma(-x.y, v.y, ar));
        ai = fma(x.x, v.y, fma(x.y, v.x, ai));
      }
    }
    L2Mem::st(A1 + (int64_t)t * jld + i, make_double2(ar, ai));
  }
  for (int s = tid_all; s <= max_sweeps; s += threads_all) L2Mem::st(w.flags + s, 0);
  sync();
  *nsel_out = ns;
}

template <class Mem, class Sync, class Jacobi, class J32 = NoJacobi32>
__device__ void svd_sector(const SvdSector& S, const Work& w, int rank, int nctas, Sync sync, int max_sweeps,
                           Jacobi jacobi, J32 j32 = J32()) {
  __shared__ double red_d[kMaxWarps][33];
  __shared__ double red_v[kMaxWarps];
  __shared__ int red_i[kMaxWarps];
  const int m = S.m, n = S.n, K = min(m, n), ld = odd_ld(n);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int tid_all = rank * blockDim.x + tid, threads_all = nctas * blockDim.x;
  const int worker = rank * nwarps + warp, workers = nctas * nwarps;
  double2* W = w.W;

  // ---- load M = diag(lambda) Theta' (row-major), column norms, identity permutation ----
  const int64_t mn = (int64_t)m * n;
  for (int64_t e = tid_all; e < mn; e += threads_all) {
    const int i = (int)(e / n), j = (int)(e % n);
    const double s = S.rowscale ? S.rowscale[i] : 1.0;
    const double2 t = S.theta[e];
    Mem::st(W + (int64_t)i * ld + j, make_double2(s * t.x, s * t.y));
  }
  for (int s = tid_all; s <= max_sweeps; s += threads_all) Mem::st(w.flags + s, 0);
  sync();
  for (int j = tid_all; j < n; j += threads_all) {
    double acc = 0.0;
    for (int i = 0; i < m; ++i) {
      const double2 x = Mem::ld(W + (int64_t)i * ld + j);
      acc = fma(x.x, x.x, fma(x.y, x.y, acc));
    }
    Mem::st(w.nu + j, acc);
    Mem::st(w.nu0 + j, acc);
    Mem::st(w.perm + j, j);
  }
  sync();
  if (tid_all == 0) {
    double f = 0.0;
    for (int j = 0; j < n; ++j) f += Mem::ld(w.nu + j);
    Mem::st(w.scal + 1, f);
  }
  sync();
  const double fro2 = Mem::ld(w.scal + 1);

  // ---- Householder QR with column pivoting: M P = Q R ---------------------------------
  for (int k = 0; k < K; ++k) {
    // pivot: largest remaining partial norm, ties to the smaller index
    double bv = -1.0;
    int bi = n;
    for (int j = k + tid_all; j < n; j += threads_all) {
      const double v = Mem::ld(w.nu + j);
      if (v > bv || (v == bv && j < bi)) { bv = v; bi = j; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = bv; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      for (int x = 1; x < nwarps; ++x)
        if (red_v[x] > bv || (red_v[x] == bv && red_i[x] < bi)) { bv = red_v[x]; bi = red_i[x]; }
      Mem::st(w.pv + rank, bv);
      Mem::st(w.pi + rank, bi);
    }
    sync();
    bv = Mem::ld(w.pv);
    bi = Mem::ld(w.pi);
    for (int x = 1; x < nctas; ++x) {
      const double v = Mem::ld(w.pv + x);
      const int ix = Mem::ld(w.pi + x);
      if (v > bv || (v == bv && ix < bi)) { bv = v; bi = ix; }
    }
    const int p = (bi < n) ? bi : k;
    if (p != k) {
      for (int i = tid_all; i < m; i += threads_all) {
        double2* rowp = W + (int64_t)i * ld;
        const double2 a = Mem::ld(rowp + k), b = Mem::ld(rowp + p);
        Mem::st(rowp + k, b);
        Mem::st(rowp + p, a);
      }
      if (tid_all == 0) {
        double a = Mem::ld(w.nu + k), b = Mem::ld(w.nu + p);
        Mem::st(w.nu + k, b); Mem::st(w.nu + p, a);
        a = Mem::ld(w.nu0 + k); b = Mem::ld(w.nu0 + p);
        Mem::st(w.nu0 + k, b); Mem::st(w.nu0 + p, a);
        const int ia = Mem::ld(w.perm + k), ib = Mem::ld(w.perm + p);
        Mem::st(w.perm + k, ib); Mem::st(w.perm + p, ia);
      }
    }
    sync();
    // reflector H = I - (2 / u^dag u) u u^dag with H x = beta e_k, |beta| = |x|
    if (worker == 0) {
      double x2 = 0.0;
      for (int i = k + lane; i < m; i += 32) {
        const double2 x = Mem::ld(W + (int64_t)i * ld + k);
        x2 = fma(x.x, x.x, fma(x.y, x.y, x2));
      }
      x2 = warp_sum(x2);
      const double xn = sqrt(x2);
      const double2 x0 = Mem::ld(W + (int64_t)k * ld + k);
      const double a0 = hypot(x0.x, x0.y);
      double2 beta;
      if (a0 > 0.0) beta = make_double2(-x0.x / a0 * xn, -x0.y / a0 * xn);
      else beta = make_double2(-xn, 0.0);
      const double uu = 2.0 * x2 + 2.0 * xn * a0;
      for (int i = k + lane; i < m; i += 32) {
        double2 x = Mem::ld(W + (int64_t)i * ld + k);
        if (i == k) x = make_double2(x.x - beta.x, x.y - beta.y);
        Mem::st(w.u + i, x);
        Mem::st(W + (int64_t)i * ld + k, i == k ? beta : make_double2(0.0, 0.0));
      }
      if (lane == 0) Mem::st(w.scal, uu > 0.0 ? 2.0 / uu : 0.0);
    }
    sync();
    // trailing update W[k:, j] -= (2/u^dag u) u (u^dag W[k:, j]) for j > k, 32 columns x 8 row chunks per CTA
    const double sc = Mem::ld(w.scal);
    const int ncols = n - k - 1;
    const int ntiles = (ncols + 31) / 32;
    if (sc != 0.0) {
      for (int tile = rank; tile < ntiles; tile += nctas) {
        const int j = k + 1 + tile * 32 + lane;
        double pr = 0.0, pim = 0.0;
        if (j < n) {
          for (int i = k + warp; i < m; i += nwarps) {
            const double2 ui = Mem::ld(w.u + i);
            const double2 x = Mem::ld(W + (int64_t)i * ld + j);
            pr = fma(ui.x, x.x, fma(ui.y, x.y, pr));      // conj(u_i) x
            pim = fma(ui.x, x.y, fma(-ui.y, x.x, pim));
          }
        }
        red_d[warp][lane] = pr;
        __syncthreads();
        double wr = 0.0;
        for (int x = 0; x < nwarps; ++x) wr += red_d[x][lane];
        __syncthreads();
        red_d[warp][lane] = pim;
        __syncthreads();
        double wi = 0.0;
        for (int x = 0; x < nwarps; ++x) wi += red_d[x][lane];
        __syncthreads();
        wr *= sc;
        wi *= sc;
        if (j < n) {
          for (int i = k + warp; i < m; i += nwarps) {
            const double2 ui = Mem::ld(w.u + i);
            double2 x = Mem::ld(W + (int64_t)i * ld + j);
            x.x -= ui.x * wr - ui.y * wi;
            x.y -= ui.x * wi + ui.y * wr;
            Mem::st(W + (int64_t)i * ld + j, x);
          }
        }
        __syncthreads();
        if (warp == 0 && j < n) {       // downdate the partial norm, recompute on cancellation
          const double2 r = Mem::ld(W + (int64_t)k * ld + j);
          double v = Mem::ld(w.nu + j) - (r.x * r.x + r.y * r.y);
          if (v <= 1.4901161193847656e-8 * Mem::ld(w.nu0 + j)) {
            v = 0.0;
            for (int i = k + 1; i < m; ++i) {
              const double2 x = Mem::ld(W + (int64_t)i * ld + j);
              v = fma(x.x, x.x, fma(x.y, x.y, v));
            }
            Mem::st(w.nu0 + j, v);
          }
          Mem::st(w.nu + j, v);
        }
      }
    } else {
      for (int tile = rank; tile < ntiles; tile += nctas) {
        const int j = k + 1 + tile * 32 + lane;
        if (warp == 0 && j < n) {
          const double2 r = Mem::ld(W + (int64_t)k * ld + j);
          Mem::st(w.nu + j, fmax(Mem::ld(w.nu + j) - (r.x * r.x + r.y * r.y), 0.0));
        }
      }
    }
    sync();
  }

  // ---- R^dag: conjugate rows 0..K-1 in place; they are the Jacobi columns ------------
  const int64_t kn = (int64_t)K * n;
  for (int64_t e = tid_all; e < kn; e += threads_all) {
    const int i = (int)(e / n), j = (int)(e % n);
    double2* a = W + (int64_t)i * ld + j;
    const double2 x = Mem::ld(a);
    Mem::st(a, make_double2(x.x, -x.y));
  }
  sync();

  // ---- wide sectors (K = m < n): R^dag = Q2 [R2; 0] by unpivoted Householder QR of its
  // K columns.  Rotations that orthogonalise the columns of R^dag orthogonalise those of
  // R2 alike (Q2 has orthonormal columns), so the Jacobi sweeps run on R2's columns,
  // length K instead of n, and Y = P Q2 [normalised columns; 0] at the end. --------------
  double2* J = W;        // the Jacobi matrix: column j at J + j * jld, length jlen
  int jlen = n, jld = ld;
  double* tau = w.nu;    // reflector scales (w.nu is free after the pivoted QR; n >= K)
  const bool wide = Mem::kCache && S.wide;   // cluster kernels only (their scratch holds R2)
  if constexpr (Mem::kCache) if (wide) {
    double2* W2 = S.work2;
    const int ld2 = odd_ld(K);
    for (int64_t e = tid_all; e < (int64_t)K * ld2; e += threads_all) Mem::st(W2 + e, make_double2(0.0, 0.0));
    sync();
    for (int k = 0; k < K; ++k) {
      double2* xk = W + (int64_t)k * ld;
      if (worker == 0) {   // H_k = I - tau_k v v^dag maps x_k[k:] to beta e_k; v overwrites x_k[k:]
        double x2 = 0.0;
        for (int i = k + lane; i < n; i += 32) {
          const double2 x = Mem::ld(xk + i);
          x2 = fma(x.x, x.x, fma(x.y, x.y, x2));
        }
        x2 = warp_sum(x2);
        const double xn = sqrt(x2);
        const double2 x0 = Mem::ld(xk + k);
        const double a0 = hypot(x0.x, x0.y);
        double2 beta;
        if (a0 > 0.0) beta = make_double2(-x0.x / a0 * xn, -x0.y / a0 * xn);
        else beta = make_double2(-xn, 0.0);
        const double uu = 2.0 * x2 + 2.0 * xn * a0;
        if (lane == 0) {
          Mem::st(xk + k, make_double2(x0.x - beta.x, x0.y - beta.y));
          Mem::st(tau + k, uu > 0.0 ? 2.0 / uu : 0.0);
          Mem::st(W2 + (int64_t)k * ld2 + k, beta);          // R2[k][k]
        }
      }
      sync();
      const double tk = Mem::ld(tau + k);
      for (int j = k + 1 + worker; j < K; j += workers) {
        double2* xj = W + (int64_t)j * ld;
        double pr = 0.0, pim = 0.0;
        if (tk != 0.0) {
          for (int i = k + lane; i < n; i += 32) {
            const double2 v = Mem::ld(xk + i), x = Mem::ld(xj + i);
            pr = fma(v.x, x.x, fma(v.y, x.y, pr));         // conj(v) x
            pim = fma(v.x, x.y, fma(-v.y, x.x, pim));
          }
          pr = warp_sum(pr) * tk;
          pim = warp_sum(pim) * tk;
        }
        for (int i = k + lane; i < n; i += 32) {
          double2 x = Mem::ld(xj + i);
          if (tk != 0.0) {
            const double2 v = Mem::ld(xk + i);
            x.x -= v.x * pr - v.y * pim;
            x.y -= v.x * pim + v.y * pr;
            Mem::st(xj + i, x);
          }
          if (i == k) Mem::st(W2 + (int64_t)j * ld2 + k, x);   // R2[k][j], final after H_k
        }
      }
      sync();
    }
    J = W2;
    jlen = K;
    jld = ld2;
  }
  for (int j = worker; j < K; j += workers) {
    const double2* a = J + (int64_t)j * jld;
    double acc = 0.0;
    for (int i = lane; i < jlen; i += 32) {
      const double2 x = Mem::ld(a + i);
      acc = fma(x.x, x.x, fma(x.y, x.y, acc));
    }
    acc = warp_sum(acc);
    if (lane == 0) Mem::st(w.nrm + j, acc);
  }
  sync();

  // ---- one-sided Jacobi on the K columns of R^dag (or R2) --------------------------------
  const double tol = kEps * (double)max(n, 32);
  const double tol2 = tol * tol;
  // floor: the rounding-noise level 32 eps |M|_F, or the caller's deflation level when higher
  const double frel = fmax(32.0 * kEps, S.floor_rel);
  const double floor2 = fmax(frel * frel * fro2, S.floor_abs * S.floor_abs);
  bool converged = false;
  int Kj = K;                    // columns the FP64 sweeps rotate
  if constexpr (std::is_same<J32, JacobiBlocks32>::value) {
    if (S.f32 && K >= 2) {       // FP32 sweeps first; the FP64 sweeps then start from J V
      int ns = K;
      mixed_precondition(S, w, J, jlen, jld, K, rank, nctas, sync, floor2, max_sweeps, j32, &ns);
      J = S.a1;
      Kj = ns;
      for (int j = worker; j < K; j += workers) {   // column norms of the new Jacobi matrix
        const double2* a = J + (int64_t)j * jld;
        double acc = 0.0;
        for (int i = lane; i < jlen; i += 32) {
          const double2 x = Mem::ld(a + i);
          acc = fma(x.x, x.x, fma(x.y, x.y, acc));
        }
        acc = warp_sum(acc);
        if (lane == 0) Mem::st(w.nrm + j, acc);
      }
      sync();
    }
  }
  const int sweep = jacobi(J, jlen, jld, Kj, w, rank, nctas, sync, tol2, floor2, max_sweeps, converged);

  // ---- singular values (noise floor -> 0), descending, ties by column index -----------
  for (int j = worker; j < K; j += workers) {
    const double2* a = J + (int64_t)j * jld;
    double acc = 0.0;
    for (int i = lane; i < jlen; i += 32) {
      const double2 x = Mem::ld(a + i);
      acc = fma(x.x, x.x, fma(x.y, x.y, acc));
    }
    acc = warp_sum(acc);
    if (lane == 0) Mem::st(w.nrm + j, acc <= floor2 ? 0.0 : sqrt(acc));
  }
  sync();
  for (int j = tid_all; j < K; j += threads_all) {
    const double vj = Mem::ld(w.nrm + j);
    const double v = isnan(vj) ? -1.0 : vj;       // NaN ranks last: ranks stay a permutation
    int rk = 0;
    for (int q = 0; q < K; ++q) {
      const double wq = Mem::ld(w.nrm + q);
      const double x = isnan(wq) ? -1.0 : wq;
      rk += (x > v) || (x == v && q < j);
    }
    Mem::st(w.ord + rk, j);
  }
  sync();
  for (int r = tid_all; r < K; r += threads_all) S.sigma[r] = Mem::ld(w.nrm + Mem::ld(w.ord + r));
  if (wide) {
    // Y[perm[j], r] = (Q2 [R2 column ord[r] / sigma_r; 0])[j]; Q2 = H_0 ... H_{K-1}, one warp per column
    for (int r = worker; r < K; r += workers) {
      const int c = Mem::ld(w.ord + r);
      const double sv = Mem::ld(w.nrm + c);
      double2* y = S.ytmp + (int64_t)r * n;
      if (sv > 0.0) {
        const double2* a = J + (int64_t)c * jld;
        for (int i = lane; i < n; i += 32) {
          double2 val = make_double2(0.0, 0.0);
          if (i < K) {
            const double2 x = Mem::ld(a + i);
            val = make_double2(x.x / sv, x.y / sv);
          }
          Mem::st(y + i, val);
        }
        __syncwarp();
        for (int k = K - 1; k >= 0; --k) {
          const double tk = Mem::ld(tau + k);
          if (tk == 0.0) continue;
          const double2* v = W + (int64_t)k * ld;
          double pr = 0.0, pim = 0.0;
          for (int i = k + lane; i < n; i += 32) {
            const double2 vv = Mem::ld(v + i), x = Mem::ld(y + i);
            pr = fma(vv.x, x.x, fma(vv.y, x.y, pr));
            pim = fma(vv.x, x.y, fma(-vv.y, x.x, pim));
          }
          pr = warp_sum(pr) * tk;
          pim = warp_sum(pim) * tk;
          for (int i = k + lane; i < n; i += 32) {
            const double2 vv = Mem::ld(v + i);
            double2 x = Mem::ld(y + i);
            x.x -= vv.x * pr - vv.y * pim;
            x.y -= vv.x * pim + vv.y * pr;
            Mem::st(y + i, x);
          }
          __syncwarp();
        }
        for (int j = lane; j < n; j += 32) S.Y[(int64_t)r * n + Mem::ld(w.perm + j)] = Mem::ld(y + j);
      } else {
        for (int j = lane; j < n; j += 32) S.Y[(int64_t)r * n + j] = make_double2(0.0, 0.0);
      }
    }
  } else {
    // Y[perm[j], r] = column ord[r] of R^dag, row j, divided by its norm
    for (int64_t e = tid_all; e < kn; e += threads_all) {
      const int r = (int)(e / n), j = (int)(e % n);
      const int c = Mem::ld(w.ord + r);
      const double sv = Mem::ld(w.nrm + c);
      double2 y = make_double2(0.0, 0.0);
      if (sv > 0.0) {
        const double2 a = Mem::ld(J + (int64_t)c * jld + j);
        y = make_double2(a.x / sv, a.y / sv);
      }
      S.Y[(int64_t)r * n + Mem::ld(w.perm + j)] = y;
    }
  }
  if (tid_all == 0) *S.status = converged ? sweep : -1;
}

struct CtaSync {
  __device__ void operator()() const { __syncthreads(); }
};
struct ClusterSync {
  __device__ void operator()() const { cluster_sync_all(); }
};

// shared-memory layout of the one-CTA kernel (offsets in bytes)
struct SmemLayout {
  int64_t W, u, nu, nu0, perm, nrm, ord, flags, pv, pi, scal, total;
};
__host__ __device__ inline SmemLayout smem_layout(int m, int n) {
  auto al = [](int64_t x) { return (x + 15) & ~int64_t(15); };
  const int K = m < n ? m : n;
  SmemLayout L;
  int64_t o = 0;
  L.W = o; o = al(o + 16LL * m * odd_ld(n));
  L.u = o; o = al(o + 16LL * m);
  L.nu = o; o = al(o + 8LL * n);
  L.nu0 = o; o = al(o + 8LL * n);
  L.perm = o; o = al(o + 4LL * n);
  L.nrm = o; o = al(o + 8LL * K);
  L.ord = o; o = al(o + 4LL * K);
  L.flags = o; o = al(o + 4LL * (kJacobiMaxSweeps + 1));
  L.pv = o; o = al(o + 8);
  L.pi = o; o = al(o + 4);
  L.scal = o; o = al(o + 16);
  L.total = o;
  return L;
}

__global__ void __launch_bounds__(kSvdThreads, 1) jacobi_cta_kernel(const SvdSector* __restrict__ secs,
                                                                    int max_sweeps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SvdSector S = secs[blockIdx.x];
  const SmemLayout L = smem_layout(S.m, S.n);
  Work w;
  w.W = reinterpret_cast<double2*>(smem_raw + L.W);
  w.u = reinterpret_cast<double2*>(smem_raw + L.u);
  w.nu = reinterpret_cast<double*>(smem_raw + L.nu);
  w.nu0 = reinterpret_cast<double*>(smem_raw + L.nu0);
  w.perm = reinterpret_cast<int*>(smem_raw + L.perm);
  w.nrm = reinterpret_cast<double*>(smem_raw + L.nrm);
  w.ord = reinterpret_cast<int*>(smem_raw + L.ord);
  w.flags = reinterpret_cast<int*>(smem_raw + L.flags);
  w.pv = reinterpret_cast<double*>(smem_raw + L.pv);
  w.pi = reinterpret_cast<int*>(smem_raw + L.pi);
  w.scal = reinterpret_cast<double*>(smem_raw + L.scal);
  svd_sector<PlainMem>(S, w, 0, 1, CtaSync{}, max_sweeps, JacobiRoundRobin<PlainMem>{});
}

__device__ __forceinline__ Work cluster_work(const SvdSector& S) {
  Work w;
  w.W = S.work;
  w.u = S.uwork;
  w.nu = S.norms;
  w.nu0 = S.norms + S.n;
  w.perm = S.order;
  w.nrm = S.norms + 2 * S.n;
  w.ord = S.order + S.n;
  w.flags = S.flags;
  w.pv = S.pivv;
  w.pi = S.flags + kJacobiMaxSweeps + 1;
  w.scal = S.pivv + kMaxCluster;
  return w;
}

__global__ void __launch_bounds__(kSvdThreads) jacobi_cluster_kernel(const SvdSector* __restrict__ secs,
                                                                     int cluster, int max_sweeps) {
  const int rank = (int)cluster_rank();
  const SvdSector S = secs[blockIdx.x / cluster];
  svd_sector<L2Mem>(S, cluster_work(S), rank, cluster, ClusterSync{}, max_sweeps, JacobiRoundRobin<L2Mem>{});
}

__global__ void __launch_bounds__(kBlockThreads, 2) jacobi_cluster_block_kernel(const SvdSector* __restrict__ secs,
                                                                                int cluster, int max_sweeps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rank = (int)cluster_rank();
  const SvdSector S = secs[blockIdx.x / cluster];
  const int K = min(S.m, S.n);
  JacobiBlocks jb;
  jb.g = S.groups;
  jb.gs = S.staged;
  jb.bsmax = (K + 2 * cluster * jb.g - 1) / (2 * cluster * jb.g);
  jb.sm = reinterpret_cast<double2*>(smem_raw);
  jb.smn = reinterpret_cast<double*>(smem_raw + 16LL * 2 * jb.gs * jb.bsmax * (S.wide ? K : S.n));
  // the FP32 sweeps of a mixed-precision sector stage columns of jlen + K <= 2 jlen FP32
  // complex values in the same area
  JacobiBlocks32 j32;
  j32.g = jb.g;
  j32.gs = jb.gs;
  j32.bsmax = jb.bsmax;
  j32.sm = reinterpret_cast<float2*>(smem_raw);
  j32.smn = reinterpret_cast<float*>(smem_raw + 8LL * 2 * jb.gs * jb.bsmax * ((((S.wide ? K : S.n) + K) + 1) & ~1));
  svd_sector<L2Mem>(S, cluster_work(S), rank, cluster, ClusterSync{}, max_sweeps, jb, j32);
}


}  // namespace

int64_t svd_smem_need(int m, int n) { return smem_layout(m, n).total; }

namespace {

constexpr int kBlockSmemMax = 110 * 1024;   // two block-Jacobi CTAs per SM
// 8 CTAs per large sector: the GPU places about twice as many 8-CTA clusters as
// 16-CTA ones, which keeps more SMs busy when a layer has hundreds of large sectors
constexpr int kBigCluster = 8;
// Kernel attributes (dynamic shared memory, non-portable clusters) apply to the current device
// only, so they are set once per device, under a lock, with that device's cluster size.
constexpr int kMaxDevices = 64;
std::mutex g_attr_mu;
bool g_attr_done[kMaxDevices] = {};
int g_big_cluster[kMaxDevices] = {};

int64_t block_smem_need(int m, int n, int cl, int g, int gs) {
  const int64_t K = std::min(m, n), bs = (K + 2 * cl * g - 1) / (2 * cl * g);
  return 16 * 2 * gs * bs * n + 16 * 2 * gs * bs + 64;   // norms, and the FP32 staging's even-stride padding
}

cudaError_t set_attrs(int* big_out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (g_attr_done[dev]) {
    *big_out = g_big_cluster[dev];
    return cudaSuccess;
  }
  e = cudaFuncSetAttribute(jacobi_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSvdSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(jacobi_cluster_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kBlockSmemMax);
  if (e != cudaSuccess) return e;
  // clusters of 16 CTAs are non-portable: use them only where the device can place them
  int big = 8;
  if (cudaFuncSetAttribute(jacobi_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess &&
      cudaFuncSetAttribute(jacobi_cluster_block_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kBlockThreads);
    cfg.dynamicSmemBytes = kBlockSmemMax;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = 16;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, jacobi_cluster_block_kernel, &cfg) == cudaSuccess && n >= 4) big = 16;
  }
  cudaGetLastError();
  g_big_cluster[dev] = big;
  g_attr_done[dev] = true;
  *big_out = big;
  return cudaSuccess;
}

cudaError_t launch_group(const SvdSector* d_secs, const SvdGroup& g, int max_sweeps, cudaStream_t st) {
  if (g.count <= 0) return cudaSuccess;
  const SvdSector* d = d_secs + g.first;
  count_launch();
  if (g.kind == kSvdSmem) {
    jacobi_cta_kernel<<<g.count, kSvdThreads, g.smem, st>>>(d, max_sweeps);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g.count * g.cl);
  cfg.blockDim = dim3(g.kind == kSvdClusterBlock ? kBlockThreads : kSvdThreads);
  cfg.dynamicSmemBytes = g.smem;
  cfg.stream = st;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = g.cl;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  if (g.kind == kSvdClusterBlock) return cudaLaunchKernelEx(&cfg, jacobi_cluster_block_kernel, d, g.cl, max_sweeps);
  return cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel, d, g.cl, max_sweeps);
}

}  // namespace

cudaError_t svd_group(std::vector<SvdSector>& secs, std::vector<SvdGroup>& groups, const SvdTune& tune) {
  int big_cluster = 0;
  cudaError_t e = set_attrs(&big_cluster);
  if (e != cudaSuccess) return e;
  // every sector gets a kernel and a cluster size
  std::vector<std::pair<int, int>> key(secs.size());
  std::vector<int64_t> smem(secs.size(), 0);
  for (size_t k = 0; k < secs.size(); ++k) {
    const SvdSector S = secs[k];
    if (S.mode == kSvdSmem) {
      key[k] = {kSvdSmem, 1};
      smem[k] = svd_smem_need(S.m, S.n);
      continue;
    }
    // blocks of about tune.bw columns (6 by default); the smallest cluster (tune.cl_min,
    // then doubling up to 8 CTAs) whose CTAs can stage all of their block pairs of a round
    // at once, so that a step offers the warp groups about K / (2 cl) * bw / 2 disjoint
    // pairs; failing that, 8 CTAs staging as many pairs as fit, with more pairs per CTA
    // when a single one does not fit
    const int bw = std::max(2, tune.bw);
    const int cn = S.wide ? std::min(S.m, S.n) : S.n;   // Jacobi column length
    int pick_cl = 0, pick_g = 0, pick_gs = 0;
    for (int cl = std::max(2, std::min(tune.cl_min, kBigCluster)); cl <= kBigCluster && !pick_cl; cl *= 2) {
      const int g = std::max(1, (std::min(S.m, S.n) + bw * cl) / (2 * bw * cl));
      if (g <= kMaxStaged && block_smem_need(S.m, cn, cl, g, g) <= kBlockSmemMax) {
        pick_cl = cl; pick_g = g; pick_gs = g;
      }
    }
    if (!pick_cl) {
      const int cl = kBigCluster;
      int g = std::max(1, (std::min(S.m, S.n) + bw * cl) / (2 * bw * cl));
      while (g < 64 && block_smem_need(S.m, cn, cl, g, 1) > kBlockSmemMax) ++g;
      int gs = 1;
      while (gs < std::min(g, kMaxStaged) && block_smem_need(S.m, cn, cl, g, gs + 1) <= kBlockSmemMax) ++gs;
      if (block_smem_need(S.m, cn, cl, g, gs) <= kBlockSmemMax) {
        pick_cl = cl; pick_g = g; pick_gs = gs;
      }
    }
    if (std::min(S.m, S.n) >= tune.c16_min_k && big_cluster >= 16) {   // a 16-CTA cluster
      const int cl = 16;
      int g = std::max(1, (std::min(S.m, S.n) + bw * cl) / (2 * bw * cl));
      while (g < 64 && block_smem_need(S.m, cn, cl, g, 1) > kBlockSmemMax) ++g;
      int gs = 1;
      while (gs < std::min(g, kMaxStaged) && block_smem_need(S.m, cn, cl, g, gs + 1) <= kBlockSmemMax) ++gs;
      if (block_smem_need(S.m, cn, cl, g, gs) <= kBlockSmemMax) {
        pick_cl = cl; pick_g = g; pick_gs = gs;
      }
    }
    if (std::min(S.m, S.n) >= tune.rr_min_k) pick_cl = 0;
    if (pick_cl) {
      key[k] = {kSvdClusterBlock, pick_cl};
      smem[k] = block_smem_need(S.m, cn, pick_cl, pick_g, pick_gs);
      secs[k].groups = pick_g;
      secs[k].staged = pick_gs;
    } else {
      key[k] = {kSvdCluster, big_cluster};
    }
  }
  // group by (kind, cluster size); the most expensive sectors first inside a group
  std::vector<size_t> idx(secs.size());
  for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
  auto cost = [&](size_t k) {
    const double C = std::min(secs[k].m, secs[k].n);
    return (double)secs[k].n * C * C + (double)secs[k].m * secs[k].n * C;
  };
  std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
    if (key[a] != key[b]) return key[a] > key[b];
    return cost(a) > cost(b);
  });
  std::vector<SvdSector> out;
  out.reserve(secs.size());
  groups.clear();
  for (size_t t = 0; t < idx.size(); ++t) {
    const size_t k = idx[t];
    if (groups.empty() || groups.back().kind != key[k].first || groups.back().cl != key[k].second) {
      SvdGroup g;
      g.kind = key[k].first;
      g.cl = key[k].second;
      g.smem = 0;
      g.first = (int)out.size();
      g.count = 0;
      groups.push_back(g);
    }
    groups.back().count++;
    groups.back().smem = std::max<int>(groups.back().smem, (int)smem[k]);
    out.push_back(secs[k]);
  }
  secs.swap(out);
  return cudaSuccess;
}

cudaError_t launch_svd_groups(const SvdSector* d_secs, const std::vector<SvdGroup>& groups, cudaStream_t st,
                              const cudaStream_t* side, int n_side, cudaEvent_t fork, const cudaEvent_t* join,
                              int max_sweeps) {
  max_sweeps = std::max(1, std::min(max_sweeps, kJacobiMaxSweeps));   // the flag arrays hold 40 sweeps
  // group 0 on st, the others on side streams when given, all joined back into st
  cudaError_t e = cudaSuccess;
  const int ng = (int)groups.size();
  if (ng == 0) return cudaSuccess;
  const bool fan = side && n_side >= ng - 1 && ng > 1;
  if (fan) {
    if ((e = cudaEventRecord(fork, st)) != cudaSuccess) return e;
    for (int g = 1; g < ng; ++g)
      if ((e = cudaStreamWaitEvent(side[g - 1], fork, 0)) != cudaSuccess) return e;
  }
  for (int g = 0; g < ng; ++g) {
    cudaStream_t s = (fan && g > 0) ? side[g - 1] : st;
    if ((e = launch_group(d_secs, groups[g], max_sweeps, s)) != cudaSuccess) return e;
  }
  if (fan) {
    for (int g = 1; g < ng; ++g) {
      if ((e = cudaEventRecord(join[g - 1], side[g - 1])) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(st, join[g - 1], 0)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

bool svd_layout(int ns, const int* m, const int* n, SvdScratchLayout& L, int cluster_min_k) {
  if (cluster_min_k < 0) cluster_min_k = svd_cluster_min_k();
  L.mode.assign(ns, kSvdSmem);
  L.work_off.assign(ns, -1);
  L.v_off.assign(ns, -1);
  L.norm_off.assign(ns, -1);
  L.ord_off.assign(ns, -1);
  L.flag_off.assign(ns, -1);
  L.piv_off.assign(ns, -1);
  L.wide.assign(ns, 0);
  L.w2_off.assign(ns, -1);
  L.yt_off.assign(ns, -1);
  for (auto* v : {&L.f32_off, &L.n32_off, &L.vd_off, &L.gm_off, &L.a1_off, &L.sel_off}) v->assign(ns, -1);
  L.smem = 0;
  const int mix_k = svd_mixed_min_k();
  int64_t off = 0;
  auto a256 = [](int64_t x) { return (x + 255) & ~int64_t(255); };
  for (int k = 0; k < ns; ++k) {
    if (m[k] < 1 || n[k] < 1) return false;
    const int64_t need = svd_smem_need(m[k], n[k]);
    if (need <= kSvdSmemMax && std::min(m[k], n[k]) < cluster_min_k) {
      L.smem = std::max<int>(L.smem, (int)need);
      continue;
    }
    const int64_t M = m[k], N = n[k], Kk = std::min(m[k], n[k]);
    L.mode[k] = kSvdCluster;
    L.work_off[k] = off; off = a256(off + 16 * M * odd_ld(n[k]));
    L.v_off[k] = off;    off = a256(off + 16 * M);                      // Householder vector
    L.norm_off[k] = off; off = a256(off + 8 * (2 * N + Kk));            // nu, nu0, nrm
    L.ord_off[k] = off;  off = a256(off + 4 * (N + Kk));                // perm, ord
    L.flag_off[k] = off; off = a256(off + 4 * (kJacobiMaxSweeps + 1 + kMaxCluster));   // flags, pivot index
    L.piv_off[k] = off;  off = a256(off + 8 * (kMaxCluster + 2));       // pivot value, scalars
    if (4LL * n[k] >= 5LL * m[k]) {   // wide: the Jacobi sweeps run on the K x K factor R2
      L.wide[k] = 1;
      L.w2_off[k] = off; off = a256(off + 16 * Kk * odd_ld((int)Kk));     // R2 / Jacobi matrix
      L.yt_off[k] = off; off = a256(off + 16 * N * Kk);                   // Q2 applied to its columns
    }
    if (mix_k > 0 && Kk >= mix_k) {   // FP32 sweeps first (see mixed_precondition)
      const int64_t jlen = L.wide[k] ? Kk : N, jld = L.wide[k] ? odd_ld((int)Kk) : odd_ld(n[k]);
      L.f32_off[k] = off; off = a256(off + 8 * (jlen + Kk + 2) * Kk);
      L.n32_off[k] = off; off = a256(off + 4 * Kk);
      L.vd_off[k] = off;  off = a256(off + 16 * Kk * Kk);
      L.gm_off[k] = off;  off = a256(off + 16 * Kk * Kk);
      L.a1_off[k] = off;  off = a256(off + 16 * jld * Kk);
      L.sel_off[k] = off; off = a256(off + 4 * (Kk + 1));
    }
  }
  L.total = off;
  return true;
}

void svd_fill_scratch(SvdSector& S, const SvdScratchLayout& L, int k, char* base) {
  S.mode = L.mode[k];
  if (S.mode != kSvdCluster) return;
  S.work = reinterpret_cast<double2*>(base + L.work_off[k]);
  S.uwork = reinterpret_cast<double2*>(base + L.v_off[k]);
  S.norms = reinterpret_cast<double*>(base + L.norm_off[k]);
  S.order = reinterpret_cast<int*>(base + L.ord_off[k]);
  S.flags = reinterpret_cast<int*>(base + L.flag_off[k]);
  S.pivv = reinterpret_cast<double*>(base + L.piv_off[k]);
  S.wide = L.wide[k];
  if (S.wide) {
    S.work2 = reinterpret_cast<double2*>(base + L.w2_off[k]);
    S.ytmp = reinterpret_cast<double2*>(base + L.yt_off[k]);
  }
  S.f32 = nullptr;
  S.fp32_sweeps = svd_mixed_sweeps();
  if (L.f32_off[k] >= 0) {
    S.f32 = reinterpret_cast<float2*>(base + L.f32_off[k]);
    S.nrm32 = reinterpret_cast<float*>(base + L.n32_off[k]);
    S.vd = reinterpret_cast<double2*>(base + L.vd_off[k]);
    S.gm = reinterpret_cast<double2*>(base + L.gm_off[k]);
    S.a1 = reinterpret_cast<double2*>(base + L.a1_off[k]);
    S.sel = reinterpret_cast<int*>(base + L.sel_off[k]);
  }
}

namespace {
std::atomic<int> g_mixed_min_k{192};
std::atomic<int> g_mixed_sweeps{8};
std::atomic<int> g_cluster_min_k{1 << 30};
}
int svd_mixed_min_k() { return g_mixed_min_k.load(); }
int svd_cluster_min_k() { return g_cluster_min_k.load(); }
int svd_mixed_sweeps() { return g_mixed_sweeps.load(); }

}  // namespace mps

extern "C" int mps_svd_mixed_min_k(int min_k) {
  if (min_k < 0) return MPS_EINVAL;
  mps::g_mixed_min_k.store(min_k);
  return MPS_OK;
}

extern "C" int mps_svd_cluster_min_k(int min_k) {
  if (min_k != 0 && min_k < 16) return MPS_EINVAL;
  mps::g_cluster_min_k.store(min_k == 0 ? (1 << 30) : min_k);
  return MPS_OK;
}

extern "C" int mps_svd_mixed_sweeps(int max_sweeps) {
  if (max_sweeps < 1 || max_sweeps > mps::kJacobiMaxSweeps) return MPS_EINVAL;
  mps::g_mixed_sweeps.store(max_sweeps);
  return MPS_OK;
}

namespace mps {

}  // namespace mps

using namespace mps;

extern "C" int64_t mps_svd_work_bytes(int n_sectors, const int* m, const int* n) {
  if (n_sectors < 0 || (n_sectors > 0 && (!m || !n))) return -1;
  SvdScratchLayout L;
  if (!svd_layout(n_sectors, m, n, L)) return -1;
  return ((int64_t)sizeof(SvdSector) * n_sectors + 255) / 256 * 256 + L.total;
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
  if (!svd_layout(n_sectors, m, n, L)) return MPS_EINVAL;
  const int64_t desc = ((int64_t)sizeof(SvdSector) * n_sectors + 255) / 256 * 256;
  if (work_bytes < desc + L.total) return MPS_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::vector<SvdSector> cta, cl;
  char* base = (char*)d_work + desc;
  for (int k = 0; k < n_sectors; ++k) {
    SvdSector S = {};
    S.theta = reinterpret_cast<const double2*>(d_mats) + mat_off[k];
    S.rowscale = d_rowscale ? d_rowscale + row_off[k] : nullptr;
    S.m = m[k];
    S.n = n[k];
    svd_fill_scratch(S, L, k, base);
    S.sigma = d_sigma + sig_off[k];
    S.Y = reinterpret_cast<double2*>(d_y) + y_off[k];
    S.status = d_status + k;
    (S.mode == kSvdCluster ? cl : cta).push_back(S);
  }
  std::vector<SvdSector> all(cta);
  all.insert(all.end(), cl.begin(), cl.end());
  std::vector<SvdGroup> groups;
  SvdTune tune;
  svd_forced_tune(tune);
  if (svd_group(all, groups, tune) != cudaSuccess) return MPS_ECUDA;
  if (cudaMemcpyAsync(d_work, all.data(), sizeof(SvdSector) * all.size(), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return MPS_ECUDA;
  const SvdSector* d_all = reinterpret_cast<const SvdSector*>(d_work);
  if (launch_svd_groups(d_all, groups, st, nullptr, 0, nullptr, nullptr) != cudaSuccess) return MPS_ECUDA;
  // the descriptors came from pageable host memory: finish before returning
  if (cudaStreamSynchronize(st) != cudaSuccess) return MPS_ECUDA;
  return MPS_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant: the scratch is a file-scope device array.  In host
// code the array's name is only a host-side stand-in, so its device address is
// looked up once per device (with that device current) and passed to the
// kernels; device code never names it.
// ---------------------------------------------------------------------------
namespace {
static __device__ __align__(256) unsigned char g_noalloc_scratch[MPS_NOALLOC_SCRATCH_BYTES];
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};
}  // namespace

extern "C" int mps_svd_sectors_noalloc(int n_sectors, const int* m, const int* n,
                                       const double* d_mats, const int64_t* mat_off,
                                       const double* d_rowscale, const int64_t* row_off,
                                       double* d_sigma, const int64_t* sig_off,
                                       double* d_y, const int64_t* y_off,
                                       int* d_status, void* cuda_stream) {
  if (n_sectors == 0) return MPS_OK;
  if (n_sectors < 0 || !m || !n || !d_mats || !mat_off || !d_sigma || !sig_off || !d_y || !y_off || !d_status)
    return MPS_EINVAL;
  if (d_rowscale && !row_off) return MPS_EINVAL;
  SvdScratchLayout L;
  if (!svd_layout(n_sectors, m, n, L)) return MPS_EINVAL;
  const int64_t desc = ((int64_t)sizeof(SvdSector) * n_sectors + 255) / 256 * 256;
  if (desc + L.total > (int64_t)MPS_NOALLOC_SCRATCH_BYTES) return MPS_ENOMEM;   // over the fixed scratch
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPS_ECUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return MPS_EINVAL;
  void* d_work = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MPS_ECUDA;
      g_noalloc_addr[dev] = p;
    }
    d_work = g_noalloc_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::vector<SvdSector> cta, cl;
  char* base = (char*)d_work + desc;
  for (int k = 0; k < n_sectors; ++k) {
    SvdSector S = {};
    S.theta = reinterpret_cast<const double2*>(d_mats) + mat_off[k];
    S.rowscale = d_rowscale ? d_rowscale + row_off[k] : nullptr;
    S.m = m[k];
    S.n = n[k];
    svd_fill_scratch(S, L, k, base);
    S.sigma = d_sigma + sig_off[k];
    S.Y = reinterpret_cast<double2*>(d_y) + y_off[k];
    S.status = d_status + k;
    (S.mode == kSvdCluster ? cl : cta).push_back(S);
  }
  std::vector<SvdSector> all(cta);
  all.insert(all.end(), cl.begin(), cl.end());
  std::vector<SvdGroup> groups;
  SvdTune tune;
  svd_forced_tune(tune);
  if (svd_group(all, groups, tune) != cudaSuccess) return MPS_ECUDA;
  if (cudaMemcpyAsync(d_work, all.data(), sizeof(SvdSector) * all.size(), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return MPS_ECUDA;
  const SvdSector* d_all = reinterpret_cast<const SvdSector*>(d_work);
  if (launch_svd_groups(d_all, groups, st, nullptr, 0, nullptr, nullptr) != cudaSuccess) return MPS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MPS_ECUDA;
  return MPS_OK;
}
