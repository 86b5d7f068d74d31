// Global top-chi truncation across all charge sectors of one update (K3).
//
// Sec. II bounds every bond by chi; the truncation is global over the middle
// charges.  Rule (the paper is silent on details; the same rule is in the
// oracle): candidates are sigma > cutoff * |sigma|_2 (strict).  If at most chi
// candidates exist all are kept.  Otherwise v = the chi-th largest candidate;
// values above v + tau are kept, values within [v - tau, v + tau] are ties and
// are taken in (charge ascending, index ascending) order until chi are kept,
// tau = 1e-11 * sigma_max.  Each sector's kept set is a prefix of its
// descending list, so the result is one count per sector.
//
// One CTA per update.  v is found exactly by bisection on the IEEE bit pattern
// of non-negative doubles (monotone as unsigned integers): each step counts,
// per sector, the values >= x by a binary search over the sorted spectrum.
// All sums are fixed-order block reductions (deterministic).
#include "mps_internal.h"

namespace mps {
namespace {

constexpr int kSelThreads = 256;

template <typename T>
__device__ T block_sum(T v, T* red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
  for (int s = kSelThreads / 2; s; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  const T r = red[0];
  __syncthreads();
  return r;
}

// number of entries of a descending array that are > x
__device__ int count_gt(const double* a, int k, double x) {
  int lo = 0, hi = k;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] > x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
// number of entries of a descending array that are >= x
__device__ int count_ge(const double* a, int k, double x) {
  int lo = 0, hi = k;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] >= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kSelThreads) select_kernel(const SelectSector* __restrict__ secs,
                                                             const SelectTask* __restrict__ tasks,
                                                             int* __restrict__ kept,
                                                             SelectResult* __restrict__ res) {
  __shared__ double dred[kSelThreads];
  __shared__ long long ired[kSelThreads];
  const SelectTask T = tasks[blockIdx.x];
  const int tid = threadIdx.x;
  const int ns = T.s1 - T.s0;
  // |sigma|^2 and sigma_max
  double part = 0.0, vmax = 0.0;
  for (int s = 0; s < ns; ++s) {
    const SelectSector S = secs[T.s0 + s];
    for (int j = tid; j < S.k; j += kSelThreads) part = fma(S.sigma[j], S.sigma[j], part);
    if (S.k > 0) vmax = fmax(vmax, S.sigma[0]);
  }
  const double total2 = block_sum(part, dred);
  SelectResult R;
  R.norm_all = sqrt(total2);
  R.band = 0;
  R.pad = 0;
  if (!(total2 > 0.0)) {
    if (tid == 0) {
      R.norm_kept = 0.0; R.trunc_err = 1.0; R.n_candidates = 0; R.status = -1; R.cut = 0.0;
      res[blockIdx.x] = R;
    }
    for (int s = tid; s < ns; s += kSelThreads) kept[T.s0 + s] = 0;
    return;
  }
  const double thr = T.cutoff * R.norm_all;
  long long nc_part = 0;
  for (int s = tid; s < ns; s += kSelThreads) {
    const SelectSector S = secs[T.s0 + s];
    const int c = count_gt(S.sigma, S.k, thr);
    kept[T.s0 + s] = c;
    nc_part += c;
  }
  const long long nc = block_sum(nc_part, ired);
  int band_total = 0;
  if (nc > T.chi) {
    // largest x with #{sigma >= x, sigma > thr} >= chi is the chi-th largest candidate
    unsigned long long lo = 0ull, hi = (unsigned long long)__double_as_longlong(vmax) + 1ull;
    while (hi - lo > 1ull) {
      const unsigned long long mid = lo + ((hi - lo) >> 1);
      const double x = __longlong_as_double((long long)mid);
      long long cnt = 0;
      for (int s = tid; s < ns; s += kSelThreads) {
        const SelectSector S = secs[T.s0 + s];
        cnt += min(count_ge(S.sigma, S.k, x), count_gt(S.sigma, S.k, thr));
      }
      cnt = block_sum(cnt, ired);
      if (cnt >= T.chi) lo = mid; else hi = mid;
    }
    const double v = __longlong_as_double((long long)lo);
    const double delta = kTieRel * vmax;
    const double upper = v + delta, lower = v - delta;
    long long above_part = 0, band_part = 0;
    for (int s = tid; s < ns; s += kSelThreads) {
      const SelectSector S = secs[T.s0 + s];
      const int cand = count_gt(S.sigma, S.k, thr);
      const int above = count_gt(S.sigma, S.k, upper);
      const int inband = min(count_ge(S.sigma, S.k, lower), cand) - above;
      above_part += above;
      band_part += inband;
    }
    const long long above_total = block_sum(above_part, ired);
    band_total = (int)block_sum(band_part, ired);
    if (tid == 0) {
      long long left = T.chi - above_total;
      for (int s = 0; s < ns; ++s) {
        const SelectSector S = secs[T.s0 + s];
        const int cand = count_gt(S.sigma, S.k, thr);
        const int above = count_gt(S.sigma, S.k, upper);
        const int inband = min(count_ge(S.sigma, S.k, lower), cand) - above;
        const long long take = min((long long)inband, left);
        kept[T.s0 + s] = above + (int)take;
        left -= take;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  // kept and discarded weight
  double kp = 0.0, dp = 0.0;
  for (int s = 0; s < ns; ++s) {
    const SelectSector S = secs[T.s0 + s];
    const int k = kept[T.s0 + s];
    for (int j = tid; j < S.k; j += kSelThreads) {
      const double w = S.sigma[j] * S.sigma[j];
      if (j < k) kp += w; else dp += w;
    }
  }
  const double kept2 = block_sum(kp, dred);
  const double disc2 = block_sum(dp, dred);
  // the cut: smallest kept value (fixed-order reduction: min is order independent anyway)
  double cmin = 1.0e308;
  for (int s = tid; s < ns; s += kSelThreads) {
    const int k = kept[T.s0 + s];
    if (k > 0) cmin = fmin(cmin, secs[T.s0 + s].sigma[k - 1]);
  }
  dred[tid] = cmin;
  __syncthreads();
  for (int s = kSelThreads / 2; s; s >>= 1) {
    if (tid < s) dred[tid] = fmin(dred[tid], dred[tid + s]);
    __syncthreads();
  }
  const double cut = dred[0];
  if (tid == 0) {
    R.cut = cut >= 1.0e308 ? 0.0 : cut;
    R.norm_kept = sqrt(kept2);
    R.trunc_err = disc2 / total2;
    R.band = band_total;
    R.n_candidates = (int)nc;
    R.status = 0;
    res[blockIdx.x] = R;
  }
}

}  // namespace

cudaError_t launch_select(const SelectSector* d_secs, const SelectTask* d_tasks, int n_tasks,
                          int* d_kept, SelectResult* d_res, cudaStream_t st) {
  if (n_tasks <= 0) return cudaSuccess;
  count_launch();
  select_kernel<<<n_tasks, kSelThreads, 0, st>>>(d_secs, d_tasks, d_kept, d_res);
  return cudaGetLastError();
}

}  // namespace mps
