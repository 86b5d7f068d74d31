// Read-only measurements of the U(1) MPS (K6, K7).
//
// K6 expect_kernel: <O_s> = sum over blocks (l, m) of site s of
//     O(l - m) * sum_a lambda^[s]_a^2 * sum_b |B^[s][l,m]_{ab}|^2,
// the local form valid for the right-canonical state with lambda the Schmidt
// values (Sec. II).  One CTA per block writes one partial; the host adds the
// partials in block order, so the result is deterministic.
//
// K7 amplitude_kernel: <i_1..i_L|psi> is, by the Kronecker deltas of the U(1)
// amplitude formula (Sec. II), the product of exactly one block per site, the one
// selected by the right-charges of the configuration.  One CTA per configuration
// runs the vector-matrix chain with the row vector in shared memory.
//
// sample_kernel: sequential sampling of occupation patterns.  In the right-canonical
// form the sites right of a bond form an isometry, so the probability of a prefix is
// the squared norm of the row vector v = B^[0][c_0, c_1] ... B^[s-1][c_{s-1}, c_s] (the
// U(1) amplitude formula of Sec. II, truncated after site s-1).  At site s each
// occupation i with a block (c_s, c_s - i) gets w_i = |v B^[s][c_s, c_s - i]|^2; i is the
// first occupation (ascending) whose cumulative w_i / sum_j w_j exceeds the caller's
// uniform u_s; v becomes v B rescaled to unit norm, and the pattern's probability is the
// product of the conditionals.  One CTA per sample: a pass computes every w_i (fixed-order
// reductions), thread 0 takes the decision, a second pass forms the chosen product.
//
// entropy_kernel: the bond entropy S_b = -sum_a lambda_a^2 ln lambda_a^2 over all
// sectors of bond b (lambda are the Schmidt values of Sec. II; zero values add
// nothing).  One CTA, a fixed-order tree reduction, so the result is deterministic.
#include "mps_internal.h"

namespace mps {
namespace {

__global__ void expect_kernel(const ExpectTask* __restrict__ tasks, double* __restrict__ partial) {
  __shared__ double red[256];
  const ExpectTask T = tasks[blockIdx.x];
  const int64_t ne = (int64_t)T.Dl * T.Dm;
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < ne; e += blockDim.x) {
    const int a = (int)(e / T.Dm);
    const double2 v = T.blk[e];
    const double w = T.lam[a] * T.lam[a];
    acc = fma(w, fma(v.x, v.x, v.y * v.y), acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = T.w * red[0];
}

__global__ void amplitude_kernel(const AmpStep* __restrict__ steps, int L, int cap,
                                 double2* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char raw[];
  double2* v = reinterpret_cast<double2*>(raw);
  double2* w = v + cap;
  const AmpStep* S = steps + (int64_t)blockIdx.x * L;
  if (threadIdx.x == 0) v[0] = make_double2(1.0, 0.0);
  __syncthreads();
  int dim = 1;
  bool zero = false;
  for (int s = 0; s < L; ++s) {
    const AmpStep st = S[s];
    if (st.blk == nullptr || st.Dl != dim) { zero = true; break; }
    for (int j = threadIdx.x; j < st.Dm; j += blockDim.x) {
      double2 acc = make_double2(0.0, 0.0);
      for (int i = 0; i < st.Dl; ++i) {
        const double2 a = v[i], b = st.blk[(int64_t)i * st.Dm + j];
        acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
        acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
      }
      w[j] = acc;
    }
    __syncthreads();
    double2* t = v; v = w; w = t;
    dim = st.Dm;
  }
  if (threadIdx.x == 0) out[blockIdx.x] = (zero || dim != 1) ? make_double2(0.0, 0.0) : v[0];
}

__global__ void entropy_kernel(const double* __restrict__ lam, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double p = lam[i] * lam[i];
    if (p > 0.0) acc -= p * log(p);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__device__ __forceinline__ double block_sum(double x, double* red) {
  red[threadIdx.x] = x;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// w[j] = sum_a v[a] B[a, j] for j < Dm (B row-major Dl x Dm); returns |w|^2 when keep, else
// only the norm (w untouched)
__device__ __forceinline__ double row_times_block(const double2* v, const SampleEntry& e, double2* w, bool keep,
                                                  double* red) {
  double part = 0.0;
  for (int j = threadIdx.x; j < e.Dm; j += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int a = 0; a < e.Dl; ++a) {
      const double2 x = v[a], b = e.blk[(int64_t)a * e.Dm + j];
      acc.x = fma(x.x, b.x, fma(-x.y, b.y, acc.x));
      acc.y = fma(x.x, b.y, fma(x.y, b.x, acc.y));
    }
    if (keep) w[j] = acc;
    part = fma(acc.x, acc.x, fma(acc.y, acc.y, part));
  }
  return block_sum(part, red);
}

__global__ void sample_kernel(const SampleEntry* __restrict__ table, const int* __restrict__ site_off, int L, int d,
                              int cap, const double* __restrict__ uniforms, int* __restrict__ configs,
                              double* __restrict__ probs) {
  extern __shared__ __align__(16) unsigned char raw[];
  double2* v = reinterpret_cast<double2*>(raw);
  double2* w = v + cap;
  __shared__ double red[256];
  __shared__ double wn[MPS_MAX_D];
  __shared__ int pick, bad;
  const int k = blockIdx.x;
  if (threadIdx.x == 0) { v[0] = make_double2(1.0, 0.0); bad = 0; }
  __syncthreads();
  int li = 0;                     // sector index of the current right-charge in its bond table
  double p = 1.0;
  for (int s = 0; s < L; ++s) {
    const SampleEntry* row = table + site_off[s] + (int64_t)li * d;
    for (int i = 0; i < d; ++i) {
      const SampleEntry e = row[i];
      const double n2 = e.blk ? row_times_block(v, e, w, false, red) : -1.0;
      if (threadIdx.x == 0) wn[i] = n2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      int last = -1;
      for (int i = 0; i < d; ++i)
        if (wn[i] >= 0.0) { tot += wn[i]; last = i; }
      int c = last;
      if (last < 0 || !(tot > 0.0)) {
        bad = 1;
      } else {
        const double u = uniforms[(int64_t)k * L + s];
        double acc = 0.0;
        for (int i = 0; i < d; ++i) {
          if (wn[i] < 0.0) continue;
          acc += wn[i] / tot;
          if (u < acc) { c = i; break; }
        }
        p *= wn[c] / tot;
      }
      pick = c;
      configs[(int64_t)k * L + s] = bad ? -1 : c;
    }
    __syncthreads();
    if (bad) break;
    const SampleEntry e = row[pick];
    const double n2 = row_times_block(v, e, w, true, red);
    const double scale = 1.0 / sqrt(n2);
    for (int j = threadIdx.x; j < e.Dm; j += blockDim.x) v[j] = make_double2(w[j].x * scale, w[j].y * scale);
    li = e.next;
    __syncthreads();
  }
  if (threadIdx.x == 0) probs[k] = bad ? 0.0 : p;
}

}  // namespace

cudaError_t launch_sample(const SampleEntry* d_table, const int* d_site_off, int L, int d, int cap,
                          const double* d_uniforms, int n, int* d_configs, double* d_probs, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const size_t smem = sizeof(double2) * 2 * (size_t)cap;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launch();
  sample_kernel<<<n, 256, smem, st>>>(d_table, d_site_off, L, d, cap, d_uniforms, d_configs, d_probs);
  return cudaGetLastError();
}

cudaError_t launch_entropy(const double* d_lambda, int n, double* d_out, cudaStream_t st) {
  count_launch();
  entropy_kernel<<<1, 256, 0, st>>>(d_lambda, n, d_out);
  return cudaGetLastError();
}

cudaError_t launch_expect(const ExpectTask* d_tasks, int n_tasks, double* d_partial, cudaStream_t st) {
  if (n_tasks <= 0) return cudaSuccess;
  count_launch();
  expect_kernel<<<n_tasks, 256, 0, st>>>(d_tasks, d_partial);
  return cudaGetLastError();
}

cudaError_t launch_amplitude(const AmpStep* d_steps, int L, int n_cfg, double2* d_out, int cap,
                             cudaStream_t st) {
  if (n_cfg <= 0) return cudaSuccess;
  const size_t smem = sizeof(double2) * 2 * (size_t)cap;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(amplitude_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launch();
  amplitude_kernel<<<n_cfg, 256, smem, st>>>(d_steps, L, cap, d_out);
  return cudaGetLastError();
}

}  // namespace mps
