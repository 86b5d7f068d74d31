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

}  // namespace

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
