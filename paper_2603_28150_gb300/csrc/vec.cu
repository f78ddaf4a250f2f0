// Vector kernels around the operator: FP64 inner products and norms (the
// adjoint test of Eq. 9, FISTA residuals, the power iteration for ||H*H||)
// and small helpers. (The FISTA proximal/momentum update of Eq. 14-15 is
// fused into the last FFT stage of the gradient, fft.cu.)
// Reductions are deterministic: fixed grid, per-block tree sums, then one
// block sums the partials in index order.
#include "pat_internal.h"

namespace pat {
namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) ws[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = l < nw ? ws[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_dot(const R* __restrict__ a, const R* __restrict__ b,
                                                int64_t n, double* __restrict__ partials) {
  pdl_wait();
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kBlock)
    acc = fma((double)a[i], (double)b[i], acc);
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_sum_partials(const double* __restrict__ partials, int n,
                                                       double* __restrict__ out) {
  pdl_wait();
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 1024) acc += partials[i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) *out = s;
}

// One block per group: out[blockIdx.x] = sum of its `per` partials.
__global__ void __launch_bounds__(256) k_group_sums(const double* __restrict__ partials, int per,
                                                    double* __restrict__ out) {
  const double* p = partials + (int64_t)blockIdx.x * per;
  pdl_wait();
  double acc = 0.0;
  for (int i = threadIdx.x; i < per; i += 256) acc += p[i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_scale(const R* __restrict__ in, R* __restrict__ out,
                                                  int64_t n, const double* __restrict__ sumsq) {
  const R s = (R)(1.0 / sqrt(*sumsq));
  for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kBlock)
    out[i] = in[i] * s;
}

int grid_for(int64_t n, int cap) {
  int64_t b = (n + kBlock - 1) / kBlock;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_partials_sum(const double* partials, int n, double* out, cudaStream_t s) {
  return launch_pdl(k_sum_partials, dim3(1), dim3(1024), 0, s, partials, n, out);
}

cudaError_t launch_group_sums(const double* partials, int per, int groups, double* out,
                              cudaStream_t s) {
  return launch_pdl(k_group_sums, dim3(groups), dim3(256), 0, s, partials, per, out);
}

cudaError_t launch_dot(const Plan& p, const void* a, const void* b, int64_t n, double* out_dev,
                       cudaStream_t s) {
  const int g = grid_for(n, kReduceBlocks);
  cudaError_t e =
      p.L.fp64 ? launch_pdl(k_dot<double>, dim3(g), dim3(kBlock), 0, s,
                            static_cast<const double*>(a), static_cast<const double*>(b), n, p.red)
               : launch_pdl(k_dot<float>, dim3(g), dim3(kBlock), 0, s,
                            static_cast<const float*>(a), static_cast<const float*>(b), n, p.red);
  if (e != cudaSuccess) return e;
  return launch_partials_sum(p.red, g, out_dev, s);
}

cudaError_t launch_scale_by_inv_norm(const Plan& p, const void* in, void* out, int64_t n,
                                     const double* sumsq_dev, cudaStream_t s) {
  const int g = grid_for(n, 152 * 16);
  if (p.L.fp64)
    k_scale<double><<<g, kBlock, 0, s>>>(static_cast<const double*>(in), static_cast<double*>(out),
                                          n, sumsq_dev);
  else
    k_scale<float><<<g, kBlock, 0, s>>>(static_cast<const float*>(in), static_cast<float*>(out), n,
                                         sumsq_dev);
  return cudaGetLastError();
}

}  // namespace pat
