#include "krylov.cuh"

namespace stm {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum in a fixed order: warp shuffles, then warp 0 over the warp totals.
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

template <typename S>
__global__ void __launch_bounds__(kRedThreads) k_multidot(const S* __restrict__ w, const S* __restrict__ V,
                                                          int64_t ldv, int k, int with_norm, int64_t n,
                                                          double* __restrict__ partial) {
  __shared__ double sh[32];
  double acc[kMaxDots];
#pragma unroll
  for (int i = 0; i < kMaxDots; ++i) acc[i] = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double wj = (double)w[j];
#pragma unroll
    for (int i = 0; i < kMaxDots - 1; ++i)
      if (i < k) acc[i] = fma(wj, (double)V[i * ldv + j], acc[i]);
    if (with_norm) acc[kMaxDots - 1] = fma(wj, wj, acc[kMaxDots - 1]);
  }
#pragma unroll
  for (int i = 0; i < kMaxDots - 1; ++i) {
    if (i < k) {  // uniform over the block
      const double r = block_sum(acc[i], sh);
      if (threadIdx.x == 0) partial[i * gridDim.x + blockIdx.x] = r;
    }
  }
  if (with_norm) {
    const double r = block_sum(acc[kMaxDots - 1], sh);
    if (threadIdx.x == 0) partial[k * gridDim.x + blockIdx.x] = r;
  }
}

__global__ void k_finish(const double* __restrict__ partial, int m, int nb, double* __restrict__ out) {
  // one warp per result, fixed order: lane-strided partial sums then a shuffle tree
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < m; i += blockDim.x >> 5) {
    double v = 0.0;
    for (int b = lane; b < nb; b += 32) v += partial[i * nb + b];
    v = warp_sum(v);
    if (lane == 0) out[i] = v;
  }
}

template <typename S>
__global__ void k_multi_axpy(S* __restrict__ w, const S* __restrict__ V, int64_t ldv, int k,
                             const double* __restrict__ h, int64_t n) {
  double hh[kMaxDots];
#pragma unroll
  for (int i = 0; i < kMaxDots; ++i) hh[i] = (i < k) ? h[i] : 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)w[j];
#pragma unroll
    for (int i = 0; i < kMaxDots; ++i)
      if (i < k) v = fma(-hh[i], (double)V[i * ldv + j], v);
    w[j] = (S)v;
  }
}

template <typename S>
__global__ void k_scale_invnorm(S* __restrict__ v, const double* __restrict__ nrm2, int64_t n) {
  const double a = 1.0 / sqrt(*nrm2);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    v[j] = (S)((double)v[j] * a);
}

template <typename S>
__global__ void k_precond(S* __restrict__ z, const S* __restrict__ v, const S* __restrict__ mass, int64_t qn3,
                          int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    z[j] = v[j] / mass[j / qn3];
}

template <typename S, typename X>
__global__ void k_precond_combine(X* __restrict__ x, const S* __restrict__ V, int64_t ldv, int k, Coef16 y,
                                  const S* __restrict__ mass, int64_t qn3, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int i = 0; i < kMaxDots; ++i)
      if (i < k) v = fma(y.c[i], (double)V[i * ldv + j], v);
    x[j] = (X)((double)x[j] + v / (double)mass[j / qn3]);
  }
}

__global__ void __launch_bounds__(kRedThreads) k_energy(const double* __restrict__ u, const double* __restrict__ mass,
                                                        int64_t n3, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double v = u[j];
    acc = fma(mass[j / n3] * v, v, acc);
  }
  const double r = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = 0.5 * r;
}

template <typename D, typename S>
__global__ void k_convert(D* __restrict__ d, const S* __restrict__ s, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    d[j] = (D)s[j];
}

inline int grid_for(int64_t n) {
  int64_t g = (n + kRedThreads - 1) / kRedThreads;
  return (int)(g < 4 * kRedBlocks ? (g < 1 ? 1 : g) : 4 * kRedBlocks);
}

}  // namespace

template <typename S>
void multidot(const S* w, const S* V, int64_t ldv, int k, bool with_norm, int64_t n, double* partial, double* out,
              cudaStream_t s) {
  k_multidot<S><<<kRedBlocks, kRedThreads, 0, s>>>(w, V, ldv, k, with_norm ? 1 : 0, n, partial);
  k_finish<<<1, 512, 0, s>>>(partial, k + (with_norm ? 1 : 0), kRedBlocks, out);
}

template <typename S>
void multi_axpy(S* w, const S* V, int64_t ldv, int k, const double* h, int64_t n, cudaStream_t s) {
  k_multi_axpy<S><<<grid_for(n), kRedThreads, 0, s>>>(w, V, ldv, k, h, n);
}

template <typename S>
void scale_by_invnorm(S* v, const double* nrm2, int64_t n, cudaStream_t s) {
  k_scale_invnorm<S><<<grid_for(n), kRedThreads, 0, s>>>(v, nrm2, n);
}

template <typename S>
void precond_apply(S* z, const S* v, const S* mass, int64_t qn3, int64_t n, cudaStream_t s) {
  k_precond<S><<<grid_for(n), kRedThreads, 0, s>>>(z, v, mass, qn3, n);
}

template <typename S, typename X>
void precond_combine(X* x, const S* V, int64_t ldv, int k, const Coef16& y, const S* mass, int64_t qn3, int64_t n,
                     cudaStream_t s) {
  k_precond_combine<S, X><<<grid_for(n), kRedThreads, 0, s>>>(x, V, ldv, k, y, mass, qn3, n);
}

void energy_brick(const double* u, const double* mass, int64_t n3, int64_t n, double* partial, double* out,
                  cudaStream_t s) {
  k_energy<<<kRedBlocks, kRedThreads, 0, s>>>(u, mass, n3, n, partial);
  k_finish<<<1, 32, 0, s>>>(partial, 1, kRedBlocks, out);
}

template <typename D, typename S>
void convert(D* dst, const S* src, int64_t n, cudaStream_t s) {
  k_convert<D, S><<<grid_for(n), kRedThreads, 0, s>>>(dst, src, n);
}

template void multidot<double>(const double*, const double*, int64_t, int, bool, int64_t, double*, double*,
                               cudaStream_t);
template void multidot<float>(const float*, const float*, int64_t, int, bool, int64_t, double*, double*,
                              cudaStream_t);
template void multi_axpy<double>(double*, const double*, int64_t, int, const double*, int64_t, cudaStream_t);
template void multi_axpy<float>(float*, const float*, int64_t, int, const double*, int64_t, cudaStream_t);
template void scale_by_invnorm<double>(double*, const double*, int64_t, cudaStream_t);
template void scale_by_invnorm<float>(float*, const double*, int64_t, cudaStream_t);
template void precond_apply<double>(double*, const double*, const double*, int64_t, int64_t, cudaStream_t);
template void precond_apply<float>(float*, const float*, const float*, int64_t, int64_t, cudaStream_t);
template void precond_combine<double, double>(double*, const double*, int64_t, int, const Coef16&, const double*,
                                              int64_t, int64_t, cudaStream_t);
template void precond_combine<float, double>(double*, const float*, int64_t, int, const Coef16&, const float*,
                                             int64_t, int64_t, cudaStream_t);
template void precond_combine<float, float>(float*, const float*, int64_t, int, const Coef16&, const float*, int64_t,
                                            int64_t, cudaStream_t);
template void convert<float, double>(float*, const double*, int64_t, cudaStream_t);
template void convert<double, float>(double*, const float*, int64_t, cudaStream_t);

}  // namespace stm
