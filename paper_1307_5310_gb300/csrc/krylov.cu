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

// Per-thread accumulator: FP64 for double storage; for float storage, FP32
// sums of 8 consecutive products flushed into an FP64 total.
template <typename S>
struct Acc;
template <>
struct Acc<double> {
  double a = 0.0;
  __device__ __forceinline__ void add(double x, double y) { a = fma(x, y, a); }
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ double get() const { return a; }
};
template <>
struct Acc<float> {
  double a = 0.0;
  float f = 0.f;
  __device__ __forceinline__ void add(float x, float y) { f = fmaf(x, y, f); }
  __device__ __forceinline__ void flush() {
    a += (double)f;
    f = 0.f;
  }
  __device__ __forceinline__ double get() const { return a + (double)f; }
};

template <typename S, int K>
__global__ void __launch_bounds__(kRedThreads) k_multidot(const S* __restrict__ w, const S* __restrict__ V,
                                                          int64_t ldv, int with_norm, int64_t n,
                                                          double* __restrict__ partial) {
  __shared__ double sh[32];
  Acc<S> acc[K + 1];
  int cnt = 0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const S wj = w[j];
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i].add(wj, V[i * ldv + j]);
    if (with_norm) acc[K].add(wj, wj);
    if (++cnt == 8) {
      cnt = 0;
#pragma unroll
      for (int i = 0; i <= K; ++i) acc[i].flush();
    }
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const double r = block_sum(acc[i].get(), sh);
    if (threadIdx.x == 0) partial[i * gridDim.x + blockIdx.x] = r;
  }
  if (with_norm) {
    const double r = block_sum(acc[K].get(), sh);
    if (threadIdx.x == 0) partial[K * gridDim.x + blockIdx.x] = r;
  }
}

template <typename S, int K>
__global__ void __launch_bounds__(kRedThreads) k_axpy_norm(S* __restrict__ w, const S* __restrict__ V, int64_t ldv,
                                                           Coef16 c, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[32];
  S cc[K > 0 ? K : 1];
#pragma unroll
  for (int i = 0; i < K; ++i) cc[i] = (S)c.c[i];
  Acc<S> acc;
  int cnt = 0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    S v = w[j];
#pragma unroll
    for (int i = 0; i < K; ++i) v = fma(-cc[i], V[i * ldv + j], v);
    if (K > 0) w[j] = v;
    acc.add(v, v);
    if (++cnt == 8) {
      cnt = 0;
      acc.flush();
    }
  }
  const double r = block_sum(acc.get(), sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = r;
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

template <bool Small>
__device__ __forceinline__ int64_t block_of(int64_t j, int64_t blk) {
  return Small ? (int64_t)((uint32_t)j / (uint32_t)blk) : j / blk;
}

template <typename S, bool Small>
__global__ void k_precond(S* __restrict__ z, const S* __restrict__ v, const S* __restrict__ inv, int64_t blk,
                          int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    z[j] = v[j] * inv[block_of<Small>(j, blk)];
}

template <typename S, typename X, int K, bool Small>
__global__ void k_precond_combine(X* __restrict__ x, const S* __restrict__ V, int64_t ldv, Coef16 y,
                                  const S* __restrict__ inv, int64_t blk, int64_t n) {
  S yy[K > 0 ? K : 1];
#pragma unroll
  for (int i = 0; i < K; ++i) yy[i] = (S)y.c[i];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    S v = S(0);
#pragma unroll
    for (int i = 0; i < K; ++i) v = fma(yy[i], V[i * ldv + j], v);
    x[j] = (X)x[j] + (X)(v * inv[block_of<Small>(j, blk)]);
  }
}

template <bool Small>
__global__ void __launch_bounds__(kRedThreads) k_energy(const double* __restrict__ u, const double* __restrict__ mass,
                                                        int64_t n3, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double v = u[j];
    acc = fma(mass[block_of<Small>(j, n3)] * v, v, acc);
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

inline bool small(int64_t n) { return n <= (int64_t)0xffffffffLL; }

template <typename S, int K>
void multidot_k(const S* w, const S* V, int64_t ldv, bool with_norm, int64_t n, double* partial, cudaStream_t s) {
  k_multidot<S, K><<<kRedBlocks, kRedThreads, 0, s>>>(w, V, ldv, with_norm ? 1 : 0, n, partial);
}

template <typename S, int K>
void axpy_k(S* w, const S* V, int64_t ldv, const Coef16& c, int64_t n, double* partial, cudaStream_t s) {
  k_axpy_norm<S, K><<<kRedBlocks, kRedThreads, 0, s>>>(w, V, ldv, c, n, partial);
}

template <typename S, typename X, int K>
void combine_k(X* x, const S* V, int64_t ldv, const Coef16& y, const S* inv, int64_t blk, int64_t n, cudaStream_t s) {
  if (small(n)) k_precond_combine<S, X, K, true><<<grid_for(n), kRedThreads, 0, s>>>(x, V, ldv, y, inv, blk, n);
  else k_precond_combine<S, X, K, false><<<grid_for(n), kRedThreads, 0, s>>>(x, V, ldv, y, inv, blk, n);
}

#define STM_SWITCH_K(k, CALL)  \
  switch (k) {                 \
    case 0: CALL(0); break;    \
    case 1: CALL(1); break;    \
    case 2: CALL(2); break;    \
    case 3: CALL(3); break;    \
    case 4: CALL(4); break;    \
    case 5: CALL(5); break;    \
    case 6: CALL(6); break;    \
    case 7: CALL(7); break;    \
    case 8: CALL(8); break;    \
    case 9: CALL(9); break;    \
    case 10: CALL(10); break;  \
    case 11: CALL(11); break;  \
    case 12: CALL(12); break;  \
    case 13: CALL(13); break;  \
    case 14: CALL(14); break;  \
    default: CALL(15); break;  \
  }

}  // namespace

template <typename S>
void multidot(const S* w, const S* V, int64_t ldv, int k, bool with_norm, int64_t n, double* partial, double* out,
              cudaStream_t s) {
#define STM_MD(K) multidot_k<S, K>(w, V, ldv, with_norm, n, partial, s)
  STM_SWITCH_K(k, STM_MD)
#undef STM_MD
  k_finish<<<1, 512, 0, s>>>(partial, k + (with_norm ? 1 : 0), kRedBlocks, out);
}

template <typename S>
void axpy_norm(S* w, const S* V, int64_t ldv, int k, const Coef16& c, int64_t n, double* partial, double* out,
               cudaStream_t s) {
#define STM_AX(K) axpy_k<S, K>(w, V, ldv, c, n, partial, s)
  STM_SWITCH_K(k, STM_AX)
#undef STM_AX
  k_finish<<<1, 32, 0, s>>>(partial, 1, kRedBlocks, out);
}

template <typename S>
void precond_apply(S* z, const S* v, const S* inv, int64_t blk, int64_t n, cudaStream_t s) {
  if (small(n)) k_precond<S, true><<<grid_for(n), kRedThreads, 0, s>>>(z, v, inv, blk, n);
  else k_precond<S, false><<<grid_for(n), kRedThreads, 0, s>>>(z, v, inv, blk, n);
}

template <typename S, typename X>
void precond_combine(X* x, const S* V, int64_t ldv, int k, const Coef16& y, const S* inv, int64_t blk, int64_t n,
                     cudaStream_t s) {
#define STM_CB(K) combine_k<S, X, K>(x, V, ldv, y, inv, blk, n, s)
  STM_SWITCH_K(k, STM_CB)
#undef STM_CB
}

void energy_brick(const double* u, const double* mass, int64_t n3, int64_t n, double* partial, double* out,
                  cudaStream_t s) {
  if (small(n)) k_energy<true><<<kRedBlocks, kRedThreads, 0, s>>>(u, mass, n3, n, partial);
  else k_energy<false><<<kRedBlocks, kRedThreads, 0, s>>>(u, mass, n3, n, partial);
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
template void axpy_norm<double>(double*, const double*, int64_t, int, const Coef16&, int64_t, double*, double*,
                                cudaStream_t);
template void axpy_norm<float>(float*, const float*, int64_t, int, const Coef16&, int64_t, double*, double*,
                               cudaStream_t);
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
