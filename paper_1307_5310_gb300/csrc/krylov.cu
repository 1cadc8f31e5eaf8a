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
// sums of the 16 products of four 16-byte chunks flushed into an FP64 total
// (the kernels call flush() after every fourth chunk: one conversion and one
// FP64 add per 16 products keeps the FP64 pipe off the critical path).
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

// 16-byte vectors: float4 / double2.  Basis columns are 16-byte aligned
// (their leading dimension is padded); a scalar loop takes the tail.
template <typename S>
struct Vec;
template <>
struct Vec<float> {
  using T = float4;
  static constexpr int W = 4;
  __device__ static float get(const float4& v, int l) { return l == 0 ? v.x : l == 1 ? v.y : l == 2 ? v.z : v.w; }
  __device__ static void set(float4& v, int l, float x) {
    if (l == 0) v.x = x; else if (l == 1) v.y = x; else if (l == 2) v.z = x; else v.w = x;
  }
};
template <>
struct Vec<double> {
  using T = double2;
  static constexpr int W = 2;
  __device__ static double get(const double2& v, int l) { return l == 0 ? v.x : v.y; }
  __device__ static void set(double2& v, int l, double x) {
    if (l == 0) v.x = x; else v.y = x;
  }
};

// chunks per loop trip: enough independent 16-byte loads in flight per thread
template <int K>
struct Unroll {
  static constexpr int U = K <= 1 ? 4 : (K <= 3 ? 2 : 1);
};

template <typename S, int K>
__global__ void __launch_bounds__(kRedThreads) k_multidot(const S* __restrict__ w, const S* __restrict__ V,
                                                          int64_t ldv, int with_norm, int64_t n,
                                                          double* __restrict__ partial, const int32_t* skip) {
  if (skip && *skip) return;
  using VT = typename Vec<S>::T;
  constexpr int W = Vec<S>::W, U = Unroll<K>::U;
  __shared__ double sh[32];
  Acc<S> acc[K + 1];
  const int64_t nv = n / W;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  const VT* w4 = reinterpret_cast<const VT*>(w);
  int chunks = 0;
  for (int64_t c0 = tid; c0 < nv; c0 += nth * U) {
    VT wv[U], vv[U][K > 0 ? K : 1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = c0 + u * nth;
      if (c < nv) {
        wv[u] = w4[c];
#pragma unroll
        for (int i = 0; i < K; ++i) vv[u][i] = reinterpret_cast<const VT*>(V + i * ldv)[c];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (c0 + u * nth < nv) {
#pragma unroll
        for (int l = 0; l < W; ++l) {
          const S x = Vec<S>::get(wv[u], l);
#pragma unroll
          for (int i = 0; i < K; ++i) acc[i].add(x, Vec<S>::get(vv[u][i], l));
          if (with_norm) acc[K].add(x, x);
        }
        if ((++chunks & 3) == 0) {
#pragma unroll
          for (int i = 0; i <= K; ++i) acc[i].flush();
        }
      }
    }
  }
  for (int64_t j = nv * W + tid; j < n; j += nth) {  // tail
    const S x = w[j];
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i].add(x, V[i * ldv + j]);
    if (with_norm) acc[K].add(x, x);
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
                                                           Coef16 c, int64_t n, double* __restrict__ partial,
                                                           const int32_t* skip, const double* cdev) {
  if (skip && *skip) return;
  using VT = typename Vec<S>::T;
  constexpr int W = Vec<S>::W, U = Unroll<K>::U;
  __shared__ double sh[32];
  S cc[K > 0 ? K : 1];
#pragma unroll
  for (int i = 0; i < K; ++i) cc[i] = (S)(cdev ? cdev[i] : c.c[i]);
  Acc<S> acc;
  const int64_t nv = n / W;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  VT* w4 = reinterpret_cast<VT*>(w);
  int chunks = 0;
  for (int64_t c0 = tid; c0 < nv; c0 += nth * U) {
    VT wv[U], vv[U][K > 0 ? K : 1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t cix = c0 + u * nth;
      if (cix < nv) {
        wv[u] = w4[cix];
#pragma unroll
        for (int i = 0; i < K; ++i) vv[u][i] = reinterpret_cast<const VT*>(V + i * ldv)[cix];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t cix = c0 + u * nth;
      if (cix < nv) {
#pragma unroll
        for (int l = 0; l < W; ++l) {
          S x = Vec<S>::get(wv[u], l);
#pragma unroll
          for (int i = 0; i < K; ++i) x = fma(-cc[i], Vec<S>::get(vv[u][i], l), x);
          Vec<S>::set(wv[u], l, x);
          acc.add(x, x);
        }
        if ((++chunks & 3) == 0) acc.flush();
        if (K > 0) w4[cix] = wv[u];
      }
    }
  }
  for (int64_t j = nv * W + tid; j < n; j += nth) {  // tail
    S x = w[j];
#pragma unroll
    for (int i = 0; i < K; ++i) x = fma(-cc[i], V[i * ldv + j], x);
    if (K > 0) w[j] = x;
    acc.add(x, x);
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
                          int64_t n, const int32_t* skip) {
  if (skip && *skip) return;
  using VT = typename Vec<S>::T;
  constexpr int W = Vec<S>::W;
  const int64_t nv = n / W;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = tid; c < nv && blk >= W; c += nth) {  // blocks of at least W entries: <= 2 per vector
    VT x = reinterpret_cast<const VT*>(v)[c];
    const int64_t j0 = c * W, b0 = block_of<Small>(j0, blk), edge = (b0 + 1) * blk;
    const S s0 = inv[b0], s1 = (j0 + W > edge) ? inv[b0 + 1] : s0;
#pragma unroll
    for (int l = 0; l < W; ++l) Vec<S>::set(x, l, Vec<S>::get(x, l) * (j0 + l < edge ? s0 : s1));
    reinterpret_cast<VT*>(z)[c] = x;
  }
  for (int64_t j = (blk >= W ? nv * W : 0) + tid; j < n; j += nth) z[j] = v[j] * inv[block_of<Small>(j, blk)];
}

template <typename S, typename X, int K, bool Small>
__global__ void k_precond_combine(X* __restrict__ x, const S* __restrict__ V, int64_t ldv, Coef16 y,
                                  const S* __restrict__ inv, int64_t blk, int64_t n, const GmresState* st) {
  // with st: k and the coefficients come from the device state (K is the largest k)
  const int kk = st ? st->k : K;
  if (kk <= 0) return;
  S yy[K > 0 ? K : 1];
#pragma unroll
  for (int i = 0; i < K; ++i) yy[i] = (S)(st ? st->yc[i] : y.c[i]);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    S v = S(0);
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i < kk) v = fma(yy[i], V[i * ldv + j], v);
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
__global__ void k_convert(D* __restrict__ d, const S* __restrict__ s, int64_t n, const int32_t* skip) {
  if (skip && *skip) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    d[j] = (D)s[j];
}


// ---- device-side GMRES control -------------------------------------------------------------
// One block of kCtrlThreads threads: the fixed-order reduction of kRedBlocks partial sums per
// value (warp i % warps sums value i lane-strided, then a shuffle tree), then thread 0 runs
// the scalar logic of the restart cycle on the state in device memory.
constexpr int kCtrlThreads = 512;

__device__ void reduce_values(const double* __restrict__ partial, int m, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < m; i += kCtrlThreads / 32) {
    double v = 0.0;
    for (int b = lane; b < kRedBlocks; b += 32) v += partial[i * kRedBlocks + b];
    v = warp_sum(v);
    if (lane == 0) out[i] = v;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kCtrlThreads) k_gm_reduce(const double* __restrict__ partial, GmresState* st,
                                                             int slot, const int32_t* skip) {
  if (skip && *skip) return;
  __shared__ double v[1];
  reduce_values(partial, 1, v);
  if (threadIdx.x == 0) st->red[slot] = v[0];
}

__global__ void k_gm_slab_start(GmresState* st, double tol, int max_it, int inexact) {
  st->ref = sqrt(st->red[0]);
  st->tol = tol;
  st->max_it = max_it;
  st->inexact = inexact;
  st->iters = 0;
  st->cycles = 0;
  st->status = 0;
  st->outer_done = 0;
  st->halt = 0;
  st->skip = 0;
  st->skip_reo = 1;
  st->k = 0;
  st->rel = 0.0;
  st->phi = 0.0;
  st->res = 0.0;
}

__global__ void k_gm_outer_check(GmresState* st) {
  st->k = 0;
  st->skip_reo = 1;
  if (st->halt) {
    st->skip = 1;
    return;
  }
  const double beta = sqrt(st->red[0]);
  const double ref = st->ref;
  st->rel = ref > 0 ? beta / ref : beta;
  if (!isfinite(st->rel)) {
    st->status = -5;  // STM_ENAN
    st->skip = 1;
    st->halt = 1;
    return;
  }
  bool done;
  if (st->inexact) {
    st->phi = sqrt(st->red[1]);
    done = st->phi <= st->tol;
  } else {
    done = st->rel <= st->tol;
  }
  if (done) st->outer_done = 1;
  st->skip = (done || st->iters >= st->max_it || beta == 0.0) ? 1 : 0;
  st->halt = st->skip;
}

__global__ void k_gm_cycle_init(GmresState* st, int slot_start, double floor_rel) {
  if (st->skip) return;
  const double b0 = sqrt(st->red[slot_start]);
  if (!(b0 > 0.0)) {
    st->skip = 1;
    st->halt = 1;
    return;
  }
  st->cycles += 1;
  // v_0 = V[0] / alpha_0 with V[0] = R = -r: alpha_0 = -|start|
  st->alpha[0] = -b0;
  st->g[0] = b0;
  const double target = st->inexact ? st->tol : st->tol * st->ref;
  st->tol_abs = fmax(target, floor_rel * b0);
}

__global__ void __launch_bounds__(kCtrlThreads) k_gm_gs(const double* __restrict__ partial, GmresState* st, int j,
                                                         int second) {
  if (second ? st->skip_reo : st->skip) return;
  __shared__ double v[kMaxDots + 1];
  reduce_values(partial, second ? j + 1 : j + 2, v);
  if (threadIdx.x == 0) {
    for (int i = 0; i <= j; ++i) {
      st->cc[i] = v[i] / (st->alpha[i] * st->alpha[i]);
      const double h = v[i] / (st->alpha[i] * st->alpha[j]);
      st->H[i * kMaxDots + j] = second ? st->H[i * kMaxDots + j] + h : h;
    }
    if (!second) st->before = v[j + 1];
  }
}

__global__ void __launch_bounds__(kCtrlThreads) k_gm_after(const double* __restrict__ partial, GmresState* st,
                                                            int reorth) {
  if (st->skip) {
    st->skip_reo = 1;
    return;
  }
  __shared__ double v[1];
  reduce_values(partial, 1, v);
  if (threadIdx.x == 0) {
    st->after = v[0];
    st->skip_reo = (reorth && v[0] < 0.5 * st->before) ? 0 : 1;
  }
}

__global__ void __launch_bounds__(kCtrlThreads) k_gm_givens(const double* __restrict__ partial, GmresState* st, int j,
                                                             int m, int reo_mode) {
  if (st->skip) return;
  __shared__ double v[1];
  const bool fresh = reo_mode ? !st->skip_reo : true;  // uniform over the block
  if (fresh) reduce_values(partial, 1, v);
  if (threadIdx.x != 0) return;
  const double after = fresh ? v[0] : st->after;
  double* H = st->H;
  if (!isfinite(after) || !isfinite(st->before)) {
    st->status = -5;  // STM_ENAN
    st->skip = 1;
    st->halt = 1;
    return;
  }
  const double nw = sqrt(after);
  st->alpha[j + 1] = st->alpha[j] < 0 ? -nw : nw;
  H[(j + 1) * kMaxDots + j] = nw / fabs(st->alpha[j]);
  for (int i = 0; i < j; ++i) {
    const double x = H[i * kMaxDots + j], y = H[(i + 1) * kMaxDots + j];
    H[i * kMaxDots + j] = st->cs[i] * x + st->sn[i] * y;
    H[(i + 1) * kMaxDots + j] = -st->sn[i] * x + st->cs[i] * y;
  }
  const double x = H[j * kMaxDots + j], y = H[(j + 1) * kMaxDots + j];
  const double r = hypot(x, y);
  st->cs[j] = r > 0 ? x / r : 1.0;
  st->sn[j] = r > 0 ? y / r : 0.0;
  H[j * kMaxDots + j] = r;
  H[(j + 1) * kMaxDots + j] = 0.0;
  st->g[j + 1] = -st->sn[j] * st->g[j];
  st->g[j] = st->cs[j] * st->g[j];
  st->iters += 1;
  st->k = j + 1;
  if (fabs(st->g[j + 1]) <= st->tol_abs || nw == 0.0 || st->iters >= st->max_it || j + 1 >= m) st->skip = 1;
}

__global__ void k_gm_backsub(GmresState* st) {
  const int k = st->k;
  double y[kMaxDots];
  for (int i = k - 1; i >= 0; --i) {
    double t = st->g[i];
    for (int l = i + 1; l < k; ++l) t -= st->H[i * kMaxDots + l] * y[l];
    y[i] = t / st->H[i * kMaxDots + i];
  }
  for (int i = 0; i < kMaxDots; ++i) st->yc[i] = i < k ? y[i] / st->alpha[i] : 0.0;
  st->res = fabs(st->g[k]);
}

inline int grid_for(int64_t n) {
  int64_t g = (n + kRedThreads - 1) / kRedThreads;
  return (int)(g < 4 * kRedBlocks ? (g < 1 ? 1 : g) : 4 * kRedBlocks);
}

inline bool small(int64_t n) { return n <= (int64_t)0xffffffffLL; }

template <typename S, int K>
void multidot_k(const S* w, const S* V, int64_t ldv, bool with_norm, int64_t n, double* partial, cudaStream_t s,
                const int32_t* skip) {
  k_multidot<S, K><<<kRedBlocks, kRedThreads, 0, s>>>(w, V, ldv, with_norm ? 1 : 0, n, partial, skip);
}

template <typename S, int K>
void axpy_k(S* w, const S* V, int64_t ldv, const Coef16& c, int64_t n, double* partial, cudaStream_t s,
            const int32_t* skip, const double* cdev) {
  k_axpy_norm<S, K><<<kRedBlocks, kRedThreads, 0, s>>>(w, V, ldv, c, n, partial, skip, cdev);
}

template <typename S, typename X, int K>
void combine_k(X* x, const S* V, int64_t ldv, const Coef16& y, const S* inv, int64_t blk, int64_t n, cudaStream_t s,
               const GmresState* st) {
  if (small(n)) k_precond_combine<S, X, K, true><<<grid_for(n), kRedThreads, 0, s>>>(x, V, ldv, y, inv, blk, n, st);
  else k_precond_combine<S, X, K, false><<<grid_for(n), kRedThreads, 0, s>>>(x, V, ldv, y, inv, blk, n, st);
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
              cudaStream_t s, const int32_t* skip) {
#define STM_MD(K) multidot_k<S, K>(w, V, ldv, with_norm, n, partial, s, skip)
  STM_SWITCH_K(k, STM_MD)
#undef STM_MD
  if (out) k_finish<<<1, 512, 0, s>>>(partial, k + (with_norm ? 1 : 0), kRedBlocks, out);
}

template <typename S>
void axpy_norm(S* w, const S* V, int64_t ldv, int k, const Coef16& c, int64_t n, double* partial, double* out,
               cudaStream_t s, const int32_t* skip, const double* cdev) {
#define STM_AX(K) axpy_k<S, K>(w, V, ldv, c, n, partial, s, skip, cdev)
  STM_SWITCH_K(k, STM_AX)
#undef STM_AX
  if (out) k_finish<<<1, 32, 0, s>>>(partial, 1, kRedBlocks, out);
}

template <typename S>
void precond_apply(S* z, const S* v, const S* inv, int64_t blk, int64_t n, cudaStream_t s, const int32_t* skip) {
  if (small(n)) k_precond<S, true><<<grid_for(n), kRedThreads, 0, s>>>(z, v, inv, blk, n, skip);
  else k_precond<S, false><<<grid_for(n), kRedThreads, 0, s>>>(z, v, inv, blk, n, skip);
}

template <typename S, typename X>
void precond_combine(X* x, const S* V, int64_t ldv, int k, const Coef16& y, const S* inv, int64_t blk, int64_t n,
                     cudaStream_t s, const GmresState* st) {
#define STM_CB(K) combine_k<S, X, K>(x, V, ldv, y, inv, blk, n, s, st)
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
void convert(D* dst, const S* src, int64_t n, cudaStream_t s, const int32_t* skip) {
  k_convert<D, S><<<grid_for(n), kRedThreads, 0, s>>>(dst, src, n, skip);
}


void gmres_reduce(const double* partial, GmresState* st, int slot, cudaStream_t s, const int32_t* skip) {
  k_gm_reduce<<<1, kCtrlThreads, 0, s>>>(partial, st, slot, skip);
}
void gmres_slab_start(GmresState* st, double tol, int max_it, int inexact, cudaStream_t s) {
  k_gm_slab_start<<<1, 1, 0, s>>>(st, tol, max_it, inexact);
}
void gmres_outer_check(GmresState* st, cudaStream_t s) { k_gm_outer_check<<<1, 1, 0, s>>>(st); }
void gmres_cycle_init(GmresState* st, int slot_start, double floor_rel, cudaStream_t s) {
  k_gm_cycle_init<<<1, 1, 0, s>>>(st, slot_start, floor_rel);
}
void gmres_gs(const double* partial, GmresState* st, int j, int second, cudaStream_t s) {
  k_gm_gs<<<1, kCtrlThreads, 0, s>>>(partial, st, j, second);
}
void gmres_after(const double* partial, GmresState* st, int reorth, cudaStream_t s) {
  k_gm_after<<<1, kCtrlThreads, 0, s>>>(partial, st, reorth);
}
void gmres_givens(const double* partial, GmresState* st, int j, int m, int reo_mode, cudaStream_t s) {
  k_gm_givens<<<1, kCtrlThreads, 0, s>>>(partial, st, j, m, reo_mode);
}
void gmres_backsub(GmresState* st, int m, cudaStream_t s) {
  (void)m;
  k_gm_backsub<<<1, 1, 0, s>>>(st);
}

template void multidot<double>(const double*, const double*, int64_t, int, bool, int64_t, double*, double*,
                               cudaStream_t, const int32_t*);
template void multidot<float>(const float*, const float*, int64_t, int, bool, int64_t, double*, double*,
                              cudaStream_t, const int32_t*);
template void axpy_norm<double>(double*, const double*, int64_t, int, const Coef16&, int64_t, double*, double*,
                                cudaStream_t, const int32_t*, const double*);
template void axpy_norm<float>(float*, const float*, int64_t, int, const Coef16&, int64_t, double*, double*,
                               cudaStream_t, const int32_t*, const double*);
template void precond_apply<double>(double*, const double*, const double*, int64_t, int64_t, cudaStream_t,
                                    const int32_t*);
template void precond_apply<float>(float*, const float*, const float*, int64_t, int64_t, cudaStream_t,
                                   const int32_t*);
template void precond_combine<double, double>(double*, const double*, int64_t, int, const Coef16&, const double*,
                                              int64_t, int64_t, cudaStream_t, const GmresState*);
template void precond_combine<float, double>(double*, const float*, int64_t, int, const Coef16&, const float*,
                                             int64_t, int64_t, cudaStream_t, const GmresState*);
template void precond_combine<float, float>(float*, const float*, int64_t, int, const Coef16&, const float*, int64_t,
                                            int64_t, cudaStream_t, const GmresState*);
template void convert<float, double>(float*, const double*, int64_t, cudaStream_t, const int32_t*);
template void convert<double, float>(double*, const float*, int64_t, cudaStream_t, const int32_t*);

}  // namespace stm
