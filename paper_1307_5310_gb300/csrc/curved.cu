#include "curved.cuh"

namespace stm {

namespace {

template <typename T>
struct CTab {
  T Lq[kMaxN][kMaxN + 1];
};

template <typename T>
CTab<T> ctab(const CurvedTables& ct) {
  CTab<T> t;
  for (int j = 0; j < kMaxN; ++j)
    for (int g = 0; g <= kMaxN; ++g) t.Lq[j][g] = (T)ct.Lq[j][g];
  return t;
}

// Jacobian DF of the trilinear map of X8 at reference point xh.
__device__ void trilinear_DF(const double* X8, const double xh[3], double DF[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) DF[i][j] = 0.0;
  for (int v = 0; v < 8; ++v) {
    const int bit[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
    double f[3], df[3];
    for (int a = 0; a < 3; ++a) {
      f[a] = bit[a] ? xh[a] : 1.0 - xh[a];
      df[a] = bit[a] ? 1.0 : -1.0;
    }
    const double dN[3] = {df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) DF[i][j] += X8[3 * v + i] * dN[j];
  }
}

template <int P>
__global__ void __launch_bounds__(256) k_metric(const double* __restrict__ X8g, const double* __restrict__ eps,
                                                const double* __restrict__ mu, int64_t ne, CurvedTables ct,
                                                double* __restrict__ Gw, double* __restrict__ Pinv, int* bad) {
  constexpr int NQ = P + 2, NQ3 = NQ * NQ * NQ;
  __shared__ double X8[24];
  __shared__ double gsum[6];
  for (int64_t e = blockIdx.x; e < ne; e += gridDim.x) {
    if (threadIdx.x < 24) X8[threadIdx.x] = X8g[e * 24 + threadIdx.x];
    __syncthreads();
    double* ge = Gw + e * 6 * NQ3;
    for (int g = threadIdx.x; g < NQ3; g += blockDim.x) {
      const int gx = g % NQ, gy = (g / NQ) % NQ, gz = g / (NQ * NQ);
      const double xh[3] = {ct.xq[gx], ct.xq[gy], ct.xq[gz]};
      double DF[3][3];
      trilinear_DF(X8, xh, DF);
      // adjugate (cofactor transpose): adj = det * DF^{-1}
      double A[3][3];
      A[0][0] = DF[1][1] * DF[2][2] - DF[1][2] * DF[2][1];
      A[0][1] = DF[0][2] * DF[2][1] - DF[0][1] * DF[2][2];
      A[0][2] = DF[0][1] * DF[1][2] - DF[0][2] * DF[1][1];
      A[1][0] = DF[1][2] * DF[2][0] - DF[1][0] * DF[2][2];
      A[1][1] = DF[0][0] * DF[2][2] - DF[0][2] * DF[2][0];
      A[1][2] = DF[0][2] * DF[1][0] - DF[0][0] * DF[1][2];
      A[2][0] = DF[1][0] * DF[2][1] - DF[1][1] * DF[2][0];
      A[2][1] = DF[0][1] * DF[2][0] - DF[0][0] * DF[2][1];
      A[2][2] = DF[0][0] * DF[1][1] - DF[0][1] * DF[1][0];
      const double J = DF[0][0] * A[0][0] + DF[0][1] * A[1][0] + DF[0][2] * A[2][0];
      if (!(J > 0.0)) atomicExch(bad, 1);
      // G = |J| DF^{-1} DF^{-T} = A A^T / J
      const double w = ct.wq[gx] * ct.wq[gy] * ct.wq[gz] / J;
      const int pr[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
      for (int k = 0; k < 6; ++k) {
        const int a = pr[k][0], b = pr[k][1];
        ge[k * NQ3 + g] = w * (A[a][0] * A[b][0] + A[a][1] * A[b][1] + A[a][2] * A[b][2]);
      }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
      double s = 0.0;
      for (int g = 0; g < NQ3; ++g) s += ge[threadIdx.x * NQ3 + g];
      gsum[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      const double m = threadIdx.x == 0 ? eps[e] : mu[e];
      const double a = m * gsum[0], b = m * gsum[1], c = m * gsum[2];
      const double d = m * gsum[3], f = m * gsum[4], h = m * gsum[5];  // xy, xz, yz
      // inverse of the symmetric [[a d f][d b h][f h c]]
      const double c00 = b * c - h * h, c01 = f * h - d * c, c02 = d * h - b * f;
      const double c11 = a * c - f * f, c12 = d * f - a * h, c22 = a * b - d * d;
      const double det = a * c00 + d * c01 + f * c02;
      double* pi = Pinv + (e * 2 + threadIdx.x) * 9;
      pi[0] = c00 / det; pi[1] = c01 / det; pi[2] = c02 / det;
      pi[3] = c01 / det; pi[4] = c11 / det; pi[5] = c12 / det;
      pi[6] = c02 / det; pi[7] = c12 / det; pi[8] = c22 / det;
    }
    __syncthreads();
  }
}

template <typename T, int P, int Q>
__global__ void __launch_bounds__(256) k_mass_curved(const T* __restrict__ um, int64_t um_es, int64_t um_cs,
                                                     const T* __restrict__ u0, int64_t u0_es, int64_t u0_cs,
                                                     const T* __restrict__ Gw, const T* __restrict__ eps,
                                                     const T* __restrict__ mu, CTab<T> L, int64_t ne,
                                                     T* __restrict__ R, const int32_t* skip) {
  if (skip && *skip) return;
  constexpr int N = P + 1, NQ = P + 2, N2 = N * N, N3 = N2 * N, NQ2 = NQ * NQ, NQ3 = NQ2 * NQ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* g6 = reinterpret_cast<T*>(smem_raw);  // [6][NQ3]
  T* b0 = g6 + 6 * NQ3;                     // [3][NQ3]
  T* b1 = b0 + 3 * NQ3;                     // [3][NQ3]
  for (int64_t e = blockIdx.x; e < ne; e += gridDim.x) {
    for (int it = threadIdx.x; it < 6 * NQ3; it += blockDim.x) g6[it] = Gw[e * 6 * NQ3 + it];
#pragma unroll 1
    for (int f = 0; f < 2; ++f) {
      const T mat = f == 0 ? eps[e] : mu[e];
#pragma unroll 1
      for (int i = 0; i < Q; ++i) {
        for (int it = threadIdx.x; it < 3 * N3; it += blockDim.x) {
          const int c = it / N3, s = it - c * N3, fc = f * 3 + c;
          T v = um[e * um_es + fc * um_cs + i * N3 + s];
          if (i == 0 && u0) v -= u0[e * u0_es + fc * u0_cs + s];
          b0[c * NQ3 + s] = v;
        }
        __syncthreads();
        for (int it = threadIdx.x; it < 3 * N2 * NQ; it += blockDim.x) {  // x: j -> gx
          const int gx = it % NQ, lk = (it / NQ) % N2, c = it / (NQ * N2);
          const T* in = b0 + c * NQ3 + lk * N;
          T acc = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) acc = fma(in[j], L.Lq[j][gx], acc);
          b1[c * NQ3 + lk * NQ + gx] = acc;
        }
        __syncthreads();
        for (int it = threadIdx.x; it < 3 * N * NQ2; it += blockDim.x) {  // y: k -> gy
          const int gx = it % NQ, gy = (it / NQ) % NQ, l = (it / NQ2) % N, c = it / (NQ2 * N);
          const T* in = b1 + c * NQ3 + l * N * NQ + gx;
          T acc = T(0);
#pragma unroll
          for (int k = 0; k < N; ++k) acc = fma(in[k * NQ], L.Lq[k][gy], acc);
          b0[c * NQ3 + (l * NQ + gy) * NQ + gx] = acc;
        }
        __syncthreads();
        for (int it = threadIdx.x; it < 3 * NQ3; it += blockDim.x) {  // z: l -> gz
          const int g2 = it % NQ2, gz = (it / NQ2) % NQ, c = it / NQ3;
          const T* in = b0 + c * NQ3 + g2;
          T acc = T(0);
#pragma unroll
          for (int l = 0; l < N; ++l) acc = fma(in[l * NQ2], L.Lq[l][gz], acc);
          b1[c * NQ3 + gz * NQ2 + g2] = acc;
        }
        __syncthreads();
        for (int g = threadIdx.x; g < NQ3; g += blockDim.x) {  // pointwise w_g G(x_g)
          const T vx = b1[g], vy = b1[NQ3 + g], vz = b1[2 * NQ3 + g];
          const T gxx = g6[g], gyy = g6[NQ3 + g], gzz = g6[2 * NQ3 + g];
          const T gxy = g6[3 * NQ3 + g], gxz = g6[4 * NQ3 + g], gyz = g6[5 * NQ3 + g];
          b0[g] = mat * fma(gxx, vx, fma(gxy, vy, gxz * vz));
          b0[NQ3 + g] = mat * fma(gxy, vx, fma(gyy, vy, gyz * vz));
          b0[2 * NQ3 + g] = mat * fma(gxz, vx, fma(gyz, vy, gzz * vz));
        }
        __syncthreads();
        for (int it = threadIdx.x; it < 3 * N * NQ2; it += blockDim.x) {  // z: gz -> l
          const int g2 = it % NQ2, l = (it / NQ2) % N, c = it / (NQ2 * N);
          const T* in = b0 + c * NQ3 + g2;
          T acc = T(0);
#pragma unroll
          for (int gz = 0; gz < NQ; ++gz) acc = fma(in[gz * NQ2], L.Lq[l][gz], acc);
          b1[c * NQ3 + l * NQ2 + g2] = acc;
        }
        __syncthreads();
        for (int it = threadIdx.x; it < 3 * N2 * NQ; it += blockDim.x) {  // y: gy -> k
          const int gx = it % NQ, k = (it / NQ) % N, l = (it / (NQ * N)) % N, c = it / (NQ * N2);
          const T* in = b1 + c * NQ3 + l * NQ2 + gx;
          T acc = T(0);
#pragma unroll
          for (int gy = 0; gy < NQ; ++gy) acc = fma(in[gy * NQ], L.Lq[k][gy], acc);
          b0[c * NQ3 + (l * N + k) * NQ + gx] = acc;
        }
        __syncthreads();
        for (int it = threadIdx.x; it < 3 * N3; it += blockDim.x) {  // x: gx -> j, write
          const int j = it % N, lk = (it / N) % N2, c = it / N3;
          const T* in = b0 + c * NQ3 + lk * NQ;
          T acc = T(0);
#pragma unroll
          for (int gx = 0; gx < NQ; ++gx) acc = fma(in[gx], L.Lq[j][gx], acc);
          R[(e * 6 + f * 3 + c) * (int64_t)(Q * N3) + i * N3 + lk * N + j] = acc;
        }
        __syncthreads();
      }
    }
  }
}

template <typename S, typename X, bool Add>
__global__ void k_precond_curved(X* __restrict__ out, const S* __restrict__ V, int64_t ldv, int k, Coef16 y,
                                 const S* __restrict__ Pinv, int64_t qn3, int64_t ne, const int32_t* skip,
                                 const GmresState* st) {
  if (skip && *skip) return;
  if (st) {
    k = st->k;
    if (k <= 0) return;
    for (int j = 0; j < kMaxDots; ++j) y.c[j] = st->yc[j];
  }
  const int64_t items = ne * 2 * qn3;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ef = it / qn3, r = it - ef * qn3;  // ef = 2 e + f
    const int64_t base = ef * 3 * qn3 + r;
    S v[3];
    for (int c = 0; c < 3; ++c) {
      if (k == 0) {
        v[c] = V[base + c * qn3];
      } else {
        S acc = S(0);
        for (int j = 0; j < k; ++j) acc = fma((S)y.c[j], V[j * ldv + base + c * qn3], acc);
        v[c] = acc;
      }
    }
    const S* pi = Pinv + ef * 9;
    for (int c = 0; c < 3; ++c) {
      const S z = fma(pi[3 * c], v[0], fma(pi[3 * c + 1], v[1], pi[3 * c + 2] * v[2]));
      if (Add) out[base + c * qn3] = (X)out[base + c * qn3] + (X)z;
      else out[base + c * qn3] = (X)z;
    }
  }
}

template <int P>
__global__ void __launch_bounds__(256) k_energy_curved(const double* __restrict__ u, const double* __restrict__ Gw,
                                                       const double* __restrict__ eps, const double* __restrict__ mu,
                                                       CTab<double> L, int64_t ne, double* __restrict__ el) {
  constexpr int N = P + 1, NQ = P + 2, N2 = N * N, N3 = N2 * N, NQ2 = NQ * NQ, NQ3 = NQ2 * NQ;
  __shared__ double b0[3 * NQ3], b1[3 * NQ3];
  __shared__ double red[32];
  for (int64_t e = blockIdx.x; e < ne; e += gridDim.x) {
    const double* ge = Gw + e * 6 * NQ3;
    double tot = 0.0;
    for (int f = 0; f < 2; ++f) {
      const double mat = f == 0 ? eps[e] : mu[e];
      for (int it = threadIdx.x; it < 3 * N3; it += blockDim.x) {
        const int c = it / N3, s = it - c * N3;
        b0[c * NQ3 + s] = u[(e * 6 + f * 3 + c) * N3 + s];
      }
      __syncthreads();
      for (int it = threadIdx.x; it < 3 * N2 * NQ; it += blockDim.x) {
        const int gx = it % NQ, lk = (it / NQ) % N2, c = it / (NQ * N2);
        double acc = 0.0;
        for (int j = 0; j < N; ++j) acc = fma(b0[c * NQ3 + lk * N + j], L.Lq[j][gx], acc);
        b1[c * NQ3 + lk * NQ + gx] = acc;
      }
      __syncthreads();
      for (int it = threadIdx.x; it < 3 * N * NQ2; it += blockDim.x) {
        const int gx = it % NQ, gy = (it / NQ) % NQ, l = (it / NQ2) % N, c = it / (NQ2 * N);
        double acc = 0.0;
        for (int k = 0; k < N; ++k) acc = fma(b1[c * NQ3 + (l * N + k) * NQ + gx], L.Lq[k][gy], acc);
        b0[c * NQ3 + (l * NQ + gy) * NQ + gx] = acc;
      }
      __syncthreads();
      for (int it = threadIdx.x; it < 3 * NQ3; it += blockDim.x) {
        const int g2 = it % NQ2, gz = (it / NQ2) % NQ, c = it / NQ3;
        double acc = 0.0;
        for (int l = 0; l < N; ++l) acc = fma(b0[c * NQ3 + l * NQ2 + g2], L.Lq[l][gz], acc);
        b1[c * NQ3 + gz * NQ2 + g2] = acc;
      }
      __syncthreads();
      double part = 0.0;
      for (int g = threadIdx.x; g < NQ3; g += blockDim.x) {
        const double vx = b1[g], vy = b1[NQ3 + g], vz = b1[2 * NQ3 + g];
        const double q = ge[g] * vx * vx + ge[NQ3 + g] * vy * vy + ge[2 * NQ3 + g] * vz * vz +
                         2.0 * (ge[3 * NQ3 + g] * vx * vy + ge[4 * NQ3 + g] * vx * vz + ge[5 * NQ3 + g] * vy * vz);
        part += q;
      }
      // fixed-order block reduction
      for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
      __syncthreads();
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        tot += 0.5 * mat * s;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) el[e] = tot;
    __syncthreads();
  }
}

}  // namespace

int launch_metric(int P, const double* X8, const double* eps, const double* mu, int64_t ne, const CurvedTables& ct,
                  double* Gw, double* Pinv, int* bad, cudaStream_t s) {
  const int grid = (int)(ne < 65536 ? ne : 65536);
  switch (P) {
#define STM_M(p) case p: k_metric<p><<<grid, 256, 0, s>>>(X8, eps, mu, ne, ct, Gw, Pinv, bad); break;
    STM_M(0) STM_M(1) STM_M(2) STM_M(3) STM_M(4) STM_M(5) STM_M(6) STM_M(7)
#undef STM_M
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

template <typename T, int P, int Q>
int mass_pq(const T* um, int64_t um_es, int64_t um_cs, const T* u0, int64_t u0_es, int64_t u0_cs, const T* Gw,
            const T* eps, const T* mu, const CurvedTables& ct, int64_t ne, T* R, cudaStream_t s,
            const int32_t* skip) {
  constexpr int NQ3 = (P + 2) * (P + 2) * (P + 2);
  const size_t sm = sizeof(T) * 12 * NQ3;
  static std::atomic<uint64_t> configured_devices{0};
  once_per_device(configured_devices, [&] {
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_mass_curved<T, P, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  });
  // grid-stride over elements, one wave of co-resident CTAs (a skipped launch costs one wave)
  static std::atomic<int> cap[64];
  const int grid = wave_grid(k_mass_curved<T, P, Q>, 256, sm, ne, cap);
  k_mass_curved<T, P, Q><<<grid, 256, sm, s>>>(um, um_es, um_cs, u0, u0_es, u0_cs, Gw, eps, mu, ctab<T>(ct), ne, R,
                                                skip);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_mass_curved(int P, int Q, const T* um, int64_t um_es, int64_t um_cs, const T* u0, int64_t u0_es,
                       int64_t u0_cs, const T* Gw, const T* eps, const T* mu, const CurvedTables& ct, int64_t ne, T* R,
                       cudaStream_t s, const int32_t* skip) {
#define STM_MQ(p, q) \
  if (P == p && Q == q) return mass_pq<T, p, q>(um, um_es, um_cs, u0, u0_es, u0_cs, Gw, eps, mu, ct, ne, R, s, skip);
#define STM_MP(p) STM_MQ(p, 1) STM_MQ(p, 2) STM_MQ(p, 3) STM_MQ(p, 4) STM_MQ(p, 5) STM_MQ(p, 6)
  STM_MP(0) STM_MP(1) STM_MP(2) STM_MP(3) STM_MP(4) STM_MP(5) STM_MP(6) STM_MP(7)
#undef STM_MP
#undef STM_MQ
  return (int)cudaErrorInvalidValue;
}

template <typename S, typename X>
void precond_curved(X* out, const S* V, int64_t ldv, int k, const double* y, const S* Pinv, int64_t qn3, int64_t ne,
                    bool add, cudaStream_t s, const int32_t* skip, const GmresState* st) {
  Coef16 yc{};
  for (int j = 0; j < k && j < kMaxDots; ++j) yc.c[j] = y[j];
  const int64_t items = ne * 2 * qn3;
  const int grid = (int)((items + 255) / 256 < 4 * kRedBlocks ? (items + 255) / 256 : 4 * kRedBlocks);
  if (add) k_precond_curved<S, X, true><<<grid, 256, 0, s>>>(out, V, ldv, k, yc, Pinv, qn3, ne, skip, st);
  else k_precond_curved<S, X, false><<<grid, 256, 0, s>>>(out, V, ldv, k, yc, Pinv, qn3, ne, skip, st);
}

int launch_energy_curved(int P, const double* u, const double* Gw, const double* eps, const double* mu,
                         const CurvedTables& ct, int64_t ne, double* el, cudaStream_t s) {
  const int grid = (int)(ne < 65536 ? ne : 65536);
  const CTab<double> L = ctab<double>(ct);
  switch (P) {
#define STM_E(p) case p: k_energy_curved<p><<<grid, 256, 0, s>>>(u, Gw, eps, mu, L, ne, el); break;
    STM_E(0) STM_E(1) STM_E(2) STM_E(3) STM_E(4) STM_E(5) STM_E(6) STM_E(7)
#undef STM_E
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

template int launch_mass_curved<double>(int, int, const double*, int64_t, int64_t, const double*, int64_t, int64_t,
                                        const double*, const double*, const double*, const CurvedTables&, int64_t,
                                        double*, cudaStream_t, const int32_t*);
template int launch_mass_curved<float>(int, int, const float*, int64_t, int64_t, const float*, int64_t, int64_t,
                                       const float*, const float*, const float*, const CurvedTables&, int64_t, float*,
                                       cudaStream_t, const int32_t*);
template void precond_curved<double, double>(double*, const double*, int64_t, int, const double*, const double*,
                                             int64_t, int64_t, bool, cudaStream_t, const int32_t*, const GmresState*);
template void precond_curved<float, float>(float*, const float*, int64_t, int, const double*, const float*, int64_t,
                                           int64_t, bool, cudaStream_t, const int32_t*, const GmresState*);
template void precond_curved<float, double>(double*, const float*, int64_t, int, const double*, const float*, int64_t,
                                            int64_t, bool, cudaStream_t, const int32_t*, const GmresState*);

}  // namespace stm
