#include "hp.cuh"

namespace stm {

namespace {

__device__ __forceinline__ void degrees(const uint8_t* pq, int64_t e, int& n3, int& q) {
  const int v = pq[e];
  const int n = (v & 15) + 1;
  n3 = n * n * n;
  q = v >> 4;
}

template <typename S>
__global__ void k_precond_hp(S* __restrict__ z, const S* __restrict__ v, const S* __restrict__ inv,
                             const int64_t* __restrict__ off, const uint8_t* __restrict__ pq, int64_t ne,
                             const int32_t* skip) {
  if (skip && *skip) return;
  for (int64_t e = blockIdx.x; e < ne; e += gridDim.x) {
    // one (field, component) block per inverse mass entry: all temporal test functions
    const int64_t o = off[e];
    const int blk = (int)((off[e + 1] - o) / 6);
    for (int it = threadIdx.x; it < 6 * blk; it += blockDim.x) z[o + it] = v[o + it] * inv[e * 6 + it / blk];
  }
}

template <typename S, typename X>
__global__ void k_combine_hp(X* __restrict__ x, const S* __restrict__ V, int64_t ldv, int k, Coef16 y,
                             const S* __restrict__ inv, const int64_t* __restrict__ off,
                             const uint8_t* __restrict__ pq, int64_t ne, const GmresState* st) {
  if (st) {
    k = st->k;
    for (int j = 0; j < kMaxDots; ++j) y.c[j] = st->yc[j];
  }
  if (k <= 0) return;
  for (int64_t e = blockIdx.x; e < ne; e += gridDim.x) {
    const int64_t o = off[e];
    const int blk = (int)((off[e + 1] - o) / 6);
    for (int it = threadIdx.x; it < 6 * blk; it += blockDim.x) {
      S acc = S(0);
      for (int j = 0; j < k; ++j) acc = fma((S)y.c[j], V[j * ldv + o + it], acc);
      x[o + it] = (X)x[o + it] + (X)(acc * inv[e * 6 + it / blk]);
    }
  }
}

__global__ void k_init_hp(double* __restrict__ x, const double* __restrict__ st, const int64_t* __restrict__ ot,
                          const int64_t* __restrict__ os, const uint8_t* __restrict__ pq, int64_t ne) {
  for (int64_t e = blockIdx.x; e < ne; e += gridDim.x) {
    int n3, q;
    degrees(pq, e, n3, q);
    // qe = N_K q temporal unknowns; mode 1 of every sub-interval = state: constant in time
    const int qe = (int)((ot[e + 1] - ot[e]) / (6 * n3));
    for (int it = threadIdx.x; it < 6 * qe * n3; it += blockDim.x) {
      const int fc = it / (qe * n3), r = it - fc * qe * n3, i = r / n3, s = r - i * n3;
      x[ot[e] + it] = (i % q == 0) ? st[os[e] + fc * n3 + s] : 0.0;
    }
  }
}

__global__ void k_extract_hp(double* __restrict__ st, const double* __restrict__ x, const int64_t* __restrict__ ot,
                             const int64_t* __restrict__ os, const uint8_t* __restrict__ pq, int64_t ne) {
  for (int64_t e = blockIdx.x; e < ne; e += gridDim.x) {
    int n3, q;
    degrees(pq, e, n3, q);
    // the slab end is mode 1 of the last sub-interval
    const int qe = (int)((ot[e + 1] - ot[e]) / (6 * n3));
    for (int it = threadIdx.x; it < 6 * n3; it += blockDim.x) {
      const int fc = it / n3, s = it - fc * n3;
      st[os[e] + it] = x[ot[e] + (fc * qe + qe - q) * n3 + s];
    }
  }
}

__global__ void k_energy_hp(const double* __restrict__ u, const double* __restrict__ mass,
                            const int64_t* __restrict__ os, const uint8_t* __restrict__ pq, int64_t ne,
                            double* __restrict__ el) {
  __shared__ double red[32];
  for (int64_t e = blockIdx.x; e < ne; e += gridDim.x) {
    int n3, q;
    degrees(pq, e, n3, q);
    double acc = 0.0;
    for (int it = threadIdx.x; it < 6 * n3; it += blockDim.x) {
      const double v = u[os[e] + it];
      acc = fma(mass[e * 6 + it / n3] * v, v, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
      el[e] = 0.5 * sum;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_hang(HangArgs<T> H) {
  if (H.skip && *H.skip) return;
  for (int64_t slot = blockIdx.x; slot < H.n_slots; slot += gridDim.x) {
    const int e = H.elem[slot], face = H.face[slot], a = face >> 1;
    int n3, q;
    degrees(H.pq, e, n3, q);
    const int N = (H.pq[e] & 15) + 1, N2 = N * N;
    const int kind = H.kind[slot];
    for (int it = threadIdx.x; it < 4 * q * N2; it += blockDim.x) {
      const int t = it % N2, r = it / N2, i = r % q, fb = r / q;  // fb = field * 2 + comp slot
      const int fld = fb >> 1, bi = fb & 1;
      const int js = t / N, jf = t - js * N;
      T acc = T(0);
      const int nsrc = kind == 0 ? 1 : 4;
      for (int k = 0; k < nsrc; ++k) {
        const int es = H.src[slot * 4 + k], sf = H.src_face[slot * 4 + k];
        const int qs = H.pq[es] >> 4, Ns = (H.pq[es] & 15) + 1;
        if (i >= qs) continue;
        const int u = H.quad[slot * 4 + k] & 1, v = H.quad[slot * 4 + k] >> 1;
        const T* ts = H.tr + H.off_tr[es] + ((((int64_t)fld * 3 + a) * 2 + (sf & 1)) * 2 + bi) * qs * Ns * Ns +
                      (int64_t)i * Ns * Ns;
        for (int ns = 0; ns < Ns; ++ns) {
          T row = T(0);
          for (int nf = 0; nf < Ns; ++nf) {
            // fine side: source modes (ns, nf) are the coarse ones; coarse side: they are fine ones
            const T tf = kind == 0 ? H.Tm[u][jf][nf] : H.Tm[u][nf][jf];
            row = fma(tf, ts[ns * Ns + nf], row);
          }
          const T tsl = kind == 0 ? H.Tm[v][js][ns] : H.Tm[v][ns][js];
          acc = fma(tsl, row, acc);
        }
      }
      H.hbuf[H.hoff[slot] + it] = T(0.5) * acc;
    }
  }
}

inline int egrid(int64_t ne) { return (int)(ne < 65536 ? ne : 65536); }

}  // namespace

template <typename S>
void precond_hp(S* z, const S* v, const S* inv, const int64_t* off_test, const uint8_t* pq, int64_t ne,
                cudaStream_t s, const int32_t* skip) {
  k_precond_hp<S><<<egrid(ne), 256, 0, s>>>(z, v, inv, off_test, pq, ne, skip);
}

template <typename S, typename X>
void combine_hp(X* x, const S* V, int64_t ldv, int k, const Coef16& y, const S* inv, const int64_t* off_test,
                const uint8_t* pq, int64_t ne, cudaStream_t s, const GmresState* st) {
  k_combine_hp<S, X><<<egrid(ne), 256, 0, s>>>(x, V, ldv, k, y, inv, off_test, pq, ne, st);
}

void init_guess_hp(double* x, const double* state, const int64_t* off_test, const int64_t* off_state,
                   const uint8_t* pq, int64_t ne, cudaStream_t s) {
  k_init_hp<<<egrid(ne), 256, 0, s>>>(x, state, off_test, off_state, pq, ne);
}

void extract_end_hp(double* state, const double* x, const int64_t* off_test, const int64_t* off_state,
                    const uint8_t* pq, int64_t ne, cudaStream_t s) {
  k_extract_hp<<<egrid(ne), 256, 0, s>>>(state, x, off_test, off_state, pq, ne);
}

void energy_hp(const double* u, const double* mass, const int64_t* off_state, const uint8_t* pq, int64_t ne,
               double* el, cudaStream_t s) {
  k_energy_hp<<<egrid(ne), 256, 0, s>>>(u, mass, off_state, pq, ne, el);
}

template <typename T>
void launch_hang(const HangArgs<T>& h, cudaStream_t s) {
  if (h.n_slots > 0) k_hang<T><<<egrid(h.n_slots), 128, 0, s>>>(h);
}
template void launch_hang<double>(const HangArgs<double>&, cudaStream_t);
template void launch_hang<float>(const HangArgs<float>&, cudaStream_t);

template void precond_hp<double>(double*, const double*, const double*, const int64_t*, const uint8_t*, int64_t,
                                 cudaStream_t, const int32_t*);
template void precond_hp<float>(float*, const float*, const float*, const int64_t*, const uint8_t*, int64_t,
                                cudaStream_t, const int32_t*);
template void combine_hp<double, double>(double*, const double*, int64_t, int, const Coef16&, const double*,
                                         const int64_t*, const uint8_t*, int64_t, cudaStream_t, const GmresState*);
template void combine_hp<float, double>(double*, const float*, int64_t, int, const Coef16&, const float*,
                                        const int64_t*, const uint8_t*, int64_t, cudaStream_t, const GmresState*);

}  // namespace stm
