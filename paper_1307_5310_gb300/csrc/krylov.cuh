// Vector kernels of the per-slab GMRES solve (Sec. 5.4) and the discrete
// energy (Eq. stability:energydef).  Storage type S is double or float; every
// dot product, norm and reduction is accumulated in double.  Reductions use a
// fixed grid and a fixed summation order, so results are bitwise
// reproducible run to run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace stm {

constexpr int kRedBlocks = 608;   // 4 x 152 SMs
constexpr int kRedThreads = 256;
constexpr int kMaxDots = 16;      // restart <= 15 basis vectors + one norm

struct Coef16 { double c[kMaxDots]; };

// partial[i * kRedBlocks + block] = block's share of sum_n w[n] * V[i*ldv + n]
// for i < k, and of sum_n w[n]^2 at i = k (if with_norm).
template <typename S>
void multidot(const S* w, const S* V, int64_t ldv, int k, bool with_norm, int64_t n,
              double* partial, double* out, cudaStream_t s);

// w[n] -= sum_{i<k} h[i] V[i*ldv + n], h on the device.
template <typename S>
void multi_axpy(S* w, const S* V, int64_t ldv, int k, const double* h, int64_t n, cudaStream_t s);

// v[n] *= 1 / sqrt(*nrm2) (nrm2 on the device).
template <typename S>
void scale_by_invnorm(S* v, const double* nrm2, int64_t n, cudaStream_t s);

// z[n] = v[n] / mass[e][fc] for the test layout with blocks of qn3 per (e, fc).
template <typename S>
void precond_apply(S* z, const S* v, const S* mass, int64_t qn3, int64_t n, cudaStream_t s);

// x[n] += (1 / mass[e][fc]) * sum_{i<k} y[i] V[i*ldv + n].
template <typename S, typename X>
void precond_combine(X* x, const S* V, int64_t ldv, int k, const Coef16& y, const S* mass,
                     int64_t qn3, int64_t n, cudaStream_t s);

// out = 1/2 sum_e sum_fc mass[e][fc] sum_s u[e][fc][s]^2 (state layout, blocks of n3).
void energy_brick(const double* u, const double* mass, int64_t n3, int64_t n, double* partial,
                  double* out, cudaStream_t s);

// dst[n] = (T) src[n]
template <typename D, typename S>
void convert(D* dst, const S* src, int64_t n, cudaStream_t s);

}  // namespace stm
