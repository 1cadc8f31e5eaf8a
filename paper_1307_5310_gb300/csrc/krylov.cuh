// Vector kernels of the per-slab GMRES solve (Sec. 5.4) and the discrete
// energy (Eq. stability:energydef).  Storage type S is double or float.
// Reductions use a fixed grid and a fixed summation order, so results are
// bitwise reproducible run to run.  With S = double every product and sum is
// FP64.  With S = float (the inner solve of the mixed-precision path) each
// thread sums products of 8 consecutive entries in FP32 and accumulates those
// partial sums in FP64; the grid and block reductions are FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace stm {

constexpr int kRedBlocks = 608;   // 4 x 152 SMs
constexpr int kRedThreads = 256;
constexpr int kMaxDots = 16;      // restart <= 15 basis vectors + one norm

struct Coef16 { double c[kMaxDots]; };

// out[i] = sum_n w[n] V[i*ldv + n] for i < k (k <= 15), and out[k] = sum_n w[n]^2
// if with_norm.  partial: (k+1) * kRedBlocks doubles of scratch.
template <typename S>
void multidot(const S* w, const S* V, int64_t ldv, int k, bool with_norm, int64_t n, double* partial, double* out,
              cudaStream_t s);

// w[n] -= sum_{i<k} c[i] V[i*ldv + n] (k may be 0), then out[0] = sum_n w[n]^2.
template <typename S>
void axpy_norm(S* w, const S* V, int64_t ldv, int k, const Coef16& c, int64_t n, double* partial, double* out,
               cudaStream_t s);

// z[n] = v[n] * inv[n / blk]  (blk = entries per (element, field, component) block).
template <typename S>
void precond_apply(S* z, const S* v, const S* inv, int64_t blk, int64_t n, cudaStream_t s);

// x[n] += inv[n / blk] * sum_{i<k} y[i] V[i*ldv + n].
template <typename S, typename X>
void precond_combine(X* x, const S* V, int64_t ldv, int k, const Coef16& y, const S* inv, int64_t blk, int64_t n,
                     cudaStream_t s);

// out = 1/2 sum_n mass[n / n3] u[n]^2 (state layout, blocks of n3 per (element, field, component)).
void energy_brick(const double* u, const double* mass, int64_t n3, int64_t n, double* partial, double* out,
                  cudaStream_t s);

// dst[n] = (D) src[n]
template <typename D, typename S>
void convert(D* dst, const S* src, int64_t n, cudaStream_t s);

}  // namespace stm
