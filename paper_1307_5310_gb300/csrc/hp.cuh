// Vector kernels for meshes whose elements have different (p, q): every
// per-element block is located through offset arrays (test layout off_test,
// state layout off_state) and the degrees pq[e] = p | q << 4.  One CTA walks
// one element's block at a time.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "krylov.cuh"

namespace stm {

// z = P^{-1} v (diagonal brick mass; test layout).
template <typename S>
void precond_hp(S* z, const S* v, const S* inv, const int64_t* off_test, const uint8_t* pq, int64_t ne,
                cudaStream_t s);

// x += P^{-1} sum_{j<k} y[j] V[j]  (test layout).
template <typename S, typename X>
void combine_hp(X* x, const S* V, int64_t ldv, int k, const Coef16& y, const S* inv, const int64_t* off_test,
                const uint8_t* pq, int64_t ne, cudaStream_t s);

// x: mode 1 (first unknown) = state, higher modes 0.
void init_guess_hp(double* x, const double* state, const int64_t* off_test, const int64_t* off_state,
                   const uint8_t* pq, int64_t ne, cudaStream_t s);

// state = mode 1 of x (the field at the slab end).
void extract_end_hp(double* state, const double* x, const int64_t* off_test, const int64_t* off_state,
                    const uint8_t* pq, int64_t ne, cudaStream_t s);

// el[e] = 1/2 sum_fc mass[e][fc] |u[e][fc]|^2 (state layout).
void energy_hp(const double* u, const double* mass, const int64_t* off_state, const uint8_t* pq, int64_t ne,
               double* el, cudaStream_t s);

}  // namespace stm
