// Vector kernels for meshes whose elements have different (p, q): every
// per-element block is located through offset arrays (test layout off_test,
// state layout off_state, ne + 1 entries: block sizes are offset differences,
// which covers N_K temporal sub-intervals) and the degrees pq[e] = p | q << 4.
// One CTA walks one element's block at a time.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "krylov.cuh"

namespace stm {

// z = P^{-1} v (diagonal brick mass; test layout).
template <typename S>
void precond_hp(S* z, const S* v, const S* inv, const int64_t* off_test, const uint8_t* pq, int64_t ne,
                cudaStream_t s, const int32_t* skip = nullptr);

// x += P^{-1} sum_{j<k} y[j] V[j]  (test layout); with st non-null k and y come from the
// device state of the GMRES cycle.
template <typename S, typename X>
void combine_hp(X* x, const S* V, int64_t ldv, int k, const Coef16& y, const S* inv, const int64_t* off_test,
                const uint8_t* pq, int64_t ne, cudaStream_t s, const GmresState* st = nullptr);

// x: mode 1 (first unknown) of every temporal sub-interval = state, higher modes 0.
void init_guess_hp(double* x, const double* state, const int64_t* off_test, const int64_t* off_state,
                   const uint8_t* pq, int64_t ne, cudaStream_t s);

// state = mode 1 of the last sub-interval of x (the field at the slab end).
void extract_end_hp(double* state, const double* x, const int64_t* off_test, const int64_t* off_state,
                    const uint8_t* pq, int64_t ne, cudaStream_t s);

// el[e] = 1/2 sum_fc mass[e][fc] |u[e][fc]|^2 (state layout).
void energy_hp(const double* u, const double* mass, const int64_t* off_state, const uint8_t* pq, int64_t ne,
               double* el, cudaStream_t s);

// 2:1 faces.  For each slot (an element face on either side of a 2:1 face)
// k_hang writes the neighbour's tangential traces as coefficients of the
// receiving element's own face basis: for a fine face the coarse trace
// restricted to its quarter (u, v), for a coarse face the four fine traces
// projected onto the coarse basis, with the transfer integrals
// T[u][j][n] = int_0^1 L_n((eta + u) / 2) L_j(eta) d eta and the factor 1/2
// from the covariant scaling and the quarter's area.  Temporal modes stop at
// min(q, q') (Eq. bilinearform:S).
template <typename T>
struct HangArgs {
  const T* tr;              // trace buffer of all elements
  const int64_t* off_tr;
  const uint8_t* pq;
  int64_t n_slots;
  const int32_t* elem;      // [slot] receiving element
  const int32_t* face;      // [slot] receiving face
  const int32_t* kind;      // [slot] 0: fine side (one coarse source), 1: coarse side (four fine sources)
  const int32_t* src;       // [slot][4] source elements
  const int32_t* src_face;  // [slot][4] source faces
  const int32_t* quad;      // [slot][4] quarter u | v << 1
  const int64_t* hoff;      // [slot] offset of the slot's output
  T* hbuf;
  T Tm[2][8][8];
  const int32_t* skip = nullptr;  // non-null: nothing is done while *skip is set
};

template <typename T>
void launch_hang(const HangArgs<T>& h, cudaStream_t s);

}  // namespace stm
