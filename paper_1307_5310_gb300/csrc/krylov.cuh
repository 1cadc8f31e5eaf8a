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

// Device-side state of the restarted GMRES slab solve (Sec. 5.4): the Hessenberg
// matrix of the current cycle with its Givens rotations, the basis scales, the stop
// tests and the flags that let a whole restart cycle run without the host.  Every
// kernel of an iteration takes `skip` (a pointer into this struct) and returns at
// once while it is set, so a cycle is a fixed launch sequence (capturable in a CUDA
// graph) whose tail is a no-op after convergence.
struct GmresState {
  double H[kMaxDots * kMaxDots];  // H[i * kMaxDots + j], column j = iteration j
  double cs[kMaxDots], sn[kMaxDots], g[kMaxDots + 1], alpha[kMaxDots + 1];
  double cc[kMaxDots];            // Gram-Schmidt coefficients of the current iteration
  double yc[kMaxDots];            // combination coefficients at the end of the cycle
  double red[4];                  // reduction results: 0 |R|^2, 1 |S R|^2, 2 |start vector|^2
  double before, after;           // |W|^2 before and after the update (DGKS test)
  double ref;                     // |R(U with unknowns 0)| of the slab (stop test R6)
  double tol;                     // relative target (exact solve) or eta budget (inexact)
  double tol_abs;                 // this cycle's stop threshold on |g|
  double rel, phi, res;           // last true relative residual, weighted norm, |g_k|
  int32_t k;                      // basis vectors used in this cycle
  int32_t skip;                   // 1: the rest of the cycle is skipped
  int32_t skip_reo;               // 1: no second Gram-Schmidt pass in this iteration
  int32_t iters;                  // GMRES iterations of the slab so far
  int32_t max_it;
  int32_t status;                 // 0, or a negative STM_* code
  int32_t outer_done;             // 1: the slab's stop test holds
  int32_t inexact;                // 1: stop on the weighted norm (eta_it), 0: on rel
  int32_t cycles;                 // restart cycles started
  int32_t halt;                   // 1: the slab solve has stopped (stop test, cap, zero residual or
                                  //    error); every later kernel of the slab is skipped
};

// out[i] = sum_n w[n] V[i*ldv + n] for i < k (k <= 15), and out[k] = sum_n w[n]^2
// if with_norm.  partial: (k+1) * kRedBlocks doubles of scratch.  out == nullptr:
// only the partial sums are written (a control kernel reduces them).
template <typename S>
void multidot(const S* w, const S* V, int64_t ldv, int k, bool with_norm, int64_t n, double* partial, double* out,
              cudaStream_t s, const int32_t* skip = nullptr);

// w[n] -= sum_{i<k} c[i] V[i*ldv + n] (k may be 0), then out[0] = sum_n w[n]^2.  With
// cdev non-null the coefficients are read from device memory instead of c.
template <typename S>
void axpy_norm(S* w, const S* V, int64_t ldv, int k, const Coef16& c, int64_t n, double* partial, double* out,
               cudaStream_t s, const int32_t* skip = nullptr, const double* cdev = nullptr);

// z[n] = v[n] * inv[n / blk]  (blk = entries per (element, field, component) block).
template <typename S>
void precond_apply(S* z, const S* v, const S* inv, int64_t blk, int64_t n, cudaStream_t s,
                   const int32_t* skip = nullptr);

// x[n] += inv[n / blk] * sum_{i<k} y[i] V[i*ldv + n].  With st non-null, k and y are
// read from the device state (st->k, st->yc) and k is the largest count.
template <typename S, typename X>
void precond_combine(X* x, const S* V, int64_t ldv, int k, const Coef16& y, const S* inv, int64_t blk, int64_t n,
                     cudaStream_t s, const GmresState* st = nullptr);

// ---- device-side GMRES control (one block each; partial: kRedBlocks sums per value) ----
// st->red[slot] = sum of the partials of one reduction (fixed order).
void gmres_reduce(const double* partial, GmresState* st, int slot, cudaStream_t s, const int32_t* skip = nullptr);
// Slab start: st->ref = sqrt(red[0]); iteration count, flags and targets reset.
void gmres_slab_start(GmresState* st, double tol, int max_it, int inexact, cudaStream_t s);
// The slab's stop test on the true residual (norm^2 in red[0], weighted norm^2 in red[1]
// if inexact, R6): sets outer_done, and skip when done, at the iteration cap or at R = 0.
void gmres_outer_check(GmresState* st, cudaStream_t s);
// Restart-cycle start (unless skipped): v_0 = start / (-|start|) with |start|^2 from
// red[slot_start], and the cycle threshold max(target, floor_rel |start|).
void gmres_cycle_init(GmresState* st, int slot_start, double floor_rel, cudaStream_t s);
// Iteration j, after the multi-dot of W with V[0..j] (+ |W|^2): H column and the
// Gram-Schmidt coefficients (second = 1: the DGKS pass, added to the column).
void gmres_gs(const double* partial, GmresState* st, int j, int second, cudaStream_t s);
// After the update's norm: with reorth, record |W|^2 and decide on a second pass.
void gmres_after(const double* partial, GmresState* st, int reorth, cudaStream_t s);
// Iteration j's Givens step; stops the cycle on |g_{j+1}| <= tol_abs, breakdown, the
// iteration cap or the end of the cycle (j = m - 1).  reo_mode = 1: |W|^2 comes from the
// second pass's partials when that pass ran, else from st->after.
void gmres_givens(const double* partial, GmresState* st, int j, int m, int reo_mode, cudaStream_t s);
// End of the cycle: y from the triangular system, yc = y / alpha.
void gmres_backsub(GmresState* st, int m, cudaStream_t s);

// out = 1/2 sum_n mass[n / n3] u[n]^2 (state layout, blocks of n3 per (element, field, component)).
void energy_brick(const double* u, const double* mass, int64_t n3, int64_t n, double* partial, double* out,
                  cudaStream_t s);

// dst[n] = (D) src[n]
template <typename D, typename S>
void convert(D* dst, const S* src, int64_t n, cudaStream_t s, const int32_t* skip = nullptr);

}  // namespace stm
