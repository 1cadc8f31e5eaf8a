// Curved (trilinear) elements: everything that depends on the metric.
//
// With the covariant transform (Sec. 2.3) the volume curl and the face terms
// are metric-free, so on curved elements only the mass term changes (Sec. 5.2,
// "mass residual"): M_G with G(x^) = |J| DF^{-1} DF^{-T} varies over the
// element and is applied by sum factorisation through the p+2 Gauss points
// per direction (R11): evaluate the coefficients at the points (three 1-D
// contractions), multiply by w_g G(x^_g), project back (three contractions).
// That is O(p^4) per temporal mode and component, O(p^5) per element.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "krylov.cuh"
#include "residual.cuh"

namespace stm {

struct CurvedTables {
  double xq[kMaxN + 1], wq[kMaxN + 1];  // p+2 Gauss points / weights on [0,1]
  double Lq[kMaxN][kMaxN + 1];          // L_j(x_g)
};

// Metric at the Gauss points of every element: Gw[e][6][NQ^3] = w_g G_g in the
// order xx, yy, zz, xy, xz, yz, and the cell-mean inverse preconditioner
// blocks Pinv[e][2][9] = (mat_f * sum_g w_g G_g)^{-1}.  bad[0] is set to 1 if
// an element has a non-positive Jacobian at a Gauss point.
int launch_metric(int P, const double* X8, const double* eps, const double* mu, int64_t ne, const CurvedTables& ct,
                  double* Gw, double* Pinv, int* bad, cudaStream_t s);

// R[e][f][c][i][s] = mat_f (M_G (u_{i+1} - delta_{i0} u_0))[c][s] for every element.
template <typename T>
int launch_mass_curved(int P, int Q, const T* um, int64_t um_es, int64_t um_cs, const T* u0, int64_t u0_es,
                       int64_t u0_cs, const T* Gw, const T* eps, const T* mu, const CurvedTables& ct, int64_t ne, T* R,
                       cudaStream_t s, const int32_t* skip = nullptr);

// The same FP32 mass term on the tensor cores (tcgen05.mma kind::tf32 with 3xTF32 split
// products, accumulators in tensor memory) for 3 <= P <= 7; cudaErrorInvalidValue for other
// degrees.  *err is set to 1 if a bounded wait of the kernel ran out (R is then incomplete).
int launch_mass_curved_tc(int P, int Q, const float* um, int64_t um_es, int64_t um_cs, const float* u0, int64_t u0_es,
                          int64_t u0_cs, const float* Gw, const float* eps, const float* mu, const CurvedTables& ct,
                          int64_t ne, float* R, cudaStream_t s, const int32_t* skip, int* err);

// z[e][f][c][i][s] = sum_d Pinv[e][f][c][d] v[e][f][d][i][s]   (add = false), or x += that (add = true);
// with k > 0, v is the combination sum_{j<k} y[j] V[j] (ldv apart).
// With skip non-null nothing is done while *skip is set; with st non-null k and y come
// from the device state of the GMRES cycle.
template <typename S, typename X>
void precond_curved(X* out, const S* V, int64_t ldv, int k, const double* y, const S* Pinv, int64_t qn3, int64_t ne,
                    bool add, cudaStream_t s, const int32_t* skip = nullptr, const GmresState* st = nullptr);

// Per-element energies 1/2 mat_f u^T M_G u of the state -> el[e].
int launch_energy_curved(int P, const double* u, const double* Gw, const double* eps, const double* mu,
                         const CurvedTables& ct, int64_t ne, double* el, cudaStream_t s);

}  // namespace stm
