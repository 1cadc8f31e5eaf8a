// Load vector of the slab residual: Gaussian current pulses (device kernel).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "residual.cuh"

namespace stm {

constexpr int kMaxSrc = 8;
constexpr int kMaxNQ = kMaxN + 1;  // p + 2 Gauss points per direction

struct GaussParams {
  int n_src;
  int Q;
  double c[kMaxSrc][3];       // centres
  double d[kMaxSrc][3];       // directions
  double inv2sx2[kMaxSrc];    // 1 / (2 sigma_x^2)
  double amp[kMaxSrc];
  double tf[kMaxSrc][kMaxQ];  // dt sum_tau w_tau L_i(xi_tau) exp(-(t - t_k)^2 / (2 sigma_t^2))
  // uneven degrees / local refinement in time: the same factors per sub-interval kk of a class
  // with N_K sub-intervals (dt / N_K each), tfk[k][kk][i]; elements of the class in elist, E
  // rows at off_test[e] with N_K q temporal test functions (null elist: uniform mesh, tf)
  int NK;
  double tfk[kMaxSrc][8][kMaxQ];
  const int32_t* elist;
  const int64_t* off_test;
  double xq[kMaxNQ], wq[kMaxNQ];
  double Lq[kMaxN][kMaxNQ];   // L_j at the spatial Gauss points
};

// b[e][0][c][i][s] += l_E for every element (E rows); b must be initialised.
int launch_load_gauss(int P, const double* X8, int64_t ne, const GaussParams& gp, double* b, cudaStream_t s);

}  // namespace stm
