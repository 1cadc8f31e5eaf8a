// Load vector L(V) = l_E(v) + l_H(w) of Eq. bilinearform:C on one slab:
//   l_E(v) = (J, v) over I_n x K,   l_H(w) = -<n x g, w> over I_n x F_b.
//
// The current J is a sum of Gaussian pulses, separable in space and time:
//   J(x, t) = sum_k amp_k d_k exp(-|x - c_k|^2 / (2 sx_k^2)) exp(-(t - t_k)^2 / (2 st_k^2)),
// so l_E[c][i][s] = sum_k T_k[i] S_k[c][s] with the temporal factor
// T_k[i] = dt sum_tau w_tau L_i(xi_tau) exp(...) (q+2 Gauss points, computed on
// the host) and the spatial projection
// S_k[c][s] = sum_g w_g phi_s(x^_g) (|J| DF^{-1} d_k)_c exp(-|x_g - c_k|^2 / (2 sx_k^2))
// with p+2 Gauss points per direction (R11), evaluated here per element with
// the trilinear map of its 8 vertices (|J| DF^{-1} = adj DF) and projected by
// three 1-D contractions.
#include <cuda_runtime.h>

#include "load.cuh"

namespace stm {

namespace {

template <int P>
__global__ void __launch_bounds__(256) k_load_gauss(const double* __restrict__ X8g, int64_t ne, GaussParams gp,
                                                    double* __restrict__ b) {
  constexpr int N = P + 1, NQ = P + 2, NQ3 = NQ * NQ * NQ, N3 = N * N * N;
  __shared__ double X8[24];
  __shared__ double f0[3][NQ3];
  __shared__ double f1[3][NQ * NQ * N];
  __shared__ double f2[3][NQ * N * N];
  const int Q = gp.Q, QE = gp.elist ? gp.NK * Q : Q;
  for (int64_t blk = blockIdx.x; blk < ne; blk += gridDim.x) {
    const int64_t e = gp.elist ? gp.elist[blk] : blk;
    if (threadIdx.x < 24) X8[threadIdx.x] = X8g[e * 24 + threadIdx.x];
    // E rows of element e (this CTA owns them)
    double* be = b + (gp.elist ? gp.off_test[e] : e * (int64_t)(6 * Q * N3));
    __syncthreads();
    for (int k = 0; k < gp.n_src; ++k) {
      // values at the quadrature points
      for (int g = threadIdx.x; g < NQ3; g += blockDim.x) {
        const int gx = g % NQ, gy = (g / NQ) % NQ, gz = g / (NQ * NQ);
        const double xh[3] = {gp.xq[gx], gp.xq[gy], gp.xq[gz]};
        double x[3] = {0, 0, 0}, DF[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int v = 0; v < 8; ++v) {
          const int bit[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
          double f[3], df[3];
          for (int a = 0; a < 3; ++a) {
            f[a] = bit[a] ? xh[a] : 1.0 - xh[a];
            df[a] = bit[a] ? 1.0 : -1.0;
          }
          const double Nv = f[0] * f[1] * f[2];
          const double dN[3] = {df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]};
          for (int i = 0; i < 3; ++i) {
            x[i] += Nv * X8[3 * v + i];
            for (int j = 0; j < 3; ++j) DF[i][j] += X8[3 * v + i] * dN[j];
          }
        }
        double r2 = 0.0;
        for (int i = 0; i < 3; ++i) r2 += (x[i] - gp.c[k][i]) * (x[i] - gp.c[k][i]);
        const double w = gp.wq[gx] * gp.wq[gy] * gp.wq[gz] * gp.amp[k] * exp(-r2 * gp.inv2sx2[k]);
        // adj(DF) d = |J| DF^{-1} d
        const double* d = gp.d[k];
        const double a00 = DF[1][1] * DF[2][2] - DF[1][2] * DF[2][1], a01 = DF[0][2] * DF[2][1] - DF[0][1] * DF[2][2],
                     a02 = DF[0][1] * DF[1][2] - DF[0][2] * DF[1][1];
        const double a10 = DF[1][2] * DF[2][0] - DF[1][0] * DF[2][2], a11 = DF[0][0] * DF[2][2] - DF[0][2] * DF[2][0],
                     a12 = DF[0][2] * DF[1][0] - DF[0][0] * DF[1][2];
        const double a20 = DF[1][0] * DF[2][1] - DF[1][1] * DF[2][0], a21 = DF[0][1] * DF[2][0] - DF[0][0] * DF[2][1],
                     a22 = DF[0][0] * DF[1][1] - DF[0][1] * DF[1][0];
        f0[0][g] = w * (a00 * d[0] + a01 * d[1] + a02 * d[2]);
        f0[1][g] = w * (a10 * d[0] + a11 * d[1] + a12 * d[2]);
        f0[2][g] = w * (a20 * d[0] + a21 * d[1] + a22 * d[2]);
      }
      __syncthreads();
      // contract x (gx -> j), then y (gy -> k), then z (gz -> l)
      for (int it = threadIdx.x; it < 3 * NQ * NQ * N; it += blockDim.x) {
        const int j = it % N, r = it / N, gyz = r % (NQ * NQ), c = r / (NQ * NQ);
        double s = 0.0;
        for (int gx = 0; gx < NQ; ++gx) s += f0[c][gyz * NQ + gx] * gp.Lq[j][gx];
        f1[c][gyz * N + j] = s;
      }
      __syncthreads();
      for (int it = threadIdx.x; it < 3 * NQ * N * N; it += blockDim.x) {
        const int j = it % N, kk = (it / N) % N, gz = (it / (N * N)) % NQ, c = it / (N * N * NQ);
        double s = 0.0;
        for (int gy = 0; gy < NQ; ++gy) s += f1[c][(gz * NQ + gy) * N + j] * gp.Lq[kk][gy];
        f2[c][(gz * N + kk) * N + j] = s;
      }
      __syncthreads();
      for (int it = threadIdx.x; it < 3 * N3; it += blockDim.x) {
        const int sidx = it % N3, c = it / N3;
        const int j = sidx % N, kk = (sidx / N) % N, l = sidx / (N * N);
        double s = 0.0;
        for (int gz = 0; gz < NQ; ++gz) s += f2[c][(gz * N + kk) * N + j] * gp.Lq[l][gz];
        if (gp.elist) {  // every temporal test function of every sub-interval
          for (int kk = 0; kk < gp.NK; ++kk)
            for (int i = 0; i < Q; ++i) be[(c * QE + kk * Q + i) * N3 + sidx] += gp.tfk[k][kk][i] * s;
        } else {
          for (int i = 0; i < Q; ++i) be[(c * Q + i) * N3 + sidx] += gp.tf[k][i] * s;
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace

int launch_load_gauss(int P, const double* X8, int64_t ne, const GaussParams& gp, double* b, cudaStream_t s) {
  const int grid = (int)(ne < 4096 * 16 ? ne : 4096 * 16);
  switch (P) {
    case 0: k_load_gauss<0><<<grid, 256, 0, s>>>(X8, ne, gp, b); break;
    case 1: k_load_gauss<1><<<grid, 256, 0, s>>>(X8, ne, gp, b); break;
    case 2: k_load_gauss<2><<<grid, 256, 0, s>>>(X8, ne, gp, b); break;
    case 3: k_load_gauss<3><<<grid, 256, 0, s>>>(X8, ne, gp, b); break;
    case 4: k_load_gauss<4><<<grid, 256, 0, s>>>(X8, ne, gp, b); break;
    case 5: k_load_gauss<5><<<grid, 256, 0, s>>>(X8, ne, gp, b); break;
    case 6: k_load_gauss<6><<<grid, 256, 0, s>>>(X8, ne, gp, b); break;
    case 7: k_load_gauss<7><<<grid, 256, 0, s>>>(X8, ne, gp, b); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

}  // namespace stm
