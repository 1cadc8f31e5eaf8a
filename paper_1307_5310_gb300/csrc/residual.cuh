// Matrix-free space-time residual on affine brick elements (Sec. 5.2).
//
// For every element K, field F in {E, H}, component c, temporal test mode
// i < q and spatial index s the residual of Eq. residual is, written in the
// reference element (the volume curl and the face terms are metric-free for
// the covariant transform of Sec. 2.3, so only the mass term sees DF):
//
//   R_E[c][i] = eps G_c (u^E_{i+1} - delta_{i0} u^E_0)
//               - dt [curl^ y^H]_c + dt/2 sum_faces [n^ x (H_K - H_K')]_c
//   R_H[c][i] = mu  G_c (u^H_{i+1} - delta_{i0} u^H_0)
//               + dt [curl^ y^E]_c - dt/2 sum_faces [n^ x (E_K - E_K')]_c
//
// with y_i = sum_m B_im u_m the temporal contraction (B_im = int L_i l_m),
// the time-derivative term A_im = int L_i l_m' = -delta_i0 (m = 0),
// delta_{i,m-1} (m >= 1) (Sec. 5.2, "mass residual"), and G = diag(hy hz/hx,
// hx hz/hy, hx hy/hz) for a brick of edge lengths (hx, hy, hz).  This is the
// paper's C_h of Eq. bilinearform:C after one integration by parts of the
// -(H, curl v) term (the "strong" form): on an interior face the central
// flux leaves half the tangential jump, on a PEC boundary face the E-equation
// term cancels and the H-equation keeps the full n x E.  The boundary data g
// and the current J enter through the load vector b that is subtracted.
//
// The 1-D operators: D_ab = int_0^1 L_a L_b' (nonzero only for a < b, b - a
// odd), face values L_a(1) = sqrt(2a+1), L_a(0) = (-1)^a sqrt(2a+1).
//
// Two kernels per launch:
//   k_prep  : y = B u for both fields (stored), and the tangential traces of
//             y on the six faces, even/odd folded: one pass along each axis
//             gives both opposite faces (X+ = e + o at x^_a = 1, X- = e - o).
//   k_apply : R = mass + per output component two line passes (one per axis
//             a != c) each doing the 1-D derivative D along a and the lift of
//             the jumps on the two faces normal to a (folded into the curl
//             operand: D_ab and the lift share the factor L_a(1)).
// and a single-pass FP32 variant (k_fused) for uniform brick meshes.
//
// Extensions carried by the same kernels: per-element degrees (HP: element
// lists per (p, q, N_K) class, offset arrays, truncated or padded neighbour
// face modes, temporal modes cut at min(q, q') for S_h of Eq.
// bilinearform:S), 2:1 faces (equivalent traces from k_hang), local
// refinement in time (TR: N_K sub-intervals per element, temporal transfer to
// neighbours with another partition), the dissipative term D_h of Sec. 4.2
// (kap), and the block-diagonal preconditioner applied on load (pinv: the launch
// computes A P^{-1} v).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "per_device.h"

namespace stm {

constexpr int kMaxN = 8;   // p <= 7
constexpr int kMaxQ = 6;   // q <= 6

template <typename T>
struct Tables {
  T B[kMaxQ][kMaxQ + 1];  // B[i][m] = int_0^1 L_i l_m
  T Dt[kMaxN][kMaxN];     // dt * D[a][b]
  T hf[kMaxN];            // dt/2 * sqrt(2a+1)
  T lv[kMaxN];            // sqrt(2a+1)
  T kq[kMaxN];            // -1 / (4 sqrt(2a+1)): folds the flux lift into the curl (k_apply)
};

template <typename T>
struct ApplyArgs {
  // every member has a default: a launch reads only what its caller set, the rest is null
  const T* um = nullptr;            // trial modes 1..q
  int64_t um_es = 0, um_cs = 0;     //   element stride, (field,component) stride; mode stride = N3
  const T* u0 = nullptr;            // trial mode 0 (slab start) or nullptr (= 0)
  int64_t u0_es = 0, u0_cs = 0;
  const T* b = nullptr;             // load vector in the test layout, or nullptr
  T* y = nullptr;                   // [ne][2][3][q][N3] scratch: temporal contraction
  T* tr = nullptr;                  // [ne][2][3 axes][2 sides][2 comps][q][N2] scratch: face traces
  T* R = nullptr;                   // [ne][2][3][q][N3] residual (test layout)
  const int32_t* nbr = nullptr;     // [ne][6]
  const T* mass = nullptr;          // [ne][2][3]: eps G_c (E rows), mu G_c (H rows); nullptr: R already
                                    //   holds the mass term (curved elements, written by k_mass_curved)
  int64_t n_elem = 0;
  Tables<T> tb{};
  // uneven (p, q): elements of one class are listed in elist; every per-element
  // block is found through offset arrays, and neighbours may belong to other classes
  const int32_t* elist = nullptr;   // [n_elem] element ids of this class (null: uniform mesh)
  const int64_t* off_um = nullptr;  // um block of element e starts at off_um[e] (+ N3 if um_trial)
  const int64_t* off_u0 = nullptr;  // u0 block of element e starts at off_u0[e]
  const int64_t* off_R = nullptr;   // test-layout offsets (R, y, b)
  const int64_t* off_tr = nullptr;  // trace-buffer offsets
  const uint8_t* pq = nullptr;      // per element: p | q << 4
  int um_trial = 0;                 // 1: um is in the trial layout (modes 0..q per component)
  int u0_state = 0;                 // 1: u0 is a state vector ([f][c][s]); 0: trial layout
  // 2:1 faces: hslot[e*6+f] >= 0 names the slot whose equivalent neighbour traces
  // (built by k_hang in the receiving element's layout [field][comp][q][N2]) start at hoff[slot]
  const int32_t* hslot = nullptr;
  const int64_t* hoff = nullptr;
  const T* hbuf = nullptr;
  // dissipative term D_h (Sec. 4.2), or nullptr: kap[e][field][face][tangential comp] =
  // alpha (c / {Z} for E, c / {Y} for H; E on PEC faces c / Z_K, H there 0) times the
  // brick's face factor h_b / h_c; scaled by dt_k at apply time
  const T* kap = nullptr;
  T dt_k = T(0);
  // local refinement in time (Sec. 2.2): this class's elements split the slab into nk equal
  // sub-intervals (the tables then hold dt / nk); nkl[e] = log2 N_K of every element (null: all 1);
  // tmat: temporal transfer matrices M^{r,o}[a][b] = int_0^1 L_a(s) L_b((o + s) / r) ds for
  // r = 2, 4, 8 (matrices 0-1, 2-5, 6-13), kMaxQ x kMaxQ each
  int nk = 1;
  const uint8_t* nkl = nullptr;
  const T* tmat = nullptr;
  // brick meshes: non-null means um holds a Krylov vector v and the launch applies A P^{-1} v,
  // with pinv[e][f][c] = 1 / (mat G_c) the inverse of the block-diagonal preconditioner
  // P = I (x) mass (Eq. preconditioner) scaling the unknown modes on load
  const T* pinv = nullptr;
  // non-null: the launch does nothing while *skip is set (device-driven GMRES cycles)
  const int32_t* skip = nullptr;
  // general affine elements (uniform meshes): mass3[e][f][6] = mat_f G with the constant
  // metric G = |J| DF^{-1} DF^{-T} in the order xx, yy, zz, xy, xz, yz; mass is then null
  const T* mass3 = nullptr;
  // set to 1 by a kernel whose bounded wait on an asynchronous copy ran out (its R is invalid)
  int* err = nullptr;
};

// Grid of a grid-stride residual kernel: at most one wave of co-resident CTAs (the
// occupancy of this kernel, block size and shared memory on the current device), so the
// elements divide evenly over the resident CTAs (no partial last wave) and a launch the
// device-side GMRES control skips costs one wave.  The occupancy is cached per device.
template <typename K>
int wave_grid(K kernel, int block, size_t smem, int64_t count, std::atomic<int>* cache) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  const int slot = (dev >= 0 && dev < 64) ? dev : 63;
  int cap = cache[slot].load(std::memory_order_relaxed);
  if (cap <= 0) {
    int per_sm = 0, sms = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 1;
    }
    cap = std::max(1, per_sm) * std::max(1, sms);
    cache[slot].store(cap, std::memory_order_relaxed);
  }
  return (int)std::max<int64_t>(1, std::min<int64_t>(count, cap));
}

// Runs f() once per CUDA device: the first time it is called with that device current.
template <typename F>
void once_per_device(std::atomic<uint64_t>& done, F&& f) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = -1;
  }
  once_for_device(done, dev, f);
}

__host__ __device__ constexpr int tmat_index(int r, int o) { return (r == 2 ? 0 : (r == 4 ? 2 : 6)) + o; }

// Element-local addressing of one element of class (P, Q).
template <typename T, int P, int Q, bool HP, bool TR = false>
struct ElemAddr {
  static constexpr int N = P + 1, N2 = N * N, N3 = N2 * N;
  int64_t e, um, um_cs, u0, u0_cs, R, tr;
  __device__ __forceinline__ ElemAddr(const ApplyArgs<T>& A, int64_t blk) {
    if (HP) {
      const int QE = TR ? A.nk * Q : Q;  // temporal test functions of the element (all sub-intervals)
      e = A.elist[blk];
      um = A.off_um[e] + (A.um_trial ? N3 : 0);
      um_cs = A.um_trial ? (QE + 1) * N3 : QE * N3;
      u0 = A.u0 ? A.off_u0[e] : 0;
      u0_cs = A.u0_state ? N3 : (QE + 1) * N3;
      R = A.off_R[e];
      tr = A.off_tr[e];
    } else {
      e = blk;
      um = e * A.um_es;
      um_cs = A.um_cs;
      u0 = e * A.u0_es;
      u0_cs = A.u0_cs;
      R = e * (int64_t)(6 * Q * N3);
      tr = e * (int64_t)(24 * Q * N2);
    }
  }
};

// Nonzero pattern of B (banded): columns 0,1 meet rows 0,1; column m >= 2 meets rows m-2 and m.
__host__ __device__ constexpr bool b_nz(int i, int m) {
  return (m <= 1) ? (i <= 1) : (i == m || i == m - 2);
}
// Nonzero pattern of D.
__host__ __device__ constexpr bool d_nz(int a, int b) { return a < b && ((b - a) & 1); }

// Row c of a symmetric 3x3 matrix stored as (xx, yy, zz, xy, xz, yz).
template <typename T>
__device__ __forceinline__ void sym3_row(const T* m, int c, T r[3]) {
  if (c == 0) { r[0] = m[0]; r[1] = m[3]; r[2] = m[4]; }
  else if (c == 1) { r[0] = m[3]; r[1] = m[1]; r[2] = m[5]; }
  else { r[0] = m[4]; r[1] = m[5]; r[2] = m[2]; }
}

// -x by flipping the sign bit on the integer pipe (keeps the FP64 pipe for the products).
__device__ __forceinline__ double neg_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}
__device__ __forceinline__ float neg_bits(float x) { return __int_as_float(__float_as_int(x) ^ (int)0x80000000u); }

// Line of the N^3 tensor along axis a at transverse position t (the spatial
// index with the a-coordinate removed, order preserved).
template <int N>
__device__ __forceinline__ void line_geom(int a, int t, int& base, int& stride) {
  if (a == 0) { base = t * N; stride = 1; }
  else if (a == 1) { base = (t / N) * N * N + (t % N); stride = N; }
  else { base = t; stride = N * N; }
}

// Largest block of the two-kernel residual passes (k_prep, k_apply) of degree (P, Q): 512
// threads where the FP64 passes' shared memory (k_apply: y of the other field and the residual
// rows, both fields per pass up to ~110 KB; k_prep: y) leaves three or fewer blocks per SM, so
// an SM still holds 32+ warps; 256 elsewhere (a 512 bound there costs registers and blocks).
__host__ __device__ constexpr int residual_max_threads(int P, int Q) {
  return (8 * 2 * (12 * Q * (P + 1) * (P + 1) * (P + 1) * 8 > 110 * 1024 ? 1 : 2) * 3 * Q * (P + 1) * (P + 1) * (P + 1) >=
              56 * 1024 ||
          8 * 6 * Q * (P + 1) * (P + 1) * (P + 1) >= 56 * 1024)
             ? 512
             : 256;
}

// TR: the mesh has elements with N_K > 1 (HP only); false compiles the one-sub-interval code
template <typename T, int P, int Q, bool HP, bool TR = false>
__global__ void __launch_bounds__(residual_max_threads(P, Q)) k_prep(ApplyArgs<T> A) {
  if (A.skip && *A.skip) return;
  constexpr int N = P + 1, N2 = N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ys = reinterpret_cast<T*>(smem_raw);  // [2][3][Q][N3]
  // A P^{-1} v (pinv set, no slab start): the inverse block-diagonal mass scales every unknown
  // mode of a (field, component) block, so it is folded into that block's B coefficients once
  // per element (6 (Q+1) Q products) instead of one multiply per coefficient
  __shared__ T Bsc[6][kMaxQ][kMaxQ + 1];
  const int nk = TR ? A.nk : 1, QE = TR ? nk * Q : Q;
  for (int64_t blk = blockIdx.x; blk < A.n_elem; blk += gridDim.x) {
    const ElemAddr<T, P, Q, HP, TR> ad(A, blk);
    if (A.pinv) {
      for (int it = threadIdx.x; it < 6 * Q * (Q + 1); it += blockDim.x) {
        const int fc = it / (Q * (Q + 1)), r = it - fc * Q * (Q + 1), i = r / (Q + 1), m = r - i * (Q + 1);
        Bsc[fc][i][m] = A.tb.B[i][m] * A.pinv[ad.e * 6 + fc];
      }
      __syncthreads();
    }
#pragma unroll 1
    for (int k = 0; k < nk; ++k) {  // temporal sub-intervals (Sec. 2.2)
    auto contract = [&](auto prec) {
      constexpr bool PRE = decltype(prec)::value;
      for (int it = threadIdx.x; it < 6 * N3; it += blockDim.x) {
        const int fc = it / N3, s = it - fc * N3;
        T u[Q + 1];
        // mode 0 of sub-interval k: the slab start, else mode 1 (end value) of sub-interval k - 1
        if (k == 0) u[0] = (!PRE && A.u0) ? A.u0[ad.u0 + fc * ad.u0_cs + s] : T(0);
        else u[0] = A.um[ad.um + fc * ad.um_cs + (k - 1) * Q * N3 + s];
#pragma unroll
        for (int m = 1; m <= Q; ++m) u[m] = A.um[ad.um + fc * ad.um_cs + (k * Q + m - 1) * N3 + s];
        T* yg = A.y + ad.R + fc * (int64_t)(QE * N3) + k * Q * N3 + s;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          T acc = T(0);
          bool first = true;
#pragma unroll
          for (int m = 0; m <= Q; ++m) {
            if (b_nz(i, m)) {
              const T bb = PRE ? Bsc[fc][i][m] : A.tb.B[i][m];
              acc = first ? bb * u[m] : fma(bb, u[m], acc);
              first = false;
            }
          }
          ys[(fc * Q + i) * N3 + s] = acc;
          yg[i * N3] = acc;
        }
      }
    };
    if (A.pinv) contract(std::true_type{});
    else contract(std::false_type{});
    __syncthreads();
    // traces: items (f, a, bi, i, t)
    for (int it = threadIdx.x; it < 12 * Q * N2; it += blockDim.x) {
      int r = it;
      const int t = r % N2; r /= N2;
      const int i = r % Q; r /= Q;
      const int bi = r % 2; r /= 2;
      const int a = r % 3;
      const int f = r / 3;
      const int b = (a == 0) ? 1 + bi : (a == 1 ? 2 * bi : bi);
      int base, stride;
      line_geom<N>(a, t, base, stride);
      const T* yl = ys + ((f * 3 + b) * Q + i) * N3 + base;
      T ev = T(0), od = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const T v = yl[j * stride];
        if (j & 1) od = fma(A.tb.lv[j], v, od);
        else ev = fma(A.tb.lv[j], v, ev);
      }
      const int64_t o = ((((int64_t)f * 3 + a) * 2 + 0) * 2 + bi) * QE + k * Q + i;
      A.tr[ad.tr + o * N2 + t] = ev - od;                 // face x^_a = 0
      A.tr[ad.tr + (o + 2 * QE) * N2 + t] = ev + od;      // face x^_a = 1
    }
    __syncthreads();
    }
  }
}

// Trace of the neighbour en across face (a, side of the element), component
// slot bi of field fp, temporal test mode i, at the element's transverse
// position t (N x N).  With uneven degrees the neighbour's orthonormal face
// modes are truncated or zero-padded and its temporal modes cut at
// min(q, q') (the projection onto the common temporal test space of
// Eq. bilinearform:S).
//
// Local refinement in time: the own test function L_i on sub-interval k and
// the neighbour's partition (N_K' sub-intervals) are nested.  The neighbour
// term <H', Pi~ L_i^k> (Pi~ onto the common test space: piecewise
// P_{min(q,q')-1} on the coarser partition) is a combination of the
// neighbour's own temporal moments y', in units of the own dt / N_K:
//   N_K' = N_K: y'_{k,i} (i < q');
//   N_K' < N_K (own finer, r = N_K/N_K', k = r k' + o): sum_{l<q~} M^{r,o}[i][l] y'_{k',l};
//   N_K' > N_K (own coarser, r = N_K'/N_K): for i < q~,
//     sum_{o<r} (1/r) sum_{j<=i} M^{r,o}[j][i] y'_{r k + o, j}.
//
// Uneven degrees: fc holds, per face of the element, the neighbour's trace
// offset, degrees p | q << 4 and N_K (k_apply keeps them in shared memory, so
// a line needs one dependent load, not three).
struct FaceCache {
  int64_t off[6];
  int pq[6], nk[6];
};

template <typename T, int N, int Q, bool HP, bool TR = false>
__device__ __forceinline__ T nbr_trace(const ApplyArgs<T>& A, int64_t en, int nside, int fp, int a, int bi, int i,
                                       int t, int k, const FaceCache& fc, int face) {
  if (!HP) {
    constexpr int N2 = N * N;
    const int64_t so = ((((int64_t)fp * 3 + a) * 2 + nside) * 2 + bi) * Q + i;
    return A.tr[en * (int64_t)(24 * Q * N2) + so * N2 + t];
  }
  const int pq = fc.pq[face];
  const int Nn = (pq & 15) + 1, qn = pq >> 4;
  const int slow = t / N, fast = t - slow * N;
  if (!TR) {  // one sub-interval everywhere
    if (i >= qn || slow >= Nn || fast >= Nn) return T(0);
    const int64_t so = ((((int64_t)fp * 3 + a) * 2 + nside) * 2 + bi) * qn + i;
    return A.tr[fc.off[face] + so * (Nn * Nn) + slow * Nn + fast];
  }
  const int qt = qn < Q ? qn : Q;
  // rows i >= qt vanish in every case (M^{r,o}[i][l] = 0 for l < i: L_i is orthogonal to P_l)
  if (i >= qt || slow >= Nn || fast >= Nn) return T(0);
  const int nkn = fc.nk[face], qen = nkn * qn, nn2 = Nn * Nn;
  const T* src = A.tr + fc.off[face] + ((((int64_t)fp * 3 + a) * 2 + nside) * 2 + bi) * qen * nn2 + slow * Nn + fast;
  if (nkn == A.nk) return src[(int64_t)(k * qn + i) * nn2];
  if (nkn < A.nk) {
    const int r = A.nk / nkn, kk = k / r, o = k - kk * r;
    const T* M = A.tmat + tmat_index(r, o) * (kMaxQ * kMaxQ) + i * kMaxQ;
    T acc = T(0);
    for (int l = i; l < qt; ++l) acc = fma(M[l], src[(int64_t)(kk * qn + l) * nn2], acc);
    return acc;
  }
  const int r = nkn / A.nk;
  T acc = T(0);
  for (int o = 0; o < r; ++o) {
    const T* M = A.tmat + tmat_index(r, o) * (kMaxQ * kMaxQ);
    for (int j = 0; j <= i; ++j) acc = fma(M[j * kMaxQ + i], src[(int64_t)((k * r + o) * qn + j) * nn2], acc);
  }
  return acc / T(r);
}

// Offset in the test layout [f][c][QE][N3] of entry w = (c, i, s) of one sub-interval's
// [3][Q][N3] block of field f, the sub-interval's rows starting at rk (per component).
template <int Q, int N3, bool HP = true>
__device__ __forceinline__ int64_t test_ofs(int64_t rk, int f, int w, int QE) {
  if constexpr (!HP) return rk + (int64_t)f * (3 * Q * N3) + w;  // one sub-interval: contiguous
  const int cc = w / (Q * N3);
  return rk + (int64_t)(f * 3 + cc) * QE * N3 + (w - cc * Q * N3);
}

// Line passes of k_apply: pass k handles, for output component c, the derivative axis
// a = (k == 0 ? (c == 0 ? 1 : 0) : (c == 2 ? 1 : 2)).  The line's term carries the sign
// s_F eps_{cab} (s_E = -1, s_H = +1), negative exactly when (f == 0) == ((c, a) cyclic).
// curl_combo maps the combination index cb (NF fields x 3 components) to (field slot fl,
// component c) with the positive lines first, and returns the sign.
template <int NF>
__device__ __forceinline__ void curl_combo(int k, int f0, int cb, int& fl, int& c, bool& neg) {
  if constexpr (NF == 2) {
    // pass 0: positive (f, c) = (0,1) (1,0) (1,2), negative (0,0) (0,2) (1,1); pass 1: the reverse
    constexpr int ord[2][6] = {{1, 3, 5, 0, 2, 4}, {0, 2, 4, 1, 3, 5}};
    const int fc = ord[k][cb];
    fl = fc / 3;
    c = fc - 3 * fl;
    neg = cb >= 3;
  } else {
    // one field per pass: (f, pass) = (0,0) and (1,1) have one positive line set, c = 1;
    // (1,0) and (0,1) have two, c = 0 and 2
    fl = 0;
    const bool one = (f0 == k);
    constexpr int ord1[3] = {1, 0, 2}, ord2[3] = {0, 2, 1};
    c = one ? ord1[cb] : ord2[cb];
    neg = one ? cb >= 1 : cb >= 2;
  }
}

// Shared memory per k_apply pass: y of the other field and the residual rows;
// both fields in one pass when that fits in ~110 KB, else one field per pass.
template <typename T, int P, int Q>
struct ApplyShape {
  static constexpr int N3 = (P + 1) * (P + 1) * (P + 1);
  static constexpr bool split = 12 * Q * N3 * sizeof(T) > 110 * 1024;
  static constexpr int NF = split ? 1 : 2;  // fields per pass
  static constexpr size_t smem = sizeof(T) * 2 * NF * 3 * Q * N3;
};

template <typename T, int P, int Q, bool HP, bool TR = false>
__global__ void __launch_bounds__(residual_max_threads(P, Q)) k_apply(ApplyArgs<T> A) {
  if (A.skip && *A.skip) return;
  constexpr int N = P + 1, N2 = N * N, N3 = N2 * N;
  constexpr int NF = ApplyShape<T, P, Q>::NF;
  constexpr int FB = 3 * Q * N3;           // one field's block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ys = reinterpret_cast<T*>(smem_raw);  // [NF][3][Q][N3]: y of the other field
  T* Rs = ys + NF * FB;                     // [NF][3][Q][N3]: residual rows
  __shared__ FaceCache fcs;                 // uneven degrees only
  const int nk = TR ? A.nk : 1, QE = TR ? nk * Q : Q;
  for (int64_t blk = blockIdx.x; blk < A.n_elem; blk += gridDim.x) {
    const ElemAddr<T, P, Q, HP, TR> ad(A, blk);
    const int64_t e = ad.e;
    const int32_t* nb = A.nbr + e * 6;
    if (HP && threadIdx.x < 6) {  // read after the first barrier below
      const int f = threadIdx.x, en = nb[f];
      fcs.off[f] = en >= 0 ? A.off_tr[en] : (en == -2 ? A.hoff[A.hslot[e * 6 + f]] : 0);
      fcs.pq[f] = en >= 0 ? A.pq[en] : 0;
      fcs.nk[f] = (en >= 0 && A.nkl) ? 1 << A.nkl[en] : 1;
    }
#pragma unroll 1
    for (int sk = 0; sk < nk; ++sk) {  // temporal sub-intervals (Sec. 2.2)
    const int64_t rk = ad.R + (int64_t)sk * Q * N3;  // sub-interval sk's rows start here (per component)
#pragma unroll 1
    for (int f0 = 0; f0 < 2; f0 += NF) {
      for (int it = threadIdx.x; it < NF * FB; it += blockDim.x) {
        const int fl = NF == 1 ? 0 : it / FB;
        ys[it] = A.y[test_ofs<Q, N3, TR>(rk, 1 - (f0 + fl), it - fl * FB, QE)];
      }
      // mass rows: items (field, component, s), the temporal modes unrolled; the variant
      // (mode 0 of the sub-interval, preconditioned input, load) is chosen once per pass so
      // no FP64 instruction is predicated
      auto mass_rows = [&](auto prevc, auto prec, auto loadc) {
        constexpr int PREV = decltype(prevc)::value;  // 0: none, 1: previous sub-interval, 2: u0
        constexpr bool PRE = decltype(prec)::value, LOAD = decltype(loadc)::value;
        for (int it = threadIdx.x; it < NF * 3 * N3; it += blockDim.x) {
          const int fcl = it / N3, s = it - fcl * N3;
          const int fl = NF == 1 ? 0 : fcl / 3, cc = fcl - 3 * fl;
          const int fc = (f0 + fl) * 3 + cc;
          const T mc = A.mass[e * 6 + fc];
          const T* uc = A.um + ad.um + fc * ad.um_cs + (int64_t)sk * Q * N3 + s;
          T* Rr = Rs + fl * FB + cc * Q * N3 + s;
          // with PRE (A P^{-1} v) the mass block times P^{-1} is the identity: the term is v
          {  // mode 0: minus mode 0 of the sub-interval (previous sub-interval's end or slab start)
            T v = PRE ? uc[0] : mc * uc[0];
            if constexpr (PREV == 1) v = PRE ? v - uc[-Q * N3] : fma(-mc, uc[-Q * N3], v);
            if constexpr (PREV == 2) v = fma(-mc, A.u0[ad.u0 + fc * ad.u0_cs + s], v);
            if constexpr (LOAD) v -= A.b[test_ofs<Q, N3, TR>(rk, f0 + fl, cc * Q * N3 + s, QE)];
            Rr[0] = v;
          }
#pragma unroll 1
          for (int i = 1; i < Q; ++i) {
            T v = PRE ? uc[i * N3] : mc * uc[i * N3];
            if constexpr (LOAD) v -= A.b[test_ofs<Q, N3, TR>(rk, f0 + fl, (cc * Q + i) * N3 + s, QE)];
            Rr[i * N3] = v;
          }
        }
      };
      if (A.mass) {
        const int prev = sk > 0 ? 1 : (A.u0 ? 2 : 0);
        const bool pre = A.pinv != nullptr, load = A.b != nullptr;
        using I0 = std::integral_constant<int, 0>;
        using I1 = std::integral_constant<int, 1>;
        using I2 = std::integral_constant<int, 2>;
        auto with_prev = [&](auto pc, auto prc) {
          if (load) mass_rows(pc, prc, std::true_type{});
          else mass_rows(pc, prc, std::false_type{});
        };
        auto with_pre = [&](auto prc) {
          if (prev == 1) with_prev(I1{}, prc);
          else if (prev == 2) with_prev(I2{}, prc);
          else with_prev(I0{}, prc);
        };
        if (pre) with_pre(std::true_type{});
        else with_pre(std::false_type{});
      } else if (A.mass3) {
        // general affine elements: the constant 3x3 metric couples the components
        for (int it = threadIdx.x; it < NF * 3 * N3; it += blockDim.x) {
          const int fcl = it / N3, s = it - fcl * N3;
          const int fl = NF == 1 ? 0 : fcl / 3, cc = fcl - 3 * fl, f = f0 + fl;
          T mr[3];
          sym3_row(A.mass3 + (e * 2 + f) * 6, cc, mr);
          const T* uf = A.um + ad.um + (int64_t)(f * 3) * ad.um_cs + s;
          T* Rr = Rs + fl * FB + cc * Q * N3 + s;
#pragma unroll 1
          for (int i = 0; i < Q; ++i) {
            T v = mr[0] * uf[i * N3];
            v = fma(mr[1], uf[ad.um_cs + i * N3], v);
            v = fma(mr[2], uf[2 * ad.um_cs + i * N3], v);
            if (i == 0 && A.u0) {
              const T* u0f = A.u0 + ad.u0 + (int64_t)(f * 3) * ad.u0_cs + s;
              v = fma(-mr[0], u0f[0], v);
              v = fma(-mr[1], u0f[ad.u0_cs], v);
              v = fma(-mr[2], u0f[2 * ad.u0_cs], v);
            }
            if (A.b) v -= A.b[test_ofs<Q, N3, TR>(rk, f, (cc * Q + i) * N3 + s, QE)];
            Rr[i * N3] = v;
          }
        }
      } else {
        // curved elements: R already holds the mass term (k_mass_curved)
        for (int it = threadIdx.x; it < NF * FB; it += blockDim.x) {
          const int fl = NF == 1 ? 0 : it / FB;
          const int w = it - fl * FB;
          const int64_t o = test_ofs<Q, N3, TR>(rk, f0 + fl, w, QE);
          Rs[it] = A.b ? A.R[o] - A.b[o] : A.R[o];
        }
      }
      __syncthreads();
#pragma unroll 1
      for (int k = 0; k < 2; ++k) {
        for (int it = threadIdx.x; it < NF * 3 * Q * N2; it += blockDim.x) {
          // lines ordered by the sign of their curl term, so that a warp rarely holds both
          const int cb = it / (Q * N2), r = it - cb * (Q * N2);
          const int i = r / N2, t = r - i * N2;
          int fl, c;
          bool neg;
          curl_combo<NF>(k, f0, cb, fl, c, neg);
          const int f = f0 + fl, fp = 1 - f;
          const int a = (k == 0) ? (c == 0 ? 1 : 0) : (c == 2 ? 1 : 2);
          const int b = 3 - c - a;
          const int bi = (a == 0) ? b - 1 : (a == 1 ? b / 2 : b);
          int base, stride;
          line_geom<N>(a, t, base, stride);
          const T* yl = ys + fl * FB + (b * Q + i) * N3 + base;
          // jumps of the tangential component b of field fp on the faces normal to a
          const int64_t so = ((((int64_t)fp * 3 + a) * 2) * 2 + bi) * QE + sk * Q + i;  // side-0 slot
          const T* tre = A.tr + ad.tr;
          const T xm = tre[so * N2 + t];
          const T xp = tre[(so + 2 * QE) * N2 + t];
          const int ep = nb[2 * a + 1], em = nb[2 * a];
          // the other side's trace: the neighbour's, or on a PEC face the mirror value (E: -own,
          // so the jump is 2 own; H: +own, jump 0) chosen by integer ops; one subtraction each
          T op, om;
          if (ep >= 0) op = nbr_trace<T, N, Q, HP, TR>(A, ep, 0, fp, a, bi, i, t, sk, fcs, 2 * a + 1);
          else if (HP && ep == -2) op = A.hbuf[fcs.off[2 * a + 1] + ((fp * 2 + bi) * Q + i) * N2 + t];
          else op = (fp == 0) ? neg_bits(xp) : xp;
          if (em >= 0) om = nbr_trace<T, N, Q, HP, TR>(A, em, 1, fp, a, bi, i, t, sk, fcs, 2 * a);
          else if (HP && em == -2) om = A.hbuf[fcs.off[2 * a] + ((fp * 2 + bi) * Q + i) * N2 + t];
          else om = (fp == 0) ? neg_bits(xm) : xm;
          const T jp = xp - op, jm = xm - om;
          const T sp = jp + jm, dm = jp - jm;
          T yv[N];
#pragma unroll
          for (int j = 0; j < N; ++j) yv[j] = yl[j * stride];
          T* Rl = Rs + fl * FB + (c * Q + i) * N3 + base;
          // the sign s_F eps_{cab} of the line's curl and flux terms is a compile-time constant
          // of each branch, carried by the table operands of the FMAs (no extra instruction);
          // lines are ordered by sign, so only the warp at the boundary runs both branches
          auto body = [&](auto negc) {
            constexpr T sg = decltype(negc)::value ? T(-1) : T(1);
            if (A.kap) {
              // D_h: alpha-weighted jumps of component c of the same field f on the two
              // faces normal to a, lifted with L_al(1) and L_al(0) = (-1)^al L_al(1);
              // on a PEC face the E jump is the own trace (E - g, g in the load)
              const int bc = (a == 0) ? c - 1 : (a == 1 ? c / 2 : c);
              const int64_t sc = ((((int64_t)f * 3 + a) * 2) * 2 + bc) * QE + sk * Q + i;
              const T zm = tre[sc * N2 + t], zp = tre[(sc + 2 * QE) * N2 + t];
              // other side: the neighbour's trace; on a PEC face 0 for E (jump = own) and own for H
              const T gop = (ep >= 0) ? nbr_trace<T, N, Q, HP, TR>(A, ep, 0, f, a, bc, i, t, sk, fcs, 2 * a + 1)
                                      : (f == 0 ? T(0) : zp);
              const T gom = (em >= 0) ? nbr_trace<T, N, Q, HP, TR>(A, em, 1, f, a, bc, i, t, sk, fcs, 2 * a)
                                      : (f == 0 ? T(0) : zm);
              const T gp = zp - gop, gm = zm - gom;
              const T* kp = A.kap + e * 24 + f * 12 + 4 * a + bc;
              const T dp = A.dt_k * kp[2] * gp, dn = A.dt_k * kp[0] * gm;
              // the central-flux lift hf[al] = (dt/2) lv[al] shares the factor lv[al]
              const T zev = fma(-sg * A.tb.hf[0], dm, dp + dn), zod = fma(-sg * A.tb.hf[0], sp, dp - dn);
#pragma unroll
              for (int al = 0; al < N; ++al) {
                T r2 = Rl[al * stride];
                r2 = fma(A.tb.lv[al], (al & 1) ? zod : zev, r2);
#pragma unroll
                for (int be = 0; be < N; ++be)
                  if (d_nz(al, be)) r2 = fma(sg * A.tb.Dt[al][be], yv[be], r2);
                Rl[al * stride] = r2;
              }
            } else {
              // Dt[a][b] = 2 dt L_a(1) L_b(1) and hf[a] = dt/2 L_a(1) share the factor L_a(1), so
              // the lift -hf[a] X of every row a but the last equals Dt[a][B] X kq[B] with B the
              // largest index of the other parity (which every such row's curl sum reaches):
              // folded into y[B] once per line instead of one FMA per row
              constexpr int B0 = ((N - 1) & 1) ? N - 1 : N - 2;  // largest odd index: even rows, X = dm
              constexpr int B1 = ((N - 1) & 1) ? N - 2 : N - 1;  // largest even index: odd rows, X = sp
              if constexpr (B0 >= 1) yv[B0] = fma(A.tb.kq[B0], dm, yv[B0]);
              if constexpr (B1 >= 2) yv[B1] = fma(A.tb.kq[B1], sp, yv[B1]);
#pragma unroll
              for (int al = 0; al < N; ++al) {
                T r2 = Rl[al * stride];
                if (al == N - 1) r2 = fma(-sg * A.tb.hf[al], (al & 1) ? sp : dm, r2);
#pragma unroll
                for (int be = 0; be < N; ++be)
                  if (d_nz(al, be)) r2 = fma(sg * A.tb.Dt[al][be], yv[be], r2);
                Rl[al * stride] = r2;
              }
            }
          };
          if (neg) body(std::true_type{});
          else body(std::false_type{});
        }
        __syncthreads();
      }
      for (int it = threadIdx.x; it < NF * FB; it += blockDim.x) {
        const int fl = NF == 1 ? 0 : it / FB;
        A.R[test_ofs<Q, N3, TR>(rk, f0 + fl, it - fl * FB, QE)] = Rs[it];
      }
      __syncthreads();
    }
    }
  }
}

// Line of the N^3 tensor along the compile-time axis A at transverse position t.
template <int N, int A>
__device__ __forceinline__ int line_base(int t) {
  if constexpr (A == 0) return t * N;
  else if constexpr (A == 1) return (t / N) * N * N + (t % N);
  else return t;
}
template <int N, int A>
constexpr int line_stride() {
  return A == 0 ? 1 : (A == 1 ? N : N * N);
}

// Calls f(std::integral_constant<int, a>) for a runtime, warp-uniform axis a.
template <typename F>
__device__ __forceinline__ void with_axis(int a, F&& f) {
  if (a == 0) f(std::integral_constant<int, 0>{});
  else if (a == 1) f(std::integral_constant<int, 1>{});
  else f(std::integral_constant<int, 2>{});
}

// The two derivative passes over the residual planes of field f, component c of one element
// (single-pass FP32 kernels): for every temporal test mode, lines along each axis a != c add the
// curl of y of the other field (component b = 3 - c - a) and the flux lift of its jumps, folded
// into the curl operand (own traces from y, the other side from the neighbour traces nt or the
// PEC mirror); with KAP also the dissipative term D_h of Sec. 4.2 (jumps of y^f_c, unfolded
// lift).  Rp: the (f, c) planes [Q][N3] in shared memory, holding the mass term; ys: y of both
// fields [2][3][Q][N3]; nt: neighbour traces [6 faces][2 fields][2 comps][Q][N2]; nb: the six
// neighbours of element e.  One warp, lanes over the lines of a pass.
template <typename T, int N, int Q, bool KAP>
__device__ __forceinline__ void fused_lines(const ApplyArgs<T>& A, int64_t e, int f, int c, const T* ys,
                                            const T* nt, const int32_t* nb, T* Rp, int lane) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const int fp = 1 - f;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int a = (k == 0) ? (c == 0 ? 1 : 0) : (c == 2 ? 1 : 2);
    const int b = 3 - c - a;
    const int bi = (a == 0) ? b - 1 : (a == 1 ? b / 2 : b);
    // sign s_F eps_{cab} of the planes' terms along a (warp-uniform)
    const bool neg = ((f == 0) == (((a - c + 3) % 3) == 1));
    const T* yb = ys + (fp * 3 + b) * Q * N3;
    const bool hasp = nb[2 * a + 1] >= 0, hasm = nb[2 * a] >= 0;
    const T* ntp = nt + ((((2 * a + 1) * 2 + fp) * 2 + bi) * Q) * N2;
    const T* ntm = nt + ((((2 * a) * 2 + fp) * 2 + bi) * Q) * N2;
    // D_h (Sec. 4.2): jumps of component c of the same field f on the faces normal to a,
    // own traces from y^f_c, the neighbour's from its staged traces; alpha-weights per face
    const int bc = (a == 0) ? c - 1 : (a == 1 ? c / 2 : c);
    const T* zb = ys + (f * 3 + c) * Q * N3;
    const T* gtp = nt + ((((2 * a + 1) * 2 + f) * 2 + bc) * Q) * N2;
    const T* gtm = nt + ((((2 * a) * 2 + f) * 2 + bc) * Q) * N2;
    const T kpp = KAP ? A.dt_k * A.kap[e * 24 + f * 12 + 4 * a + 2 + bc] : T(0);
    const T kpm = KAP ? A.dt_k * A.kap[e * 24 + f * 12 + 4 * a + bc] : T(0);
    auto lines = [&](auto ac, auto negc) {
      constexpr int AX = decltype(ac)::value, ST = line_stride<N, AX>();
      constexpr T sg = decltype(negc)::value ? T(-1) : T(1);
      for (int t = lane; t < N2; t += 32) {
        const int base = line_base<N, AX>(t);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const T* yl = yb + i * N3 + base;
          T yv[N];
          T ev = T(0), od = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            yv[j] = yl[j * ST];
            if (j & 1) od = fma(A.tb.lv[j], yv[j], od);
            else ev = fma(A.tb.lv[j], yv[j], ev);
          }
          const T xp = ev + od, xm = ev - od;  // own traces at x^_a = 1 and 0
          // other side: neighbour trace, or the PEC mirror (E: -own, H: +own)
          const T op = hasp ? ntp[i * N2 + t] : ((fp == 0) ? neg_bits(xp) : xp);
          const T om = hasm ? ntm[i * N2 + t] : ((fp == 0) ? neg_bits(xm) : xm);
          const T jp = xp - op, jm = xm - om;
          const T sp = jp + jm, dm = jp - jm;
          T* Rl = Rp + i * N3 + base;
          if constexpr (KAP) {
            // own traces of y^f_c; on a PEC face the E jump is the own trace (E - g, g in
            // the load) and the H jump 0; lifted with L_al(1) and L_al(0) = (-1)^al L_al(1)
            const T* zl = zb + i * N3 + base;
            T ze = T(0), zo = T(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
              if (j & 1) zo = fma(A.tb.lv[j], zl[j * ST], zo);
              else ze = fma(A.tb.lv[j], zl[j * ST], ze);
            }
            const T zp = ze + zo, zm = ze - zo;
            const T gop = hasp ? gtp[i * N2 + t] : (f == 0 ? T(0) : zp);
            const T gom = hasm ? gtm[i * N2 + t] : (f == 0 ? T(0) : zm);
            const T dp = kpp * (zp - gop), dn = kpm * (zm - gom);
            const T zev = fma(-sg * A.tb.hf[0], dm, dp + dn), zod = fma(-sg * A.tb.hf[0], sp, dp - dn);
#pragma unroll
            for (int al = 0; al < N; ++al) {
              T r2 = Rl[al * ST];
              r2 = fma(A.tb.lv[al], (al & 1) ? zod : zev, r2);
#pragma unroll
              for (int be = 0; be < N; ++be)
                if (d_nz(al, be)) r2 = fma(sg * A.tb.Dt[al][be], yv[be], r2);
              Rl[al * ST] = r2;
            }
          } else {
            // flux lift folded into the curl operand as in k_apply
            constexpr int B0 = ((N - 1) & 1) ? N - 1 : N - 2, B1 = ((N - 1) & 1) ? N - 2 : N - 1;
            if constexpr (B0 >= 1) yv[B0] = fma(A.tb.kq[B0], dm, yv[B0]);
            if constexpr (B1 >= 2) yv[B1] = fma(A.tb.kq[B1], sp, yv[B1]);
#pragma unroll
            for (int al = 0; al < N; ++al) {
              T r2 = Rl[al * ST];
              if (al == N - 1) r2 = fma(-sg * A.tb.hf[al], (al & 1) ? sp : dm, r2);
#pragma unroll
              for (int be = 0; be < N; ++be)
                if (d_nz(al, be)) r2 = fma(sg * A.tb.Dt[al][be], yv[be], r2);
              Rl[al * ST] = r2;
            }
          }
        }
      }
    };
    with_axis(a, [&](auto ac) {
      if (neg) lines(ac, std::true_type{});
      else lines(ac, std::false_type{});
    });
    __syncwarp();
  }
}

// Single-pass variant (used for FP32, where the kernel is bound by memory
// traffic, not arithmetic): one CTA per element at a time reads its own
// coefficients once, recomputes the six neighbour face traces from the
// neighbours' coefficients (face neighbours sit close in memory, so these
// reads mostly hit L2), forms its own traces in registers inside the line
// loop, and writes R.  No y or trace scratch goes through HBM.
//
// Work split: (a) all threads form y = B u and the mass rows of the element in
// shared memory; (b) one warp per (face, field) forms the neighbour's traces on
// that face; (c) every warp owns the residual planes of one (field, component):
// it runs both line passes (one per derivative axis) over all temporal modes
// with only warp synchronisation and stores them to HBM.  Two CTA barriers per
// element.  Line axes are
// dispatched warp-uniformly to compile-time strides, so every load of a line
// has an immediate offset.
template <typename T, int P, int Q, bool PRE, bool KAP = false>
__global__ void __launch_bounds__(192) k_fused(ApplyArgs<T> A) {
  if (A.skip && *A.skip) return;
  constexpr int N = P + 1, N2 = N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ys = reinterpret_cast<T*>(smem_raw);  // [2][3][Q][N3] temporal contraction
  T* Rs = ys + 6 * Q * N3;                  // [2][3][Q][N3] residual planes
  T* nt = Rs + 6 * Q * N3;                  // [6 faces][2 fields][2 comps][Q][N2] neighbour traces
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int um_cs = (int)A.um_cs, u0_cs = (int)A.u0_cs;
  for (int64_t e = blockIdx.x; e < A.n_elem; e += gridDim.x) {
    const int32_t* nb = A.nbr + e * 6;
    const T* ume = A.um + e * A.um_es;
    const T* u0e = A.u0 ? A.u0 + e * A.u0_es : nullptr;
    const int64_t re = e * (int64_t)(6 * Q * N3);
    // (a) own coefficients: temporal contraction and the mass term
    for (int it = threadIdx.x; it < 6 * N3; it += blockDim.x) {
      const int fc = it / N3, s = it - fc * N3;
      const T* up = ume + fc * um_cs + s;
      T u[Q + 1], v[Q];
      u[0] = u0e ? u0e[fc * u0_cs + s] : T(0);
#pragma unroll
      for (int m = 1; m <= Q; ++m) u[m] = v[m - 1] = up[(m - 1) * N3];
      if constexpr (PRE) {
        const T sc = A.pinv[e * 6 + fc];
#pragma unroll
        for (int m = 1; m <= Q; ++m) u[m] *= sc;
      }
      const T mc = A.mass ? A.mass[e * 6 + fc] : T(0);
      T* yo = ys + fc * Q * N3 + s;
      T* ro = Rs + fc * Q * N3 + s;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        T acc = T(0);
        bool first = true;
#pragma unroll
        for (int m = 0; m <= Q; ++m) {
          if (b_nz(i, m)) {
            acc = first ? A.tb.B[i][m] * u[m] : fma(A.tb.B[i][m], u[m], acc);
            first = false;
          }
        }
        yo[i * N3] = acc;
        const int64_t o = re + (fc * Q + i) * N3 + s;
        T w;
        if (A.mass) {
          // with PRE the mass block times P^{-1} is the identity: the term is v itself
          w = PRE ? v[i] : mc * u[i + 1];
          if (i == 0 && u0e) w = fma(-mc, u[0], w);
        } else if (A.mass3) {
          // general affine elements: the constant 3x3 metric couples the components
          const int f = fc >= 3 ? 1 : 0, c = fc - 3 * f;
          T mr[3];
          sym3_row(A.mass3 + (e * 2 + f) * 6, c, mr);
          const T* uf = ume + (f * 3) * um_cs + i * N3 + s;
          w = mr[0] * uf[0];
          w = fma(mr[1], uf[um_cs], w);
          w = fma(mr[2], uf[2 * um_cs], w);
          if (i == 0 && u0e) {
            const T* u0f = u0e + (f * 3) * u0_cs + s;
            w = fma(-mr[0], u0f[0], w);
            w = fma(-mr[1], u0f[u0_cs], w);
            w = fma(-mr[2], u0f[2 * u0_cs], w);
          }
        } else {
          w = A.R[o];  // curved elements: the mass term is already in R
        }
        if (A.b) w -= A.b[o];
        ro[i * N3] = w;
      }
    }
    // (b) neighbour traces: one warp per (face, field), both tangential components, lanes over t
    for (int task = warp; task < 12; task += nwarp) {
      const int fld = task & 1, face = task >> 1;
      const int a = face >> 1, side = face & 1;
      const int64_t en = nb[face];
      if (en < 0) continue;  // warp-uniform
      const T* ue = A.um + en * A.um_es;
      const T* u0e2 = A.u0 ? A.u0 + en * A.u0_es : nullptr;
#pragma unroll 1
      for (int bi = 0; bi < 2; ++bi) {
      const int b = (a == 0) ? 1 + bi : (a == 1 ? 2 * bi : bi);
      const T* un = ue + (fld * 3 + b) * um_cs;
      const T* u0n = u0e2 ? u0e2 + (fld * 3 + b) * u0_cs : nullptr;
      const T sc = PRE ? A.pinv[en * 6 + fld * 3 + b] : T(1);
      T* nto = nt + ((task * 2 + bi) * Q) * N2;
      with_axis(a, [&](auto ac) {
        constexpr int AX = decltype(ac)::value, ST = line_stride<N, AX>();
        for (int t = lane; t < N2; t += 32) {
          const int base = line_base<N, AX>(t);
          // the neighbour across face (a, side) meets it with its face (a, 1 - side):
          // L_j(0) = (-1)^j L_j(1) for side 1, L_j(1) for side 0
          T tu[Q + 1];
          tu[0] = T(0);
          if (u0n) {
            T ev = T(0), od = T(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
              if (j & 1) od = fma(A.tb.lv[j], u0n[base + j * ST], od);
              else ev = fma(A.tb.lv[j], u0n[base + j * ST], ev);
            }
            tu[0] = side ? ev - od : ev + od;
          }
          const T* ul = un + base;
#pragma unroll
          for (int m = 1; m <= Q; ++m) {
            T ev = T(0), od = T(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
              if (j & 1) od = fma(A.tb.lv[j], ul[(m - 1) * N3 + j * ST], od);
              else ev = fma(A.tb.lv[j], ul[(m - 1) * N3 + j * ST], ev);
            }
            tu[m] = (side ? ev - od : ev + od) * sc;
          }
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            T acc = T(0);
#pragma unroll
            for (int m = 0; m <= Q; ++m)
              if (b_nz(i, m)) acc = fma(A.tb.B[i][m], tu[m], acc);
            nto[i * N2 + t] = acc;
          }
        }
      });
      }
    }
    __syncthreads();
    // (c) residual planes: one warp per (field, component) at a time, all Q temporal test
    //     modes of it, so the axis, sign, pointers and line geometry are set up once per pass
    for (int fc = warp; fc < 6; fc += nwarp) {
      const int f = fc >= 3 ? 1 : 0, c = fc - 3 * f;
      T* Rp = Rs + fc * Q * N3;
      fused_lines<T, N, Q, KAP>(A, e, f, c, ys, nt, nb, Rp, lane);
      // the Q planes of (f, c) are contiguous in R
      T* Rg = A.R + re + fc * Q * N3;
      for (int s2 = lane; s2 < Q * N3; s2 += 32) Rg[s2] = Rp[s2];
    }
    __syncthreads();
  }
}

// ---- bulk copies shared -> global through the tensor memory accelerator (bulk groups) ----
// Orders this thread's earlier shared-memory writes before later async-proxy reads of them.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// bytes: a multiple of 16; dst and src 16-byte aligned.
__device__ __forceinline__ void bulk_store(float* dst, const float* src, int bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst),
               "r"((uint32_t)__cvta_generic_to_shared(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// Waits (in hardware) until this thread's committed bulk copies have read their sources / completed.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// ---- bulk copies global -> shared, completed on an mbarrier (transaction bytes) ----
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(bar)),
               "r"(bytes)
               : "memory");
}
// bytes: a multiple of 16; dst and src 16-byte aligned.
__device__ __forceinline__ void bulk_load(float* dst, const float* src, int bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          (uint32_t)__cvta_generic_to_shared(dst)),
      "l"(src), "r"(bytes), "r"((uint32_t)__cvta_generic_to_shared(bar))
      : "memory");
}
// Polls the barrier's phase `parity` at most `tries` times; true once it has completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int tries) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
  for (int k = 0; k < tries; ++k) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Staging of n floats at src (4-byte aligned) into a 16-byte aligned shared-memory slot: float
// k lands at the returned pointer + k, which sits at the same offset modulo 16 bytes as src.
// stage_bytes: the bytes of the 16-byte aligned body, which the caller announces on the
// barrier before the copies are issued.  stage_warp_bulk (one warp): lane 0 issues the body as
// one bulk copy completing on `bar`; the at most 3 + 3 floats around it move by plain loads and
// stores (visible to the warp after the barrier wait and a __syncwarp).
__device__ __forceinline__ int stage_bytes(const float* src, int n) {
  const int mis = (int)((reinterpret_cast<uintptr_t>(src) >> 2) & 3);
  const int head = min((4 - mis) & 3, n);
  return ((n - head) >> 2) * 16;
}
__device__ __forceinline__ const float* stage_warp_bulk(float* slot, const float* src, int n, int lane,
                                                        uint64_t* bar) {
  const int mis = (int)((reinterpret_cast<uintptr_t>(src) >> 2) & 3);
  float* dst = slot + mis;
  const int head = min((4 - mis) & 3, n);
  const int nb = (n - head) >> 2;
  const int t0 = head + 4 * nb;
  if (lane == 0 && nb > 0) bulk_load(dst + head, src + head, nb * 16, bar);
  if (lane < head) dst[lane] = src[lane];
  if (lane >= 4 && lane - 4 < n - t0) dst[t0 + lane - 4] = src[t0 + lane - 4];
  return dst;
}

// Floats of a staging slot for n floats: n plus up to 3 of alignment shift, rounded to 16 bytes.
__host__ __device__ constexpr int stage_slot(int n) { return (n + 6) & ~3; }

// Shared memory of k_fused_kry: k_fused's (the residual block with 4 floats of slack) plus six
// warps' two staging slots each.
__host__ __device__ constexpr size_t kry_stage_offset(int P, int Q) {
  return ((sizeof(float) * (12 * Q * (P + 1) * (P + 1) * (P + 1) + 4 + 24 * Q * (P + 1) * (P + 1))) + 15) &
         ~size_t(15);
}
__host__ __device__ constexpr size_t fused_kry_smem(int P, int Q) {
  return kry_stage_offset(P, Q) + sizeof(float) * 12 * stage_slot(Q * (P + 1) * (P + 1) * (P + 1)) + 6 * 8;
}

// Single-pass FP32 Krylov operator on uniform meshes (no slab-start mode, no load): the inner
// operator of the mixed-precision solve.  MODE 0: A P^{-1} v on bricks (P^{-1} on load, the
// mass term is v itself); MODE 1: A z on curved elements, the mass term already in R (the
// tensor-core or CUDA-core curved mass, z = P^{-1} v from the 3x3 block pass); MODE 2: A z on
// general affine elements (constant 3x3 metric mass).  Same arithmetic as k_fused,
// specialised:
//  (a) forms y = sc B v and the mass term with no branches on the generic inputs;
//  (b) stages each neighbour's two tangential component blocks into shared memory by bulk
//      copies (one warp per (face, field), two batches of six, completion on the warp's
//      mbarrier with bounded polling) and forms its face traces from there, so the strided
//      trace reads hit shared memory, not L1/L2;
//  (c) the line passes (fused_lines, shared with k_fused; with KAP the dissipative term D_h);
//  (d) the residual block leaves shared memory by one bulk copy (completion by bulk-group
//      waits, no polling), placed in shared memory at its offset modulo 16 bytes in R so only
//      the at most 3 + 3 floats around the 16-byte aligned body need plain stores.
// Launched with 192 threads (six warps).
template <int P, int Q, bool KAP = false, int MODE = 0>
__global__ void __launch_bounds__(192) k_fused_kry(ApplyArgs<float> A) {
  using T = float;
  if (A.skip && *A.skip) return;
  constexpr int N = P + 1, N2 = N * N, N3 = N2 * N, SS = stage_slot(Q * N3);
  constexpr int EB = 6 * Q * N3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // [2][3][Q][N3] residual planes (start: the mass term), placed per element at the offset modulo
  // 16 bytes of its block in R (4 floats of slack), so the block leaves by one bulk copy
  T* Rb = reinterpret_cast<T*>(smem_raw);
  T* ys = Rb + EB + 4;  // [2][3][Q][N3] temporal contraction
  T* nt = ys + EB;      // [6 faces][2 fields][2 comps][Q][N2] neighbour traces
  T* stg = reinterpret_cast<T*>(smem_raw + kry_stage_offset(P, Q));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* slot = stg + warp * 2 * SS;  // this warp's two component slots
  // this warp's barrier for its staging copies (after the slots; 8-byte aligned)
  uint64_t* bar = reinterpret_cast<uint64_t*>(stg + 12 * SS) + warp;
  __shared__ int failed;  // a bounded wait ran out: every warp leaves at the next barrier
  if (threadIdx.x == 0) failed = 0;
  if (lane == 0) mbar_init(bar, 1);
  mbar_init_fence();
  __syncthreads();
  uint32_t parity = 0;
  const int um_cs = (int)A.um_cs;
  // issues the copies of task (face, fld) = (task >> 1, task & 1): the neighbour's two
  // tangential components; returns false (nothing issued) on a boundary face
  auto issue = [&](int64_t e, int task, const T** src) -> bool {
    const int face = task >> 1, fld = task & 1, a = face >> 1;
    const int64_t en = A.nbr[e * 6 + face];
    if (en < 0) return false;
    const T* ue = A.um + en * A.um_es;
    // this warp's reads of the slots (generic proxy) come before the next bulk writes into them
    fence_proxy_async_smem();
    __syncwarp();
    const T* cs[2];
    int bytes = 0;
#pragma unroll
    for (int bi = 0; bi < 2; ++bi) {
      const int b = (a == 0) ? 1 + bi : (a == 1 ? 2 * bi : bi);
      cs[bi] = ue + (fld * 3 + b) * um_cs;
      bytes += stage_bytes(cs[bi], Q * N3);
    }
    if (lane == 0) mbar_arrive_tx(bar, bytes);  // announced before the copies can complete
#pragma unroll
    for (int bi = 0; bi < 2; ++bi) src[bi] = stage_warp_bulk(slot + bi * SS, cs[bi], Q * N3, lane, bar);
    return true;
  };
  // waits for the batch's copies (bounded: 1 << 22 polls), then makes the plain-stored floats
  // of the other lanes visible; false if the wait ran out
  bool my_fail = false;  // this warp's copies of the batch that timed out may still be in flight
  auto arrived = [&]() -> bool {
    const bool ok = mbar_wait(bar, parity, 1 << 22);
    parity ^= 1;
    __syncwarp();
    if (!ok) {
      my_fail = true;
      if (lane == 0) {
        failed = 1;
        if (A.err) atomicExch(A.err, 1);
      }
    }
    return ok;
  };
  // the traces of task `task` from the staged blocks
  auto traces = [&](int64_t e, int task, const T* const* src) {
    const int face = task >> 1, fld = task & 1, a = face >> 1, side = face & 1;
    const int64_t en = A.nbr[e * 6 + face];
#pragma unroll
    for (int bi = 0; bi < 2; ++bi) {
      const int b = (a == 0) ? 1 + bi : (a == 1 ? 2 * bi : bi);
      const T sc = MODE == 0 ? A.pinv[en * 6 + fld * 3 + b] : T(1);
      T* nto = nt + ((task * 2 + bi) * Q) * N2;
      const T* ub = src[bi];
      with_axis(a, [&](auto ac) {
        constexpr int AX = decltype(ac)::value, ST = line_stride<N, AX>();
        // the neighbour meets face (a, side) with its face (a, 1 - side): L_j(0) = (-1)^j L_j(1)
        auto run = [&](auto sidec) {
          constexpr bool S1 = decltype(sidec)::value;
          for (int t = lane; t < N2; t += 32) {
            const T* ul = ub + line_base<N, AX>(t);
            T tu[Q];
#pragma unroll
            for (int m = 0; m < Q; ++m) {
              T acc = T(0);
#pragma unroll
              for (int j = 0; j < N; ++j) {
                const T w = (S1 && (j & 1)) ? -A.tb.lv[j] : A.tb.lv[j];
                acc = fma(w, ul[m * N3 + j * ST], acc);
              }
              tu[m] = acc;
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
              T acc = T(0);
#pragma unroll
              for (int m = 1; m <= Q; ++m)
                if (b_nz(i, m)) acc = fma(A.tb.B[i][m], tu[m - 1], acc);
              nto[i * N2 + t] = sc * acc;
            }
          }
        };
        if (side) run(std::true_type{});
        else run(std::false_type{});
      });
    }
  };
  for (int64_t e = blockIdx.x; e < A.n_elem; e += gridDim.x) {
    const int32_t* nb = A.nbr + e * 6;
    const T* ume = A.um + e * A.um_es;
    T* Rg = A.R + e * (int64_t)EB;
    const int shift = (int)((reinterpret_cast<uintptr_t>(Rg) >> 2) & 3);
    T* Rs = Rb + shift;
    // the first batch of neighbour copies in flight while the own block is contracted
    const T* src[2];
    bool have = issue(e, warp, src);
    // the previous element's residual has left shared memory (its bulk copy has read it)
    if (threadIdx.x == 0) bulk_wait_read();
    __syncthreads();
    // (a) y = sc B v and the mass term: on bricks with P^{-1} on load (MODE 0) v itself (the
    //     mass block times P^{-1} is the identity), on curved elements (MODE 1) the term already
    //     in R, on general affine elements (MODE 2) the constant 3x3 metric mass of v
    for (int it = threadIdx.x; it < 6 * N3; it += 192) {
      const int fc = it / N3, s = it - fc * N3;
      const T* up = ume + fc * um_cs + s;
      T v[Q];
#pragma unroll
      for (int m = 0; m < Q; ++m) v[m] = up[m * N3];
      const T sc = MODE == 0 ? A.pinv[e * 6 + fc] : T(1);
      T* yo = ys + fc * Q * N3 + s;
      T* ro = Rs + fc * Q * N3 + s;
      T mr[3] = {T(0), T(0), T(0)};
      const T* uf = ume + s;
      if constexpr (MODE == 2) {
        const int f = fc >= 3 ? 1 : 0, c = fc - 3 * f;
        sym3_row(A.mass3 + (e * 2 + f) * 6, c, mr);
        uf += (f * 3) * um_cs;
      }
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        T acc = T(0);
#pragma unroll
        for (int m = 1; m <= Q; ++m)
          if (b_nz(i, m)) acc = fma(A.tb.B[i][m], v[m - 1], acc);
        yo[i * N3] = sc * acc;
        if constexpr (MODE == 0) ro[i * N3] = v[i];
        if constexpr (MODE == 1) ro[i * N3] = Rg[(fc * Q + i) * N3 + s];
        if constexpr (MODE == 2)
          ro[i * N3] = fma(mr[2], uf[2 * um_cs + i * N3], fma(mr[1], uf[um_cs + i * N3], mr[0] * uf[i * N3]));
      }
    }
    // (b) neighbour traces: two batches of six (face, field) tasks, one per warp
    bool ok = true;
    if (have) {
      ok = arrived();
      if (ok) traces(e, warp, src);
      __syncwarp();  // the slots are refilled next
    }
    if (ok) {
      have = issue(e, warp + 6, src);
      if (have && arrived()) traces(e, warp + 6, src);
    }
    __syncthreads();
    if (failed) break;  // uniform: read after the barrier
    // (c) residual planes: one warp per (field, component), all Q temporal test modes
    {
      const int f = warp >= 3 ? 1 : 0, c = warp - 3 * f;
      fused_lines<T, N, Q, KAP>(A, e, f, c, ys, nt, nb, Rs + warp * Q * N3, lane);
    }
    // (d) the residual block to R: the 16-byte aligned body by one bulk copy, the at most 3 + 3
    //     floats around it by plain stores
    fence_proxy_async_smem();
    __syncthreads();
    const int head = min((4 - shift) & 3, EB), nb16 = (EB - head) >> 2, t0 = head + 4 * nb16;
    if (threadIdx.x == 0) {
      if (nb16 > 0) bulk_store(Rg + head, Rs + head, nb16 * 16);
      bulk_commit();
    } else if (threadIdx.x <= head) {
      Rg[threadIdx.x - 1] = Rs[threadIdx.x - 1];
    } else if (threadIdx.x > 4 && threadIdx.x - 5 < EB - t0) {
      Rg[t0 + threadIdx.x - 5] = Rs[t0 + threadIdx.x - 5];
    }
  }
  if (threadIdx.x == 0) bulk_wait_all();
  if (my_fail && lane == 0) mbar_wait(bar, parity ^ 1, 1 << 22);  // let a late copy land before exit
}


// Optional CUDA events recorded before k_prep, between the kernels and after
// k_apply (all null: no timing).
struct LaunchEvents {
  cudaEvent_t start = nullptr, mid = nullptr, stop = nullptr;
};

// Shared memory of the single-pass FP32 kernel (y and residual planes of both fields, the
// neighbour traces), and whether it is used: at most 64 KB, so that at least three CTAs share
// an SM; larger (p, q) run the two-kernel structure in FP32 (trace pass, then apply).
__host__ __device__ constexpr size_t fused_smem(int P, int Q) {
  return sizeof(float) * (2 * 6 * Q * (P + 1) * (P + 1) * (P + 1) + 24 * Q * (P + 1) * (P + 1));
}
__host__ __device__ constexpr bool fused_fits(int P, int Q) { return fused_smem(P, Q) <= 64 * 1024; }

template <typename T, int P, int Q>
int launch_residual_pq(const ApplyArgs<T>& args, cudaStream_t s, int grid, const LaunchEvents& ev, int phase = 0,
                       int block = 256) {
  constexpr int N = P + 1, N3 = N * N * N;
  constexpr int N2 = N * N;
  const size_t sm_prep = sizeof(T) * 6 * Q * N3;
  const size_t sm_apply = ApplyShape<T, P, Q>::smem;
  const size_t sm_fused = 2 * sm_prep + sizeof(T) * 24 * Q * N2;
  // kernel attributes are per device: set them once on every device this instantiation launches on
  static std::atomic<uint64_t> configured_devices{0};
  // the dynamic shared-memory limit is set for every size: static shared memory (k_prep's
  // folded coefficients, k_apply's face cache) counts against the same 48 KB default
  once_per_device(configured_devices, [&] {
    cudaFuncSetAttribute(k_prep<T, P, Q, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_prep);
    cudaFuncSetAttribute(k_prep<T, P, Q, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_prep);
    cudaFuncSetAttribute(k_prep<T, P, Q, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_prep);
    cudaFuncSetAttribute(k_apply<T, P, Q, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_apply);
    cudaFuncSetAttribute(k_apply<T, P, Q, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_apply);
    cudaFuncSetAttribute(k_apply<T, P, Q, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_apply);
    if constexpr (sizeof(T) == 4) {
      cudaFuncSetAttribute(k_fused<T, P, Q, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fused);
      cudaFuncSetAttribute(k_fused<T, P, Q, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fused);
      cudaFuncSetAttribute(k_fused<T, P, Q, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fused);
      cudaFuncSetAttribute(k_fused<T, P, Q, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fused);
      cudaFuncSetAttribute(k_fused_kry<P, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fused_kry_smem(P, Q));
      cudaFuncSetAttribute(k_fused_kry<P, Q, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fused_kry_smem(P, Q));
      cudaFuncSetAttribute(k_fused_kry<P, Q, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fused_kry_smem(P, Q));
      cudaFuncSetAttribute(k_fused_kry<P, Q, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fused_kry_smem(P, Q));
    }
    cudaGetLastError();
  });
  const bool hp = args.elist != nullptr;
  if constexpr (sizeof(T) == 4 && fused_fits(P, Q)) {
    if (!hp) {
      // single pass: ev.start/ev.stop bracket k_fused (reported in the apply slot)
      if (ev.start) cudaEventRecord(ev.start, s);
      if (ev.mid) cudaEventRecord(ev.mid, s);
      // six warps: the 6 Q residual planes and the 24 neighbour-trace tasks divide evenly
      constexpr int kFusedThreads = 192;
      (void)block;
      static std::atomic<int> cap_t[64], cap_f[64], cap_k[64], cap_dt[64], cap_df[64], cap_dk[64];
      // the Krylov operator of the mixed-precision solve (no slab-start mode, no load): bricks with
      // P^{-1} on load (mode 0), curved with the mass term in R (mode 1), general affine (mode 2)
      const int kmode = (args.pinv && args.mass && !args.mass3) ? 0 : (!args.pinv && !args.mass && !args.mass3 ? 1 : (!args.pinv && args.mass3 ? 2 : -1));
      const bool krylov = fused_kry_smem(P, Q) <= 74 * 1024 && !args.u0 && !args.b && kmode >= 0;
      if (args.kap) {
        // the dissipative term D_h (Sec. 4.2) in the same single pass
        if (krylov && kmode == 0)
          k_fused_kry<P, Q, true><<<wave_grid(k_fused_kry<P, Q, true>, kFusedThreads, fused_kry_smem(P, Q), grid,
                                              cap_dk),
                                    kFusedThreads, fused_kry_smem(P, Q), s>>>(args);
        else if (args.pinv)
          k_fused<T, P, Q, true, true><<<wave_grid(k_fused<T, P, Q, true, true>, kFusedThreads, sm_fused, grid, cap_dt),
                                         kFusedThreads, sm_fused, s>>>(args);
        else
          k_fused<T, P, Q, false, true>
              <<<wave_grid(k_fused<T, P, Q, false, true>, kFusedThreads, sm_fused, grid, cap_df), kFusedThreads,
                 sm_fused, s>>>(args);
      } else if (krylov) {
        const size_t smk = fused_kry_smem(P, Q);
        static std::atomic<int> cap_k1[64], cap_k2[64];
        if (kmode == 0)
          k_fused_kry<P, Q><<<wave_grid(k_fused_kry<P, Q>, kFusedThreads, smk, grid, cap_k), kFusedThreads, smk, s>>>(
              args);
        else if (kmode == 1)
          k_fused_kry<P, Q, false, 1><<<wave_grid(k_fused_kry<P, Q, false, 1>, kFusedThreads, smk, grid, cap_k1),
                                        kFusedThreads, smk, s>>>(args);
        else
          k_fused_kry<P, Q, false, 2><<<wave_grid(k_fused_kry<P, Q, false, 2>, kFusedThreads, smk, grid, cap_k2),
                                        kFusedThreads, smk, s>>>(args);
      } else if (args.pinv)
        k_fused<T, P, Q, true><<<wave_grid(k_fused<T, P, Q, true>, kFusedThreads, sm_fused, grid, cap_t),
                                 kFusedThreads, sm_fused, s>>>(args);
      else
        k_fused<T, P, Q, false><<<wave_grid(k_fused<T, P, Q, false>, kFusedThreads, sm_fused, grid, cap_f),
                                  kFusedThreads, sm_fused, s>>>(args);
      if (ev.stop) cudaEventRecord(ev.stop, s);
      return (int)cudaGetLastError();
    }
  }
  // one-wave grids, cached per (kernel, block size: 64, 128, 256 or 512) and device
  static std::atomic<int> cap_p[3][4][64], cap_a[3][4][64];
  block = std::min(block, residual_max_threads(P, Q));
  const int bs = block <= 64 ? 0 : (block <= 128 ? 1 : (block <= 256 ? 2 : 3));
  if (phase != 2) {
    if (ev.start) cudaEventRecord(ev.start, s);
    if (hp && args.nkl) {
      auto k = k_prep<T, P, Q, true, true>;
      k<<<wave_grid(k, block, sm_prep, grid, cap_p[0][bs]), block, sm_prep, s>>>(args);
    } else if (hp) {
      auto k = k_prep<T, P, Q, true>;
      k<<<wave_grid(k, block, sm_prep, grid, cap_p[1][bs]), block, sm_prep, s>>>(args);
    } else {
      auto k = k_prep<T, P, Q, false>;
      k<<<wave_grid(k, block, sm_prep, grid, cap_p[2][bs]), block, sm_prep, s>>>(args);
    }
    if (ev.mid) cudaEventRecord(ev.mid, s);
  }
  if (phase != 1) {
    if (hp && args.nkl) {
      auto k = k_apply<T, P, Q, true, true>;
      k<<<wave_grid(k, block, sm_apply, grid, cap_a[0][bs]), block, sm_apply, s>>>(args);
    } else if (hp) {
      auto k = k_apply<T, P, Q, true>;
      k<<<wave_grid(k, block, sm_apply, grid, cap_a[1][bs]), block, sm_apply, s>>>(args);
    } else {
      auto k = k_apply<T, P, Q, false>;
      k<<<wave_grid(k, block, sm_apply, grid, cap_a[2][bs]), block, sm_apply, s>>>(args);
    }
    if (ev.stop) cudaEventRecord(ev.stop, s);
  }
  return (int)cudaGetLastError();
}

}  // namespace stm
