// Curved-element mass term in FP32 on the 5th-generation tensor cores (tcgen05,
// 3xTF32 split products, accumulators in tensor memory).
//
// The mass residual of a curved element (Sec. 5.2, "mass residual") is, per
// element, field f and temporal test mode i, the sum-factorised chain
//   v_c  = u_{i+1,c} - delta_{i0} u_{0,c}                         (c = x, y, z)
//   T_c  = (V (x) V (x) V) v_c         at the (p+2)^3 Gauss points
//   W_c  = mat_f sum_d w_g G_cd(x_g) T_d                          (pointwise)
//   R_c  = (V^T (x) V^T (x) V^T) W_c
// with V[g][j] = L_j(x_g).  Each of the six 1-D contractions is a GEMM whose
// rows are the tensor's lines along the contracted axis (K = p+1 or p+2 <= 9,
// padded to 8 or 16) and whose columns are the p+2 or p+1 outputs (padded to
// 16): D[rows x 16] = A[rows x K] B^T with B = V (forward) or V^T (backward).
// The rows of one (element, field, mode) job (at most 3 (p+2)^2 = 243) form
// one or two M = 128 tiles.
//
// One CTA of 128 threads (4 warps, one per TMEM lane quarter) runs one job at
// a time: the threads write the stage's A operand into shared memory (K-major
// core-matrix layout, no swizzle) as TF32 high and low parts, one thread issues
// 3 MMAs per tile and K block (hi.hi + hi.lo + lo.hi, FP32 accumulation in
// TMEM), commits to an mbarrier, and every thread reads its D row back with
// tcgen05.ld and scatters it, transposed, into the next stage's A operand.
// Every wait is bounded: a timed-out wait sets *err and the CTA stops after
// releasing its tensor memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "curved.cuh"

namespace stm {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcCols = 32;  // TMEM columns per CTA: up to two 128 x 16 accumulator tiles

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle; lbo = bytes between core matrices
// adjacent along K, sbo = bytes between 8-row groups (descriptor version 1).
__device__ __forceinline__ uint64_t mat_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32 with FP32 accumulation, both operands K-major.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(16 >> 3) << 17) |
                                ((uint32_t)(128 >> 4) << 24);

// Byte offset of element (r, k) in a K-major operand of ROWS rows: 8-row x 16-byte core
// matrices with the rows of a K group of 4 values contiguous (16 bytes apart, 8-row groups
// 128 bytes apart) and the K groups ROWS * 16 bytes apart, so consecutive rows are 16 bytes
// apart whatever the K width.
template <int ROWS>
__device__ __forceinline__ uint32_t core_ofs(int r, int k) {
  return (uint32_t)((k >> 2) * (ROWS * 16) + r * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t y;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
  return __uint_as_float(y);
}

// x = hi + lo with both parts TF32 (3xTF32: hi.hi + hi.lo + lo.hi keeps FP32 accuracy)
__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, uint32_t ofs, float x) {
  const float h = tf32_rna(x);
  *reinterpret_cast<float*>(hi + ofs) = h;
  *reinterpret_cast<float*>(lo + ofs) = tf32_rna(x - h);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdescTf32), "r"(acc));
}

__device__ __forceinline__ void sync_for_mma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Bounded wait for the mbarrier phase; returns false when the bound ran out.
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t phase) {
  uint32_t ok = 0;
  for (int it = 0; it < (1 << 22) && !ok; ++it)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mbar), "r"(phase)
        : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

struct TcTabs {
  float L[kMaxN][kMaxN + 1];  // L_j(x_g)
};

template <int P, int Q>
struct TcShape {
  static constexpr int N = P + 1, NQ = P + 2, N2 = N * N, N3 = N2 * N, NQ2 = NQ * NQ, NQ3 = NQ2 * NQ;
  static constexpr int KWB = NQ <= 8 ? 8 : 16;   // K width of the backward contractions
  static constexpr int ROWS = 3 * NQ2;           // largest stage (3 components)
  static constexpr int NT = (ROWS + 127) / 128;  // M = 128 tiles
  static constexpr int AROWS = NT * 128;          // rows of the A operand buffer
  static constexpr int ABYTES = NT * 128 * 16 * 4;
  // shared memory: A hi, A lo, B forward hi/lo (16 x 8), B backward hi/lo (16 x 16), T3 [3][NQ3]
  static constexpr int OFS_ALO = ABYTES, OFS_BF = 2 * ABYTES, OFS_BB = OFS_BF + 2 * 512, OFS_T3 = OFS_BB + 2 * 1024;
  static constexpr int SMEM = OFS_T3 + 3 * NQ3 * 4;
};

template <int P, int Q>
__global__ void __launch_bounds__(kTcThreads) k_mass_tc(const float* __restrict__ um, int64_t um_es, int64_t um_cs,
                                                        const float* __restrict__ u0, int64_t u0_es, int64_t u0_cs,
                                                        const float* __restrict__ Gw, const float* __restrict__ eps,
                                                        const float* __restrict__ mu, TcTabs tb, int64_t ne,
                                                        float* __restrict__ R, const int32_t* skip, int* err) {
  using S = TcShape<P, Q>;
  constexpr int N = S::N, NQ = S::NQ, N2 = S::N2, N3 = S::N3, NQ2 = S::NQ2, NQ3 = S::NQ3, NT = S::NT;
  if (skip && *skip) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* Ahi = sm;
  unsigned char* Alo = sm + S::OFS_ALO;
  unsigned char* Bf = sm + S::OFS_BF;   // hi, then lo (512 bytes each)
  unsigned char* Bb = sm + S::OFS_BB;   // hi, then lo (1024 bytes each)
  float* T3 = reinterpret_cast<float*>(sm + S::OFS_T3);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5;
  // operands: A zero (padding must be finite), B tables split into TF32 parts
  for (int k = tid; k < S::OFS_BF / 4; k += kTcThreads) reinterpret_cast<float*>(sm)[k] = 0.f;
  for (int k = tid; k < 16 * 8; k += kTcThreads) {
    const int n = k / 8, kk = k % 8;  // forward: B[n = g][k = j] = L_j(x_g)
    const float v = (n < NQ && kk < N) ? tb.L[kk][n] : 0.f;
    put_split(Bf, Bf + 512, core_ofs<16>(n, kk), v);
  }
  for (int k = tid; k < 16 * S::KWB; k += kTcThreads) {
    const int n = k / S::KWB, kk = k % S::KWB;  // backward: B[n = j][k = g] = L_j(x_g)
    const float v = (n < N && kk < NQ) ? tb.L[n][kk] : 0.f;
    put_split(Bb, Bb + 1024, core_ofs<16>(n, kk), v);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    failed = 0;
  }
  sync_for_mma();
  const uint32_t tmem = tmem_base, mb = smem_u32(&mbar);
  uint32_t phase = 0;
  const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo), bf = smem_u32(Bf), bb = smem_u32(Bb);
  float d[NT][16];
  // one stage: MMAs over all tiles from the A operand (K width KW) and B, results to d
  auto stage = [&](int KW, uint32_t bhi, uint32_t blo) -> bool {
    sync_for_mma();
    if (tid == 0) {
      // K groups of 4 values: A ones S::AROWS * 16 bytes apart, B ones 16 * 16; 8-row groups 128
      constexpr uint32_t lboa = S::AROWS * 16, lbob = 16 * 16;
#pragma unroll
      for (int t = 0; t < NT; ++t)
        for (int kb = 0; kb < KW / 8; ++kb) {
          const uint32_t ao = (uint32_t)t * 128 * 16 + kb * 2 * lboa;
          const uint64_t dah = mat_desc(a_hi + ao, lboa, 128), dal = mat_desc(a_lo + ao, lboa, 128);
          const uint64_t dbh = mat_desc(bhi + kb * 2 * lbob, lbob, 128), dbl = mat_desc(blo + kb * 2 * lbob, lbob, 128);
          const uint32_t dt = tmem + 16 * t;
          mma_tf32(dt, dah, dbh, kb > 0 ? 1u : 0u);
          mma_tf32(dt, dah, dbl, 1u);
          mma_tf32(dt, dal, dbh, 1u);
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
    }
    const bool ok = wait_phase(mb, phase);
    phase ^= 1u;
    if (!ok) failed = 1;
    __syncthreads();  // every thread takes the same decision
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (failed) return false;
#pragma unroll
    for (int t = 0; t < NT; ++t) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 16 * t, d[t]);
    return true;
  };
  bool alive = true;
  for (int64_t e = blockIdx.x; e < ne && alive; e += gridDim.x) {
#pragma unroll 1
    for (int job = 0; job < 2 * Q && alive; ++job) {
      const int f = job / Q, i = job - f * Q;
      const float mat = f == 0 ? eps[e] : mu[e];
      // S1: rows (c, l, k), K = j: v_c = u_{i+1,c} - delta_{i0} u_{0,c}
      for (int x = tid; x < 3 * N3; x += kTcThreads) {
        const int c = x / N3, s = x - c * N3;
        float v = um[e * um_es + (f * 3 + c) * um_cs + i * N3 + s];
        if (i == 0 && u0) v -= u0[e * u0_es + (f * 3 + c) * u0_cs + s];
        put_split(Ahi, Alo, core_ofs<S::AROWS>(x / N, s % N), v);
      }
      if (!(alive = stage(8, bf, bf + 512))) break;
      // S1 -> S2: row (c, l, k), column gx  ->  row (c, l, gx), column k
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int r = 128 * t + tid;
        if (r < 3 * N2) {
          const int cl = r / N, k = r - cl * N;
#pragma unroll
          for (int g = 0; g < NQ; ++g) put_split(Ahi, Alo, core_ofs<S::AROWS>(cl * NQ + g, k), d[t][g]);
        }
      }
      if (!(alive = stage(8, bf, bf + 512))) break;
      // S2 -> S3: row (c, l, gx), column gy  ->  row (c, gy, gx), column l
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int r = 128 * t + tid;
        if (r < 3 * N * NQ) {
          const int c = r / (N * NQ), rem = r - c * N * NQ, l = rem / NQ, gx = rem - l * NQ;
#pragma unroll
          for (int g = 0; g < NQ; ++g) put_split(Ahi, Alo, core_ofs<S::AROWS>((c * NQ + g) * NQ + gx, l), d[t][g]);
        }
      }
      if (!(alive = stage(8, bf, bf + 512))) break;
      // S3: row (c, gy, gx), column gz = value T_c at g = (gz NQ + gy) NQ + gx
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int r = 128 * t + tid;
        if (r < 3 * NQ2) {
          const int c = r / NQ2, g2 = r - c * NQ2;
#pragma unroll
          for (int g = 0; g < NQ; ++g) T3[c * NQ3 + g * NQ2 + g2] = d[t][g];
        }
      }
      __syncthreads();
      // pointwise W_c = mat sum_d w G_cd T_d  ->  B1 operand: row (c, gy, gx), column gz
      const float* ge = Gw + e * 6 * NQ3;
      for (int g = tid; g < NQ3; g += kTcThreads) {
        const float vx = T3[g], vy = T3[NQ3 + g], vz = T3[2 * NQ3 + g];
        const float gxx = ge[g], gyy = ge[NQ3 + g], gzz = ge[2 * NQ3 + g];
        const float gxy = ge[3 * NQ3 + g], gxz = ge[4 * NQ3 + g], gyz = ge[5 * NQ3 + g];
        const int gz = g / NQ2, g2 = g - gz * NQ2;
        put_split(Ahi, Alo, core_ofs<S::AROWS>(g2, gz), mat * fmaf(gxx, vx, fmaf(gxy, vy, gxz * vz)));
        put_split(Ahi, Alo, core_ofs<S::AROWS>(NQ2 + g2, gz), mat * fmaf(gxy, vx, fmaf(gyy, vy, gyz * vz)));
        put_split(Ahi, Alo, core_ofs<S::AROWS>(2 * NQ2 + g2, gz), mat * fmaf(gxz, vx, fmaf(gyz, vy, gzz * vz)));
      }
      if (!(alive = stage(S::KWB, bb, bb + 1024))) break;
      // B1 -> B2: row (c, gy, gx), column l  ->  row (c, l, gx), column gy
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int r = 128 * t + tid;
        if (r < 3 * NQ2) {
          const int c = r / NQ2, rem = r - c * NQ2, gy = rem / NQ, gx = rem - gy * NQ;
#pragma unroll
          for (int l = 0; l < N; ++l) put_split(Ahi, Alo, core_ofs<S::AROWS>((c * N + l) * NQ + gx, gy), d[t][l]);
        }
      }
      if (!(alive = stage(S::KWB, bb, bb + 1024))) break;
      // B2 -> B3: row (c, l, gx), column k  ->  row (c, l, k), column gx
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int r = 128 * t + tid;
        if (r < 3 * N * NQ) {
          const int cl = r / NQ, gx = r - cl * NQ;
#pragma unroll
          for (int k = 0; k < N; ++k) put_split(Ahi, Alo, core_ofs<S::AROWS>(cl * N + k, gx), d[t][k]);
        }
      }
      if (!(alive = stage(S::KWB, bb, bb + 1024))) break;
      // B3: row (c, l, k), column j  ->  R[e][f][c][i][(l N + k) N + j]
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int r = 128 * t + tid;
        if (r < 3 * N2) {
          const int c = r / N2, lk = r - c * N2;
          float* Rr = R + ((e * 6 + f * 3 + c) * (int64_t)Q + i) * N3 + lk * N;
#pragma unroll
          for (int j = 0; j < N; ++j) Rr[j] = d[t][j];
        }
      }
    }
  }
  if (!alive && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

template <int P, int Q>
int mass_tc_pq(const float* um, int64_t um_es, int64_t um_cs, const float* u0, int64_t u0_es, int64_t u0_cs,
               const float* Gw, const float* eps, const float* mu, const CurvedTables& ct, int64_t ne, float* R,
               cudaStream_t s, const int32_t* skip, int* err) {
  using S = TcShape<P, Q>;
  static std::atomic<uint64_t> configured_devices{0};
  once_per_device(configured_devices, [&] {
    cudaFuncSetAttribute(k_mass_tc<P, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
  });
  TcTabs tb;
  for (int j = 0; j < kMaxN; ++j)
    for (int g = 0; g <= kMaxN; ++g) tb.L[j][g] = (float)ct.Lq[j][g];
  // one wave of co-resident CTAs: shared memory and the 512 TMEM columns (kTcCols per CTA)
  // bound the CTAs per SM (the occupancy calculator does not model tensor memory)
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = std::max(1, std::min(512 / kTcCols, (227 * 1024) / (S::SMEM + 2048)));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ne, (int64_t)per_sm * sms));
  k_mass_tc<P, Q><<<grid, kTcThreads, S::SMEM, s>>>(um, um_es, um_cs, u0, u0_es, u0_cs, Gw, eps, mu, tb, ne, R, skip,
                                                    err);
  return (int)cudaGetLastError();
}

}  // namespace

int launch_mass_curved_tc(int P, int Q, const float* um, int64_t um_es, int64_t um_cs, const float* u0, int64_t u0_es,
                          int64_t u0_cs, const float* Gw, const float* eps, const float* mu, const CurvedTables& ct,
                          int64_t ne, float* R, cudaStream_t s, const int32_t* skip, int* err) {
#define STM_TQ(p, q)                                                                                         \
  if (P == p && Q == q)                                                                                      \
    return mass_tc_pq<p, q>(um, um_es, um_cs, u0, u0_es, u0_cs, Gw, eps, mu, ct, ne, R, s, skip, err);
#define STM_TP(p) STM_TQ(p, 1) STM_TQ(p, 2) STM_TQ(p, 3) STM_TQ(p, 4) STM_TQ(p, 5) STM_TQ(p, 6)
  STM_TP(3) STM_TP(4) STM_TP(5) STM_TP(6) STM_TP(7)
#undef STM_TP
#undef STM_TQ
  return (int)cudaErrorInvalidValue;
}

}  // namespace stm
