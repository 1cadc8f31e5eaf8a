// Residual apply that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA graph
// that is being captured, a host that has handed all device memory to its
// own pool allocator, or an embedding that forbids allocation after start-up
// (a real-time or safety-certified loop).  For them this unit keeps the
// residual kernels' scratch (the temporal contraction y, the face traces and
// the element mass factors) in one file-scope device array of fixed size,
// STM_NOALLOC_SCRATCH_BYTES, that every GPU which loads the library holds
// until the process exits.  The caller passes every input and output as
// device pointers.
//
// The device address of the array is looked up once per device with
// cudaGetSymbolAddress (host code cannot use the array's name as a device
// pointer) on the first call made with that device current.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "residual.cuh"
#include "stm.h"

namespace stm {
template <typename T>
int launch_residual(int P, int Q, const ApplyArgs<T>& a, cudaStream_t s, int grid, const LaunchEvents& ev);
template <typename T>
Tables<T> make_tables(int P, int Q, double dt);
}  // namespace stm

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[STM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return STM_EDEVICE;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      fprintf(stderr, "stm_residual_apply_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
      return STM_EDEVICE;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return STM_OK;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

__global__ void k_noalloc_mass(const double* __restrict__ h, const double* __restrict__ eps,
                               const double* __restrict__ mu, double* __restrict__ mass, int64_t ne) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    const double hx = h[3 * e], hy = h[3 * e + 1], hz = h[3 * e + 2];
    const double G[3] = {hy * hz / hx, hx * hz / hy, hx * hy / hz};
    for (int c = 0; c < 3; ++c) {
      mass[6 * e + c] = eps[e] * G[c];
      mass[6 * e + 3 + c] = mu[e] * G[c];
    }
  }
}

}  // namespace

extern "C" int32_t stm_residual_apply_noalloc(int64_t n_elem, int32_t p, int32_t q, double dt, const int32_t* nbr,
                                              const double* h, const double* eps, const double* mu, const double* U,
                                              double* R, int64_t stream) {
  if (n_elem <= 0 || p < 0 || p > 7 || q < 1 || q > stm::kMaxQ || !(dt > 0) || !nbr || !h || !eps || !mu || !U ||
      !R)
    return STM_EINVAL;
  const int64_t n = p + 1, n2 = n * n, n3 = n2 * n;
  // bound the element count before forming any product: past this count the scratch
  // cannot fit, and below it none of the sums below can overflow
  const size_t per_elem = sizeof(double) * (6 + 6 * (size_t)q * n3 + 24 * (size_t)q * n2);
  const size_t cap = (size_t)STM_NOALLOC_SCRATCH_BYTES;
  size_t need = 0;
  size_t need_mass = 0, need_y = 0;
  if ((uint64_t)n_elem <= cap / per_elem) {
    need_mass = round256(sizeof(double) * 6 * (size_t)n_elem);
    need_y = round256(sizeof(double) * 6 * (size_t)q * n3 * (size_t)n_elem);
    const size_t need_tr = round256(sizeof(double) * 24 * (size_t)q * n2 * (size_t)n_elem);
    need = need_mass + need_y + need_tr;
  }
  if (need == 0 || need > cap) {
    fprintf(stderr,
            "stm_residual_apply_noalloc: %lld elements of degree (p=%d, q=%d) need %zu bytes of scratch per element, "
            "more in total than the fixed %zu bytes (STM_NOALLOC_SCRATCH_BYTES)\n",
            (long long)n_elem, p, q, per_elem, cap);
    return STM_EINVAL;
  }
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  unsigned char* b = static_cast<unsigned char*>(base);
  double* mass = reinterpret_cast<double*>(b);
  double* y = reinterpret_cast<double*>(b + need_mass);
  double* tr = reinterpret_cast<double*>(b + need_mass + need_y);
  cudaStream_t s = (cudaStream_t)(intptr_t)stream;

  const int grid_m = (int)((n_elem + 255) / 256 < 4096 ? (n_elem + 255) / 256 : 4096);
  k_noalloc_mass<<<grid_m, 256, 0, s>>>(h, eps, mu, mass, n_elem);

  stm::ApplyArgs<double> a{};
  const int64_t tes = 6 * (q + 1) * n3, tcs = (q + 1) * n3;
  a.um = U + n3;
  a.um_es = tes;
  a.um_cs = tcs;
  a.u0 = U;
  a.u0_es = tes;
  a.u0_cs = tcs;
  a.b = nullptr;
  a.y = y;
  a.tr = tr;
  a.R = R;
  a.nbr = nbr;
  a.mass = mass;
  a.n_elem = n_elem;
  a.tb = stm::make_tables<double>(p, q, dt);
  const int grid = (int)(n_elem < (1 << 30) ? n_elem : (1 << 30));
  const int e = stm::launch_residual<double>(p, q, a, s, grid, stm::LaunchEvents{});
  if (e) {
    fprintf(stderr, "stm_residual_apply_noalloc: launch failed: %s\n", cudaGetErrorString((cudaError_t)e));
    return STM_EDEVICE;
  }
  return STM_OK;
}
