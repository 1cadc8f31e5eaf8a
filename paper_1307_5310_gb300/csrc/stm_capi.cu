// C ABI of the slab library (declared in include/stm.h).
//
// A context owns the device copy of the mesh data (face neighbours, the
// element mass factors eps G_c / mu G_c), the state (spatial coefficients of
// E and H at the current time), the scratch of the residual kernels and the
// GMRES workspace.  All device work is ordered on one stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "curved.cuh"
#include "hp.cuh"
#include "krylov.cuh"
#include "load.cuh"
#include "residual.cuh"
#include "stm.h"

namespace stm {
#define STM_DECL_P(k)                                                                                  \
  template <typename T>                                                                                \
  int launch_residual_p##k(int Q, const ApplyArgs<T>& a, cudaStream_t s, int grid, const LaunchEvents& ev, \
                           int phase, int block);
STM_DECL_P(0)
STM_DECL_P(1)
STM_DECL_P(2)
STM_DECL_P(3)
STM_DECL_P(4)
STM_DECL_P(5)
STM_DECL_P(6)
STM_DECL_P(7)
#undef STM_DECL_P

// phase: 0 = both kernels, 1 = k_prep only, 2 = k_apply only (uneven-degree meshes run
// every class's k_prep before any k_apply, which reads neighbour traces of other classes)
template <typename T>
int launch_residual_ph(int P, int Q, const ApplyArgs<T>& a, cudaStream_t s, int grid, const LaunchEvents& ev,
                       int phase, int block) {
  switch (P) {
    case 0: return launch_residual_p0<T>(Q, a, s, grid, ev, phase, block);
    case 1: return launch_residual_p1<T>(Q, a, s, grid, ev, phase, block);
    case 2: return launch_residual_p2<T>(Q, a, s, grid, ev, phase, block);
    case 3: return launch_residual_p3<T>(Q, a, s, grid, ev, phase, block);
    case 4: return launch_residual_p4<T>(Q, a, s, grid, ev, phase, block);
    case 5: return launch_residual_p5<T>(Q, a, s, grid, ev, phase, block);
    case 6: return launch_residual_p6<T>(Q, a, s, grid, ev, phase, block);
    case 7: return launch_residual_p7<T>(Q, a, s, grid, ev, phase, block);
    default: return -1;
  }
}

template <typename T>
int launch_residual(int P, int Q, const ApplyArgs<T>& a, cudaStream_t s, int grid, const LaunchEvents& ev) {
  return launch_residual_ph<T>(P, Q, a, s, grid, ev, 0, 256);
}

// 1-D tables from their closed forms (Sec. 5.1-5.2): B_im = int L_i l_m with
// l_m = (P_m - P_{m-2}) / (2 sqrt(2m-1)) in terms of the classical Legendre
// polynomials P on [-1,1] mapped to [0,1]; D_ab = int L_a L_b' =
// 2 sqrt(2a+1) sqrt(2b+1) for a < b with b - a odd; L_a(1) = sqrt(2a+1).
template <typename T>
Tables<T> make_tables(int P, int Q, double dt) {
  Tables<T> t;
  std::memset(&t, 0, sizeof(t));
  const int N = P + 1;
  double B[kMaxQ][kMaxQ + 1] = {};
  B[0][0] = 0.5;
  B[0][1] = 0.5;
  if (Q >= 2) {
    B[1][0] = -0.5 / std::sqrt(3.0);
    B[1][1] = 0.5 / std::sqrt(3.0);
  }
  for (int m = 2; m <= Q; ++m) {
    if (m <= Q - 1) B[m][m] = 0.5 / (std::sqrt(2.0 * m - 1) * std::sqrt(2.0 * m + 1));
    B[m - 2][m] = -0.5 / (std::sqrt(2.0 * m - 1) * std::sqrt(2.0 * m - 3));
  }
  for (int i = 0; i < kMaxQ; ++i)
    for (int m = 0; m <= kMaxQ; ++m) t.B[i][m] = (T)B[i][m];
  for (int a = 0; a < N; ++a) {
    t.lv[a] = (T)std::sqrt(2.0 * a + 1);
    t.kq[a] = (T)(-0.25 / std::sqrt(2.0 * a + 1));
    t.hf[a] = (T)(0.5 * dt * std::sqrt(2.0 * a + 1));
    for (int b = 0; b < N; ++b)
      if (d_nz(a, b)) t.Dt[a][b] = (T)(dt * 2.0 * std::sqrt(2.0 * a + 1) * std::sqrt(2.0 * b + 1));
  }
  return t;
}

template Tables<double> make_tables<double>(int, int, double);
template int launch_residual<double>(int, int, const ApplyArgs<double>&, cudaStream_t, int, const LaunchEvents&);

// Gauss-Legendre rule on [0,1] by Newton's method on the Legendre polynomial.
void gauss01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1) * z * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < n; ++k) {
      const double p2 = ((2.0 * k + 1) * z * p1 - k * p0) / (k + 1);
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Orthonormal Legendre L_0..L_{n-1} on [0,1] at xi.
void legendre01(int n, double xi, double* out) {
  const double s = 2.0 * xi - 1.0;
  double p0 = 1.0, p1 = s;
  for (int k = 0; k < n; ++k) {
    double pk;
    if (k == 0) pk = 1.0;
    else if (k == 1) pk = s;
    else {
      pk = ((2.0 * (k - 1) + 1) * s * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    out[k] = pk * std::sqrt(2.0 * k + 1);
  }
}

}  // namespace stm

using namespace stm;

struct stm_ctx {
  int device = 0;
  int sms = 1;  // streaming multiprocessors of the device
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t ne = 0;
  int P = 0, Q = 0, N = 0, N2 = 0, N3 = 0;
  int geometry = STM_GEOM_BRICK;
  int64_t n_trial = 0, n_test = 0, n_state = 0;
  stm_opts opts{};
  std::string err;
  std::vector<double> h_x0, h_h, h_mass;  // [ne][3], [ne][3], [ne][6]
  std::vector<double> h_mass3;             // general affine: [ne][2][6]
  std::vector<double> h_eps, h_mu;         // [ne]
  // dissipative term D_h (Sec. 4.2): per element [field][face][tangential comp] coefficients
  double* kap64 = nullptr;
  float* kap32 = nullptr;
  std::vector<double> h_kap;
  // inexact solve (Sec. 5.3): per (element, field, component) weights sqrt(4 c_f / (dt G_c))
  double* sw64 = nullptr;
  float* sw32 = nullptr;
  double sw_dt = 0.0;
  int32_t* nbr = nullptr;
  double* mass64 = nullptr;
  float* mass32 = nullptr;
  double* y64 = nullptr;
  double* tr64 = nullptr;
  float* y32 = nullptr;
  float* tr32 = nullptr;
  double* state = nullptr;
  double t = 0.0;
  double* red_partial = nullptr;
  double* red_out = nullptr;
  double* h_pinned = nullptr;  // small pinned staging for reductions
  void* tmp_in = nullptr;
  size_t tmp_in_bytes = 0;
  void* tmp_out = nullptr;
  size_t tmp_out_bytes = 0;
  void* tmp_op = nullptr;  // P^{-1} V of stm_operator_apply on curved and affine meshes
  size_t tmp_op_bytes = 0;
  // inverse mass factors 1 / (eps G_c), 1 / (mu G_c): the preconditioner of Eq. preconditioner
  double* inv64 = nullptr;
  float* inv32 = nullptr;
  // GMRES workspace: FP64 basis (plain path) or FP32 basis + FP64 residual (mixed path)
  double* V = nullptr;
  int64_t V_len = 0;
  double* z = nullptr;
  int64_t z_len = 0;
  double* x = nullptr;
  int64_t x_len = 0;
  float* V32 = nullptr;
  int64_t V32_len = 0;
  float* z32 = nullptr;
  int64_t z32_len = 0;
  // geometry: vertices of every element; curved metric
  std::vector<double> h_X8;  // [ne][8][3]
  std::vector<int32_t> h_nbr;  // [ne][6]
  // uneven (p, q): per-element degrees, block offsets and the (p, q) classes
  bool hp = false;
  std::vector<int> h_p, h_q;
  std::vector<int64_t> h_off_trial, h_off_test, h_off_state, h_off_tr;
  uint8_t* pq = nullptr;
  int64_t *off_trial = nullptr, *off_test = nullptr, *off_state = nullptr, *off_tr = nullptr;
  struct Class {
    int P, Q;
    int64_t count;
    int32_t* elist;
    int block;
    int NK = 1;  // temporal sub-intervals of the class's elements
  };
  // local refinement in time: N_K per element (log2 on the device) and the temporal transfer tables
  std::vector<int> h_nk;
  bool ltr = false;
  uint8_t* nkl = nullptr;
  double* tmat64 = nullptr;
  float* tmat32 = nullptr;
  std::vector<Class> classes;
  int64_t n_tr = 0;
  // 2:1 faces: slots (receiving element faces) and their sources
  int64_t n_slots = 0, n_hbuf = 0;
  int32_t *hslot = nullptr, *s_elem = nullptr, *s_face = nullptr, *s_kind = nullptr, *s_src = nullptr,
          *s_srcface = nullptr, *s_quad = nullptr;
  int64_t* hoff = nullptr;
  double* hbuf64 = nullptr;
  float* hbuf32 = nullptr;
  double Tm[2][8][8] = {};
  // uniform-mesh block size (autotuned), CUDA graphs of multi-class applies
  int block = 256;
  cudaStream_t cap_stream = nullptr;
  // uneven (p, q): the class kernels of one phase run side by side on these streams
  static constexpr int kAux = 4;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kAux] = {};
  std::vector<int> class_order;  // classes by decreasing work, dealt round-robin to aux
  struct GraphKey {
    int prec, um_layout, u0_layout, pre;
    const void *um, *u0, *b, *R;
    double dt;
    bool operator<(const GraphKey& o) const {
      return std::tie(prec, um_layout, u0_layout, pre, um, u0, b, R, dt) <
             std::tie(o.prec, o.um_layout, o.u0_layout, o.pre, o.um, o.u0, o.b, o.R, o.dt);
    }
  };
  std::map<GraphKey, cudaGraphExec_t> graphs;
  double* X8 = nullptr;
  double *eps64 = nullptr, *mu64 = nullptr;
  float *eps32 = nullptr, *mu32 = nullptr;
  double* Gw64 = nullptr;  // [ne][6][(p+2)^3]
  float* Gw32 = nullptr;
  double* Pinv64 = nullptr;  // [ne][2][9]
  float* Pinv32 = nullptr;
  double* mass3_64 = nullptr;  // general affine elements: [ne][2][6] mat * G (constant metric)
  float* mass3_32 = nullptr;
  int* tc_err = nullptr;       // trilinear meshes: set by the tensor-core mass kernel if a wait ran out
  int* wait_err = nullptr;     // set by the FP32 Krylov kernel if a bounded wait on its copies ran out
  double* el = nullptr;      // per-element energies (curved)
  CurvedTables ct{};
  // load vector L (Gaussian currents, boundary data g), cached per (t0, dt)
  std::vector<stm_gauss_src> srcs;
  stm_st_field_fn gfn = nullptr;
  void* guser = nullptr;
  stm_st_field_fn jfn = nullptr;  // current density J(x, t) sampled on the host
  void* juser = nullptr;
  double* load64 = nullptr;
  float* load32 = nullptr;
  bool load_valid = false;
  double load_t0 = 0.0, load_dt = 0.0;
  // device-side GMRES control (Sec. 5.4): state in device memory, a pinned copy for the
  // one host read per restart cycle, and CUDA graphs of whole cycles keyed by
  // (precision, dt, load pointer)
  GmresState* gst = nullptr;
  GmresState* h_gst = nullptr;
  struct CycleGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
  };
  std::map<std::tuple<int, double, const void*, int>, CycleGraph> cycle_graphs;
  // instrumentation: kernel launch count, optional per-launch event timing
  int64_t launches = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Timed { cudaEvent_t a, b, c; int prec; };
  std::vector<Timed> timed;
  // while profiling: index into `timed` at the start of each GMRES iteration of the current
  // cycle (the entries of iterations the device skipped are dropped after the cycle)
  std::vector<size_t> it_marks;
};

#define STM_CK(call)                                                                              \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) {                                                                      \
      c->err = std::string(#call) + ": " + cudaGetErrorString(e_);                                \
      return STM_EDEVICE;                                                                         \
    }                                                                                             \
  } while (0)

namespace {

int fail(stm_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int ensure(stm_ctx* c, void** p, size_t* have, size_t need) {
  if (*have >= need) return STM_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, need) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, STM_ENOMEM, "device allocation of " + std::to_string(need) + " bytes failed");
  }
  *have = need;
  return STM_OK;
}

template <typename T>
int ensure_scratch(stm_ctx* c, T** y, T** tr) {
  if (*y) return STM_OK;
  const size_t ny = (size_t)c->n_test;
  const size_t nt = (size_t)c->n_tr;
  if (cudaMalloc((void**)y, ny * sizeof(T)) != cudaSuccess || cudaMalloc((void**)tr, nt * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, STM_ENOMEM, "scratch allocation failed");
  }
  return STM_OK;
}

template <typename T>
const T* mass_ptr(stm_ctx* c);
template <>
const double* mass_ptr<double>(stm_ctx* c) { return c->mass64; }
template <>
const float* mass_ptr<float>(stm_ctx* c) { return c->mass32; }

// curved element data in the working precision: 0 = w G at the Gauss points, 1 = eps, 2 = mu, 3 = Pinv
template <typename T>
const T* curved_ptr(stm_ctx* c, int which);
template <>
const double* curved_ptr<double>(stm_ctx* c, int which) {
  const double* p[4] = {c->Gw64, c->eps64, c->mu64, c->Pinv64};
  return p[which];
}
template <>
const float* curved_ptr<float>(stm_ctx* c, int which) {
  const float* p[4] = {c->Gw32, c->eps32, c->mu32, c->Pinv32};
  return p[which];
}

template <typename T>
const T* hbuf_ptr(stm_ctx* c);
template <>
const double* hbuf_ptr<double>(stm_ctx* c) { return c->hbuf64; }
template <>
const float* hbuf_ptr<float>(stm_ctx* c) { return c->hbuf32; }

template <typename T>
int scratch(stm_ctx* c, T** y, T** tr);
template <>
int scratch<double>(stm_ctx* c, double** y, double** tr) {
  int rc = ensure_scratch<double>(c, &c->y64, &c->tr64);
  *y = c->y64;
  *tr = c->tr64;
  return rc;
}
template <>
int scratch<float>(stm_ctx* c, float** y, float** tr) {
  int rc = ensure_scratch<float>(c, &c->y32, &c->tr32);
  *y = c->y32;
  *tr = c->tr32;
  return rc;
}

enum Layout { L_TRIAL = 0, L_TEST = 1, L_STATE = 2 };

template <typename T>
int record_events(stm_ctx* c, LaunchEvents& ev) {
  if (!c->profiling) return STM_OK;
  while (c->ev_pool.size() < c->ev_used + 3) {
    cudaEvent_t x;
    if (cudaEventCreate(&x) != cudaSuccess) return fail(c, STM_EDEVICE, "event creation failed");
    c->ev_pool.push_back(x);
  }
  ev.start = c->ev_pool[c->ev_used];
  ev.mid = c->ev_pool[c->ev_used + 1];
  ev.stop = c->ev_pool[c->ev_used + 2];
  c->ev_used += 3;
  c->timed.push_back({ev.start, ev.mid, ev.stop, sizeof(T) == 8 ? 0 : 1});
  return STM_OK;
}

// R = A(um; u0) - b on the context stream.  um holds the unknown modes 1..q, in
// the trial layout (um_layout = L_TRIAL, mode 0 skipped) or the test layout;
// u0 is mode 0 (trial layout or a state vector) or null; b is the load or null.
template <typename T>
const T* pinv_ptr(stm_ctx* c) {
  if constexpr (sizeof(T) == 8) return c->inv64;
  else return c->inv32;
}

template <typename T>
const T* tmat_ptr(stm_ctx* c) {
  if constexpr (sizeof(T) == 8) return c->tmat64;
  else return c->tmat32;
}

template <typename T>
const T* kap_ptr(stm_ctx* c) {
  if constexpr (sizeof(T) == 8) return c->kap64;
  else return c->kap32;
}

// Whether the residual kernels of precision T use the y / trace scratch: all but the
// single-pass FP32 kernel (uniform meshes, with or without D_h, shared memory within fused_fits).
template <typename T>
bool needs_scratch(const stm_ctx* c) {
  return sizeof(T) == 8 || c->hp || !fused_fits(c->P, c->Q);
}

// Upper bound of the residual kernels' grids (grid-stride loops over elements): the launch
// sizes each grid to one wave of co-resident CTAs (wave_grid in residual.cuh).
int res_grid(const stm_ctx* c, int64_t count) {
  (void)c;
  return (int)std::max<int64_t>(1, std::min<int64_t>(count, 1 << 30));
}

__global__ void k_copy_words(double* __restrict__ dst, const double* __restrict__ src, int64_t n, int vec);

// Moves n doubles between host and device memory on the context stream (to_device: src on the
// host, dst on the device; otherwise the reverse).  Host memory the device addresses directly
// (page-locked by stm_host_alloc or cudaMallocHost, or registered) is read or written by a copy
// kernel: its concurrent requests keep the host link busy where a copy-engine transfer of a
// large buffer stalls on its first touch after other device work; other host memory goes
// through cudaMemcpyAsync.
int host_transfer(stm_ctx* c, double* dst, const double* src, int64_t n, bool to_device) {
  const void* host = to_device ? (const void*)src : (const void*)dst;
  cudaPointerAttributes at{};
  const bool mapped = cudaPointerGetAttributes(&at, host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                      at.devicePointer != nullptr;
  cudaGetLastError();
  if (mapped && n > 0) {
    double* hd = (double*)at.devicePointer;
    double* d = to_device ? dst : hd;
    const double* s = to_device ? hd : src;
    const int vec = ((reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(s)) & 15) == 0 ? 1 : 0;
    const int64_t blocks = std::min<int64_t>((int64_t)c->sms * 16, std::max<int64_t>(1, (n / 2 + 255) / 256));
    k_copy_words<<<(int)blocks, 256, 0, c->stream>>>(d, s, n, vec);
    c->launches += 1;
    STM_CK(cudaGetLastError());
    return STM_OK;
  }
  STM_CK(cudaMemcpyAsync(dst, src, n * sizeof(double), to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost,
                         c->stream));
  return STM_OK;
}

// STM_ETIMEOUT if a bounded wait of the FP32 Krylov kernel on its asynchronous copies ran out
// (the flag stays set: every later result of the context is suspect), else STM_OK.
int check_wait_err(stm_ctx* c) {
  int h = 0;
  if (cudaMemcpyAsync(&h, c->wait_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    return fail(c, STM_EDEVICE, std::string("error flag read: ") + cudaGetErrorString(e));
  }
  return h ? fail(c, STM_ETIMEOUT, "FP32 Krylov kernel: a bounded wait on its copies ran out") : STM_OK;
}

// Default threads per block of the two-kernel residual passes of degree (P, Q): the kernels'
// largest block (residual_max_threads: 512 where shared memory limits the blocks per SM, else
// 256).  The autotuner may replace it.
int default_block(int P, int Q) { return residual_max_threads(P, Q); }

template <typename T>
int apply(stm_ctx* c, double dt, const T* um, int um_layout, const T* u0, int u0_layout, const T* b, T* R,
          bool pre = false, const int32_t* skip = nullptr) {
  T *y = nullptr, *tr = nullptr;
  if (needs_scratch<T>(c)) {  // the uniform FP32 single-pass kernel needs none
    int rc = scratch<T>(c, &y, &tr);
    if (rc) return rc;
  }
  ApplyArgs<T> a{};
  a.b = b;
  a.y = y;
  a.tr = tr;
  a.R = R;
  a.nbr = c->nbr;
  a.mass = mass_ptr<T>(c);
  a.kap = kap_ptr<T>(c);
  a.dt_k = (T)dt;
  a.pinv = pre ? pinv_ptr<T>(c) : nullptr;
  a.skip = skip;
  a.err = c->wait_err;
  const int N3 = c->N3, Q = c->Q;
  if (c->hp) {
    a.um = um;
    a.u0 = u0;
    a.off_um = um_layout == L_TRIAL ? c->off_trial : c->off_test;
    a.um_trial = um_layout == L_TRIAL;
    a.off_u0 = u0_layout == L_STATE ? c->off_state : c->off_trial;
    a.u0_state = u0_layout == L_STATE;
    a.off_R = c->off_test;
    a.off_tr = c->off_tr;
    a.pq = c->pq;
    a.nkl = c->nkl;
    a.tmat = tmat_ptr<T>(c);
    // no graph of its own inside a capture of a whole GMRES cycle (captures do not nest)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    STM_CK(cudaStreamIsCapturing(c->stream, &cap));
    const bool use_graph = c->opts.graph && !c->profiling && cap == cudaStreamCaptureStatusNone && !skip;
    typename stm_ctx::GraphKey key{sizeof(T) == 8 ? 0 : 1, um_layout, u0_layout, pre ? 1 : 0, um, u0, b, R, dt};
    if (use_graph) {
      auto it = c->graphs.find(key);
      if (it != c->graphs.end()) {
        c->launches += 2 * (int64_t)c->classes.size() + (c->n_slots > 0);
        STM_CK(cudaGraphLaunch(it->second, c->stream));
        return STM_OK;
      }
      if (!c->cap_stream) STM_CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
      STM_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    }
    cudaStream_t ls = use_graph ? c->cap_stream : c->stream;
    LaunchEvents ev, none;
    int rc = record_events<T>(c, ev);
    if (rc) return rc;
    a.hslot = c->hslot;
    a.hoff = c->hoff;
    a.hbuf = hbuf_ptr<T>(c);
    // the classes of one phase are independent: fork them over the auxiliary streams (largest
    // first, round-robin) and join before the next phase; the timed profile keeps them in order
    const bool conc = !c->profiling && c->classes.size() > 1;
    if (conc && !c->fork_ev) {
      bool ok = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) == cudaSuccess;
      for (int k = 0; ok && k < stm_ctx::kAux; ++k)
        ok = cudaStreamCreateWithFlags(&c->aux[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->join_ev[k], cudaEventDisableTiming) == cudaSuccess;
      if (!ok) {  // leave nothing half made: the next call tries again
        cudaGetLastError();
        for (int k = 0; k < stm_ctx::kAux; ++k) {
          if (c->aux[k]) cudaStreamDestroy(c->aux[k]);
          if (c->join_ev[k]) cudaEventDestroy(c->join_ev[k]);
          c->aux[k] = nullptr;
          c->join_ev[k] = nullptr;
        }
        if (c->fork_ev) cudaEventDestroy(c->fork_ev);
        c->fork_ev = nullptr;
        return fail(c, STM_EDEVICE, "auxiliary stream set-up failed");
      }
    }
    if (c->class_order.size() != c->classes.size()) {
      c->class_order.resize(c->classes.size());
      for (size_t k = 0; k < c->classes.size(); ++k) c->class_order[k] = (int)k;
      auto work = [&](int k) {
        const auto& cl = c->classes[k];
        const double n = cl.P + 1.0;
        return (double)cl.count * n * n * n * n * cl.Q * cl.NK;
      };
      std::stable_sort(c->class_order.begin(), c->class_order.end(), [&](int x, int y) { return work(x) > work(y); });
    }
    auto fork = [&]() -> cudaError_t {
      cudaError_t e = cudaEventRecord(c->fork_ev, ls);
      for (int k = 0; e == cudaSuccess && k < stm_ctx::kAux; ++k) e = cudaStreamWaitEvent(c->aux[k], c->fork_ev, 0);
      return e;
    };
    auto join = [&]() -> cudaError_t {
      cudaError_t e = cudaSuccess;
      for (int k = 0; k < stm_ctx::kAux; ++k) {
        const cudaError_t e1 = cudaEventRecord(c->join_ev[k], c->aux[k]);
        const cudaError_t e2 = cudaStreamWaitEvent(ls, c->join_ev[k], 0);
        if (e == cudaSuccess) e = (e1 != cudaSuccess) ? e1 : e2;
      }
      return e;
    };
    for (int phase = 1; phase <= 2; ++phase) {
      if (phase == 2 && c->n_slots > 0) {
        // 2:1 faces: equivalent neighbour traces from all classes' traces
        HangArgs<T> h;
        h.tr = tr;
        h.off_tr = c->off_tr;
        h.pq = c->pq;
        h.n_slots = c->n_slots;
        h.elem = c->s_elem;
        h.face = c->s_face;
        h.kind = c->s_kind;
        h.src = c->s_src;
        h.src_face = c->s_srcface;
        h.quad = c->s_quad;
        h.hoff = c->hoff;
        h.hbuf = const_cast<T*>(hbuf_ptr<T>(c));
        h.skip = skip;
        for (int u = 0; u < 2; ++u)
          for (int j = 0; j < 8; ++j)
            for (int nn = 0; nn < 8; ++nn) h.Tm[u][j][nn] = (T)c->Tm[u][j][nn];
        launch_hang<T>(h, ls);
        c->launches += 1;
      }
      cudaError_t fe = conc ? fork() : cudaSuccess;
      for (size_t j = 0; j < c->classes.size(); ++j) {
        const size_t k = conc ? (size_t)c->class_order[j] : j;
        const auto& cl = c->classes[k];
        a.elist = cl.elist;
        a.n_elem = cl.count;
        a.nk = cl.NK;
        a.tb = make_tables<T>(cl.P, kMaxQ, dt / cl.NK);  // sub-interval length dt / N_K
        LaunchEvents e2 = none;
        if (!conc) {
          if (phase == 1 && k == 0) e2.start = ev.start;
          if (phase == 1 && k + 1 == c->classes.size()) e2.mid = ev.mid;
          if (phase == 2 && k + 1 == c->classes.size()) e2.stop = ev.stop;
        }
        const int grid = res_grid(c, cl.count);
        const int e = fe != cudaSuccess ? (int)fe
                                        : launch_residual_ph<T>(cl.P, cl.Q, a, conc ? c->aux[j % stm_ctx::kAux] : ls,
                                                                grid, e2, phase, cl.block);
        c->launches += 1;
        if (e) {
          if (conc) join();  // the forked streams rejoin the origin before the capture ends
          if (use_graph) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(c->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();  // the invalidated capture leaves no error behind
          }
          return fail(c, STM_EDEVICE, std::string("residual launch: ") + cudaGetErrorString((cudaError_t)e));
        }
      }
      if (conc) {
        const cudaError_t je = join();
        if (je != cudaSuccess) {
          if (use_graph) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(c->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
          }
          return fail(c, STM_EDEVICE, std::string("class join: ") + cudaGetErrorString(je));
        }
      }
    }
    if (use_graph) {
      cudaGraph_t g = nullptr;
      STM_CK(cudaStreamEndCapture(c->cap_stream, &g));
      cudaGraphExec_t ex = nullptr;
      const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) return fail(c, STM_EDEVICE, std::string("graph instantiate: ") + cudaGetErrorString(ie));
      if (c->graphs.size() > 64) {
        for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
        c->graphs.clear();
      }
      c->graphs[key] = ex;
      STM_CK(cudaGraphLaunch(ex, c->stream));
    }
    return STM_OK;
  }
  // uniform mesh: strides
  a.um = um_layout == L_TRIAL ? um + N3 : um;
  a.um_es = um_layout == L_TRIAL ? 6LL * (Q + 1) * N3 : 6LL * Q * N3;
  a.um_cs = um_layout == L_TRIAL ? (int64_t)(Q + 1) * N3 : (int64_t)Q * N3;
  a.u0 = u0;
  a.u0_es = u0_layout == L_STATE ? 6LL * N3 : 6LL * (Q + 1) * N3;
  a.u0_cs = u0_layout == L_STATE ? (int64_t)N3 : (int64_t)(Q + 1) * N3;
  if (c->geometry == STM_GEOM_AFFINE) {
    a.mass = nullptr;  // the constant 3x3 metric mass, inside the residual kernels
    if constexpr (sizeof(T) == 8) a.mass3 = c->mass3_64;
    else a.mass3 = c->mass3_32;
  }
  if (c->geometry == STM_GEOM_TRILINEAR) {
    // curved: the metric-dependent mass term goes first into R; the residual kernels add the rest
    int em;
    if constexpr (sizeof(T) == 4) {
      if (!c->opts.no_tensor_cores && c->P >= 3 && c->tc_err)
        em = launch_mass_curved_tc(c->P, c->Q, a.um, a.um_es, a.um_cs, a.u0, a.u0_es, a.u0_cs, c->Gw32, c->eps32,
                                   c->mu32, c->ct, c->ne, R, c->stream, skip, c->tc_err);
      else
        em = launch_mass_curved<T>(c->P, c->Q, a.um, a.um_es, a.um_cs, a.u0, a.u0_es, a.u0_cs, curved_ptr<T>(c, 0),
                                   curved_ptr<T>(c, 1), curved_ptr<T>(c, 2), c->ct, c->ne, R, c->stream, skip);
    } else {
      em = launch_mass_curved<T>(c->P, c->Q, a.um, a.um_es, a.um_cs, a.u0, a.u0_es, a.u0_cs, curved_ptr<T>(c, 0),
                                 curved_ptr<T>(c, 1), curved_ptr<T>(c, 2), c->ct, c->ne, R, c->stream, skip);
    }
    c->launches += 1;
    if (em) return fail(c, STM_EDEVICE, std::string("curved mass launch: ") + cudaGetErrorString((cudaError_t)em));
    a.mass = nullptr;
  }
  a.n_elem = c->ne;
  a.tb = make_tables<T>(c->P, c->Q, dt);
  const int grid = res_grid(c, c->ne);
  LaunchEvents ev;
  int rc = record_events<T>(c, ev);
  if (rc) return rc;
  c->launches += 2;
  const int e = launch_residual_ph<T>(c->P, c->Q, a, c->stream, grid, ev, 0, c->block);
  if (e) return fail(c, STM_EDEVICE, std::string("residual launch: ") + cudaGetErrorString((cudaError_t)e));
  return STM_OK;
}

// Linear operator on the unknowns (Krylov layout, modes 1..q), no u0, no load.
template <typename T>
int linop(stm_ctx* c, double dt, const T* xin, T* out, const int32_t* skip = nullptr) {
  return apply<T>(c, dt, xin, L_TEST, nullptr, L_STATE, nullptr, out, false, skip);
}

// A P^{-1} v in one residual launch (uniform brick meshes): the kernels scale v by the
// inverse block-diagonal mass on load instead of a separate preconditioner pass
template <typename T>
int linop_pre(stm_ctx* c, double dt, const T* v, T* out, const int32_t* skip = nullptr) {
  return apply<T>(c, dt, v, L_TEST, nullptr, L_STATE, nullptr, out, true, skip);
}

// R(U) = A U - b with mode 0 = state (FP64), modes 1..q = xin and the load b (or none).
int resid64(stm_ctx* c, double dt, const double* xin, const double* b, double* out, const int32_t* skip = nullptr) {
  return apply<double>(c, dt, xin, L_TEST, c->state, L_STATE, b, out, false, skip);
}

// l_E(v) = (J, v) over I_n x K for a current density sampled on the host (Eq.
// bilinearform:C), added into the E rows of hb (test layout, per-element
// offsets).  With the covariant test functions v = DF^{-T} phi_s e_c,
// J . v |J| = (adj(DF) J)_c phi_s, so per element: values a = adj(DF) J at the
// (p+2)^3 Gauss points times q+2 Gauss points on each of the element's N_K
// time sub-intervals, weighted and contracted with L_i of the sub-interval,
// then projected on phi_s by three 1-D contractions.  The trilinear map of the
// 8 vertices covers bricks and curved elements alike; p, q and N_K are the
// element's own.
void add_host_current(stm_ctx* c, double t0, double dt, stm_st_field_fn fn, void* user, std::vector<double>& hb) {
  struct Rule {
    std::vector<double> x, w, L;  // points, weights, L_j(x_g) at [g * n + j]
  };
  auto rule = [](int npts, int nfun) {
    Rule r;
    gauss01(npts, r.x, r.w);
    r.L.resize((size_t)npts * nfun);
    for (int g = 0; g < npts; ++g) legendre01(nfun, r.x[g], &r.L[(size_t)g * nfun]);
    return r;
  };
  std::vector<Rule> space(8), time(kMaxQ + 1);
  for (int P = 0; P < 8; ++P) space[P] = rule(P + 2, P + 1);
  for (int q = 1; q <= kMaxQ; ++q) time[q] = rule(q + 2, q);
  auto pts_of = [&](int64_t e) {
    const int nq = c->h_p[e] + 2;
    return (int64_t)(c->h_q[e] + 2) * c->h_nk[e] * nq * nq * nq;
  };
  std::vector<double> xtp, jv, adj, F, G1, G2;
  for (int64_t e0 = 0; e0 < c->ne;) {
    // a chunk of elements with about 2^20 space-time points
    int64_t e1 = e0, np = 0;
    std::vector<int64_t> start;
    while (e1 < c->ne && (np == 0 || np + pts_of(e1) <= (1 << 20))) {
      start.push_back(np);
      np += pts_of(e1++);
    }
    xtp.resize(4 * np);
    jv.resize(3 * np);
    for (int64_t e = e0; e < e1; ++e) {
      const int P = c->h_p[e], q = c->h_q[e], nk = c->h_nk[e], nq = P + 2, nq3 = nq * nq * nq, nt = q + 2;
      const Rule& sr = space[P];
      const Rule& tr = time[q];
      const double* X = &c->h_X8[24 * e];
      for (int g = 0; g < nq3; ++g) {
        const double xh[3] = {sr.x[g % nq], sr.x[(g / nq) % nq], sr.x[g / (nq * nq)]};
        double x[3] = {0, 0, 0};
        for (int v = 0; v < 8; ++v) {
          const int bit[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
          double Nv = 1.0;
          for (int a = 0; a < 3; ++a) Nv *= bit[a] ? xh[a] : 1.0 - xh[a];
          for (int i = 0; i < 3; ++i) x[i] += Nv * X[3 * v + i];
        }
        for (int k = 0; k < nk; ++k)
          for (int tq = 0; tq < nt; ++tq) {
            double* pt = &xtp[4 * (start[e - e0] + ((int64_t)k * nt + tq) * nq3 + g)];
            pt[0] = x[0];
            pt[1] = x[1];
            pt[2] = x[2];
            pt[3] = t0 + dt * (k + tr.x[tq]) / nk;
          }
      }
    }
    fn(user, np, xtp.data(), jv.data());
    for (int64_t e = e0; e < e1; ++e) {
      const int P = c->h_p[e], q = c->h_q[e], nk = c->h_nk[e], N = P + 1, N3 = N * N * N, nq = P + 2,
                nq3 = nq * nq * nq, nt = q + 2, QE = nk * q;
      const Rule& sr = space[P];
      const Rule& tr = time[q];
      const double* X = &c->h_X8[24 * e];
      // adj(DF) = |J| DF^{-1} (cofactor transpose) at the spatial points
      adj.resize(9 * (size_t)nq3);
      for (int g = 0; g < nq3; ++g) {
        const double xh[3] = {sr.x[g % nq], sr.x[(g / nq) % nq], sr.x[g / (nq * nq)]};
        double DF[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int v = 0; v < 8; ++v) {
          const int bit[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
          double fa[3], dfa[3];
          for (int a = 0; a < 3; ++a) {
            fa[a] = bit[a] ? xh[a] : 1.0 - xh[a];
            dfa[a] = bit[a] ? 1.0 : -1.0;
          }
          const double dN[3] = {dfa[0] * fa[1] * fa[2], fa[0] * dfa[1] * fa[2], fa[0] * fa[1] * dfa[2]};
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) DF[i][j] += X[3 * v + i] * dN[j];
        }
        double* A = &adj[9 * (size_t)g];
        A[0] = DF[1][1] * DF[2][2] - DF[1][2] * DF[2][1];
        A[1] = DF[0][2] * DF[2][1] - DF[0][1] * DF[2][2];
        A[2] = DF[0][1] * DF[1][2] - DF[0][2] * DF[1][1];
        A[3] = DF[1][2] * DF[2][0] - DF[1][0] * DF[2][2];
        A[4] = DF[0][0] * DF[2][2] - DF[0][2] * DF[2][0];
        A[5] = DF[0][2] * DF[1][0] - DF[0][0] * DF[1][2];
        A[6] = DF[1][0] * DF[2][1] - DF[1][1] * DF[2][0];
        A[7] = DF[0][1] * DF[2][0] - DF[0][0] * DF[2][1];
        A[8] = DF[0][0] * DF[1][1] - DF[0][1] * DF[1][0];
      }
      // F[c][k q + i][g] = sum_tau w_tau (dt/N_K) L_i(tau) w_g (adj(DF) J)_c
      F.assign(3 * (size_t)QE * nq3, 0.0);
      for (int k = 0; k < nk; ++k)
        for (int tq = 0; tq < nt; ++tq)
          for (int g = 0; g < nq3; ++g) {
            const double* J = &jv[3 * (start[e - e0] + ((int64_t)k * nt + tq) * nq3 + g)];
            const double* A = &adj[9 * (size_t)g];
            const double w = dt / nk * tr.w[tq] * sr.w[g % nq] * sr.w[(g / nq) % nq] * sr.w[g / (nq * nq)];
            for (int cc = 0; cc < 3; ++cc) {
              const double a = w * (A[3 * cc] * J[0] + A[3 * cc + 1] * J[1] + A[3 * cc + 2] * J[2]);
              for (int i = 0; i < q; ++i)
                F[((size_t)cc * QE + k * q + i) * nq3 + g] += tr.L[(size_t)tq * q + i] * a;
            }
          }
      // project on phi_s = L_j(x^) L_k(y^) L_l(z^): contract x, then y, then z
      for (int ci = 0; ci < 3 * QE; ++ci) {
        const double* f0 = &F[(size_t)ci * nq3];
        G1.assign((size_t)nq * nq * N, 0.0);
        for (int gz = 0; gz < nq; ++gz)
          for (int gy = 0; gy < nq; ++gy)
            for (int j = 0; j < N; ++j) {
              double acc = 0.0;
              for (int gx = 0; gx < nq; ++gx) acc += f0[(gz * nq + gy) * nq + gx] * sr.L[(size_t)gx * N + j];
              G1[(gz * nq + gy) * N + j] = acc;
            }
        G2.assign((size_t)nq * N * N, 0.0);
        for (int gz = 0; gz < nq; ++gz)
          for (int kk = 0; kk < N; ++kk)
            for (int j = 0; j < N; ++j) {
              double acc = 0.0;
              for (int gy = 0; gy < nq; ++gy) acc += G1[(gz * nq + gy) * N + j] * sr.L[(size_t)gy * N + kk];
              G2[(gz * N + kk) * N + j] = acc;
            }
        // E rows of the element: field 0, (component, temporal index) = ci
        double* row = &hb[(size_t)c->h_off_test[e] + (size_t)ci * N3];
        for (int l = 0; l < N; ++l)
          for (int kk = 0; kk < N; ++kk)
            for (int j = 0; j < N; ++j) {
              double acc = 0.0;
              for (int gz = 0; gz < nq; ++gz) acc += G2[(gz * N + kk) * N + j] * sr.L[(size_t)gz * N + l];
              row[(l * N + kk) * N + j] += acc;
            }
      }
    }
    e0 = e1;
  }
}

// l_H(w) = -<n x g, w> over I_n x F_b (Eq. bilinearform:C) for boundary data g
// sampled on the host, added into the H rows of hb; with D_h (Sec. 4.2) also the
// g part of <alpha_E n x (E - g), n x v> into the E rows.  In the reference face
// (Nanson, covariant transform) <n x g, w> = int int (n^ x g^) . w^ with
// g^ = DF^T g.  Per boundary face: (p+2)^2 Gauss points and q+2 in time on each
// of the element's N_K sub-intervals, with the element's own p, q and N_K.
void add_host_boundary(stm_ctx* c, double t0, double dt, std::vector<double>& hb) {
  struct Rule {
    std::vector<double> x, w, L;
  };
  auto rule = [](int npts, int nfun) {
    Rule r;
    gauss01(npts, r.x, r.w);
    r.L.resize((size_t)npts * nfun);
    for (int g = 0; g < npts; ++g) legendre01(nfun, r.x[g], &r.L[(size_t)g * nfun]);
    return r;
  };
  std::vector<Rule> space(8), time(kMaxQ + 1);
  for (int P = 0; P < 8; ++P) space[P] = rule(P + 2, P + 1);
  for (int q = 1; q <= kMaxQ; ++q) time[q] = rule(q + 2, q);
  std::vector<int64_t> faces;
  for (int64_t e = 0; e < c->ne; ++e)
    for (int f = 0; f < 6; ++f)
      if (c->h_nbr[6 * e + f] == -1) faces.push_back(6 * e + f);
  auto pts_of = [&](int64_t e) {
    const int nq = c->h_p[e] + 2;
    return (int64_t)(c->h_q[e] + 2) * c->h_nk[e] * nq * nq;
  };
  std::vector<double> xtp, gv, DFs;
  for (size_t f0 = 0; f0 < faces.size();) {
    size_t f1 = f0;
    int64_t np = 0;
    std::vector<int64_t> start;
    while (f1 < faces.size() && (np == 0 || np + pts_of(faces[f1] / 6) <= (1 << 20))) {
      start.push_back(np);
      np += pts_of(faces[f1++] / 6);
    }
    xtp.resize(4 * np);
    gv.resize(3 * np);
    DFs.resize(9 * np);
    for (size_t fi = f0; fi < f1; ++fi) {
      const int64_t e = faces[fi] / 6;
      const int f = (int)(faces[fi] % 6), d = f / 2, sd = f % 2;
      const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
      const int nq = c->h_p[e] + 2, nt = c->h_q[e] + 2, nk = c->h_nk[e];
      const Rule& sr = space[c->h_p[e]];
      const Rule& tr = time[c->h_q[e]];
      const double* X = &c->h_X8[24 * e];
      for (int u = 0; u < nq; ++u)
        for (int v = 0; v < nq; ++v) {
          double xh[3];
          xh[d] = sd;
          xh[a1] = sr.x[u];
          xh[a2] = sr.x[v];
          double x[3] = {0, 0, 0}, DF[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
          for (int vv = 0; vv < 8; ++vv) {
            const int bit[3] = {vv & 1, (vv >> 1) & 1, (vv >> 2) & 1};
            double fa[3], dfa[3];
            for (int a = 0; a < 3; ++a) {
              fa[a] = bit[a] ? xh[a] : 1.0 - xh[a];
              dfa[a] = bit[a] ? 1.0 : -1.0;
            }
            const double Nv = fa[0] * fa[1] * fa[2];
            const double dN[3] = {dfa[0] * fa[1] * fa[2], fa[0] * dfa[1] * fa[2], fa[0] * fa[1] * dfa[2]};
            for (int i = 0; i < 3; ++i) {
              x[i] += Nv * X[3 * vv + i];
              for (int j = 0; j < 3; ++j) DF[3 * i + j] += X[3 * vv + i] * dN[j];
            }
          }
          for (int k = 0; k < nk; ++k)
            for (int tq = 0; tq < nt; ++tq) {
              const int64_t idx = start[fi - f0] + (((int64_t)k * nt + tq) * nq + u) * nq + v;
              xtp[4 * idx] = x[0];
              xtp[4 * idx + 1] = x[1];
              xtp[4 * idx + 2] = x[2];
              xtp[4 * idx + 3] = t0 + dt * (k + tr.x[tq]) / nk;
              std::copy(DF, DF + 9, &DFs[9 * idx]);
            }
        }
    }
    c->gfn(c->guser, np, xtp.data(), gv.data());
    for (size_t fi = f0; fi < f1; ++fi) {
      const int64_t e = faces[fi] / 6;
      const int f = (int)(faces[fi] % 6), d = f / 2, sd = f % 2;
      const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
      const int P = c->h_p[e], q = c->h_q[e], nk = c->h_nk[e], N = P + 1, N3 = N * N * N, nq = P + 2, nt = q + 2;
      const int QE = nk * q;
      const Rule& sr = space[P];
      const Rule& tr = time[q];
      double Lside[kMaxN];
      legendre01(N, sd ? 1.0 : 0.0, Lside);
      const double sgn = sd ? 1.0 : -1.0;  // n^ = sgn e_d
      const double nv[3] = {d == 0 ? sgn : 0.0, d == 1 ? sgn : 0.0, d == 2 ? sgn : 0.0};
      const int64_t off = c->h_off_test[e];
      // adds wi * phi_s at the face point (u, v) to the rows (field fld, component cc, index ti)
      auto lift = [&](int fld, int cc, int ti, double wi, int u, int v) {
        double* row = &hb[off + ((int64_t)(fld * 3 + cc) * QE + ti) * N3];
        for (int al = 0; al < N; ++al)
          for (int j1 = 0; j1 < N; ++j1)
            for (int j2 = 0; j2 < N; ++j2) {
              int ix[3];
              ix[d] = al;
              ix[a1] = j1;
              ix[a2] = j2;
              row[(ix[2] * N + ix[1]) * N + ix[0]] += wi * Lside[al] * sr.L[(size_t)u * N + j1] * sr.L[(size_t)v * N + j2];
            }
      };
      for (int k = 0; k < nk; ++k)
        for (int tq = 0; tq < nt; ++tq)
          for (int u = 0; u < nq; ++u)
            for (int v = 0; v < nq; ++v) {
              const int64_t idx = start[fi - f0] + (((int64_t)k * nt + tq) * nq + u) * nq + v;
              const double* DF = &DFs[9 * idx];
              const double* g = &gv[3 * idx];
              double gh[3];
              for (int cc = 0; cc < 3; ++cc) gh[cc] = DF[0 * 3 + cc] * g[0] + DF[1 * 3 + cc] * g[1] + DF[2 * 3 + cc] * g[2];
              const double ng[3] = {nv[1] * gh[2] - nv[2] * gh[1], nv[2] * gh[0] - nv[0] * gh[2],
                                    nv[0] * gh[1] - nv[1] * gh[0]};  // n^ x g^
              const double w = dt / nk * tr.w[tq] * sr.w[u] * sr.w[v];
              if (c->opts.c_diss > 0) {
                for (int bc = 0; bc < 2; ++bc) {
                  const int cc = (d == 0) ? bc + 1 : (d == 1 ? 2 * bc : bc);
                  const double kg = c->h_kap[e * 24 + f * 2 + bc] * gh[cc];
                  for (int i = 0; i < q; ++i) lift(0, cc, k * q + i, w * tr.L[(size_t)tq * q + i] * kg, u, v);
                }
              }
              for (int cc = 0; cc < 3; ++cc) {
                if (ng[cc] == 0.0) continue;
                for (int i = 0; i < q; ++i) lift(1, cc, k * q + i, -w * tr.L[(size_t)tq * q + i] * ng[cc], u, v);
              }
            }
    }
    f0 = f1;
  }
}

// Load vector b = L on the slab (t0, t0 + dt] (Eq. bilinearform:C): Gaussian
// currents on the device, boundary data g on the host.  Returns null when no
// source and no boundary data are set (L = 0).  Cached per (t0, dt).
int build_load(stm_ctx* c, double t0, double dt, const double** out) {
  *out = nullptr;
  if (c->srcs.empty() && !c->gfn && !c->jfn) return STM_OK;

  if (c->load_valid && c->load_t0 == t0 && c->load_dt == dt) {
    *out = c->load64;
    return STM_OK;
  }
  const int64_t n = c->n_test;
  if (!c->load64) {
    if (cudaMalloc(&c->load64, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->load32, n * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, STM_ENOMEM, "load vector allocation failed");
    }
  }
  if (c->hp) {
    // uneven degrees or N_K: the host callbacks (J, g) are sampled and projected on the
    // host per element with its own p, q and N_K; the Gaussian pulses are projected on the
    // device, one launch per (p, q, N_K) class
    if (c->jfn || c->gfn) {
      std::vector<double> hb(n, 0.0);
      if (c->jfn) add_host_current(c, t0, dt, c->jfn, c->juser, hb);
      if (c->gfn) add_host_boundary(c, t0, dt, hb);
      STM_CK(cudaMemcpyAsync(c->load64, hb.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      STM_CK(cudaStreamSynchronize(c->stream));
    } else {
      STM_CK(cudaMemsetAsync(c->load64, 0, n * sizeof(double), c->stream));
    }
    for (const auto& cl : c->classes) {
      if (c->srcs.empty()) break;
      const int nqc = cl.P + 2, ntc = cl.Q + 2, NKc = cl.NK;
      const double dk = dt / NKc;
      std::vector<double> xq, wq, xt, wt;
      gauss01(nqc, xq, wq);
      gauss01(ntc, xt, wt);
      GaussParams gp;
      std::memset(&gp, 0, sizeof(gp));
      gp.n_src = (int)c->srcs.size();
      gp.Q = cl.Q;
      gp.NK = NKc;
      gp.elist = cl.elist;
      gp.off_test = c->off_test;
      for (int g = 0; g < nqc; ++g) {
        gp.xq[g] = xq[g];
        gp.wq[g] = wq[g];
        double L[kMaxN];
        legendre01(cl.P + 1, xq[g], L);
        for (int j = 0; j <= cl.P; ++j) gp.Lq[j][g] = L[j];
      }
      for (int k = 0; k < gp.n_src; ++k) {
        const stm_gauss_src& sr = c->srcs[k];
        for (int i = 0; i < 3; ++i) {
          gp.c[k][i] = sr.centre[i];
          gp.d[k][i] = sr.dir[i];
        }
        gp.inv2sx2[k] = 1.0 / (2.0 * sr.sigma_x * sr.sigma_x);
        gp.amp[k] = sr.amp;
        for (int kk = 0; kk < NKc; ++kk)
          for (int i = 0; i < cl.Q; ++i) {
            double acc = 0.0;
            for (int tq = 0; tq < ntc; ++tq) {
              double Lt[kMaxQ];
              legendre01(cl.Q, xt[tq], Lt);
              const double tt = t0 + dk * (kk + xt[tq]) - sr.t0;
              acc += wt[tq] * Lt[i] * std::exp(-tt * tt / (2.0 * sr.sigma_t * sr.sigma_t));
            }
            gp.tfk[k][kk][i] = dk * acc;
          }
      }
      const int e = launch_load_gauss(cl.P, c->X8, cl.count, gp, c->load64, c->stream);
      c->launches += 1;
      if (e) return fail(c, STM_EDEVICE, std::string("load kernel: ") + cudaGetErrorString((cudaError_t)e));
    }
    convert<float, double>(c->load32, c->load64, n, c->stream);
    c->launches += 1;
    STM_CK(cudaGetLastError());
    c->load_valid = true;
    c->load_t0 = t0;
    c->load_dt = dt;
    *out = c->load64;
    return STM_OK;
  }
  const int P = c->P, Q = c->Q, N = c->N, nq = P + 2, nt = Q + 2;
  std::vector<double> xq, wq, xt, wt;
  gauss01(nq, xq, wq);
  gauss01(nt, xt, wt);
  std::vector<double> Lq(nq * N), Lt(nt * Q > 0 ? nt * kMaxQ : 1);
  for (int g = 0; g < nq; ++g) legendre01(N, xq[g], &Lq[g * N]);
  for (int g = 0; g < nt; ++g) legendre01(Q, xt[g], &Lt[g * kMaxQ]);
  if (c->gfn || c->jfn) {
    std::vector<double> hb(n, 0.0);
    if (c->jfn) add_host_current(c, t0, dt, c->jfn, c->juser, hb);
    if (c->gfn) add_host_boundary(c, t0, dt, hb);
    STM_CK(cudaMemcpyAsync(c->load64, hb.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    STM_CK(cudaStreamSynchronize(c->stream));
  } else {
    STM_CK(cudaMemsetAsync(c->load64, 0, n * sizeof(double), c->stream));
  }
  if (!c->srcs.empty()) {
    GaussParams gp;
    std::memset(&gp, 0, sizeof(gp));
    gp.n_src = (int)c->srcs.size();
    gp.Q = Q;
    for (int g = 0; g < nq; ++g) {
      gp.xq[g] = xq[g];
      gp.wq[g] = wq[g];
      for (int j = 0; j < N; ++j) gp.Lq[j][g] = Lq[g * N + j];
    }
    for (int k = 0; k < gp.n_src; ++k) {
      const stm_gauss_src& sr = c->srcs[k];
      for (int i = 0; i < 3; ++i) {
        gp.c[k][i] = sr.centre[i];
        gp.d[k][i] = sr.dir[i];
      }
      gp.inv2sx2[k] = 1.0 / (2.0 * sr.sigma_x * sr.sigma_x);
      gp.amp[k] = sr.amp;
      for (int i = 0; i < Q; ++i) {
        double acc = 0.0;
        for (int tq = 0; tq < nt; ++tq) {
          const double t = t0 + dt * xt[tq] - sr.t0;
          acc += wt[tq] * Lt[tq * kMaxQ + i] * std::exp(-t * t / (2.0 * sr.sigma_t * sr.sigma_t));
        }
        gp.tf[k][i] = dt * acc;
      }
    }
    const int e = launch_load_gauss(P, c->X8, c->ne, gp, c->load64, c->stream);
    c->launches += 1;
    if (e) return fail(c, STM_EDEVICE, std::string("load kernel: ") + cudaGetErrorString((cudaError_t)e));
  }
  convert<float, double>(c->load32, c->load64, n, c->stream);
  c->launches += 1;
  c->load_valid = true;
  c->load_t0 = t0;
  c->load_dt = dt;
  *out = c->load64;
  return STM_OK;
}

// Peak probe of the FP64 pipe: independent chains of dependent FMAs per thread
// (enough to hide the pipe latency), no memory traffic; the result is stored so
// the chains are not removed.
constexpr int kProbeChains = 8;
__global__ void __launch_bounds__(256) k_fma_probe(double* out, int iters, double a) {
  double v[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) v[k] = threadIdx.x * 1e-3 + k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) v[k] = fma(v[k], a, 1e-7);
  }
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) acc += v[k];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = acc;
}

// dst[i] = src[i] for n 8-byte words, one side in host memory the device addresses directly
// (page-locked or registered): the SMs' many concurrent requests stream over the host link
// without the copy engines' first-touch stalls.  vec: both pointers 16-byte aligned.
__global__ void k_copy_words(double* __restrict__ dst, const double* __restrict__ src, int64_t n, int vec) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  if (vec) {
    const int64_t n2 = n / 2;
    double2* d2 = reinterpret_cast<double2*>(dst);
    const double2* s2 = reinterpret_cast<const double2*>(src);
    for (int64_t i = tid; i < n2; i += nth) d2[i] = s2[i];
    if (tid == 0 && (n & 1)) dst[n - 1] = src[n - 1];
  } else {
    for (int64_t i = tid; i < n; i += nth) dst[i] = src[i];
  }
}

__global__ void k_init_guess(double* x, const double* state, int64_t q, int64_t n3, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = j / n3, s = j - blk * n3;
    const int64_t fc = blk / q, i = blk - fc * q;
    x[j] = (i == 0) ? state[fc * n3 + s] : 0.0;
  }
}

__global__ void k_extract_end(double* state, const double* x, int64_t q, int64_t n3, int64_t n) {
  // end of the slab: l_1(1) = 1, l_m(1) = 0 otherwise, so u(t0+dt) = mode 1 = Krylov index 0
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t fc = j / n3, s = j - fc * n3;
    state[j] = x[(fc * q) * n3 + s];
  }
}

int grid1(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

// ||v||^2 (fixed-order reduction, FP64 accumulation).
template <typename S>
int norm2(stm_ctx* c, S* v, int64_t n, double* out) {
  axpy_norm<S>(v, v, 0, 0, Coef16{}, n, c->red_partial, c->red_out, c->stream);
  c->launches += 2;
  STM_CK(cudaMemcpyAsync(c->h_pinned, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  STM_CK(cudaStreamSynchronize(c->stream));
  *out = c->h_pinned[0];
  return STM_OK;
}

// One restart cycle of right-preconditioned GMRES on the unknowns (Sec. 5.4),
// with the basis kept unnormalised: v_i = V_i / alpha_i (alpha_i signed).
// On entry V[0] holds the start vector with v_0 = V[0] / a0 the normalised
// residual r / |r|, |a0| = |r|.  Classical Gram-Schmidt (one fused dot pass,
// one fused update + norm pass), with an optional second pass when the norm
// drops below 1/sqrt(2) of its value before the update.  Returns the number k
// of basis vectors used and the coefficients yc[i] such that the correction
// is P^{-1} sum_{i<k} yc[i] V[i]; *res is the residual norm estimate |g_k|.
// Weights of the iteration-error bound of Sec. 5.3 (Eq. a_posteriori:iteration):
// eta_it^2 = 4 sum_n [(2 t_N/eps_min + dt^2/(2 t_N eps_min)) |R_E|^2_{W'} + (same, mu) |R_H|^2_{W'}],
// with the dual norm on the test space |R|^2_{W'} = R^T M_W^{-1} R and, on
// bricks, M_W = dt diag(G_c) (orthonormal test basis in time and space).  So
// eta-contribution^2 of a slab = |S R|_2^2 with S = diag(sqrt(4 c_f / (dt G_c))).
int build_eta_weights(stm_ctx* c, double dt) {
  if (c->sw64 && c->sw_dt == dt) return STM_OK;
  const double emin = *std::min_element(c->h_eps.begin(), c->h_eps.end());
  const double mmin = *std::min_element(c->h_mu.begin(), c->h_mu.end());
  const double tN = c->opts.t_final;
  const double cf[2] = {2 * tN / emin + dt * dt / (2 * tN * emin), 2 * tN / mmin + dt * dt / (2 * tN * mmin)};
  std::vector<double> w(6 * c->ne);
  std::vector<float> w32(6 * c->ne);
  for (int64_t e = 0; e < c->ne; ++e)
    for (int fc = 0; fc < 6; ++fc) {
      const double mat = fc < 3 ? c->h_eps[e] : c->h_mu[e];
      const double G = c->h_mass[6 * e + fc] / mat;
      w[6 * e + fc] = std::sqrt(4.0 * cf[fc / 3] / (dt * G));
      w32[6 * e + fc] = (float)w[6 * e + fc];
    }
  if (!c->sw64) {
    if (cudaMalloc(&c->sw64, w.size() * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->sw32, w32.size() * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, STM_ENOMEM, "weight allocation failed");
    }
  }
  STM_CK(cudaMemcpy(c->sw64, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
  STM_CK(cudaMemcpy(c->sw32, w32.data(), w32.size() * sizeof(float), cudaMemcpyHostToDevice));
  c->sw_dt = dt;
  return STM_OK;
}

template <typename S>
const S* sw_ptr(stm_ctx* c);
template <>
const double* sw_ptr<double>(stm_ctx* c) { return c->sw64; }
template <>
const float* sw_ptr<float>(stm_ctx* c) { return c->sw32; }

// v <- S v (per-block weights), in place
template <typename S>
void scale_blocks(stm_ctx* c, S* v, const S* w, int64_t n, const int32_t* skip = nullptr) {
  if (c->hp) precond_hp<S>(v, v, w, c->off_test, c->pq, c->ne, c->stream, skip);
  else precond_apply<S>(v, v, w, (int64_t)c->Q * c->N3, n, c->stream, skip);
  c->launches += 1;
}

// The m iterations of one restart cycle of right-preconditioned GMRES (Sec. 5.4) on the
// unknowns, launched without any host synchronisation: the Gram-Schmidt coefficients,
// the Hessenberg column, the Givens rotations and the stop test live in the device
// state c->gst, and every kernel of an iteration is skipped once the cycle has stopped.
// The basis is kept unnormalised: v_i = V_i / alpha_i (alpha_i signed), V[0] holds the
// start vector (set up by gmres_cycle_init).  Classical Gram-Schmidt (one fused dot pass,
// one fused update + norm pass), with an optional second pass when the norm drops below
// 1/sqrt(2) of its value before the update.  At the end st->yc holds the coefficients
// such that the correction is P^{-1} sum_{i<k} yc[i] V[i].
template <typename S>
int gmres_iterations(stm_ctx* c, double dt, S* V, int64_t ldv, S* z, int64_t n) {
  const int m = c->opts.restart;
  const int64_t qn3 = (int64_t)c->Q * c->N3;
  GmresState* st = c->gst;
  const int32_t* skip = &st->skip;
  int rc;
  c->it_marks.assign(m + 1, c->timed.size());
  for (int j = 0; j < m; ++j) {
    c->it_marks[j] = c->timed.size();
    S* W = V + (size_t)(j + 1) * ldv;
    const S* Vj = V + (size_t)j * ldv;
    if (c->geometry != STM_GEOM_BRICK) {  // 3x3 blocks of the (cell-mean) metric mass
      precond_curved<S, S>(z, Vj, 0, 0, nullptr, curved_ptr<S>(c, 3), qn3, c->ne, false, c->stream, skip);
      c->launches += 1;
      if ((rc = linop<S>(c, dt, z, W, skip))) return rc;
    } else {
      // bricks: P^{-1} on load inside the residual kernels (one multiply per unknown in the
      // temporal contraction; the mass term of A P^{-1} v is v itself), no separate pass
      if ((rc = linop_pre<S>(c, dt, Vj, W, skip))) return rc;
    }
    if (c->opts.eta_tol > 0) scale_blocks<S>(c, W, sw_ptr<S>(c), n, skip);  // residual space weighted by S
    multidot<S>(W, V, ldv, j + 1, true, n, c->red_partial, nullptr, c->stream, skip);
    gmres_gs(c->red_partial, st, j, 0, c->stream);
    axpy_norm<S>(W, V, ldv, j + 1, Coef16{}, n, c->red_partial, nullptr, c->stream, skip, st->cc);
    c->launches += 4;
    if (c->opts.reorth) {
      const int32_t* skip2 = &st->skip_reo;
      gmres_after(c->red_partial, st, 1, c->stream);
      multidot<S>(W, V, ldv, j + 1, false, n, c->red_partial, nullptr, c->stream, skip2);
      gmres_gs(c->red_partial, st, j, 1, c->stream);
      axpy_norm<S>(W, V, ldv, j + 1, Coef16{}, n, c->red_partial, nullptr, c->stream, skip2, st->cc);
      c->launches += 4;
    }
    gmres_givens(c->red_partial, st, j, m, c->opts.reorth ? 1 : 0, c->stream);
    c->launches += 1;
  }
  c->it_marks[m] = c->timed.size();
  gmres_backsub(st, m, c->stream);
  c->launches += 1;
  STM_CK(cudaGetLastError());
  return STM_OK;
}

template <typename T>
int ensure_buf(stm_ctx* c, T** p, int64_t* have, int64_t need) {
  if (*have >= need) return STM_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc((void**)p, (size_t)need * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, STM_ENOMEM, "solver workspace allocation failed");
  }
  *have = need;
  return STM_OK;
}

// One restart cycle of the slab solve: the true FP64 residual R(u0, x) and the slab's stop
// test, then (unless it holds) m GMRES iterations and x += P^{-1} sum yc V; no host
// synchronisation.  Mixed precision: the FP32 inner cycle works on the rounded FP64
// residual and the FP64 residual of the next cycle refines it (iterative refinement).
int launch_cycle(stm_ctx* c, double dt, const double* b, bool mixed, int64_t ldv) {
  const int m = c->opts.restart;
  const int64_t n = c->n_test;
  const int64_t qn3 = (int64_t)c->Q * c->N3;
  const bool curved = c->geometry != STM_GEOM_BRICK;  // trilinear or general affine: 3x3 blocks
  const bool inexact = c->opts.eta_tol > 0;
  GmresState* st = c->gst;
  int rc;
  double* R64 = mixed ? c->z : c->V;
  // once the slab has stopped (st->halt), this cycle's kernels are all no-ops
  const int32_t* halt = &st->halt;
  if ((rc = resid64(c, dt, c->x, b, R64, halt))) return rc;
  axpy_norm<double>(R64, R64, 0, 0, Coef16{}, n, c->red_partial, nullptr, c->stream, halt);
  gmres_reduce(c->red_partial, st, 0, c->stream, halt);
  c->launches += 2;
  if (inexact) {  // GMRES then works on the weighted residual S R
    scale_blocks<double>(c, R64, c->sw64, n, halt);
    axpy_norm<double>(R64, R64, 0, 0, Coef16{}, n, c->red_partial, nullptr, c->stream, halt);
    gmres_reduce(c->red_partial, st, 1, c->stream, halt);
    c->launches += 2;
  }
  gmres_outer_check(st, c->stream);
  c->launches += 1;
  if (!mixed) {
    // V[0] = R = -r, so v_0 = V[0] / (-beta)
    gmres_cycle_init(st, inexact ? 1 : 0, 0.0, c->stream);
    c->launches += 1;
    if ((rc = gmres_iterations<double>(c, dt, c->V, ldv, c->z, n))) return rc;
    if (curved) precond_curved<double, double>(c->x, c->V, ldv, 0, nullptr, c->Pinv64, qn3, c->ne, true, c->stream,
                                               nullptr, st);
    else if (c->hp) combine_hp<double, double>(c->x, c->V, ldv, m, Coef16{}, c->inv64, c->off_test, c->pq, c->ne,
                                               c->stream, st);
    else precond_combine<double, double>(c->x, c->V, ldv, m, Coef16{}, c->inv64, qn3, n, c->stream, st);
  } else {
    // FP32 inner GMRES(m) cycle on A d = r, started from the rounded FP64 residual; the inner
    // target is the outer one or what FP32 can resolve (1e-6 of the start), whichever is larger
    convert<float, double>(c->V32, R64, n, c->stream, &st->skip);
    axpy_norm<float>(c->V32, c->V32, 0, 0, Coef16{}, n, c->red_partial, nullptr, c->stream, &st->skip);
    gmres_reduce(c->red_partial, st, 2, c->stream, &st->skip);
    gmres_cycle_init(st, 2, 1e-6, c->stream);
    c->launches += 4;
    if ((rc = gmres_iterations<float>(c, dt, c->V32, ldv, c->z32, n))) return rc;
    if (curved) precond_curved<float, double>(c->x, c->V32, ldv, 0, nullptr, c->Pinv32, qn3, c->ne, true, c->stream,
                                              nullptr, st);
    else if (c->hp) combine_hp<float, double>(c->x, c->V32, ldv, m, Coef16{}, c->inv32, c->off_test, c->pq, c->ne,
                                              c->stream, st);
    else precond_combine<float, double>(c->x, c->V32, ldv, m, Coef16{}, c->inv32, qn3, n, c->stream, st);
  }
  c->launches += 1;
  STM_CK(cudaGetLastError());
  return STM_OK;
}

void drop_cycle_graphs(stm_ctx* c) {
  for (auto& kv : c->cycle_graphs) cudaGraphExecDestroy(kv.second.exec);
  c->cycle_graphs.clear();
}

// Runs `cycles` restart cycles: captured once per (precision, dt, load pointer, cycles) into a
// CUDA graph on the capture stream and replayed on the context stream (directly launched
// while profiling, whose events are recorded around individual kernels).
int run_cycles(stm_ctx* c, double dt, const double* b, bool mixed, int64_t ldv, int cycles) {
  if (c->profiling) {
    for (int k = 0; k < cycles; ++k) {
      const int rc = launch_cycle(c, dt, b, mixed, ldv);
      if (rc) return rc;
    }
    return STM_OK;
  }
  const auto key = std::make_tuple(mixed ? 1 : 0, dt, (const void*)b, cycles);
  auto it = c->cycle_graphs.find(key);
  if (it == c->cycle_graphs.end()) {
    if (!c->cap_stream) STM_CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    if (c->cycle_graphs.size() >= 16) drop_cycle_graphs(c);
    const int64_t l0 = c->launches;
    cudaStream_t orig = c->stream;
    STM_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
    c->stream = c->cap_stream;
    int rc = STM_OK;
    for (int k = 0; k < cycles && !rc; ++k) rc = launch_cycle(c, dt, b, mixed, ldv);
    c->stream = orig;
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g);
    const int64_t count = c->launches - l0;
    c->launches = l0;
    if (rc || ee != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return rc ? rc : fail(c, STM_EDEVICE, std::string("cycle capture: ") + cudaGetErrorString(ee));
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return fail(c, STM_EDEVICE, std::string("cycle graph: ") + cudaGetErrorString(ie));
    stm_ctx::CycleGraph cg;
    cg.exec = ex;
    cg.launches = count;
    it = c->cycle_graphs.emplace(key, cg).first;
  }
  c->launches += it->second.launches;
  STM_CK(cudaGraphLaunch(it->second.exec, c->stream));
  return STM_OK;
}

}  // namespace

extern "C" {

const char* stm_last_error(stm_ctx* c) { return c ? c->err.c_str() : "null context"; }

int32_t stm_create(stm_ctx** out, const stm_mesh* m, const stm_opts* o) {
  if (!out || !m) return STM_EINVAL;
  *out = nullptr;
  stm_ctx* c = new stm_ctx();
  auto bad = [&](int code, const std::string& msg) {
    fprintf(stderr, "stm_create: %s\n", msg.c_str());
    delete c;
    return code;
  };
  if (m->n_elem <= 0 || !m->vert || !m->hex || !m->nbr || !m->p || !m->q || !m->eps || !m->mu)
    return bad(STM_EINVAL, "mesh has missing arrays or no elements");
  c->ne = m->n_elem;
  c->P = m->p[0];
  c->Q = m->q[0];
  c->block = default_block(c->P, c->Q);
  c->h_p.resize(c->ne);
  c->h_q.resize(c->ne);
  for (int64_t e = 0; e < c->ne; ++e) {
    c->h_p[e] = m->p[e];
    c->h_q[e] = m->q[e];
    if (m->p[e] > 7) return bad(STM_EINVAL, "p must be 0..7");
    if (m->q[e] < 1 || m->q[e] > kMaxQ) return bad(STM_EINVAL, "q must be 1..6");
    if (m->p[e] != c->P || m->q[e] != c->Q) c->hp = true;
  }
  c->h_nk.assign(c->ne, 1);
  for (int64_t e = 0; m->nk && e < c->ne; ++e) {
    const int v = m->nk[e];
    if (v != 1 && v != 2 && v != 4 && v != 8) return bad(STM_EINVAL, "N_K must be 1, 2, 4 or 8");
    c->h_nk[e] = v;
    if (v > 1) c->ltr = c->hp = true;  // local refinement in time runs through the per-element kernels
  }
  for (int64_t k = 0; k < 6 * c->ne; ++k)
    if (m->nbr[k] == -2) c->hp = true;  // 2:1 faces run through the per-element-offset kernels
  if (c->ltr) {
    for (int64_t k = 0; k < 6 * c->ne; ++k)
      if (m->nbr[k] == -2) return bad(STM_EUNSUPPORTED, "local refinement in time is not built for 2:1 faces");
    if (o && o->c_diss != 0.0) return bad(STM_EUNSUPPORTED, "the dissipative term needs N_K = 1");
  }
  if (c->hp && m->geometry != STM_GEOM_BRICK)
    return bad(STM_EUNSUPPORTED, "uneven (p, q) and 2:1 faces are handled on brick meshes only");
  if (o && o->c_diss != 0.0) {
    if (!(o->c_diss > 0)) return bad(STM_EINVAL, "c_diss must be >= 0");
    if (m->geometry != STM_GEOM_BRICK) return bad(STM_EUNSUPPORTED, "the dissipative term is built for brick meshes");
    for (int64_t e = 0; e < c->ne; ++e)
      if (m->q[e] != c->Q) return bad(STM_EUNSUPPORTED, "the dissipative term needs a uniform q");
    for (int64_t k = 0; k < 6 * c->ne; ++k)
      if (m->nbr[k] == -2) return bad(STM_EUNSUPPORTED, "the dissipative term is not built for 2:1 faces");
  }
  if (m->n_hang < 0 || (m->n_hang > 0 && !m->hang)) return bad(STM_EINVAL, "bad hang list");
  if (m->geometry != STM_GEOM_BRICK && m->geometry != STM_GEOM_AFFINE && m->geometry != STM_GEOM_TRILINEAR)
    return bad(STM_EINVAL, "unknown geometry");
  // trilinear and general affine elements share the vertex-based set-up (metric, faces)
  const bool curved = m->geometry != STM_GEOM_BRICK;
  const bool affine = m->geometry == STM_GEOM_AFFINE;
  c->geometry = m->geometry;
  c->N = c->P + 1;
  c->N2 = c->N * c->N;
  c->N3 = c->N2 * c->N;
  {
    // per-element block offsets of the trial, test, state and trace layouts
    c->h_off_trial.assign(c->ne + 1, 0);
    c->h_off_test.assign(c->ne + 1, 0);
    c->h_off_state.assign(c->ne + 1, 0);
    c->h_off_tr.assign(c->ne + 1, 0);
    for (int64_t e = 0; e < c->ne; ++e) {
      const int64_t n = c->h_p[e] + 1, n2 = n * n, n3 = n2 * n, q = (int64_t)c->h_nk[e] * c->h_q[e];
      c->h_off_trial[e + 1] = c->h_off_trial[e] + 6 * (q + 1) * n3;
      c->h_off_test[e + 1] = c->h_off_test[e] + 6 * q * n3;
      c->h_off_state[e + 1] = c->h_off_state[e] + 6 * n3;
      c->h_off_tr[e + 1] = c->h_off_tr[e] + 24 * q * n2;
    }
  }
  c->n_trial = c->h_off_trial[c->ne];
  c->n_test = c->h_off_test[c->ne];
  c->n_state = c->h_off_state[c->ne];
  c->n_tr = c->h_off_tr[c->ne];
  if (o) c->opts = *o;
  else {
    c->opts.precision = STM_FP64;
    c->opts.tol = 1e-12;
    c->opts.restart = 10;
    c->opts.max_it = 500;
    c->opts.deterministic = 1;
    c->opts.stream = 0;
    c->opts.reorth = 1;
    c->opts.graph = 1;
  }
  if (c->opts.restart < 1 || c->opts.restart > kMaxDots - 1)
    return bad(STM_EINVAL, "restart must be 1..15");
  // element geometry: vertices of every element; bricks must be axis-aligned boxes
  c->h_x0.resize(3 * c->ne);
  c->h_h.resize(3 * c->ne);
  c->h_mass.resize(6 * c->ne);
  c->h_X8.resize(24 * c->ne);
  for (int64_t e = 0; e < c->ne; ++e) {
    const int64_t* hv = m->hex + 8 * e;
    for (int v = 0; v < 8; ++v) {
      if (hv[v] < 0 || hv[v] >= m->n_vert) return bad(STM_EINVAL, "vertex id out of range");
      for (int d = 0; d < 3; ++d) c->h_X8[24 * e + 3 * v + d] = m->vert[3 * hv[v] + d];
    }
    if (!(m->eps[e] > 0) || !(m->mu[e] > 0)) return bad(STM_EINVAL, "eps and mu must be positive");
    c->h_eps.push_back(m->eps[e]);
    c->h_mu.push_back(m->mu[e]);
    const double* v0 = m->vert + 3 * hv[0];
    const double* v7 = m->vert + 3 * hv[7];
    double h[3];
    for (int d = 0; d < 3; ++d) h[d] = v7[d] - v0[d];
    if (curved) {
      for (int d = 0; d < 3; ++d) {
        c->h_x0[3 * e + d] = v0[d];
        c->h_h[3 * e + d] = h[d];
        c->h_mass[6 * e + d] = 1.0;
        c->h_mass[6 * e + 3 + d] = 1.0;
      }
      if (affine) {
        // parallelepiped: DF = [x_1 - x_0, x_2 - x_0, x_4 - x_0] and x_v = x_0 + DF bits(v)
        double DF[3][3];
        for (int d = 0; d < 3; ++d)
          for (int k = 0; k < 3; ++k) DF[d][k] = m->vert[3 * hv[1 << k] + d] - v0[d];
        double scale = 0.0;
        for (int d = 0; d < 3; ++d)
          for (int k = 0; k < 3; ++k) scale = std::max(scale, std::fabs(DF[d][k]));
        for (int v = 0; v < 8; ++v)
          for (int d = 0; d < 3; ++d) {
            const double x = v0[d] + DF[d][0] * (v & 1) + DF[d][1] * ((v >> 1) & 1) + DF[d][2] * ((v >> 2) & 1);
            if (std::fabs(m->vert[3 * hv[v] + d] - x) > 1e-10 * scale)
              return bad(STM_EUNSUPPORTED, "element is not a parallelepiped (use STM_GEOM_TRILINEAR)");
          }
        // G = |J| DF^{-1} DF^{-T} = adj(DF) adj(DF)^T / J, J = det DF
        double A[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            A[j][i] = DF[i1][j1] * DF[i2][j2] - DF[i1][j2] * DF[i2][j1];  // cofactor transpose
          }
        const double J = DF[0][0] * A[0][0] + DF[0][1] * A[1][0] + DF[0][2] * A[2][0];
        if (!(J > 0)) return bad(STM_EINVAL, "element map with non-positive Jacobian");
        const int pr[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
        double g[6];
        for (int k = 0; k < 6; ++k) {
          const int a = pr[k][0], b = pr[k][1];
          g[k] = (A[a][0] * A[b][0] + A[a][1] * A[b][1] + A[a][2] * A[b][2]) / J;
        }
        for (int k = 0; k < 6; ++k) c->h_mass3.push_back(m->eps[e] * g[k]);
        for (int k = 0; k < 6; ++k) c->h_mass3.push_back(m->mu[e] * g[k]);
      }
      continue;
    }
    for (int d = 0; d < 3; ++d)
      if (!(h[d] > 0)) return bad(STM_EINVAL, "element with non-positive extent (vertex order)");
    const double tol = 1e-10 * std::max(h[0], std::max(h[1], h[2]));
    for (int v = 0; v < 8; ++v) {
      const double* x = m->vert + 3 * hv[v];
      const int bit[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
      for (int d = 0; d < 3; ++d)
        if (std::fabs(x[d] - (v0[d] + bit[d] * h[d])) > tol)
          return bad(STM_EUNSUPPORTED, "element is not an axis-aligned box (use STM_GEOM_TRILINEAR)");
    }
    const double G[3] = {h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2]};
    for (int d = 0; d < 3; ++d) {
      c->h_x0[3 * e + d] = v0[d];
      c->h_h[3 * e + d] = h[d];
      c->h_mass[6 * e + d] = m->eps[e] * G[d];
      c->h_mass[6 * e + 3 + d] = m->mu[e] * G[d];
    }
  }
  std::vector<int32_t> nb(6 * c->ne);
  for (int64_t e = 0; e < c->ne; ++e) {
    for (int f = 0; f < 6; ++f) {
      const int64_t e2 = m->nbr[6 * e + f];
      if (e2 < -2 || e2 >= c->ne) return bad(STM_EINVAL, "neighbour id out of range");
      if (e2 == -2 && curved) return bad(STM_EUNSUPPORTED, "2:1 faces are handled on brick meshes only");
      if (e2 >= 0) {
        const int d = f / 2, s = f % 2;
        if (m->nbr[6 * e2 + (2 * d + 1 - s)] != e) return bad(STM_EINVAL, "neighbour lists are not symmetric");
        bool ok = true;
        if (curved) {
          // conforming, same parametrisation: face (d, s) of e and face (d, 1-s) of e2 have the
          // same four vertices in the same reference order
          int k1 = 0;
          int64_t va[4], vb[4];
          for (int v = 0; v < 8; ++v) {
            if (((v >> d) & 1) == s) va[k1++] = m->hex[8 * e + v];
          }
          int k2 = 0;
          for (int v = 0; v < 8; ++v) {
            if (((v >> d) & 1) == 1 - s) vb[k2++] = m->hex[8 * e2 + v];
          }
          for (int k = 0; k < 4; ++k) ok = ok && va[k] == vb[k];
        } else {
          // conforming: the two boxes share the whole face
          const double tol = 1e-10 * c->h_h[3 * e + d];
          const double face = c->h_x0[3 * e + d] + (s ? c->h_h[3 * e + d] : 0.0);
          const double face2 = c->h_x0[3 * e2 + d] + (s ? 0.0 : c->h_h[3 * e2 + d]);
          ok = std::fabs(face - face2) <= tol;
          for (int t = 0; t < 3; ++t)
            if (t != d)
              ok = ok && std::fabs(c->h_x0[3 * e + t] - c->h_x0[3 * e2 + t]) <= tol &&
                   std::fabs(c->h_h[3 * e + t] - c->h_h[3 * e2 + t]) <= tol;
        }
        if (!ok) return bad(STM_EUNSUPPORTED, "non-conforming face (hanging nodes) are not handled");
      }
      nb[6 * e + f] = (int32_t)e2;
    }
  }
  c->h_nbr = nb;
  // 2:1 faces: validate the hang rows and build one slot per receiving element face
  std::vector<int32_t> hslot(6 * c->ne, -1), s_elem, s_face, s_kind, s_src, s_srcface, s_quad;
  std::vector<int64_t> hoff;
  {
    auto slot_of = [&](int64_t e, int f, int kind) -> int {
      int32_t& sl = hslot[6 * e + f];
      if (sl < 0) {
        sl = (int32_t)s_elem.size();
        s_elem.push_back((int32_t)e);
        s_face.push_back(f);
        s_kind.push_back(kind);
        for (int k = 0; k < 4; ++k) {
          s_src.push_back(-1);
          s_srcface.push_back(-1);
          s_quad.push_back(-1);
        }
      }
      return s_kind[sl] == kind ? sl : -1;
    };
    for (int64_t r = 0; r < m->n_hang; ++r) {
      const int64_t* H = m->hang + 6 * r;
      const int64_t eb = H[0], es = H[2];
      const int fb = (int)H[1], fs = (int)H[3], u = (int)H[4], v = (int)H[5];
      if (eb < 0 || eb >= c->ne || es < 0 || es >= c->ne || fb < 0 || fb > 5 || fs < 0 || fs > 5 || (u & ~1) ||
          (v & ~1) || fb / 2 != fs / 2 || fb % 2 == fs % 2 || m->nbr[6 * eb + fb] != -2 || m->nbr[6 * es + fs] != -2)
        return bad(STM_EINVAL, "inconsistent row in the hang list");
      const int d = fb / 2, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      const double* xb = &c->h_x0[3 * eb];
      const double* hb = &c->h_h[3 * eb];
      const double* xs = &c->h_x0[3 * es];
      const double* hs = &c->h_h[3 * es];
      const double tol = 1e-9 * hb[t1];
      const double pb = xb[d] + (fb % 2 ? hb[d] : 0.0), ps = xs[d] + (fs % 2 ? hs[d] : 0.0);
      if (std::fabs(pb - ps) > tol || std::fabs(2 * hs[t1] - hb[t1]) > tol || std::fabs(2 * hs[t2] - hb[t2]) > tol ||
          std::fabs(xs[t1] - (xb[t1] + u * hs[t1])) > tol || std::fabs(xs[t2] - (xb[t2] + v * hs[t2])) > tol)
        return bad(STM_EINVAL, "hang row does not describe a quarter of the coarse face");
      const int sb = slot_of(eb, fb, 1), ss = slot_of(es, fs, 0);
      if (sb < 0 || ss < 0) return bad(STM_EINVAL, "a face is both coarse and fine side of 2:1 faces");
      const int q4 = u | (v << 1);
      if (s_src[4 * sb + q4] >= 0 || s_src[4 * ss] >= 0) return bad(STM_EINVAL, "duplicate row in the hang list");
      s_src[4 * sb + q4] = (int32_t)es;
      s_srcface[4 * sb + q4] = fs;
      s_quad[4 * sb + q4] = q4;
      s_src[4 * ss] = (int32_t)eb;
      s_srcface[4 * ss] = fb;
      s_quad[4 * ss] = q4;
    }
    for (int64_t k = 0; k < 6 * c->ne; ++k)
      if (m->nbr[k] == -2 && hslot[k] < 0) return bad(STM_EINVAL, "a face marked -2 has no row in the hang list");
    for (size_t sl = 0; sl < s_elem.size(); ++sl)
      for (int k = 0; k < (s_kind[sl] ? 4 : 1); ++k)
        if (s_src[4 * sl + k] < 0) return bad(STM_EINVAL, "a coarse 2:1 face lacks one of its four fine faces");
    int64_t off = 0;
    for (size_t sl = 0; sl < s_elem.size(); ++sl) {
      hoff.push_back(off);
      const int64_t n = c->h_p[s_elem[sl]] + 1;
      off += 4LL * c->h_q[s_elem[sl]] * n * n;
    }
    c->n_slots = (int64_t)s_elem.size();
    c->n_hbuf = off;
    // transfer integrals T[u][j][n] = int_0^1 L_n((eta + u) / 2) L_j(eta) d eta (exact Gauss rule)
    std::vector<double> xg, wg;
    gauss01(10, xg, wg);
    for (int u = 0; u < 2; ++u)
      for (size_t g = 0; g < xg.size(); ++g) {
        double Lj[8], Ln[8];
        legendre01(8, xg[g], Lj);
        legendre01(8, 0.5 * (xg[g] + u), Ln);
        for (int j = 0; j < 8; ++j)
          for (int n = 0; n < 8; ++n) c->Tm[u][j][n] += wg[g] * Ln[n] * Lj[j];
      }
  }
  if (cudaGetDevice(&c->device) != cudaSuccess) return bad(STM_EDEVICE, "no CUDA device");
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || c->sms < 1)
    return bad(STM_EDEVICE, "device attribute query failed");
  // 0 is the CUDA default stream, so work is ordered with a caller that uses it
  c->stream = (cudaStream_t)(intptr_t)c->opts.stream;
  std::vector<float> m32(c->h_mass.begin(), c->h_mass.end());
  std::vector<double> i64(c->h_mass.size());
  for (size_t k = 0; k < i64.size(); ++k) i64[k] = 1.0 / c->h_mass[k];
  std::vector<float> i32(i64.begin(), i64.end());
  bool ok = cudaMalloc(&c->nbr, nb.size() * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&c->mass64, c->h_mass.size() * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->mass32, m32.size() * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->inv64, i64.size() * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->inv32, i32.size() * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&c->state, c->n_state * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->red_partial, (kMaxDots + 1) * kRedBlocks * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->red_out, (kMaxDots + 1) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->wait_err, sizeof(int)) == cudaSuccess && cudaMemset(c->wait_err, 0, sizeof(int)) == cudaSuccess &&
            cudaMallocHost(&c->h_pinned, (kMaxDots + 1) * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    stm_destroy(c);
    fprintf(stderr, "stm_create: device allocation failed\n");
    return STM_ENOMEM;
  }
  cudaMemcpy(c->nbr, nb.data(), nb.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  cudaMemcpy(c->mass64, c->h_mass.data(), c->h_mass.size() * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(c->mass32, m32.data(), m32.size() * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(c->inv64, i64.data(), i64.size() * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(c->inv32, i32.data(), i32.size() * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemset(c->state, 0, c->n_state * sizeof(double));
  // vertices (load kernel, curved metric) and, for curved elements, the metric at the Gauss points
  ok = cudaMalloc(&c->X8, c->h_X8.size() * sizeof(double)) == cudaSuccess;
  if (ok) cudaMemcpy(c->X8, c->h_X8.data(), c->h_X8.size() * sizeof(double), cudaMemcpyHostToDevice);
  {
    std::vector<double> xq, wq;
    gauss01(c->P + 2, xq, wq);
    for (int g = 0; g < c->P + 2; ++g) {
      c->ct.xq[g] = xq[g];
      c->ct.wq[g] = wq[g];
      double L[kMaxN];
      legendre01(c->N, xq[g], L);
      for (int j = 0; j < c->N; ++j) c->ct.Lq[j][g] = L[j];
    }
  }
  if (ok && curved) {
    const int64_t nq3 = (int64_t)(c->P + 2) * (c->P + 2) * (c->P + 2);
    std::vector<float> e32(m->eps, m->eps + c->ne), m32b(m->mu, m->mu + c->ne);
    int* bad_d = nullptr;
    ok = cudaMalloc(&c->eps64, c->ne * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&c->mu64, c->ne * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&c->eps32, c->ne * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&c->mu32, c->ne * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&c->Gw64, c->ne * 6 * nq3 * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&c->Gw32, c->ne * 6 * nq3 * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&c->Pinv64, c->ne * 18 * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&c->Pinv32, c->ne * 18 * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&c->el, c->ne * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&bad_d, sizeof(int)) == cudaSuccess;
    if (ok) {
      cudaMemcpy(c->eps64, m->eps, c->ne * sizeof(double), cudaMemcpyHostToDevice);
      cudaMemcpy(c->mu64, m->mu, c->ne * sizeof(double), cudaMemcpyHostToDevice);
      cudaMemcpy(c->eps32, e32.data(), c->ne * sizeof(float), cudaMemcpyHostToDevice);
      cudaMemcpy(c->mu32, m32b.data(), c->ne * sizeof(float), cudaMemcpyHostToDevice);
      cudaMemset(bad_d, 0, sizeof(int));
      launch_metric(c->P, c->X8, c->eps64, c->mu64, c->ne, c->ct, c->Gw64, c->Pinv64, bad_d, 0);
      convert<float, double>(c->Gw32, c->Gw64, c->ne * 6 * nq3, 0);
      convert<float, double>(c->Pinv32, c->Pinv64, c->ne * 18, 0);
      int bad_h = 0;
      cudaMemcpy(&bad_h, bad_d, sizeof(int), cudaMemcpyDeviceToHost);
      cudaFree(bad_d);
      if (!affine) {
        ok = cudaMalloc(&c->tc_err, sizeof(int)) == cudaSuccess;
        if (ok) cudaMemset(c->tc_err, 0, sizeof(int));
      }
      if (affine) {
        std::vector<float> m3(c->h_mass3.begin(), c->h_mass3.end());
        ok = cudaMalloc(&c->mass3_64, c->h_mass3.size() * sizeof(double)) == cudaSuccess &&
             cudaMalloc(&c->mass3_32, m3.size() * sizeof(float)) == cudaSuccess;
        if (ok) {
          cudaMemcpy(c->mass3_64, c->h_mass3.data(), c->h_mass3.size() * sizeof(double), cudaMemcpyHostToDevice);
          cudaMemcpy(c->mass3_32, m3.data(), m3.size() * sizeof(float), cudaMemcpyHostToDevice);
        }
      }
      if (bad_h) {
        stm_destroy(c);
        fprintf(stderr, "stm_create: an element map has a non-positive Jacobian\n");
        return STM_EINVAL;
      }
    }
  }
  if (!ok || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    stm_destroy(c);
    fprintf(stderr, "stm_create: device setup failed\n");
    return ok ? STM_EDEVICE : STM_ENOMEM;
  }
  if (c->hp) {
    std::vector<uint8_t> pq(c->ne);
    for (int64_t e = 0; e < c->ne; ++e) pq[e] = (uint8_t)(c->h_p[e] | (c->h_q[e] << 4));
    bool okh = cudaMalloc(&c->pq, c->ne) == cudaSuccess &&
               cudaMalloc(&c->off_trial, (c->ne + 1) * sizeof(int64_t)) == cudaSuccess &&
               cudaMalloc(&c->off_test, (c->ne + 1) * sizeof(int64_t)) == cudaSuccess &&
               cudaMalloc(&c->off_state, (c->ne + 1) * sizeof(int64_t)) == cudaSuccess &&
               cudaMalloc(&c->off_tr, (c->ne + 1) * sizeof(int64_t)) == cudaSuccess &&
               cudaMalloc(&c->el, c->ne * sizeof(double)) == cudaSuccess;
    // (p, q) classes, element lists in mesh order
    auto lg2 = [](int v) { return v == 1 ? 0 : (v == 2 ? 1 : (v == 4 ? 2 : 3)); };
    std::vector<std::vector<int32_t>> lists(8 * (kMaxQ + 1) * 4);
    for (int64_t e = 0; e < c->ne; ++e)
      lists[(c->h_p[e] * (kMaxQ + 1) + c->h_q[e]) * 4 + lg2(c->h_nk[e])].push_back((int32_t)e);
    for (int pp = 0; pp < 8 && okh; ++pp)
      for (int qq = 1; qq <= kMaxQ && okh; ++qq)
        for (int lk = 0; lk < 4 && okh; ++lk) {
          const auto& L = lists[(pp * (kMaxQ + 1) + qq) * 4 + lk];
          if (L.empty()) continue;
          stm_ctx::Class cl{pp, qq, (int64_t)L.size(), nullptr, default_block(pp, qq)};
          cl.NK = 1 << lk;
          okh = cudaMalloc(&cl.elist, L.size() * sizeof(int32_t)) == cudaSuccess;
          if (okh) cudaMemcpy(cl.elist, L.data(), L.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
          c->classes.push_back(cl);
        }
    if (okh && c->ltr) {
      // per-element log2 N_K and the temporal transfer matrices M^{r,o}[a][b] =
      // int_0^1 L_a(s) L_b((o + s) / r) ds by Gauss quadrature (exact: degree <= 2 kMaxQ)
      std::vector<uint8_t> nkl(c->ne);
      for (int64_t e = 0; e < c->ne; ++e) nkl[e] = (uint8_t)lg2(c->h_nk[e]);
      std::vector<double> tm(14 * kMaxQ * kMaxQ, 0.0), xg, wg;
      gauss01(kMaxQ + 1, xg, wg);
      for (int r = 2; r <= 8; r *= 2)
        for (int oo = 0; oo < r; ++oo)
          for (size_t g = 0; g < xg.size(); ++g) {
            double La[kMaxN], Lb[kMaxN];
            legendre01(kMaxQ, xg[g], La);
            legendre01(kMaxQ, (oo + xg[g]) / r, Lb);
            for (int aa = 0; aa < kMaxQ; ++aa)
              for (int bb = 0; bb < kMaxQ; ++bb) tm[(tmat_index(r, oo) * kMaxQ + aa) * kMaxQ + bb] += wg[g] * La[aa] * Lb[bb];
          }
      std::vector<float> tm32(tm.begin(), tm.end());
      okh = cudaMalloc(&c->nkl, c->ne) == cudaSuccess &&
            cudaMalloc(&c->tmat64, tm.size() * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->tmat32, tm.size() * sizeof(float)) == cudaSuccess;
      if (okh) {
        cudaMemcpy(c->nkl, nkl.data(), c->ne, cudaMemcpyHostToDevice);
        cudaMemcpy(c->tmat64, tm.data(), tm.size() * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(c->tmat32, tm32.data(), tm32.size() * sizeof(float), cudaMemcpyHostToDevice);
      }
    }
    if (okh && c->n_slots > 0) {
      const size_t ns = (size_t)c->n_slots;
      okh = cudaMalloc(&c->hslot, 6 * c->ne * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&c->s_elem, ns * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&c->s_face, ns * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&c->s_kind, ns * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&c->s_src, 4 * ns * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&c->s_srcface, 4 * ns * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&c->s_quad, 4 * ns * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&c->hoff, ns * sizeof(int64_t)) == cudaSuccess &&
            cudaMalloc(&c->hbuf64, c->n_hbuf * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&c->hbuf32, c->n_hbuf * sizeof(float)) == cudaSuccess;
      if (okh) {
        cudaMemcpy(c->hslot, hslot.data(), 6 * c->ne * sizeof(int32_t), cudaMemcpyHostToDevice);
        cudaMemcpy(c->s_elem, s_elem.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice);
        cudaMemcpy(c->s_face, s_face.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice);
        cudaMemcpy(c->s_kind, s_kind.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice);
        cudaMemcpy(c->s_src, s_src.data(), 4 * ns * sizeof(int32_t), cudaMemcpyHostToDevice);
        cudaMemcpy(c->s_srcface, s_srcface.data(), 4 * ns * sizeof(int32_t), cudaMemcpyHostToDevice);
        cudaMemcpy(c->s_quad, s_quad.data(), 4 * ns * sizeof(int32_t), cudaMemcpyHostToDevice);
        cudaMemcpy(c->hoff, hoff.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice);
      }
    }
    if (okh) {
      cudaMemcpy(c->pq, pq.data(), c->ne, cudaMemcpyHostToDevice);
      cudaMemcpy(c->off_trial, c->h_off_trial.data(), (c->ne + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
      cudaMemcpy(c->off_test, c->h_off_test.data(), (c->ne + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
      cudaMemcpy(c->off_state, c->h_off_state.data(), (c->ne + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
      cudaMemcpy(c->off_tr, c->h_off_tr.data(), (c->ne + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    }
    if (!okh || cudaGetLastError() != cudaSuccess) {
      cudaGetLastError();
      stm_destroy(c);
      fprintf(stderr, "stm_create: device setup of the (p, q) classes failed\n");
      return STM_ENOMEM;
    }
  }
  if (c->opts.c_diss > 0) {
    // D_h coefficients: alpha_E = c / {sqrt(mu/eps)}, alpha_H = c / {sqrt(eps/mu)} on interior
    // faces; alpha_E = c sqrt(eps/mu) of the element and no H term on PEC faces.  On a brick the
    // tangential product <E_c, v_c> over a face normal to a is (h_b / h_c) times the reference one.
    std::vector<double> k64(24 * c->ne);
    for (int64_t e = 0; e < c->ne; ++e) {
      const double Ze = std::sqrt(c->h_mu[e] / c->h_eps[e]);
      for (int face = 0; face < 6; ++face) {
        const int a = face / 2;
        const int32_t e2 = c->h_nbr[6 * e + face];
        double al[2];
        if (e2 >= 0) {
          const double Z2 = std::sqrt(c->h_mu[e2] / c->h_eps[e2]);
          al[0] = c->opts.c_diss / (0.5 * (Ze + Z2));
          al[1] = c->opts.c_diss / (0.5 * (1.0 / Ze + 1.0 / Z2));
        } else {
          al[0] = c->opts.c_diss / Ze;
          al[1] = 0.0;
        }
        for (int bc = 0; bc < 2; ++bc) {
          const int cc = (a == 0) ? bc + 1 : (a == 1 ? 2 * bc : bc), bb = 3 - a - cc;
          const double geo = c->h_h[3 * e + bb] / c->h_h[3 * e + cc];
          for (int f = 0; f < 2; ++f) k64[e * 24 + f * 12 + face * 2 + bc] = al[f] * geo;
        }
      }
    }
    std::vector<float> k32(k64.begin(), k64.end());
    c->h_kap = k64;
    if (cudaMalloc(&c->kap64, k64.size() * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->kap32, k32.size() * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      stm_destroy(c);
      fprintf(stderr, "stm_create: allocation of the dissipation coefficients failed\n");
      return STM_ENOMEM;
    }
    cudaMemcpy(c->kap64, k64.data(), k64.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->kap32, k32.data(), k32.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (curved) {  // the diagonal brick factors do not apply
    cudaFree(c->mass64);
    cudaFree(c->mass32);
    c->mass64 = nullptr;
    c->mass32 = nullptr;
  }
  *out = c;
  return STM_OK;
}

int32_t stm_destroy(stm_ctx* c) {
  if (!c) return STM_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  void* ptrs[] = {c->nbr,     c->mass64,  c->mass32, c->y64,   c->tr64, c->y32, c->tr32,
                  c->state,   c->red_partial, c->red_out, c->tmp_in, c->tmp_out, c->tmp_op, c->V, c->z,
                  c->x,       c->V32,     c->z32,    c->inv64, c->inv32, c->X8, c->eps64, c->mu64,
                  c->eps32,   c->mu32,    c->Gw64,   c->Gw32,  c->Pinv64, c->Pinv32, c->el, c->load64, c->load32,
                  c->sw64,    c->sw32,    c->kap64,  c->kap32, c->nkl,    c->tmat64, c->tmat32,
                  c->mass3_64, c->mass3_32, c->tc_err, c->wait_err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  void* hp_ptrs[] = {c->pq,     c->off_trial, c->off_test, c->off_state, c->off_tr, c->hslot,  c->s_elem,
                     c->s_face, c->s_kind,    c->s_src,    c->s_srcface, c->s_quad, c->hoff,   c->hbuf64,
                     c->hbuf32};
  for (void* p : hp_ptrs)
    if (p) cudaFree(p);
  for (auto& k : c->classes)
    if (k.elist) cudaFree(k.elist);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  drop_cycle_graphs(c);
  if (c->gst) cudaFree(c->gst);
  if (c->h_gst) cudaFreeHost(c->h_gst);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (int k = 0; k < stm_ctx::kAux; ++k) {
    if (c->aux[k]) cudaStreamDestroy(c->aux[k]);
    if (c->join_ev[k]) cudaEventDestroy(c->join_ev[k]);
  }
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return STM_OK;
}

int32_t stm_sizes(stm_ctx* c, int64_t* n_trial, int64_t* n_test, int64_t* n_state) {
  if (!c) return STM_EINVAL;
  if (n_trial) *n_trial = c->n_trial;
  if (n_test) *n_test = c->n_test;
  if (n_state) *n_state = c->n_state;
  return STM_OK;
}

int32_t stm_residual_apply(stm_ctx* c, double t0, double dt, const void* U, void* R, int32_t prec, int32_t mem) {
  if (!c || !U || !R) return STM_EINVAL;
  if (!(dt > 0)) return fail(c, STM_EINVAL, "dt must be positive");
  if (prec != STM_FP64 && prec != STM_FP32) return fail(c, STM_EINVAL, "prec must be STM_FP64 or STM_FP32");
  if (mem != STM_MEM_HOST && mem != STM_MEM_DEVICE) return fail(c, STM_EINVAL, "bad memory kind");
  const size_t es = prec == STM_FP64 ? sizeof(double) : sizeof(float);
  const void* Ud = U;
  void* Rd = R;
  if (mem == STM_MEM_HOST) {
    int rc = ensure(c, &c->tmp_in, &c->tmp_in_bytes, c->n_trial * es);
    if (!rc) rc = ensure(c, &c->tmp_out, &c->tmp_out_bytes, c->n_test * es);
    if (rc) return rc;
    STM_CK(cudaMemcpyAsync(c->tmp_in, U, c->n_trial * es, cudaMemcpyHostToDevice, c->stream));
    Ud = c->tmp_in;
    Rd = c->tmp_out;
  }
  const double* b = nullptr;
  int rc = build_load(c, t0, dt, &b);
  if (rc) return rc;
  if (prec == STM_FP64) {
    const double* u = (const double*)Ud;
    rc = apply<double>(c, dt, u, L_TRIAL, u, L_TRIAL, b, (double*)Rd);
  } else {
    const float* u = (const float*)Ud;
    rc = apply<float>(c, dt, u, L_TRIAL, u, L_TRIAL, b ? c->load32 : nullptr, (float*)Rd);
  }
  if (rc) return rc;
  if (mem == STM_MEM_HOST) {
    STM_CK(cudaMemcpyAsync(R, c->tmp_out, c->n_test * es, cudaMemcpyDeviceToHost, c->stream));
    STM_CK(cudaStreamSynchronize(c->stream));
  }
  STM_CK(cudaGetLastError());
  return STM_OK;
}

int32_t stm_operator_apply(stm_ctx* c, double dt, const void* V, void* W, int32_t pre, int32_t prec, int32_t mem) {
  if (!c || !V || !W) return STM_EINVAL;
  if (!(dt > 0)) return fail(c, STM_EINVAL, "dt must be positive");
  if (prec != STM_FP64 && prec != STM_FP32) return fail(c, STM_EINVAL, "prec must be STM_FP64 or STM_FP32");
  if (mem != STM_MEM_HOST && mem != STM_MEM_DEVICE) return fail(c, STM_EINVAL, "bad memory kind");
  if (pre != 0 && pre != 1) return fail(c, STM_EINVAL, "pre must be 0 or 1");
  const size_t es = prec == STM_FP64 ? sizeof(double) : sizeof(float);
  const void* Vd = V;
  void* Wd = W;
  if (mem == STM_MEM_HOST) {
    int rc = ensure(c, &c->tmp_in, &c->tmp_in_bytes, c->n_test * es);
    if (!rc) rc = ensure(c, &c->tmp_out, &c->tmp_out_bytes, c->n_test * es);
    if (rc) return rc;
    STM_CK(cudaMemcpyAsync(c->tmp_in, V, c->n_test * es, cudaMemcpyHostToDevice, c->stream));
    Vd = c->tmp_in;
    Wd = c->tmp_out;
  }
  auto run = [&](auto tag) -> int {
    using S = decltype(tag);
    const S* v = (const S*)Vd;
    S* w = (S*)Wd;
    if (!pre) return linop<S>(c, dt, v, w);
    if (c->geometry != STM_GEOM_BRICK) {
      // 3x3 blocks of the (cell-mean) metric mass, then the operator, as in the GMRES cycle
      int rc = ensure(c, &c->tmp_op, &c->tmp_op_bytes, c->n_test * sizeof(S));
      if (rc) return rc;
      S* z = (S*)c->tmp_op;
      precond_curved<S, S>(z, v, 0, 0, nullptr, curved_ptr<S>(c, 3), (int64_t)c->Q * c->N3, c->ne, false,
                           c->stream);
      c->launches += 1;
      return linop<S>(c, dt, z, w);
    }
    return linop_pre<S>(c, dt, v, w);
  };
  int rc = prec == STM_FP64 ? run(double{}) : run(float{});
  if (!rc && prec == STM_FP32 && pre) rc = check_wait_err(c);
  if (rc) return rc;
  if (mem == STM_MEM_HOST) {
    STM_CK(cudaMemcpyAsync(W, c->tmp_out, c->n_test * es, cudaMemcpyDeviceToHost, c->stream));
    STM_CK(cudaStreamSynchronize(c->stream));
  }
  STM_CK(cudaGetLastError());
  return STM_OK;
}

int32_t stm_set_state(stm_ctx* c, double t, const void* u, int32_t mem) {
  if (!c || !u) return STM_EINVAL;
  if (mem == STM_MEM_HOST) {
    int rc = host_transfer(c, c->state, (const double*)u, c->n_state, true);
    if (rc) return rc;
  } else {
    STM_CK(cudaMemcpyAsync(c->state, u, c->n_state * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  }
  STM_CK(cudaStreamSynchronize(c->stream));
  c->t = t;
  return STM_OK;
}

int32_t stm_get_state(stm_ctx* c, double* t, void* u, int32_t mem) {
  if (!c || !u) return STM_EINVAL;
  if (mem == STM_MEM_HOST) {
    int rc = host_transfer(c, (double*)u, c->state, c->n_state, false);
    if (rc) return rc;
  } else {
    STM_CK(cudaMemcpyAsync(u, c->state, c->n_state * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  }
  STM_CK(cudaStreamSynchronize(c->stream));
  if (t) *t = c->t;
  return STM_OK;
}

}  // extern "C"

// Covariant L2 projection on trilinear elements: mat_f M_G u = mat_f (F, v) per
// element, with the metric mass M_G of the residual (G = |J| DF^{-1} DF^{-T} at the
// (p+2)^3 Gauss points) and the right side (F, v) = sum_g w_g (adj(DF) F)_c phi_s by
// the same rule.  The element systems are solved together by conjugate gradients
// on the device (the metric-mass kernel as operator, the cell-mean blocks as
// preconditioner); the result is the state.
int project_curved(stm_ctx* c, double t, stm_field_fn E0, stm_field_fn H0, void* user) {
  const int P = c->P, N = c->N, N3 = c->N3, nq = P + 2, nq3 = nq * nq * nq;
  const int64_t n = c->n_state;
  std::vector<double> xq, wq, Lq(nq * N);
  gauss01(nq, xq, wq);
  for (int g = 0; g < nq; ++g) legendre01(N, xq[g], &Lq[g * N]);
  std::vector<double> rhs(n, 0.0), pts, val, adj, F(3 * (size_t)nq3), G1, G2;
  const int64_t chunk = std::max<int64_t>(1, (1 << 20) / nq3);
  for (int64_t e0 = 0; e0 < c->ne; e0 += chunk) {
    const int64_t e1 = std::min<int64_t>(c->ne, e0 + chunk), cnt = e1 - e0;
    pts.resize(3 * cnt * nq3);
    val.resize(3 * cnt * nq3);
    adj.resize(9 * cnt * nq3);
    for (int64_t e = e0; e < e1; ++e) {
      const double* X = &c->h_X8[24 * e];
      for (int g = 0; g < nq3; ++g) {
        const double xh[3] = {xq[g % nq], xq[(g / nq) % nq], xq[g / (nq * nq)]};
        double x[3] = {0, 0, 0}, DF[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int v = 0; v < 8; ++v) {
          const int bit[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
          double fa[3], dfa[3];
          for (int a = 0; a < 3; ++a) {
            fa[a] = bit[a] ? xh[a] : 1.0 - xh[a];
            dfa[a] = bit[a] ? 1.0 : -1.0;
          }
          const double Nv = fa[0] * fa[1] * fa[2];
          const double dN[3] = {dfa[0] * fa[1] * fa[2], fa[0] * dfa[1] * fa[2], fa[0] * fa[1] * dfa[2]};
          for (int i = 0; i < 3; ++i) {
            x[i] += Nv * X[3 * v + i];
            for (int j = 0; j < 3; ++j) DF[i][j] += X[3 * v + i] * dN[j];
          }
        }
        const int64_t k = (e - e0) * nq3 + g;
        for (int i = 0; i < 3; ++i) pts[3 * k + i] = x[i];
        double* A = &adj[9 * k];  // adj(DF) = |J| DF^{-1}
        A[0] = DF[1][1] * DF[2][2] - DF[1][2] * DF[2][1];
        A[1] = DF[0][2] * DF[2][1] - DF[0][1] * DF[2][2];
        A[2] = DF[0][1] * DF[1][2] - DF[0][2] * DF[1][1];
        A[3] = DF[1][2] * DF[2][0] - DF[1][0] * DF[2][2];
        A[4] = DF[0][0] * DF[2][2] - DF[0][2] * DF[2][0];
        A[5] = DF[0][2] * DF[1][0] - DF[0][0] * DF[1][2];
        A[6] = DF[1][0] * DF[2][1] - DF[1][1] * DF[2][0];
        A[7] = DF[0][1] * DF[2][0] - DF[0][0] * DF[2][1];
        A[8] = DF[0][0] * DF[1][1] - DF[0][1] * DF[1][0];
      }
    }
    for (int f = 0; f < 2; ++f) {
      stm_field_fn fn = f == 0 ? E0 : H0;
      if (!fn) continue;
      fn(user, cnt * nq3, pts.data(), val.data());
      for (int64_t e = e0; e < e1; ++e) {
        const double mat = f == 0 ? c->h_eps[e] : c->h_mu[e];
        for (int g = 0; g < nq3; ++g) {
          const int64_t k = (e - e0) * nq3 + g;
          const double* A = &adj[9 * k];
          const double* v = &val[3 * k];
          const double w = mat * wq[g % nq] * wq[(g / nq) % nq] * wq[g / (nq * nq)];
          for (int cc = 0; cc < 3; ++cc) F[(size_t)cc * nq3 + g] = w * (A[3 * cc] * v[0] + A[3 * cc + 1] * v[1] + A[3 * cc + 2] * v[2]);
        }
        for (int cc = 0; cc < 3; ++cc) {  // three 1-D contractions onto phi_s
          const double* f0 = &F[(size_t)cc * nq3];
          G1.assign((size_t)nq * nq * N, 0.0);
          for (int gz = 0; gz < nq; ++gz)
            for (int gy = 0; gy < nq; ++gy)
              for (int j = 0; j < N; ++j) {
                double acc = 0.0;
                for (int gx = 0; gx < nq; ++gx) acc += f0[(gz * nq + gy) * nq + gx] * Lq[gx * N + j];
                G1[(gz * nq + gy) * N + j] = acc;
              }
          G2.assign((size_t)nq * N * N, 0.0);
          for (int gz = 0; gz < nq; ++gz)
            for (int kk = 0; kk < N; ++kk)
              for (int j = 0; j < N; ++j) {
                double acc = 0.0;
                for (int gy = 0; gy < nq; ++gy) acc += G1[(gz * nq + gy) * N + j] * Lq[gy * N + kk];
                G2[(gz * N + kk) * N + j] = acc;
              }
          double* row = &rhs[(size_t)c->h_off_state[e] + (size_t)(f * 3 + cc) * N3];
          for (int l = 0; l < N; ++l)
            for (int kk = 0; kk < N; ++kk)
              for (int j = 0; j < N; ++j) {
                double acc = 0.0;
                for (int gz = 0; gz < nq; ++gz) acc += G2[(gz * N + kk) * N + j] * Lq[gz * N + l];
                row[(l * N + kk) * N + j] = acc;
              }
        }
      }
    }
  }
  // CG on the device: x, r, p, Ap, z and the right side b; restarted from the true residual
  // b - M x (at most three times) until that is below 1e-15 |b| (the recursively updated
  // residual of CG drifts away from the true one near round-off)
  double* buf = nullptr;
  if (cudaMalloc(&buf, 6 * (size_t)n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, STM_ENOMEM, "projection work vectors");
  }
  double *x = buf, *r = buf + n, *pv = buf + 2 * n, *Ap = buf + 3 * n, *z = buf + 4 * n, *bd = buf + 5 * n;
  auto dot = [&](const double* a, const double* b, double* out) -> int {
    multidot<double>(a, b, 0, 1, false, n, c->red_partial, c->red_out, c->stream);
    c->launches += 2;
    STM_CK(cudaMemcpyAsync(c->h_pinned, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    STM_CK(cudaStreamSynchronize(c->stream));
    *out = c->h_pinned[0];
    return STM_OK;
  };
  auto mass = [&](const double* in, double* out) -> int {
    const int em = launch_mass_curved<double>(P, 1, in, 6LL * N3, N3, nullptr, 0, 0, c->Gw64, c->eps64, c->mu64,
                                              c->ct, c->ne, out, c->stream);
    c->launches += 1;
    return em ? fail(c, STM_EDEVICE, "projection mass launch") : STM_OK;
  };
  int rc = STM_OK;
  do {
    if (cudaMemsetAsync(x, 0, n * sizeof(double), c->stream) != cudaSuccess ||
        cudaMemcpyAsync(bd, rhs.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(r, bd, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
      rc = fail(c, STM_EDEVICE, "projection copies");
      break;
    }
    double rr0;
    if ((rc = dot(r, r, &rr0))) break;
    for (int restart = 0; restart < 4 && rr0 > 0 && !rc; ++restart) {
      if (restart > 0) {  // true residual r = b - M x
        if ((rc = mass(x, Ap))) break;
        STM_CK(cudaMemcpyAsync(r, bd, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        Coef16 cm{};
        cm.c[0] = 1.0;
        axpy_norm<double>(r, Ap, 0, 1, cm, n, c->red_partial, c->red_out, c->stream);
        c->launches += 2;
        STM_CK(cudaMemcpyAsync(c->h_pinned, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        STM_CK(cudaStreamSynchronize(c->stream));
        if (!(c->h_pinned[0] > 1e-30 * rr0)) break;  // |b - M x| <= 1e-15 |b|
      }
      precond_curved<double, double>(z, r, 0, 0, nullptr, c->Pinv64, N3, c->ne, false, c->stream);
      STM_CK(cudaMemcpyAsync(pv, z, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      double rz;
      if ((rc = dot(r, z, &rz))) break;
      for (int it = 0; it < 1000; ++it) {
        if ((rc = mass(pv, Ap))) break;
        double pAp;
        if ((rc = dot(pv, Ap, &pAp))) break;
        const double alpha = rz / pAp;
        Coef16 ca{}, cr{};
        ca.c[0] = -alpha;
        cr.c[0] = alpha;
        axpy_norm<double>(x, pv, 0, 1, ca, n, c->red_partial, c->red_out, c->stream);  // x += alpha p
        axpy_norm<double>(r, Ap, 0, 1, cr, n, c->red_partial, c->red_out, c->stream);  // r -= alpha Ap
        c->launches += 4;
        STM_CK(cudaMemcpyAsync(c->h_pinned, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        STM_CK(cudaStreamSynchronize(c->stream));
        if (!(c->h_pinned[0] > 1e-32 * rr0)) break;  // |r| <= 1e-16 |b| (or not finite: stop)
        precond_curved<double, double>(z, r, 0, 0, nullptr, c->Pinv64, N3, c->ne, false, c->stream);
        c->launches += 1;
        double rz1;
        if ((rc = dot(r, z, &rz1))) break;
        Coef16 cb{};
        cb.c[0] = -rz1 / rz;
        rz = rz1;
        axpy_norm<double>(z, pv, 0, 1, cb, n, c->red_partial, c->red_out, c->stream);  // z += beta p
        c->launches += 2;
        std::swap(pv, z);
      }
    }
    if (rc) break;
    STM_CK(cudaMemcpyAsync(c->state, x, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    STM_CK(cudaStreamSynchronize(c->stream));
    c->t = t;
  } while (false);
  cudaFree(buf);
  return rc;
}

extern "C" {

int32_t stm_set_initial(stm_ctx* c, double t, stm_field_fn E0, stm_field_fn H0, void* user) {
  // Covariant L2 projection on a brick: u_c[s] = h_c int_K^ phi_s (F_c o F_K) dx^,
  // by the tensor Gauss rule with p+2 points per direction (per element degree).
  if (!c) return STM_EINVAL;
  if (c->geometry != STM_GEOM_BRICK) return project_curved(c, t, E0, H0, user);
  std::vector<std::vector<double>> xg(9), wg(9), Lg(9);
  for (int P = 0; P <= 7; ++P) {
    const int nq = P + 2, N = P + 1;
    gauss01(nq, xg[P], wg[P]);
    Lg[P].resize(nq * N);
    for (int g = 0; g < nq; ++g) legendre01(N, xg[P][g], &Lg[P][g * N]);
  }
  std::vector<double> u(c->n_state, 0.0), pts, val;
  std::vector<int64_t> pstart;
  int64_t e0 = 0;
  while (e0 < c->ne) {
    // a chunk of elements with about 2^20 quadrature points
    int64_t e1 = e0, np = 0;
    pstart.clear();
    while (e1 < c->ne && (np == 0 || np < (1 << 20))) {
      const int nq = c->h_p[e1] + 2;
      pstart.push_back(np);
      np += (int64_t)nq * nq * nq;
      ++e1;
    }
    pts.resize(3 * np);
    val.resize(3 * np);
    for (int64_t e = e0; e < e1; ++e) {
      const int P = c->h_p[e], nq = P + 2;
      for (int gz = 0; gz < nq; ++gz)
        for (int gy = 0; gy < nq; ++gy)
          for (int gx = 0; gx < nq; ++gx) {
            const int64_t k = (pstart[e - e0] + (gz * nq + gy) * nq + gx) * 3;
            pts[k + 0] = c->h_x0[3 * e + 0] + c->h_h[3 * e + 0] * xg[P][gx];
            pts[k + 1] = c->h_x0[3 * e + 1] + c->h_h[3 * e + 1] * xg[P][gy];
            pts[k + 2] = c->h_x0[3 * e + 2] + c->h_h[3 * e + 2] * xg[P][gz];
          }
    }
    for (int f = 0; f < 2; ++f) {
      stm_field_fn fn = f == 0 ? E0 : H0;
      if (!fn) continue;
      fn(user, np, pts.data(), val.data());
      for (int64_t e = e0; e < e1; ++e) {
        const int P = c->h_p[e], nq = P + 2, N = P + 1, N3 = N * N * N;
        const double* L = Lg[P].data();
        for (int cc = 0; cc < 3; ++cc) {
          double* ue = &u[c->h_off_state[e] + (f * 3 + cc) * N3];
          const double hc = c->h_h[3 * e + cc];
          for (int gz = 0; gz < nq; ++gz)
            for (int gy = 0; gy < nq; ++gy)
              for (int gx = 0; gx < nq; ++gx) {
                const double v = val[(pstart[e - e0] + (gz * nq + gy) * nq + gx) * 3 + cc] * hc * wg[P][gx] *
                                 wg[P][gy] * wg[P][gz];
                for (int l = 0; l < N; ++l)
                  for (int k = 0; k < N; ++k) {
                    const double lk = L[gz * N + l] * L[gy * N + k] * v;
                    for (int j = 0; j < N; ++j) ue[(l * N + k) * N + j] += lk * L[gx * N + j];
                  }
              }
        }
      }
    }
    e0 = e1;
  }
  return stm_set_state(c, t, u.data(), STM_MEM_HOST);
}

int32_t stm_energy(stm_ctx* c, double* energy) {
  if (!c || !energy) return STM_EINVAL;
  if (c->geometry != STM_GEOM_BRICK || c->hp) {
    if (c->hp) {
      energy_hp(c->state, c->mass64, c->off_state, c->pq, c->ne, c->el, c->stream);
    } else {
      const int e = launch_energy_curved(c->P, c->state, c->Gw64, c->eps64, c->mu64, c->ct, c->ne, c->el, c->stream);
      if (e) return fail(c, STM_EDEVICE, "curved energy launch failed");
    }
    c->launches += 1;
    std::vector<double> el(c->ne);
    STM_CK(cudaMemcpyAsync(el.data(), c->el, c->ne * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    STM_CK(cudaStreamSynchronize(c->stream));
    double sum = 0.0;
    for (double v : el) sum += v;  // fixed order
    *energy = sum;
    return STM_OK;
  }
  energy_brick(c->state, c->mass64, c->N3, c->n_state, c->red_partial, c->red_out, c->stream);
  c->launches += 2;
  STM_CK(cudaMemcpyAsync(c->h_pinned, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  STM_CK(cudaStreamSynchronize(c->stream));
  *energy = c->h_pinned[0];
  return STM_OK;
}

int32_t stm_slab_solve(stm_ctx* c, double dt, stm_solve_report* rep) {
  if (!c) return STM_EINVAL;
  if (!(dt > 0)) return fail(c, STM_EINVAL, "dt must be positive");
  const bool mixed = c->opts.precision == STM_MIXED;
  if (!mixed && c->opts.precision != STM_FP64) return fail(c, STM_EINVAL, "opts.precision must be FP64 or MIXED");
  const int m = c->opts.restart;
  const int64_t n = c->n_test;
  int rc;
  // FP64 buffers: x (unknowns), z (work / residual); basis in FP64 or FP32
  // basis columns start on 16-byte (here 512-byte) boundaries for vector loads
  const int64_t ldv = (n + 63) / 64 * 64;
  if ((rc = ensure_buf<double>(c, &c->x, &c->x_len, n)) || (rc = ensure_buf<double>(c, &c->z, &c->z_len, n))) return rc;
  if (mixed) {
    if ((rc = ensure_buf<float>(c, &c->V32, &c->V32_len, (m + 1) * ldv)) ||
        (rc = ensure_buf<float>(c, &c->z32, &c->z32_len, n)))
      return rc;
  } else if ((rc = ensure_buf<double>(c, &c->V, &c->V_len, (m + 1) * ldv))) {
    return rc;
  }
  if (!c->gst) {
    if (cudaMalloc((void**)&c->gst, sizeof(GmresState)) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_gst, sizeof(GmresState)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, STM_ENOMEM, "GMRES state allocation failed");
    }
    STM_CK(cudaMemsetAsync(c->gst, 0, sizeof(GmresState), c->stream));
  }
  if (mixed && needs_scratch<float>(c)) {  // FP32 residual scratch, allocated before any capture
    float *y32 = nullptr, *tr32 = nullptr;
    if ((rc = scratch<float>(c, &y32, &tr32))) return rc;
  }
  const double* b = nullptr;
  if ((rc = build_load(c, c->t, dt, &b))) return rc;
  // inexact solve: stop when this slab's share of eta_it (Sec. 5.3) is below eta_tol / sqrt(slabs)
  const bool inexact = c->opts.eta_tol > 0;
  double target = c->opts.tol;
  if (inexact) {
    if (c->geometry != STM_GEOM_BRICK) return fail(c, STM_EUNSUPPORTED, "the inexact solve is built for brick meshes");
    for (const auto& k : c->classes)  // the bound needs one temporal degree everywhere
      if (k.Q != c->classes[0].Q) return fail(c, STM_EUNSUPPORTED, "the inexact solve needs a uniform q");
    if (c->ltr) return fail(c, STM_EUNSUPPORTED, "the inexact solve needs N_K = 1 (no local refinement in time)");
    if (!(c->opts.t_final > 0)) return fail(c, STM_EINVAL, "opts.t_final must be positive for the inexact solve");
    if ((rc = build_eta_weights(c, dt))) return rc;
    const double nslab = std::max(1.0, std::round(c->opts.t_final / dt));
    target = c->opts.eta_tol / std::sqrt(nslab);
  }
  GmresState* st = c->gst;
  // reference: ||R(U^(0))|| with all unknowns zero (R6), kept on the device
  STM_CK(cudaMemsetAsync(c->x, 0, n * sizeof(double), c->stream));
  if ((rc = resid64(c, dt, c->x, b, c->z))) return rc;
  axpy_norm<double>(c->z, c->z, 0, 0, Coef16{}, n, c->red_partial, nullptr, c->stream);
  gmres_reduce(c->red_partial, st, 0, c->stream);
  gmres_slab_start(st, target, c->opts.max_it, inexact ? 1 : 0, c->stream);
  c->launches += 3;
  // initial guess: u_1 = u_0, higher modes 0 (or all unknowns 0: x is already zero)
  if (!c->opts.zero_guess) {
    if (c->hp) init_guess_hp(c->x, c->state, c->off_test, c->off_state, c->pq, c->ne, c->stream);
    else k_init_guess<<<grid1(n), 256, 0, c->stream>>>(c->x, c->state, c->Q, c->N3, n);
    c->launches += 1;
  }
  // restart cycles, each one launch sequence (a replayed CUDA graph unless profiling) and one
  // read of the device state: the stop test, the iteration count and the error status
  bool done = false;
  const int per = c->profiling ? 1 : std::max(1, (int)c->opts.cycles_per_launch);
  const int max_launches = c->opts.max_it + 2;  // every cycle but the last makes >= 1 iteration
  for (int cyc = 0; cyc < max_launches; ++cyc) {
    if ((rc = run_cycles(c, dt, b, mixed, ldv, per))) return rc;
    STM_CK(cudaMemcpyAsync(c->h_gst, st, sizeof(GmresState), cudaMemcpyDeviceToHost, c->stream));
    STM_CK(cudaStreamSynchronize(c->stream));
    const GmresState& h = *c->h_gst;
    if (c->profiling && c->it_marks.size() == (size_t)m + 1) {
      // the residual launches of iterations the device skipped did no work: not timed
      const size_t k = (size_t)std::max(0, std::min(h.k, m));
      c->timed.erase(c->timed.begin() + (std::ptrdiff_t)c->it_marks[k],
                     c->timed.begin() + (std::ptrdiff_t)c->it_marks[m]);
      c->it_marks.clear();
    }
    if (h.status < 0) return fail(c, h.status, "non-finite value in the slab solve");
    if (h.halt) {  // the stop test held, or no progress is possible (iteration cap, zero residual)
      done = h.outer_done != 0;
      break;
    }
  }
  if (c->tc_err) {  // a bounded wait of the tensor-core mass kernel ran out: no valid result
    int h_err = 0;
    STM_CK(cudaMemcpyAsync(&h_err, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    STM_CK(cudaStreamSynchronize(c->stream));
    if (h_err) return fail(c, STM_ETIMEOUT, "tensor-core mass kernel: a bounded wait ran out");
  }
  if (int rc = check_wait_err(c)) return rc;
  if (c->hp) extract_end_hp(c->state, c->x, c->off_test, c->off_state, c->pq, c->ne, c->stream);
  else k_extract_end<<<grid1(c->n_state), 256, 0, c->stream>>>(c->state, c->x, c->Q, c->N3, c->n_state);
  c->launches += 1;
  STM_CK(cudaGetLastError());
  c->t += dt;
  double en = 0.0;
  if ((rc = stm_energy(c, &en))) return rc;
  if (rep) {
    rep->iterations = c->h_gst->iters;
    rep->restarts = c->h_gst->cycles;
    rep->rel_residual = c->h_gst->rel;
    rep->energy = en;
    rep->eta2 = inexact ? c->h_gst->phi * c->h_gst->phi : 0.0;
  }
  return done ? STM_OK : STM_ENOTCONV;
}

int32_t stm_set_source_gauss(stm_ctx* c, const stm_gauss_src* src, int32_t n_src) {
  if (!c || n_src < 0 || n_src > kMaxSrc || (n_src > 0 && !src)) return STM_EINVAL;
  for (int k = 0; k < n_src; ++k)
    if (!(src[k].sigma_x > 0) || !(src[k].sigma_t > 0)) return fail(c, STM_EINVAL, "source widths must be positive");
  c->srcs.assign(src, src + n_src);
  c->load_valid = false;
  return STM_OK;
}

int32_t stm_set_boundary(stm_ctx* c, stm_st_field_fn g, void* user) {
  if (!c) return STM_EINVAL;
  c->gfn = g;
  c->guser = user;
  c->load_valid = false;
  return STM_OK;
}

int32_t stm_set_source(stm_ctx* c, stm_st_field_fn J, void* user) {
  if (!c) return STM_EINVAL;
  c->jfn = J;
  c->juser = user;
  c->load_valid = false;
  return STM_OK;
}

int32_t stm_dof_layout(stm_ctx* c, int64_t* off_trial, int64_t* off_test, int64_t* off_state) {
  if (!c) return STM_EINVAL;
  const size_t n = (size_t)c->ne + 1;
  if (off_trial) std::copy(c->h_off_trial.begin(), c->h_off_trial.begin() + n, off_trial);
  if (off_test) std::copy(c->h_off_test.begin(), c->h_off_test.begin() + n, off_test);
  if (off_state) std::copy(c->h_off_state.begin(), c->h_off_state.begin() + n, off_state);
  return STM_OK;
}

}  // extern "C"

// Autotuner: for every (p, q) class (or the whole uniform mesh) time the
// residual kernels with 64, 128, 256 and 512 threads per block on the context's
// own data layout and keep the fastest; later applies use it.
template <typename T>
int autotune_prec(stm_ctx* c, double dt, int reps, std::vector<double>& best_ms) {
  T *U = nullptr, *R = nullptr;
  if (cudaMalloc(&U, c->n_trial * sizeof(T)) != cudaSuccess || cudaMalloc(&R, c->n_test * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    if (U) cudaFree(U);
    return fail(c, STM_ENOMEM, "autotune buffers");
  }
  cudaMemsetAsync(U, 0, c->n_trial * sizeof(T), c->stream);
  const bool saved_graph = c->opts.graph != 0;
  c->opts.graph = 0;
  int rc = apply<T>(c, dt, U, L_TRIAL, U, L_TRIAL, nullptr, R);  // warm up, traces for every class
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int cands[4] = {64, 128, 256, 512};
  const size_t ncl = c->hp ? c->classes.size() : 1;
  best_ms.assign(ncl, 0.0);
  for (size_t k = 0; k < ncl && rc == STM_OK; ++k) {
    double best = 1e30;
    int bb = 256;
    const int P = c->hp ? c->classes[k].P : c->P, Q = c->hp ? c->classes[k].Q : c->Q;
    for (int cb : cands) {
      if (cb > residual_max_threads(P, Q)) continue;  // beyond the kernels' launch bound
      if (c->hp) c->classes[k].block = cb;
      else c->block = cb;
      float ms = 0.f;
      cudaEventRecord(e0, c->stream);
      for (int r = 0; r < reps && rc == STM_OK; ++r) {
        if (!c->hp) {
          rc = apply<T>(c, dt, U, L_TRIAL, U, L_TRIAL, nullptr, R);
        } else {
          // this class alone (its trace pass, then its apply pass; other classes' traces are current)
          const auto& cl = c->classes[k];
          T *y = nullptr, *tr = nullptr;
          scratch<T>(c, &y, &tr);
          ApplyArgs<T> a{};
          a.y = y;
          a.tr = tr;
          a.R = R;
          a.nbr = c->nbr;
          a.mass = mass_ptr<T>(c);
          a.um = U;
          a.u0 = U;
          a.off_um = c->off_trial;
          a.um_trial = 1;
          a.off_u0 = c->off_trial;
          a.off_R = c->off_test;
          a.off_tr = c->off_tr;
          a.pq = c->pq;
          a.hslot = c->hslot;
          a.hoff = c->hoff;
          a.hbuf = hbuf_ptr<T>(c);
          a.elist = cl.elist;
          a.n_elem = cl.count;
          a.nk = cl.NK;
          a.nkl = c->nkl;
          a.tmat = tmat_ptr<T>(c);
          a.kap = kap_ptr<T>(c);
          a.dt_k = (T)dt;
          a.tb = make_tables<T>(cl.P, kMaxQ, dt / cl.NK);
          const int grid = res_grid(c, cl.count);
          LaunchEvents none;
          if (launch_residual_ph<T>(cl.P, cl.Q, a, c->stream, grid, none, 1, cb) ||
              launch_residual_ph<T>(cl.P, cl.Q, a, c->stream, grid, none, 2, cb))
            rc = fail(c, STM_EDEVICE, "autotune launch");
        }
      }
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bb = cb;
      }
    }
    if (c->hp) c->classes[k].block = bb;
    else c->block = bb;
    best_ms[k] = best / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(U);
  cudaFree(R);
  c->opts.graph = saved_graph;
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);  // launch shapes changed
  c->graphs.clear();
  return rc;
}

extern "C" {

int32_t stm_autotune(stm_ctx* c, double dt, int32_t reps, int32_t n_max, int32_t* P, int32_t* Q, int32_t* block,
                     double* ms, int32_t* n_out) {
  if (!c || !(dt > 0) || reps < 1) return STM_EINVAL;
  std::vector<double> best;
  int rc = autotune_prec<double>(c, dt, reps, best);
  if (rc) return rc;
  drop_cycle_graphs(c);  // captured cycles hold the old block sizes
  const int ncl = c->hp ? (int)c->classes.size() : 1;
  if (n_out) *n_out = ncl;
  for (int k = 0; k < ncl && k < n_max; ++k) {
    if (P) P[k] = c->hp ? c->classes[k].P : c->P;
    if (Q) Q[k] = c->hp ? c->classes[k].Q : c->Q;
    if (block) block[k] = c->hp ? c->classes[k].block : c->block;
    if (ms) ms[k] = best[k];
  }
  return STM_OK;
}

int32_t stm_host_alloc(void** ptr, int64_t bytes) {
  if (!ptr || bytes <= 0) return STM_EINVAL;
  *ptr = nullptr;
  if (cudaMallocHost(ptr, (size_t)bytes) != cudaSuccess) {
    cudaGetLastError();
    return STM_ENOMEM;
  }
  return STM_OK;
}

int32_t stm_host_free(void* ptr) {
  if (ptr && cudaFreeHost(ptr) != cudaSuccess) {
    cudaGetLastError();
    return STM_EINVAL;
  }
  return STM_OK;
}

int32_t stm_fp64_probe(double* tflops) {
  if (!tflops) return STM_EINVAL;
  *tflops = 0.0;
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return STM_EDEVICE;
  const int grid = sms * 8, block = 256, iters = 4096;
  double* out = nullptr;
  if (cudaMalloc(&out, (size_t)grid * block * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return STM_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_probe<<<grid, block>>>(out, iters, 1.0 + 1e-9);  // warm-up
  cudaEventRecord(e0);
  k_fma_probe<<<grid, block>>>(out, iters, 1.0 + 1e-9);
  cudaEventRecord(e1);
  const cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return STM_EDEVICE;
  *tflops = 2.0 * kProbeChains * (double)iters * grid * block / (ms * 1e-3) / 1e12;
  return STM_OK;
}

int32_t stm_launch_count(stm_ctx* c, int64_t* n) {
  if (!c || !n) return STM_EINVAL;
  *n = c->launches;
  return STM_OK;
}

int32_t stm_profile_enable(stm_ctx* c, int32_t on) {
  if (!c) return STM_EINVAL;
  STM_CK(cudaStreamSynchronize(c->stream));
  c->profiling = on != 0;
  c->timed.clear();
  c->ev_used = 0;
  return STM_OK;
}

int32_t stm_profile_read(stm_ctx* c, double* ms, int64_t* count) {
  if (!c || !ms || !count) return STM_EINVAL;
  STM_CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 4; ++k) {
    ms[k] = 0.0;
    count[k] = 0;
  }
  for (const auto& t : c->timed) {
    float a = 0.f, b = 0.f;
    STM_CK(cudaEventElapsedTime(&a, t.a, t.b));
    STM_CK(cudaEventElapsedTime(&b, t.b, t.c));
    ms[2 * t.prec] += a;
    ms[2 * t.prec + 1] += b;
    count[2 * t.prec] += 1;
    count[2 * t.prec + 1] += 1;
  }
  return STM_OK;
}

}  // extern "C"
