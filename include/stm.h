/*
 * stm.h -- C ABI of the space-time hp-DG Maxwell slab library (GB300, sm_103a).
 *
 * The library evaluates, matrix-free on the GPU, the space-time residual of
 * Lilienthal, Schnepp & Weiland's non-dissipative space-time hp-DG method
 * for the time-dependent Maxwell equations, and solves the per-slab systems
 * with restarted GMRES.
 *
 * Problem (Eq. maxwell, Sec. 1):   eps E_t - curl H = J,  mu H_t + curl E = 0
 * in Omega x (0,T],  n x E = n x g on the boundary,  E = E0, H = H0 at t = 0,
 * eps and mu element-wise constant (Sec. 3, Theorem 3.1).
 *
 * Discretisation (Sec. 2.3, Sec. 5.1): per hexahedron K and time slab
 * (t0, t0 + dt], trial functions DF^{-T} l_m(xi) L_j(x^) L_k(y^) L_l(z^) e_c
 * (m = 0..q, continuous in time), test functions DF^{-T} L_i(xi) L_j L_k L_l e_c
 * (i = 0..q-1), with L the orthonormal Legendre polynomials on [0,1] and l_m
 * the integrated Legendre polynomials (Eq. def:ilegendre).
 *
 * Coefficient layouts (all arrays are dense, element after element):
 *   trial  U[e][field 0=E,1=H][component x,y,z][mode m = 0..q][s]
 *   test   R[e][field][component][mode i = 0..q-1][s]
 *   state  u[e][field][component][s]          (spatial coefficients at a time)
 * with s = (l (p+1) + k)(p+1) + j, j the x^ degree.  Mode 0 of U is the field
 * at the slab start and mode 1 the field at the slab end (l_0(1) = 0,
 * l_1(1) = 1, l_m(0) = l_m(1) = 0 for m >= 2); modes 1..q are the slab
 * unknowns, so the unknown vector has the test layout.
 *
 * Status codes: 0 = STM_OK; negative = failure, nothing written; positive =
 * a result with a warning.  stm_last_error() returns a message for the last
 * failure of a context.  A context is not thread-safe.
 *
 * Memory: the library never frees caller memory.  STM_MEM_HOST pointers are
 * host arrays copied in and out inside the call; STM_MEM_DEVICE pointers are
 * device arrays on the context's device that the caller keeps alive until the
 * call's stream work has finished.  Calls are ordered on the context stream.
 */
#ifndef STM_H
#define STM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STM_OK 0
#define STM_EINVAL (-1)       /* invalid argument or mesh                       */
#define STM_ENOMEM (-2)       /* device allocation failed                        */
#define STM_EDEVICE (-3)      /* CUDA error                                      */
#define STM_ETIMEOUT (-4)     /* a bounded device wait ran out                   */
#define STM_ENAN (-5)         /* non-finite value detected                       */
#define STM_EUNSUPPORTED (-6) /* mesh or option outside what this build handles */
#define STM_ECANCELLED (-7)   /* request cancelled (server destroyed while queued)  */
#define STM_ENOTCONV 1        /* solver stopped at max_it; best iterate kept     */

#define STM_GEOM_BRICK 0     /* axis-aligned boxes (affine, diagonal DF)          */
#define STM_GEOM_AFFINE 1    /* parallelepipeds: x = x_0 + DF x^ with a constant,
                                general DF (vertex v at x_0 + DF (v&1, v>>1&1,
                                v>>2&1)); the mass term uses the constant 3x3
                                metric G = |J| DF^{-1} DF^{-T} (Sec. 5.2, "mass
                                residual"); same face rule as TRILINEAR          */
#define STM_GEOM_TRILINEAR 2 /* trilinear maps from the 8 vertices (curved); face 2d+1
                                of e and face 2d of its neighbour must have the same
                                four vertex ids in the same reference order         */

#define STM_FP64 0  /* residual apply / solve in double precision             */
#define STM_FP32 1  /* residual apply in single precision (float arrays)       */
#define STM_MIXED 2 /* slab solve: FP32 inner GMRES, FP64 outer refinement     */

#define STM_MEM_HOST 0
#define STM_MEM_DEVICE 1

typedef struct stm_ctx stm_ctx;

/* Mesh and data of the problem statement (Sec. 1-2).  Host arrays, copied by
 * stm_create; the caller keeps ownership. */
typedef struct {
  int64_t n_elem, n_vert;
  const double *vert;  /* [n_vert][3] vertex coordinates                          */
  const int64_t *hex;  /* [n_elem][8] vertex ids, vertex v at reference corner
                          (v&1, v>>1&1, v>>2&1)                                   */
  const int64_t *nbr;  /* [n_elem][6] element across face 2d+s (axis d, s = 1 at
                          x^_d = 1), -1 on the boundary, -2 on either side of a
                          2:1 face (see hang); face 2d+1 of e must meet face 2d
                          of nbr                                                  */
  int64_t n_hang;      /* rows of hang (0 = conforming mesh)                       */
  const int64_t *hang; /* [n_hang][6] 2:1 faces of brick meshes: coarse element,
                          coarse face, fine element, fine face, u, v -- the fine
                          face is the quarter (u, v) of the coarse face, u along
                          the lower and v along the higher tangential axis; every
                          coarse face of this kind has four rows               */
  const uint8_t *p;    /* [n_elem] spatial degree (isotropic), 0..7              */
  const uint8_t *q;    /* [n_elem] temporal degree, 1..6                         */
  const double *eps;   /* [n_elem] permittivity, > 0                             */
  const double *mu;    /* [n_elem] permeability, > 0                             */
  int32_t geometry;    /* STM_GEOM_*                                              */
  const uint8_t *nk;   /* [n_elem] temporal sub-intervals N_K of the slab (local
                          refinement in time, Sec. 2.2): 1, 2, 4 or 8; NULL = all
                          1.  Element K then carries N_K q unknown temporal modes
                          per (field, component, spatial index): trial layout
                          [f][c][1 + N_K q][s] (index 0 the slab start, 1 + k q
                          + m - 1 mode m of sub-interval k), test layout
                          [f][c][N_K q][s].  Brick meshes without 2:1 faces   */
} stm_mesh;

typedef struct {
  int32_t precision;     /* STM_FP64 | STM_MIXED for stm_slab_solve               */
  double tol;            /* relative residual target of the slab solve            */
  int32_t restart;       /* GMRES restart length n_r (Sec. 5.4: 10)               */
  int32_t max_it;        /* iteration cap per slab                                */
  int32_t deterministic; /* 1: fixed-order reductions (bitwise reproducible)      */
  int64_t stream;        /* cudaStream_t as integer; 0 = the CUDA default stream  */
  int32_t reorth;        /* 1: second Gram-Schmidt pass when the norm drops below
                            1/sqrt(2) of its value (DGKS test); 0: never           */
  int32_t graph;         /* 1: on meshes with several (p, q) classes or 2:1 faces,
                            capture each residual apply (all launches) once in a
                            CUDA graph per (buffers, dt) and replay it             */
  double eta_tol;        /* > 0: inexact solve (Sec. 5.3, brick meshes): a slab
                            stops once its share of the guaranteed iteration-error
                            bound eta_it of Eq. a_posteriori:iteration is at most
                            eta_tol / sqrt(t_final / dt); tol is then unused       */
  double t_final;        /* final time t_N of the bound (inexact solve)             */
  double c_diss;         /* >= 0: adds the dissipative upwind term D_h of Sec. 4.2
                            with alpha_E = c/{sqrt(mu/eps)}, alpha_H = c/{sqrt(eps/mu)}
                            (0: the non-dissipative method).  Brick meshes with one
                            q and no 2:1 faces; else stm_create returns
                            STM_EUNSUPPORTED                                        */
  int32_t zero_guess;    /* 1: GMRES starts each slab from all unknowns 0; 0 (default):
                            from u_1 = u_0, higher modes 0 (the field held constant
                            over the slab).  The converged solution is the same     */
  int32_t no_tensor_cores; /* 1: the FP32 mass term of trilinear elements runs on the
                            CUDA cores; 0 (default): on the tensor cores (3xTF32)
                            for 3 <= p <= 7                                         */
  int32_t cycles_per_launch; /* GMRES restart cycles per CUDA-graph launch of the slab
                            solve, each followed by one host read of the solver state
                            (<= 1: one); cycles after the stop test are skipped on
                            the device, so a value above the cycles a slab needs runs
                            the whole solve as one graph launch and one host read   */
} stm_opts;

typedef struct {
  int32_t iterations;      /* GMRES iterations (inner iterations in STM_MIXED)   */
  int32_t restarts;        /* restart cycles (outer refinements in STM_MIXED)    */
  double rel_residual;     /* final ||R(U)||_2 / ||R(U^(0))||_2, FP64            */
  double energy;           /* discrete energy at the slab end (Eq. stability:energydef) */
  double eta2;             /* inexact solve: this slab's term of eta_it^2, i.e.
                              4 c_E |R_E|^2_{W'} + 4 c_H |R_H|^2_{W'} at the
                              returned iterate (sum over slabs = eta_it^2)          */
} stm_solve_report;

/* Create a context on the current CUDA device.  Validates the mesh, copies
 * connectivity, degrees and materials to the device and precomputes the
 * element metric.  Returns STM_EINVAL for invalid input (degrees out of
 * range, non-positive materials, bad ids) and STM_EUNSUPPORTED for a
 * combination this build does not handle: uneven (p, q), 2:1 faces or N_K > 1
 * on trilinear meshes; N_K > 1 together with 2:1 faces; the dissipative term
 * with trilinear geometry, uneven q, 2:1 faces or N_K > 1. */
int32_t stm_create(stm_ctx **ctx, const stm_mesh *mesh, const stm_opts *opts);
int32_t stm_destroy(stm_ctx *ctx);
const char *stm_last_error(stm_ctx *ctx);

/* Number of trial coefficients (U), test coefficients (R, unknowns) and state
 * coefficients (u) of the whole mesh. */
int32_t stm_sizes(stm_ctx *ctx, int64_t *n_trial, int64_t *n_test, int64_t *n_state);

/* Residual R_h(V) = B_h(U, V) - L(V) of Eq. residual (Sec. 5) for every test
 * basis function V, with B_h = C_h + S_h (Eq. bilinearform:C, bilinearform:S)
 * on the slab (t0, t0 + dt].  U: trial layout, R: test layout, both of type
 * double (prec = STM_FP64) or float (prec = STM_FP32).  Boundary data and
 * sources set with stm_set_* enter through L; by default g = 0 (PEC), J = 0. */
int32_t stm_residual_apply(stm_ctx *ctx, double t0, double dt, const void *U, void *R,
                           int32_t prec, int32_t mem);

/* The operator the slab's GMRES iterates on (Sec. 5.4): W = A P^{-1} V (pre = 1)
 * or W = A V (pre = 0).  A is the linear part of the residual of Eq. residual as
 * a function of the unknown temporal modes 1..q (slab start mode 0 = 0, no load
 * L), P the block-diagonal preconditioner of Eq. preconditioner (the time-
 * derivative terms (eps d_t E, v) + (mu d_t H, w)); on trilinear and general
 * affine meshes P^{-1} is the cell-mean 3x3 block inverse the solver uses, and
 * on time-refined meshes (N_K > 1, where the form couples each sub-interval to
 * the end value of the one before) the inverse of its diagonal blocks, as in
 * the solver.  V and
 * W: n_test entries in the test layout (stm_sizes), double (prec = STM_FP64) or
 * float (prec = STM_FP32), in host (mem = STM_MEM_HOST, copied through device
 * buffers the context owns) or device memory (STM_MEM_DEVICE, caller-owned; V is
 * not modified, V and W must not overlap).  Returns STM_EINVAL for a null
 * pointer, dt <= 0 or a bad prec/mem/pre value, STM_ENOMEM when a staging
 * buffer cannot be allocated, STM_EDEVICE on a CUDA error, STM_ETIMEOUT if a
 * bounded device wait of the FP32 kernel on its asynchronous copies ran out (W
 * is then invalid; the call synchronises the stream to read that flag when
 * prec = STM_FP32 and pre = 1). */
int32_t stm_operator_apply(stm_ctx *ctx, double dt, const void *V, void *W, int32_t pre,
                           int32_t prec, int32_t mem);

/* Set the state (spatial coefficients of E and H at time t, state layout,
 * double).  The next slab starts from it.  With mem = STM_MEM_HOST, host memory
 * the device addresses directly (from stm_host_alloc, cudaMallocHost or
 * registered) is moved by a copy kernel over the host link, other host memory
 * by the copy engines; both calls return when the transfer is complete. */
int32_t stm_set_state(stm_ctx *ctx, double t, const void *u, int32_t mem);
int32_t stm_get_state(stm_ctx *ctx, double *t, void *u, int32_t mem);

/* L2 projection of E0(x), H0(x) onto the covariant spatial spaces (initial
 * data of Eq. maxwell), evaluated by the callback at p+2 Gauss points per
 * direction; becomes the state at time t.  Either callback may be NULL (0).
 * Bricks: the diagonal mass is inverted directly.  Trilinear meshes: the
 * element systems with the metric mass (the same (p+2)^3 rule as the
 * residual) are solved by conjugate gradients on the device, restarted from
 * the true residual until that is below 1e-15 of the right side (at most
 * three restarts); STM_EDEVICE / STM_ENOMEM on failure. */
typedef void (*stm_field_fn)(void *user, int64_t npts, const double *x /*[npts][3]*/,
                             double *out /*[npts][3]*/);
int32_t stm_set_initial(stm_ctx *ctx, double t, stm_field_fn E0, stm_field_fn H0, void *user);

/* Current density J of Eq. maxwell as a sum of Gaussian pulses (at most 8):
 *   J(x, t) = sum_k amp_k dir_k exp(-|x - centre_k|^2 / (2 sigma_x^2)) exp(-(t - t0_k)^2 / (2 sigma_t^2)).
 * It enters the load l_E(v) = (J, v) of Eq. bilinearform:C, integrated on the
 * device with p+2 Gauss points per direction and q+2 in time (on meshes with
 * uneven degrees or N_K > 1 each element with its own p, q and sub-intervals,
 * one launch per (p, q, N_K) class).
 * n_src = 0 removes all sources.  The array is copied. */
typedef struct {
  double centre[3], dir[3];
  double sigma_x, t0, sigma_t, amp;
} stm_gauss_src;
int32_t stm_set_source_gauss(stm_ctx *ctx, const stm_gauss_src *src, int32_t n_src);

/* Boundary data g of Eq. maxwell (n x E = n x g): l_H(w) = -<n x g, w> on the
 * boundary faces (Eq. bilinearform:C).  The callback gets npts space-time
 * points x[k] = (x, y, z, t) and writes g there; it is called on the host once
 * per slab (p+2 Gauss points per face direction, q+2 in time on each of the
 * element's N_K sub-intervals, with each element's own p and q).  With the
 * dissipative term (opts.c_diss > 0) g also enters the E rows through
 * <alpha_E n x (E - g), n x v>.  NULL = PEC (g = 0). */
typedef void (*stm_st_field_fn)(void *user, int64_t npts, const double *xt /*[npts][4]*/,
                                double *out /*[npts][3]*/);
int32_t stm_set_boundary(stm_ctx *ctx, stm_st_field_fn g, void *user);

/* Current density J of Eq. maxwell sampled on the host: l_E(v) = (J, v) over
 * I_n x K (Eq. bilinearform:C), by (p+2)^3 Gauss points per element and q+2 in
 * time; the callback gets npts space-time points (x, y, z, t) and writes J.
 * Added to the Gaussian sources of stm_set_source_gauss.  Any mesh: on uneven
 * (p, q) or time-refined meshes each element uses its own degrees and N_K
 * sub-intervals (there the boundary data are assembled on the host the same
 * way; Gaussian sources are projected on the device per (p, q, N_K) class);
 * NULL removes it.  The library keeps the
 * pointer; the caller keeps the callback alive while the context uses it. */
int32_t stm_set_source(stm_ctx *ctx, stm_st_field_fn J, void *user);

/* Per-element block offsets ([n_elem + 1] each, filled when non-NULL) of the
 * trial layout (stm_residual_apply's U), the test layout (R, unknowns) and the
 * state layout (stm_set_state / stm_get_state). */
int32_t stm_dof_layout(stm_ctx *ctx, int64_t *off_trial, int64_t *off_test, int64_t *off_state);

/* Solve one slab (Sec. 5.4): find modes 1..q of U with R_h(U) = 0 by GMRES
 * (restart opts.restart, right preconditioned by the time-derivative terms of
 * Eq. preconditioner), starting from the state; on return the state is the
 * field at t + dt.  opts.precision selects FP64 or mixed precision.  Returns
 * STM_ETIMEOUT (state not advanced) if a bounded device wait of a kernel ran
 * out. */
int32_t stm_slab_solve(stm_ctx *ctx, double dt, stm_solve_report *rep);

/* Discrete energy 1/2 int eps E.E + mu H.H of the state (Eq. stability:energydef), FP64. */
int32_t stm_energy(stm_ctx *ctx, double *energy);

/* Autotuner (the paper has no counterpart): for every (p, q) class of the mesh
 * (one class on uniform meshes) time the residual kernels with 64, 128, 256
 * and 512 threads per block, reps times each, on scratch data of the mesh's
 * own layout, and keep the fastest for later applies (before any autotune call
 * a class uses 512 threads where the FP64 passes' shared memory leaves three or
 * fewer blocks per SM, else 256).  Reports per class (up to
 * n_max) the degrees, the chosen block size and its time in ms; *n_out = the
 * number of classes.  Allocates scratch buffers for the duration of the call. */
int32_t stm_autotune(stm_ctx *ctx, double dt, int32_t reps, int32_t n_max, int32_t *P, int32_t *Q,
                     int32_t *block, double *ms, int32_t *n_out);

/* Page-locked host buffers for STM_MEM_HOST arguments (the paper has no
 * counterpart): copies from and to them run at full host-device bandwidth.
 * stm_host_free releases a buffer from stm_host_alloc. */
int32_t stm_host_alloc(void **ptr, int64_t bytes);
int32_t stm_host_free(void *ptr);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (a register-only
 * kernel of independent FMA chains, about 10 ms); the paper has no counterpart:
 * it is the denominator against which a benchmark can put the FP64 residual. */
int32_t stm_fp64_probe(double *tflops);

/* Number of kernels this context has launched (residual, Krylov, energy). */
int32_t stm_launch_count(stm_ctx *ctx, int64_t *n);

/* Instrumentation: while enabled, CUDA events are recorded on the context
 * stream around every residual kernel launch.  stm_profile_enable resets the
 * record.  stm_profile_read synchronises the stream and returns the summed
 * durations in ms and the launch counts of [k_prep FP64, k_apply FP64,
 * k_prep FP32, k_apply FP32] (arrays of 4). */
int32_t stm_profile_enable(stm_ctx *ctx, int32_t on);
int32_t stm_profile_read(stm_ctx *ctx, double *ms, int64_t *count);

/* ---- Request server (continuous batching of slab-solve requests) ----------
 * The paper solves one problem; serving many is this library's addition.  A
 * request describes a problem on the unit cube: an n^3 mesh of bricks
 * (elements numbered with x fastest), degrees p and q, eps/mu of the first
 * material box containing an element's centre (background 1), Gaussian
 * current pulses, and either cavity initial data (kind 0: E0 = (0, 0,
 * sin pi x sin pi y), H0 = 0, the TM_11 mode of Sec. 6.1.1) or a field at
 * rest (kind 1, driven by the sources); PEC walls.  It asks for n_slabs slab
 * solves of size dt.  Requests queue FIFO; `workers` threads each admit the
 * head request when its estimated device footprint fits the remaining
 * hbm_budget_bytes (a request larger than the budget starts alone), run it on
 * their own CUDA stream (so admitted requests overlap on the device), keep
 * its fields and Krylov state on the device, and free it when done.  Results
 * are identical whether a request runs alone or among others (fixed-order
 * reductions, independent contexts).  The server is thread-safe. */
typedef struct stm_server stm_server;
typedef struct {
  int32_t workers;          /* concurrent requests (1..64)                          */
  int64_t hbm_budget_bytes; /* admission budget; <= 0: 80% of free device memory   */
  int32_t precision;        /* STM_FP64 | STM_MIXED                                 */
  double tol;               /* relative residual per slab                           */
  int32_t restart, max_it;
} stm_server_opts;
typedef struct {
  int32_t n, p, q, n_slabs;
  double dt;
  int32_t kind;             /* 0 cavity, 1 scattering (zero initial field)          */
  int32_t n_boxes;          /* material boxes, at most 4                            */
  double boxes[4][8];       /* lo x,y,z, hi x,y,z, eps, mu                          */
  int32_t n_src;            /* Gaussian current pulses, at most 8                   */
  stm_gauss_src src[8];
} stm_request;
typedef struct {
  int32_t status;           /* 0 done, 1 queued, 2 running, ENOTCONV (>0) done with
                               warning, < 0 failed (others are unaffected)           */
  int32_t iterations;       /* GMRES iterations over all slabs                      */
  double energy;            /* discrete energy at the final time                    */
  double t_final;
  double latency_ms;        /* submission to completion                             */
  double queue_ms;          /* submission to admission                              */
  double max_rel_residual;
  int64_t n_state;          /* length of the final state                            */
  int64_t footprint_bytes;  /* device footprint estimated at admission              */
} stm_result;
typedef struct {
  int64_t submitted, completed, failed, running, queued;
  int64_t peak_admitted_bytes, hbm_budget_bytes;
  double p50_ms, p99_ms;    /* latency percentiles of completed requests            */
  double solves_per_s;      /* slab solves completed per second since the first submission */
  double wall_s;
} stm_stats;
int32_t stm_server_create(stm_server **srv, const stm_server_opts *opts);
int32_t stm_server_submit(stm_server *srv, const stm_request *req, int64_t *ticket);
/* Current result of a ticket; once done, state_out (host, n_state doubles) may
 * receive the final state.  stm_server_wait blocks until the ticket is done. */
int32_t stm_server_poll(stm_server *srv, int64_t ticket, stm_result *res, double *state_out);
int32_t stm_server_wait(stm_server *srv, int64_t ticket, stm_result *res, double *state_out);
int32_t stm_server_stats(stm_server *srv, stm_stats *st);
/* Cancels queued requests, waits for running ones, frees everything. */
int32_t stm_server_destroy(stm_server *srv);

/* Residual apply that allocates no device memory (the paper has no
 * counterpart; this is a service for callers that cannot call cudaMalloc,
 * e.g. code inside a CUDA graph being captured, or a host whose device memory
 * all belongs to its own pool).  Same result as stm_residual_apply with
 * prec = STM_FP64 on an STM_GEOM_BRICK mesh of uniform (p, q), 0 <= p <= 7,
 * 1 <= q <= 6, with PEC and no sources, but without a context: every argument
 * is a device pointer the caller owns.
 *   nbr [n_elem][6] int32 face neighbours (as stm_mesh.nbr, -1 = boundary);
 *   h   [n_elem][3] edge lengths of the axis-aligned boxes;
 *   eps, mu [n_elem]; U trial layout, R test layout (both double).
 * Scratch lives in one static device array of STM_NOALLOC_SCRATCH_BYTES,
 * held by every GPU that loads the library until the process exits.  A call
 * needs 8 (6 + 6 q (p+1)^3 + 24 q (p+1)^2) bytes per element (each of the three
 * parts rounded up to 256 bytes); a larger request, degrees out of range or a
 * null pointer return STM_EINVAL (the size case with a message on stderr)
 * before any CUDA call, and nothing is launched.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the array, so calls that overlap on the GPU (different streams, or other
 * threads) race; calls ordered on one stream do not.  Everything the kernels
 * read from the scratch is written by the same call first.  Work is queued on
 * `stream` (0 = the default stream) and the call returns without waiting. */
#define STM_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int32_t stm_residual_apply_noalloc(int64_t n_elem, int32_t p, int32_t q, double dt, const int32_t *nbr,
                                   const double *h, const double *eps, const double *mu, const double *U,
                                   double *R, int64_t stream);

#ifdef __cplusplus
}
#endif

#endif /* STM_H */
