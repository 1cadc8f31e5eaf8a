// Request server: continuous batching of slab-solve requests on one GPU.
//
// Each request describes a problem (an n^3 brick mesh of the unit cube,
// degrees p and q, piecewise-constant eps/mu boxes, Gaussian current pulses,
// cavity or scattering initial data) and a number of slabs.  Requests wait in
// a FIFO queue; a worker thread admits the head request when a worker slot is
// free and its estimated device footprint fits the remaining HBM budget, then
// builds the mesh, creates a context on its own CUDA stream and marches the
// slabs.  Workers run concurrently, so the kernels of admitted requests
// overlap on the device; finished requests release their footprint.  Field
// state and Krylov workspace stay resident on the device for the life of the
// request; host traffic is the initial data and, on request, the final state.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "stm.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  int64_t ticket = 0;
  stm_request req{};
  stm_result res{};
  int64_t bytes = 0;
  Clock::time_point t_submit, t_start, t_end;
  std::vector<double> state;  // final state (host copy)
};

void tm11_E(void*, int64_t n, const double* x, double* out) {
  for (int64_t k = 0; k < n; ++k) {
    out[3 * k] = 0.0;
    out[3 * k + 1] = 0.0;
    out[3 * k + 2] = std::sin(M_PI * x[3 * k]) * std::sin(M_PI * x[3 * k + 1]);
  }
}

}  // namespace

struct stm_server {
  stm_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> queue;
  std::map<int64_t, Job*> jobs;
  std::vector<std::thread> workers;
  int64_t next_ticket = 1;
  int64_t admitted_bytes = 0, peak_bytes = 0;
  int64_t completed = 0, failed = 0, running = 0, submitted = 0;
  bool stop = false;
  int device = 0;
  Clock::time_point t0;
  bool started = false;
  std::vector<double> latencies;
  Clock::time_point last_done;
  int64_t slabs_done = 0;
};

namespace {

// Device footprint of one request (bytes): residual scratch, state, load,
// GMRES basis and vectors in the working precision.
int64_t footprint(const stm_request& r, const stm_server_opts& o) {
  const int64_t ne = (int64_t)r.n * r.n * r.n;
  const int64_t n = r.p + 1, n2 = n * n, n3 = n2 * n;
  const int64_t test = ne * 6 * r.q * n3, state = ne * 6 * n3, tr = ne * 24 * r.q * n2;
  const int64_t m = o.restart;
  int64_t b = 8 * (test + tr) + 8 * 2 * state + 8 * 2 * test + 8 * test + 4 * test + ne * 512;
  if (o.precision == STM_MIXED) b += 4 * (m + 1) * test + 4 * test;
  else b += 8 * (m + 1) * test;
  return b + (64 << 20);
}

// Unit-cube n^3 brick mesh, elements numbered with x fastest, face neighbours,
// and eps/mu from the first material box containing the element centre.
struct MeshBuf {
  std::vector<double> vert, eps, mu;
  std::vector<int64_t> hex, nbr;
  std::vector<uint8_t> p, q;
  stm_mesh m{};
};

void build_mesh(const stm_request& r, MeshBuf& b) {
  const int n = r.n;
  const int64_t nv1 = n + 1, ne = (int64_t)n * n * n;
  b.vert.resize(3 * nv1 * nv1 * nv1);
  for (int64_t k = 0; k <= n; ++k)
    for (int64_t j = 0; j <= n; ++j)
      for (int64_t i = 0; i <= n; ++i) {
        const int64_t v = (k * nv1 + j) * nv1 + i;
        b.vert[3 * v] = (double)i / n;
        b.vert[3 * v + 1] = (double)j / n;
        b.vert[3 * v + 2] = (double)k / n;
      }
  b.hex.resize(8 * ne);
  b.nbr.resize(6 * ne);
  b.eps.assign(ne, 1.0);
  b.mu.assign(ne, 1.0);
  b.p.assign(ne, (uint8_t)r.p);
  b.q.assign(ne, (uint8_t)r.q);
  for (int64_t k = 0; k < n; ++k)
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i) {
        const int64_t e = (k * n + j) * n + i;
        for (int v = 0; v < 8; ++v)
          b.hex[8 * e + v] = ((k + ((v >> 2) & 1)) * nv1 + (j + ((v >> 1) & 1))) * nv1 + (i + (v & 1));
        const int64_t ijk[3] = {i, j, k};
        for (int d = 0; d < 3; ++d)
          for (int s = 0; s < 2; ++s) {
            int64_t c[3] = {i, j, k};
            c[d] += s ? 1 : -1;
            b.nbr[6 * e + 2 * d + s] = (c[d] < 0 || c[d] >= n) ? -1 : (c[2] * n + c[1]) * n + c[0];
          }
        const double xc[3] = {(ijk[0] + 0.5) / n, (ijk[1] + 0.5) / n, (ijk[2] + 0.5) / n};
        for (int bx = 0; bx < r.n_boxes && bx < 4; ++bx) {
          const double* B = r.boxes[bx];
          if (xc[0] >= B[0] && xc[0] <= B[3] && xc[1] >= B[1] && xc[1] <= B[4] && xc[2] >= B[2] && xc[2] <= B[5]) {
            b.eps[e] = B[6];
            b.mu[e] = B[7];
            break;
          }
        }
      }
  b.m.n_elem = ne;
  b.m.n_vert = nv1 * nv1 * nv1;
  b.m.vert = b.vert.data();
  b.m.hex = b.hex.data();
  b.m.nbr = b.nbr.data();
  b.m.p = b.p.data();
  b.m.q = b.q.data();
  b.m.eps = b.eps.data();
  b.m.mu = b.mu.data();
  b.m.geometry = STM_GEOM_BRICK;
}

void run_job(stm_server* S, Job* J, cudaStream_t stream) {
  const stm_request& r = J->req;
  MeshBuf mb;
  build_mesh(r, mb);
  stm_opts o{};
  o.precision = S->opts.precision;
  o.tol = S->opts.tol;
  o.restart = S->opts.restart;
  o.max_it = S->opts.max_it;
  o.deterministic = 1;
  o.stream = (int64_t)(intptr_t)stream;
  o.reorth = 0;
  stm_ctx* c = nullptr;
  int rc = stm_create(&c, &mb.m, &o);
  if (rc != STM_OK) {
    J->res.status = rc;
    return;
  }
  if (r.n_src > 0) rc = stm_set_source_gauss(c, r.src, std::min(r.n_src, 8));
  if (rc == STM_OK && r.kind == 0) rc = stm_set_initial(c, 0.0, tm11_E, nullptr, nullptr);
  int iters = 0;
  double maxres = 0.0;
  for (int k = 0; rc >= 0 && k < r.n_slabs; ++k) {
    stm_solve_report rep{};
    rc = stm_slab_solve(c, r.dt, &rep);
    iters += rep.iterations;
    maxres = std::max(maxres, rep.rel_residual);
    J->res.energy = rep.energy;
  }
  J->res.iterations = iters;
  J->res.max_rel_residual = maxres;
  int64_t nt = 0, nts = 0, nst = 0;
  stm_sizes(c, &nt, &nts, &nst);
  J->res.n_state = nst;
  if (rc >= 0) {
    J->state.resize(nst);
    double t = 0.0;
    stm_get_state(c, &t, J->state.data(), STM_MEM_HOST);
    J->res.t_final = t;
  }
  stm_destroy(c);
  J->res.status = rc < 0 ? rc : (rc == STM_ENOTCONV ? STM_ENOTCONV : STM_OK);
}

void worker_main(stm_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t stream;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  for (;;) {
    Job* J = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // FIFO admission: the head request starts once its footprint fits (a request larger
      // than the whole budget starts when nothing else runs)
      auto fits = [&] {
        return !S->queue.empty() && (S->admitted_bytes + S->queue.front()->bytes <= S->opts.hbm_budget_bytes ||
                                     S->admitted_bytes == 0);
      };
      S->cv_work.wait(lk, [&] { return S->stop || fits(); });
      if (S->stop) break;
      J = S->queue.front();
      S->queue.pop_front();
      S->admitted_bytes += J->bytes;
      S->peak_bytes = std::max(S->peak_bytes, S->admitted_bytes);
      ++S->running;
      J->res.status = 2;
      J->t_start = Clock::now();
    }
    run_job(S, J, stream);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      J->t_end = Clock::now();
      S->admitted_bytes -= J->bytes;
      --S->running;
      J->res.latency_ms = std::chrono::duration<double, std::milli>(J->t_end - J->t_submit).count();
      J->res.queue_ms = std::chrono::duration<double, std::milli>(J->t_start - J->t_submit).count();
      if (J->res.status < 0) ++S->failed;
      else {
        ++S->completed;
        S->slabs_done += J->req.n_slabs;
        S->latencies.push_back(J->res.latency_ms);
      }
      S->last_done = J->t_end;
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
  cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

int32_t stm_server_create(stm_server** out, const stm_server_opts* o) {
  if (!out || !o || o->workers < 1 || o->workers > 64 || o->restart < 1 || o->restart > 15) return STM_EINVAL;
  stm_server* S = new stm_server();
  S->opts = *o;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return STM_EDEVICE;
  }
  if (S->opts.hbm_budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    S->opts.hbm_budget_bytes = (int64_t)(0.8 * (double)fr);
  }
  for (int k = 0; k < o->workers; ++k) S->workers.emplace_back(worker_main, S);
  *out = S;
  return STM_OK;
}

int32_t stm_server_submit(stm_server* S, const stm_request* r, int64_t* ticket) {
  if (!S || !r || !ticket) return STM_EINVAL;
  Job* J = new Job();
  J->req = *r;
  J->t_submit = Clock::now();
  const bool ok = r->n >= 1 && r->n <= 512 && r->p >= 0 && r->p <= 7 && r->q >= 1 && r->q <= 6 && r->n_slabs >= 0 &&
                  r->dt > 0 && r->n_boxes >= 0 && r->n_boxes <= 4 && r->n_src >= 0 && r->n_src <= 8;
  std::lock_guard<std::mutex> lk(S->mu);
  J->ticket = S->next_ticket++;
  *ticket = J->ticket;
  S->jobs[J->ticket] = J;
  ++S->submitted;
  if (!S->started) {
    S->started = true;
    S->t0 = J->t_submit;
  }
  if (!ok) {
    J->res.status = STM_EINVAL;
    J->t_end = J->t_start = J->t_submit;
    ++S->failed;
    S->cv_done.notify_all();
    return STM_OK;
  }
  J->bytes = footprint(*r, S->opts);
  J->res.footprint_bytes = J->bytes;
  J->res.status = 1;
  S->queue.push_back(J);
  S->cv_work.notify_all();
  return STM_OK;
}

int32_t stm_server_poll(stm_server* S, int64_t ticket, stm_result* res, double* state_out) {
  if (!S || !res) return STM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return STM_EINVAL;
  *res = it->second->res;
  if (state_out && res->status >= 0 && res->status != 1 && res->status != 2 && !it->second->state.empty())
    std::memcpy(state_out, it->second->state.data(), it->second->state.size() * sizeof(double));
  return STM_OK;
}

int32_t stm_server_wait(stm_server* S, int64_t ticket, stm_result* res, double* state_out) {
  if (!S || !res) return STM_EINVAL;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return STM_EINVAL;
    Job* J = it->second;
    S->cv_done.wait(lk, [&] { return J->res.status != 1 && J->res.status != 2; });
  }
  return stm_server_poll(S, ticket, res, state_out);
}

int32_t stm_server_stats(stm_server* S, stm_stats* st) {
  if (!S || !st) return STM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = S->submitted;
  st->completed = S->completed;
  st->failed = S->failed;
  st->running = S->running;
  st->queued = (int64_t)S->queue.size();
  st->peak_admitted_bytes = S->peak_bytes;
  st->hbm_budget_bytes = S->opts.hbm_budget_bytes;
  std::vector<double> l = S->latencies;
  std::sort(l.begin(), l.end());
  if (!l.empty()) {
    auto pct = [&](double p) {
      const size_t k = (size_t)std::ceil(p * l.size());
      return l[std::min(l.size() - 1, k > 0 ? k - 1 : 0)];
    };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    st->wall_s = std::chrono::duration<double>(S->last_done - S->t0).count();
    st->solves_per_s = st->wall_s > 0 ? (double)S->slabs_done / st->wall_s : 0.0;
  }
  return STM_OK;
}

int32_t stm_server_destroy(stm_server* S) {
  if (!S) return STM_OK;
  {
    // queued requests are cancelled; running ones finish
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (Job* J : S->queue) J->res.status = STM_ECANCELLED;
    S->queue.clear();
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->jobs) delete kv.second;
  delete S;
  return STM_OK;
}

}  // extern "C"
