// server.cu -- continuous-batching solve server behind eb_server_* (host
// code only; no counterpart in the paper).  One worker thread per server owns
// the device work: it admits queued requests while the memory budget and slot
// count allow, and advances all admitted instances together with batch_step
// (one cooperative persistent launch per step, every instance with its own CTA
// group and barrier), `step_iters` FP64 outer iterations at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "eb_internal.h"

using namespace ebp;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  unsigned long long ticket = 0;
  eb_geom_desc desc{};
  std::vector<eb_prim> prims;
  std::vector<eb_csg> nodes;
  std::vector<double> rhs, sigma;
  long long ncell = 0;
  long long estimate = 0;  // device bytes assumed at admission
  double t_submit = 0.0;
};

struct Active {
  std::unique_ptr<Request> req;
  eb_geom* G = nullptr;
  eb_poisson* P = nullptr;
  double* d_fields = nullptr;  // rhs [2n] | sigma [n] | phi [2n]
  long long bytes = 0;
  int cycles = 0, iters = 0;
  double rel = 0.0, bnorm = 0.0;
};

struct Done {
  std::vector<double> phi;
  eb_solve_info info{};
};

// Upper estimate of the device bytes of one instance before it is built: per
// cell the FP64 solution and right-hand side of both phases (32 B), the
// caller-side fields (40 B), the inner-precision hierarchy (<= 32 B x 8/7..4/3),
// geometry arrays per level (~12 B) and the FP64 level copies of the
// multi-launch path (<= 43 B); cut cells and sparse rows stay well inside the
// slack; plus the node labels, a fixed part for the small buffers and the
// dense bottom inverse: coarsening halves even sizes down to 8 cells but may
// stop earlier on the geometry, so any bottom of at most 1024 unknowns is
// possible unless the finest grid alone is already larger at the deepest
// level it could reach.  (Set-up scratch of the inverse is transient.)
long long estimate_bytes(const eb_geom_desc& d) {
  long long n = 1, nodes = 1, deepest = 2;
  for (int k = 0; k < d.dim; ++k) {
    n *= d.n[k];
    nodes *= d.n[k] + 1;
    int m = d.n[k];
    while (m % 2 == 0 && m / 2 >= 8) m /= 2;
    deepest *= m;
  }
  long long inv = deepest > 1024 ? 0 : 1024ll * 1024ll * 8ll;
  return n * 200 + nodes + (8ll << 20) + inv;
}

}  // namespace

struct eb_server {
  eb_server_opts o{};
  long long budget = 0;
  cudaStream_t s = nullptr;
  std::mutex m;
  std::condition_variable cv_work, cv_done;
  std::deque<std::unique_ptr<Request>> queue;
  std::unordered_map<unsigned long long, Done> done;
  std::unordered_map<unsigned long long, int> state;  // 0 queued, 1 active, 2 done
  unsigned long long next_ticket = 1;
  bool stop = false;
  // statistics (under m)
  long long submitted = 0, completed = 0, failed = 0, n_active = 0, steps = 0, misses = 0;
  long long used = 0, peak = 0, cells_done = 0;
  double t_first = 0.0, t_last = 0.0;
  std::vector<double> latencies;
  std::thread worker;

  void finish(Active& a, eb_status st, bool copy);
  bool admit_one(std::vector<Active>& act);
  void run();
};

extern "C" void eb_server_opts_default(eb_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->hbm_budget_bytes = 0.0;
  o->max_slots = 64;
  o->queue_cap = 1 << 16;
  o->step_iters = 1;
  o->device = 0;
  eb_solver_opts_default(&o->solver);
}

// result of an instance: phi and info copied to the host, device memory freed
void eb_server::finish(Active& a, eb_status st, bool copy) {
  Done d;
  long long n = a.req->ncell;
  if (copy && a.P && st != EB_ERR_CUDA) {
    d.phi.resize(2 * n);
    double* d_phi = a.d_fields + 3 * n;
    eb_status c = batch_copy_out(a.P, d_phi, s);
    cudaError_t e = c == EB_OK ? cudaMemcpyAsync(d.phi.data(), d_phi, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, s)
                               : cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = EB_ERR_CUDA;
      d.phi.clear();
    }
  }
  d.info.status = st;
  d.info.outer_iters = a.iters;
  d.info.vcycles = a.cycles;
  d.info.rel_res = a.rel;
  d.info.bnorm = a.bnorm;
  if (a.P) eb_poisson_destroy(a.P);
  if (a.G) eb_geom_destroy(a.G);
  if (a.d_fields) cudaFree(a.d_fields);
  double t = now_s();
  std::lock_guard<std::mutex> lk(m);
  used -= a.bytes;
  --n_active;
  if (st == EB_OK) {
    ++completed;
    cells_done += n;
    latencies.push_back((t - a.req->t_submit) * 1e3);
    t_last = t;
  } else {
    ++failed;
  }
  state[a.req->ticket] = 2;
  done.emplace(a.req->ticket, std::move(d));
  cv_done.notify_all();
}

// Admits the request at the head of the queue if a slot and the budget allow;
// returns false when nothing was admitted.
bool eb_server::admit_one(std::vector<Active>& act) {
  std::unique_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(m);
    if (queue.empty() || (int)act.size() >= o.max_slots) return false;
    Request& head = *queue.front();
    bool alone_too_big = head.estimate > budget;
    if (!alone_too_big && used + head.estimate > budget) return false;  // wait for memory to free up
    r = std::move(queue.front());
    queue.pop_front();
    ++n_active;
    state[r->ticket] = 1;
    if (!alone_too_big) used += r->estimate;  // reserved until the real size is known
    peak = std::max(peak, used);
    if (t_first == 0.0) t_first = now_s();
  }
  Active a;
  a.req = std::move(r);
  Request& q = *a.req;
  if (q.estimate > budget) {
    set_error("request larger than the server's memory budget");
    finish(a, EB_ERR_OOM, false);
    return true;
  }
  a.bytes = q.estimate;  // accounted until replaced by the measured size
  eb_status st = eb_geom_build(&q.desc, s, &a.G);
  if (st == EB_OK) {
    eb_solver_opts so = o.solver;
    so.launch_mode = 0;
    st = eb_poisson_setup(a.G, &so, s, &a.P);
  }
  long long n = q.ncell;
  if (st == EB_OK) {
    cudaError_t e = cudaMalloc((void**)&a.d_fields, 5 * n * sizeof(double));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(a.d_fields, q.rhs.data(), 2 * n * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !q.sigma.empty())
      e = cudaMemcpyAsync(a.d_fields + 2 * n, q.sigma.data(), n * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.d_fields + 3 * n, 0, 2 * n * sizeof(double), s);
    if (e != cudaSuccess) st = cuda_fail(e, "server fields");
  }
  if (st == EB_OK)
    st = batch_prepare(a.P, a.d_fields, q.sigma.empty() ? nullptr : a.d_fields + 2 * n, a.d_fields + 3 * n, s);
  if (st == EB_OK && cudaStreamSynchronize(s) != cudaSuccess) st = EB_ERR_CUDA;
  if (st != EB_OK) {
    finish(a, st, false);
    return true;
  }
  eb_geom_info gi;
  eb_geom_query(a.G, &gi);
  long long real = gi.device_bytes + poisson_device_bytes(a.P) + 5 * n * (long long)sizeof(double);
  {
    std::lock_guard<std::mutex> lk(m);
    used += real - a.bytes;
    a.bytes = real;
    if (real > q.estimate) ++misses;
    peak = std::max(peak, used);
  }
  act.push_back(std::move(a));
  return true;
}

void eb_server::run() {
  cudaSetDevice(o.device);
  std::vector<Active> act;
  for (;;) {
    while (admit_one(act)) {
    }
    if (act.empty()) {
      std::unique_lock<std::mutex> lk(m);
      if (stop && queue.empty()) break;
      cv_work.wait_for(lk, std::chrono::milliseconds(20));
      continue;
    }
    std::vector<eb_poisson*> Ps(act.size());
    for (size_t i = 0; i < act.size(); ++i) Ps[i] = act[i].P;
    eb_status st = batch_step(Ps.data(), (int)Ps.size(), nullptr, nullptr, nullptr, false, false, o.step_iters, s,
                              nullptr);
    {
      std::lock_guard<std::mutex> lk(m);
      ++steps;
    }
    std::vector<Active> keep;
    for (Active& a : act) {
      eb_status fin = EB_OK;
      bool end = false;
      if (st != EB_OK) {
        fin = st;
        end = true;
      } else {
        eb_solve_info inf;
        batch_info(a.P, &inf);
        a.iters += inf.outer_iters;
        a.cycles += inf.vcycles;
        a.rel = inf.rel_res;
        a.bnorm = inf.bnorm;
        if (inf.status == 7) {  // step limit reached: continue at the next step unless capped
          if (a.cycles + o.solver.inner_cycles > o.solver.max_cycles) {
            fin = EB_ERR_NOT_CONVERGED;
            end = true;
          }
        } else {
          fin = (eb_status)inf.status;
          end = true;
        }
      }
      if (end) finish(a, fin, fin == EB_OK || fin == EB_ERR_NOT_CONVERGED);
      else keep.push_back(std::move(a));
    }
    act.swap(keep);
  }
}

static eb_status copy_request(const eb_geom_desc* d, const double* h_rhs, const double* h_sigma, Request& r) {
  if (!d || !h_rhs || d->dim < 2 || d->dim > 3 || d->n_prims < 0 || d->n_prims > EB_MAX_PRIMS || d->n_nodes < 0 ||
      d->n_nodes > EB_MAX_NODES || (d->n_prims && !d->prims) || (d->n_nodes && !d->nodes)) {
    set_error("invalid request");
    return EB_ERR_INVALID;
  }
  long long n = 1;
  for (int k = 0; k < d->dim; ++k) {
    if (d->n[k] < 1 || d->n[k] > (1 << 16)) {
      set_error("invalid request size");
      return EB_ERR_INVALID;
    }
    n *= d->n[k];
  }
  r.desc = *d;
  r.prims.assign(d->prims, d->prims + d->n_prims);
  r.nodes.assign(d->nodes, d->nodes + d->n_nodes);
  r.desc.prims = r.prims.data();
  r.desc.nodes = r.nodes.data();
  r.ncell = n;
  r.rhs.assign(h_rhs, h_rhs + 2 * n);
  if (h_sigma) r.sigma.assign(h_sigma, h_sigma + n);
  r.estimate = estimate_bytes(*d);
  return EB_OK;
}

extern "C" eb_status eb_server_create(const eb_server_opts* o, eb_server** out) {
  if (!out) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  *out = nullptr;
  eb_server_opts opt;
  if (o) opt = *o;
  else eb_server_opts_default(&opt);
  if (opt.max_slots < 1 || opt.max_slots > 1024 || opt.queue_cap < 1 || opt.step_iters < 1 ||
      opt.solver.max_cycles < 1 || opt.solver.inner_cycles < 1) {
    set_error("invalid server options");
    return EB_ERR_INVALID;
  }
  cudaError_t e = cudaSetDevice(opt.device);
  size_t fr = 0, tot = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
  if (e != cudaSuccess) return cuda_fail(e, "server device");
  eb_server* S = new eb_server();
  S->o = opt;
  S->budget = opt.hbm_budget_bytes > 0.0 ? (long long)opt.hbm_budget_bytes : (long long)(fr / 2);
  e = cudaStreamCreateWithFlags(&S->s, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete S;
    return cuda_fail(e, "server stream");
  }
  S->worker = std::thread([S] { S->run(); });
  *out = S;
  return EB_OK;
}

extern "C" eb_status eb_server_submit(eb_server* S, const eb_geom_desc* desc, const double* h_rhs,
                                      const double* h_sigma, unsigned long long* ticket) {
  if (!S || !ticket) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  auto r = std::make_unique<Request>();
  eb_status st = copy_request(desc, h_rhs, h_sigma, *r);
  if (st != EB_OK) return st;
  std::lock_guard<std::mutex> lk(S->m);
  if (S->stop) {
    set_error("server stopping");
    return EB_ERR_INVALID;
  }
  if ((int)S->queue.size() >= S->o.queue_cap) {
    set_error("server queue full");
    return EB_ERR_BUSY;
  }
  r->ticket = S->next_ticket++;
  r->t_submit = now_s();
  *ticket = r->ticket;
  S->state[r->ticket] = 0;
  S->queue.push_back(std::move(r));
  ++S->submitted;
  S->cv_work.notify_one();
  return EB_OK;
}

static eb_status take_result(eb_server* S, unsigned long long ticket, double* h_phi, eb_solve_info* info) {
  auto it = S->done.find(ticket);
  Done& d = it->second;
  if (h_phi && !d.phi.empty()) std::memcpy(h_phi, d.phi.data(), d.phi.size() * sizeof(double));
  if (info) *info = d.info;
  S->done.erase(it);
  S->state.erase(ticket);
  return EB_OK;
}

extern "C" eb_status eb_server_poll(eb_server* S, unsigned long long ticket, double* h_phi, eb_solve_info* info) {
  if (!S) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(S->m);
  auto it = S->state.find(ticket);
  if (it == S->state.end()) {
    set_error("unknown ticket");
    return EB_ERR_INVALID;
  }
  if (it->second != 2) return EB_ERR_BUSY;
  return take_result(S, ticket, h_phi, info);
}

extern "C" eb_status eb_server_wait(eb_server* S, unsigned long long ticket, double timeout_s, double* h_phi,
                                    eb_solve_info* info) {
  if (!S) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  std::unique_lock<std::mutex> lk(S->m);
  auto ready = [&] {
    auto it = S->state.find(ticket);
    return it == S->state.end() || it->second == 2;
  };
  // NaN, negative and infinite timeouts become 0 and 1e7 s: the clock arithmetic must not overflow
  const double t = std::isfinite(timeout_s) ? std::min(std::max(0.0, timeout_s), 1e7) : (timeout_s > 0 ? 1e7 : 0.0);
  S->cv_done.wait_for(lk, std::chrono::duration<double>(t), ready);
  auto it = S->state.find(ticket);
  if (it == S->state.end()) {
    set_error("unknown ticket");
    return EB_ERR_INVALID;
  }
  if (it->second != 2) return EB_ERR_BUSY;
  return take_result(S, ticket, h_phi, info);
}

extern "C" eb_status eb_server_query(eb_server* S, eb_server_stats* out) {
  if (!S || !out) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(S->m);
  std::memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->queued = (long long)S->queue.size();
  out->active = S->n_active;
  std::vector<double> l = S->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    size_t k = (size_t)std::min<double>((double)l.size() - 1, std::ceil(q * (double)l.size()) - 1);
    return l[k];
  };
  out->p50_ms = pct(0.50);
  out->p99_ms = pct(0.99);
  out->cells_completed = S->cells_done;
  double span = S->t_last - S->t_first;
  out->cells_per_s = span > 0.0 ? (double)S->cells_done / span : 0.0;
  out->hbm_budget = S->budget;
  out->hbm_used = S->used;
  out->hbm_peak = S->peak;
  out->steps = S->steps;
  out->estimate_misses = S->misses;
  return EB_OK;
}

extern "C" void eb_server_destroy(eb_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->m);
    S->stop = true;
    S->cv_work.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  if (S->s) cudaStreamDestroy(S->s);
  delete S;
}
