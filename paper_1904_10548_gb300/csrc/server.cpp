// Serving: continuous batching of solve requests over resident factor
// handles (include/rapidnet.h, rapidnet_server_*).
//
// A model (network x tree x cost) is served by slots.  A slot is one factor
// handle with its own stream, device buffers for a request's data and
// results, and the last dual it computed.  Worker threads take queued
// requests in arrival order as soon as a slot of the request's model is
// free, opening a new slot when the device-memory budget allows; the solve
// runs on the slot's stream, so requests that arrive while others run
// overlap with them on the device.  Slots of one model are identical
// handles (same step size), so a result does not depend on which slot, or
// which other requests, ran alongside it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "rn_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Slot {
  rn_factor *f = nullptr;
  cudaStream_t stream = nullptr;
  double *x0 = nullptr, *q = nullptr, *dem = nullptr, *alp = nullptr;
  double *u = nullptr, *x = nullptr, *y = nullptr, *ylast = nullptr;
  bool busy = false, has_last = false;
};

struct Model {
  std::vector<double> A, B, Gd, E, Ed, xmin, xmax, xs, umin, umax, alpha0, Wu, prob;
  std::vector<int> stage_ptr, anc;
  rn_network net{};
  rn_tree tree{};
  rn_cost cost{};
  rn_opts opts{};
  int nx = 0, nu = 0, nd = 0, n = 0;
  long long slot_bytes = 0;
  std::vector<std::unique_ptr<Slot>> slots;
};

struct Request {
  long long ticket = 0;
  int key = 0;
  std::vector<double> x0, q, dem, alp, u, x, y;
  int max_iters = 0, warm = 0;
  double tol = 0.0;
  Clock::time_point t0;
  bool done = false;
  int status = RN_OK;
  rn_result res{};
  double latency = 0.0;
};

}  // namespace

struct rn_server {
  rn_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> queue;
  std::map<long long, std::unique_ptr<Request>> reqs;
  std::vector<std::unique_ptr<Model>> models;
  std::vector<std::thread> workers;
  bool stop = false;
  long long next_ticket = 1, submitted = 0, completed = 0, rejected = 0, bytes = 0;
  std::vector<double> latencies;
};

namespace {

void free_slot(Slot *s) {
  if (s->f) rapidnet_factor_free(s->f);
  for (double *p : {s->x0, s->q, s->dem, s->alp, s->u, s->x, s->y, s->ylast})
    if (p) cudaFree(p);
  if (s->stream) cudaStreamDestroy(s->stream);
  s->f = nullptr;
}

// one more slot of model m (a factor handle with the model's step size)
int open_slot(rn_server *sv, Model &m, std::unique_ptr<Slot> &out) {
  std::unique_ptr<Slot> s(new Slot());
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    rn::set_error("server: stream creation failed: %s", cudaGetErrorString(e));
    return RN_ERR_CUDA;
  }
  rn_opts o = m.opts;
  o.device = sv->opts.device;
  o.stream = s->stream;
  int rc = rapidnet_factor(&m.net, &m.tree, &m.cost, &o, &s->f);
  if (rc) {
    free_slot(s.get());
    return rc;
  }
  const size_t ny = 2 * (size_t)m.nx + m.nu;
  const size_t sizes[8] = {(size_t)m.nx, (size_t)m.nu, (size_t)m.n * m.nd, (size_t)m.n * m.nu,
                           (size_t)m.n * m.nu, (size_t)m.n * m.nx, (size_t)m.n * ny,
                           (size_t)m.n * ny};
  double **ptrs[8] = {&s->x0, &s->q, &s->dem, &s->alp, &s->u, &s->x, &s->y, &s->ylast};
  for (int k = 0; k < 8; ++k) {
    e = cudaMalloc(ptrs[k], sizes[k] * sizeof(double));
    if (e != cudaSuccess) {
      free_slot(s.get());
      rn::set_error("server: cudaMalloc failed: %s", cudaGetErrorString(e));
      return RN_ERR_NOMEM;
    }
  }
  out = std::move(s);
  return RN_OK;
}

void run_request(Model &m, Slot &s, Request &r) {
  const size_t ny = 2 * (size_t)m.nx + m.nu;
  auto fail = [&](int st) { r.status = st; };
  if (cudaMemcpyAsync(s.x0, r.x0.data(), m.nx * sizeof(double), cudaMemcpyHostToDevice,
                      s.stream) != cudaSuccess ||
      cudaMemcpyAsync(s.q, r.q.data(), m.nu * sizeof(double), cudaMemcpyHostToDevice,
                      s.stream) != cudaSuccess ||
      cudaMemcpyAsync(s.dem, r.dem.data(), r.dem.size() * sizeof(double), cudaMemcpyHostToDevice,
                      s.stream) != cudaSuccess ||
      cudaMemcpyAsync(s.alp, r.alp.data(), r.alp.size() * sizeof(double), cudaMemcpyHostToDevice,
                      s.stream) != cudaSuccess) {
    fail(RN_ERR_CUDA);
    return;
  }
  rn_result res{};
  res.u = s.u;
  res.x = s.x;
  res.y = s.y;
  const int st = rapidnet_solve_device(s.f, s.x0, s.q, s.dem, s.alp, r.max_iters, r.tol,
                                       (r.warm && s.has_last) ? s.ylast : nullptr, &res);
  r.status = st;
  r.res = res;
  if (st < 0) return;
  r.u.resize((size_t)m.n * m.nu);
  r.x.resize((size_t)m.n * m.nx);
  r.y.resize((size_t)m.n * ny);
  if (cudaMemcpyAsync(s.ylast, s.y, (size_t)m.n * ny * sizeof(double), cudaMemcpyDeviceToDevice,
                      s.stream) != cudaSuccess ||
      cudaMemcpyAsync(r.u.data(), s.u, r.u.size() * sizeof(double), cudaMemcpyDeviceToHost,
                      s.stream) != cudaSuccess ||
      cudaMemcpyAsync(r.x.data(), s.x, r.x.size() * sizeof(double), cudaMemcpyDeviceToHost,
                      s.stream) != cudaSuccess ||
      cudaMemcpyAsync(r.y.data(), s.y, r.y.size() * sizeof(double), cudaMemcpyDeviceToHost,
                      s.stream) != cudaSuccess ||
      cudaStreamSynchronize(s.stream) != cudaSuccess) {
    fail(RN_ERR_CUDA);
    return;
  }
  s.has_last = true;
}

void worker(rn_server *sv) {
  cudaSetDevice(sv->opts.device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    // the first queued request that can start: a free slot of its model, or
    // room in the budget for a new one
    Request *r = nullptr;
    Slot *slot = nullptr;
    bool open = false;
    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
      Model &m = *sv->models[(*it)->key];
      for (auto &s : m.slots)
        if (!s->busy) {
          slot = s.get();
          break;
        }
      if (!slot && sv->bytes + m.slot_bytes <= sv->opts.budget_bytes) open = true;
      if (slot || open) {
        r = *it;
        sv->queue.erase(it);
        break;
      }
    }
    if (!r) {
      if (sv->stop && sv->queue.empty()) return;
      sv->cv_work.wait(lk);
      continue;
    }
    Model &m = *sv->models[r->key];
    std::unique_ptr<Slot> fresh;
    if (open) {
      sv->bytes += m.slot_bytes;
      lk.unlock();
      const int rc = open_slot(sv, m, fresh);
      lk.lock();
      if (rc) {
        sv->bytes -= m.slot_bytes;
        r->status = rc;
        r->done = true;
        sv->completed++;
        sv->cv_done.notify_all();
        continue;
      }
      fresh->busy = true;
      slot = fresh.get();
      m.slots.push_back(std::move(fresh));
    } else {
      slot->busy = true;
    }
    lk.unlock();
    run_request(m, *slot, *r);
    const double lat = std::chrono::duration<double>(Clock::now() - r->t0).count();
    lk.lock();
    slot->busy = false;
    r->latency = lat;
    r->done = true;
    sv->completed++;
    sv->latencies.push_back(lat);
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
}

}  // namespace

extern "C" int rapidnet_server_create(const rn_server_opts *opts, rn_server **out) {
  rn::clear_error();
  if (!out) {
    rn::set_error("server_create: out is NULL");
    return RN_ERR_INVAL;
  }
  *out = nullptr;
  std::unique_ptr<rn_server> sv(new (std::nothrow) rn_server());
  if (!sv) return RN_ERR_NOMEM;
  if (opts) sv->opts = *opts;
  if (sv->opts.budget_bytes <= 0) sv->opts.budget_bytes = 8LL << 30;
  if (sv->opts.max_queue <= 0) sv->opts.max_queue = 4096;
  if (sv->opts.workers <= 0) sv->opts.workers = 8;
  if (cudaSetDevice(sv->opts.device) != cudaSuccess) {
    rn::set_error("server_create: cudaSetDevice(%d) failed", sv->opts.device);
    return RN_ERR_CUDA;
  }
  for (int k = 0; k < sv->opts.workers; ++k) sv->workers.emplace_back(worker, sv.get());
  *out = sv.release();
  return RN_OK;
}

extern "C" int rapidnet_server_add_model(rn_server *sv, const rn_network *net,
                                         const rn_tree *tree, const rn_cost *cost,
                                         const rn_opts *opts, int *key) {
  rn::clear_error();
  if (!sv || !net || !tree || !cost || !key) {
    rn::set_error("server_add_model: NULL argument");
    return RN_ERR_INVAL;
  }
  if (net->nx < 1 || net->nu < 1 || net->nd < 1 || net->ne < 0 || tree->n_nodes < 2 ||
      tree->N < 1) {
    rn::set_error("server_add_model: bad sizes");
    return RN_ERR_INVAL;
  }
  std::unique_ptr<Model> m(new Model());
  const int nx = net->nx, nu = net->nu, nd = net->nd, ne = net->ne, n = tree->n_nodes;
  auto cp = [](const double *p, size_t k) {
    return p ? std::vector<double>(p, p + k) : std::vector<double>();
  };
  m->A = cp(net->A, (size_t)nx * nx);
  m->B = cp(net->B, (size_t)nx * nu);
  m->Gd = cp(net->Gd, (size_t)nx * nd);
  m->E = cp(net->E, (size_t)ne * nu);
  m->Ed = cp(net->Ed, (size_t)ne * nd);
  m->xmin = cp(net->xmin, nx);
  m->xmax = cp(net->xmax, nx);
  m->xs = cp(net->xs, nx);
  m->umin = cp(net->umin, nu);
  m->umax = cp(net->umax, nu);
  m->alpha0 = cp(cost->alpha0, nu);
  m->Wu = cp(cost->Wu, (size_t)nu * nu);
  m->prob = cp(tree->prob, n);
  if (!tree->stage_ptr || !tree->anc) {
    rn::set_error("server_add_model: NULL tree arrays");
    return RN_ERR_INVAL;
  }
  m->stage_ptr.assign(tree->stage_ptr, tree->stage_ptr + tree->N + 2);
  m->anc.assign(tree->anc, tree->anc + n);
  auto ptr = [](std::vector<double> &v) { return v.empty() ? nullptr : v.data(); };
  m->net = rn_network{nx, nu, nd, ne, ptr(m->A), ptr(m->B), ptr(m->Gd), ptr(m->E), ptr(m->Ed),
                      ptr(m->xmin), ptr(m->xmax), ptr(m->xs), ptr(m->umin), ptr(m->umax)};
  m->tree = rn_tree{tree->N, n, m->stage_ptr.data(), m->anc.data(), ptr(m->prob)};
  m->cost = rn_cost{cost->W_alpha, ptr(m->alpha0), ptr(m->Wu), cost->Ws, cost->Wx};
  m->opts = opts ? *opts : rn_opts{};
  // RN_FACTOR_AUTO as in rapidnet_factor: the shared-operator kernels
  // wherever they apply, else (A != I, RN_PREC_FP32, a refused layout in
  // FP64) the per-node form, whose solves occupy the whole device with one
  // cooperative launch each and so run one at a time
  m->nx = nx;
  m->nu = nu;
  m->nd = nd;
  m->n = n;
  std::unique_ptr<Slot> first;
  int rc = open_slot(sv, *m, first);
  if (rc) return rc;
  rn_factor_info info{};
  rapidnet_factor_info(first->f, &info);
  m->opts.gamma = info.gamma;  // every later slot reuses the step size
  const size_t ny = 2 * (size_t)nx + nu;
  m->slot_bytes = info.device_bytes +
                  (long long)sizeof(double) * ((size_t)nx + nu + (size_t)n * (nd + nu + nu + nx + 2 * ny));
  m->slots.push_back(std::move(first));
  long long extra = 0;
  for (int k = 1; k < sv->opts.slots_per_model; ++k) {
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (sv->bytes + (2 + k) * m->slot_bytes > sv->opts.budget_bytes) break;
    }
    std::unique_ptr<Slot> more;
    if (open_slot(sv, *m, more)) break;
    m->slots.push_back(std::move(more));
    extra += m->slot_bytes;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->bytes += m->slot_bytes + extra;
  *key = (int)sv->models.size();
  sv->models.push_back(std::move(m));
  return RN_OK;
}

extern "C" int rapidnet_server_submit(rn_server *sv, int key, const double *x0, const double *q,
                                      const double *demand, const double *alpha, int max_iters,
                                      double tol, int warm, long long *ticket) {
  rn::clear_error();
  if (!sv || !x0 || !q || !demand || !alpha || !ticket || max_iters < 1) {
    rn::set_error("server_submit: NULL argument or max_iters < 1");
    return RN_ERR_INVAL;
  }
  std::unique_ptr<Request> r(new Request());
  const Model *mp = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (key < 0 || key >= (int)sv->models.size()) {
      rn::set_error("server_submit: unknown model key %d", key);
      return RN_ERR_INVAL;
    }
    if ((int)sv->queue.size() >= sv->opts.max_queue) {
      sv->rejected++;
      rn::set_error("server_submit: queue full (%d), retry later", sv->opts.max_queue);
      return RN_ERR_NOMEM;
    }
    mp = sv->models[key].get();
  }
  const Model &m = *mp;
  r->key = key;
  r->x0.assign(x0, x0 + m.nx);
  r->q.assign(q, q + m.nu);
  r->dem.assign(demand, demand + (size_t)m.n * m.nd);
  r->alp.assign(alpha, alpha + (size_t)m.n * m.nu);
  r->max_iters = max_iters;
  r->tol = tol;
  r->warm = warm;
  r->t0 = Clock::now();
  std::lock_guard<std::mutex> lk(sv->mu);
  r->ticket = sv->next_ticket++;
  *ticket = r->ticket;
  sv->queue.push_back(r.get());
  sv->reqs[r->ticket] = std::move(r);
  sv->submitted++;
  sv->cv_work.notify_one();
  return RN_OK;
}

extern "C" int rapidnet_server_wait(rn_server *sv, long long ticket, double timeout_s,
                                    rn_result *out, double *latency_s) {
  rn::clear_error();
  if (!sv) {
    rn::set_error("server_wait: NULL server");
    return RN_ERR_INVAL;
  }
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) {
    rn::set_error("server_wait: unknown ticket %lld", ticket);
    return RN_ERR_INVAL;
  }
  Request *r = it->second.get();
  auto ready = [&] { return r->done; };
  if (timeout_s < 0) {
    sv->cv_done.wait(lk, ready);
  } else if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    rn::set_error("server_wait: ticket %lld not done yet", ticket);
    return RN_ERR_TIMEOUT;
  }
  const int st = r->status;
  if (out) {
    double *u = out->u, *x = out->x, *y = out->y;
    *out = r->res;
    out->u = u;
    out->x = x;
    out->y = y;
    if (u && !r->u.empty()) std::memcpy(u, r->u.data(), r->u.size() * sizeof(double));
    if (x && !r->x.empty()) std::memcpy(x, r->x.data(), r->x.size() * sizeof(double));
    if (y && !r->y.empty()) std::memcpy(y, r->y.data(), r->y.size() * sizeof(double));
  }
  if (latency_s) *latency_s = r->latency;
  sv->reqs.erase(it);
  return st;
}

extern "C" int rapidnet_server_stats(rn_server *sv, rn_server_stats *st) {
  rn::clear_error();
  if (!sv || !st) {
    rn::set_error("server_stats: NULL argument");
    return RN_ERR_INVAL;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  st->submitted = sv->submitted;
  st->completed = sv->completed;
  st->rejected = sv->rejected;
  st->models = (int)sv->models.size();
  st->slots = 0;
  for (auto &m : sv->models) st->slots += (int)m->slots.size();
  st->bytes_in_use = sv->bytes;
  std::vector<double> l = sv->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) {
    if (l.empty()) return 0.0;
    size_t i = (size_t)std::min<double>(l.size() - 1, std::max(0.0, p * (l.size() - 1) + 0.5));
    return l[i];
  };
  st->p50_s = pct(0.50);
  st->p99_s = pct(0.99);
  double s = 0.0;
  for (double v : l) s += v;
  st->mean_s = l.empty() ? 0.0 : s / l.size();
  return RN_OK;
}

extern "C" void rapidnet_server_destroy(rn_server *sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto &t : sv->workers) t.join();
  cudaSetDevice(sv->opts.device);
  for (auto &m : sv->models)
    for (auto &s : m->slots) free_slot(s.get());
  delete sv;
}
