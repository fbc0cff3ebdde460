// Served stream: a request server with continuous batching on one device.
//
// Requests are independent time-stepping problems (heat, wave, Schroedinger;
// any grid size and interface curve).  The server keeps every admitted
// request's domain tables, time-level fields, Krylov workspace, boundary
// data and source on the device until the request completes, and advances
// all resident requests together: each tick is one lockstep batch step
// (grouped tcgen05 passes over all instances' tiles, one CUDA graph per
// GMRES iteration).  Between ticks, completed requests are retired (result
// copied to the caller's host buffer, device memory freed) and arrived
// requests are admitted first come first served while a slot is free and
// their exact device bytes fit the budget and the free device memory.
// Host plan building (geometry, cut edges, coefficient tables: Procedure 1,
// Sec. 3.3) is the expensive host part of admission; worker threads start it
// as soon as a request has arrived, while the device is busy with the
// resident requests.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

using namespace kfbi;

namespace {

struct PlanJob {
  int stage = 0;  // 0 waiting, 1 building, 2 built (guarded by the server mutex)
  Plan plan;
  kfbi_status status = KFBI_OK;
  std::string err;
};

struct Req {
  kfbi_request r{};
  int id = 0;
  int state = KFBI_REQ_QUEUED;
  kfbi_status status = KFBI_OK;
  double admitted = -1.0, finished = -1.0;
  int admit_tick = -1, finish_tick = -1;
  std::shared_ptr<PlanJob> job;
  kfbi_domain* D = nullptr;
  kfbi_state* S = nullptr;
  double* d_g = nullptr;    // steps x gstride Dirichlet data
  double* d_src = nullptr;  // heat source profile or Schroedinger potential, (M-1)^2
  size_t gstride = 0;       // doubles per step of d_g
  std::vector<double> coef; // heat source coefficients per step
  int steps_done = 0, max_iters = 0;
  double max_res = 0.0;
  long long bytes = 0;
};

using Clock = std::chrono::steady_clock;

}  // namespace

struct kfbi_server {
  kfbi_server_desc desc{};
  cudaStream_t st = nullptr;
  kfbi_batch* B = nullptr;
  std::vector<std::unique_ptr<Req>> reqs;
  std::vector<int> queue;     // not yet admitted, ordered by (arrival, id)
  std::vector<int> resident;  // in admission order
  bool set_changed = false;
  long long budget = 0, used = 0;
  double* d_stage = nullptr;  // staging for initial grids and results
  size_t stage_cap = 0;       // doubles
  kfbi_server_stats stats{};
  Clock::time_point t0;
  bool wall = false;  // run(): workers read the wall clock
  // plan workers
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  double published_now = -1e300;
  std::vector<std::thread> workers;
  std::string err;

  double clock_now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

double worker_now(kfbi_server* S) { return S->wall ? S->clock_now() : S->published_now; }

// The earliest arrived request whose plan nobody has started (server mutex held).
Req* next_plan_job(kfbi_server* S, double now) {
  for (int id : S->queue) {
    Req& q = *S->reqs[id];
    if (q.r.arrival > now) return nullptr;  // queue is ordered by arrival
    if (q.job->stage == 0) return &q;
  }
  return nullptr;
}

void build_job(PlanJob* job, const kfbi_domain_desc& desc) {
  std::string err;
  Plan plan;
  kfbi_status s = build_plan(desc, plan, err);
  job->plan = std::move(plan);
  job->status = s;
  job->err = err;
}

void worker_loop(kfbi_server* S) {
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    Req* q = next_plan_job(S, worker_now(S));
    if (!q) {
      S->cv.wait_for(lk, std::chrono::milliseconds(1));
      continue;
    }
    std::shared_ptr<PlanJob> job = q->job;
    const kfbi_domain_desc desc = q->r.domain;
    job->stage = 1;
    lk.unlock();
    build_job(job.get(), desc);
    lk.lock();
    job->stage = 2;
    S->cv.notify_all();
  }
}

void ensure_stage(kfbi_server* S, size_t doubles) {
  if (doubles <= S->stage_cap) return;
  if (S->d_stage) KFBI_CUDA(cudaFree(S->d_stage));
  S->d_stage = nullptr;
  S->stage_cap = 0;
  KFBI_CUDA(cudaMalloc(&S->d_stage, doubles * sizeof(double)));
  S->stage_cap = doubles;
}

void release(kfbi_server* S, Req& q) {
  if (q.S) kfbi_state_destroy(q.S);
  if (q.D) kfbi_destroy_domain(q.D);
  if (q.d_g) cudaFree(q.d_g);
  if (q.d_src) cudaFree(q.d_src);
  q.S = nullptr;
  q.D = nullptr;
  q.d_g = nullptr;
  q.d_src = nullptr;
  S->used -= q.bytes;
  q.job.reset();
}

void fail(kfbi_server* S, Req& q, kfbi_status s, double now) {
  release(S, q);
  q.state = KFBI_REQ_FAILED;
  q.status = s;
  q.finished = now;
  q.finish_tick = S->stats.ticks;
  S->stats.failed++;
}

// Bytes of a request's own device data besides its domain and state.
long long data_bytes(const kfbi_request& r, const Plan& P) {
  const int planes = r.equation == KFBI_SCHRODINGER ? 2 : 1;
  long long b = (long long)r.steps * planes * P.nb * (long long)sizeof(double);
  const bool has_grid = (r.equation == KFBI_HEAT && r.src_profile) || r.equation == KFBI_SCHRODINGER;
  if (has_grid) b += (long long)P.n1 * P.n1 * (long long)sizeof(double);
  return b;
}

template <class T>
void upload(T* dst, const void* src, size_t n, kfbi_server* S) {
  KFBI_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, S->st));
  S->stats.h2d_bytes += (long long)(n * sizeof(T));
}

// Make request q resident (domain, state, data, initial fields).
void make_resident(kfbi_server* S, Req& q, double now) {
  const Plan& P = q.job->plan;
  const kfbi_request& r = q.r;
  const int planes = r.equation == KFBI_SCHRODINGER ? 2 : 1;
  const size_t grid = (size_t)P.n1 * P.n1;
  q.D = domain_from_plan(P, S->st);
  kfbi_status s = kfbi_state_create(q.D, r.equation, &q.S);
  if (s != KFBI_OK) throw Status{s, kfbi_last_error(q.D)};
  q.gstride = (size_t)planes * P.nb;
  KFBI_CUDA(cudaMalloc(&q.d_g, (size_t)r.steps * q.gstride * sizeof(double)));
  upload<double>(q.d_g, r.g, (size_t)r.steps * q.gstride, S);
  const double* grid_src = r.equation == KFBI_HEAT ? r.src_profile
                           : r.equation == KFBI_SCHRODINGER ? r.potential : nullptr;
  if (grid_src) {
    KFBI_CUDA(cudaMalloc(&q.d_src, grid * sizeof(double)));
    upload<double>(q.d_src, grid_src, grid, S);
  }
  if (r.equation == KFBI_HEAT) {
    q.coef.assign(r.steps, 1.0);
    if (r.src_coef) q.coef.assign(r.src_coef, r.src_coef + r.steps);
  }
  // initial fields through the staging buffer
  const int nfields = r.equation == KFBI_WAVE ? 4 : (r.equation == KFBI_HEAT && r.src_init ? 3 : 2);
  ensure_stage(S, nfields * planes * grid);
  double* f0 = S->d_stage;
  double* f1 = f0 + planes * grid;
  double* f2 = f1 + planes * grid;
  double* f3 = f2 + planes * grid;
  upload<double>(f0, r.u0, planes * grid, S);
  upload<double>(f1, r.lap_u0, planes * grid, S);
  if (r.equation == KFBI_HEAT) {
    if (r.src_init) upload<double>(f2, r.src_init, grid, S);
    s = kfbi_state_init_heat(q.S, r.dt, f0, f1, r.src_init ? f2 : nullptr, S->st);
  } else if (r.equation == KFBI_WAVE) {
    upload<double>(f2, r.u1, grid, S);
    upload<double>(f3, r.lap_u1, grid, S);
    s = kfbi_state_init_wave(q.S, r.dt, r.theta, f0, f1, f2, f3, S->st);
  } else {
    s = kfbi_state_init_schrodinger(q.S, r.dt, f0, f1, S->st);
  }
  if (s != KFBI_OK) throw Status{s, kfbi_last_error(q.D)};
  KFBI_CUDA(cudaStreamSynchronize(S->st));
  q.bytes = kfbi_domain_device_bytes(q.D) + kfbi_state_device_bytes(q.S) + data_bytes(r, P);
  q.state = KFBI_REQ_RESIDENT;
  q.admitted = now;
  q.admit_tick = S->stats.ticks;
}

// First come first served admission at time now.
void admit(kfbi_server* S, double now) {
  while (!S->queue.empty()) {
    Req& q = *S->reqs[S->queue.front()];
    if (q.r.arrival > now) return;
    if ((int)S->resident.size() >= S->desc.max_resident) return;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (q.job->stage == 0) {
        // nobody took it yet: build here
        q.job->stage = 1;
        lk.unlock();
        build_job(q.job.get(), q.r.domain);
        lk.lock();
        q.job->stage = 2;
      } else if (q.job->stage == 1) {
        // a worker is building it: wait only when the device would idle
        if (!S->resident.empty()) return;
        S->cv.wait(lk, [&] { return q.job->stage == 2; });
      }
    }
    S->queue.erase(S->queue.begin());
    if (q.job->status != KFBI_OK) {
      S->err = "request " + std::to_string(q.id) + ": " + q.job->err;
      fail(S, q, q.job->status, now);
      continue;
    }
    const Plan& P = q.job->plan;
    const long long need = kfbi::domain_bytes_for(P) +
                           state_bytes_for(((P.n1 + 127) / 128) * 128, P.nb, q.r.equation) +
                           data_bytes(q.r, P);
    if (need > S->budget) {
      S->err = "request " + std::to_string(q.id) + " needs more device memory than the budget";
      fail(S, q, KFBI_ERR_OOM, now);
      continue;
    }
    size_t free_b = 0, total_b = 0;
    KFBI_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (S->used + need > S->budget || need + S->desc.hbm_reserve_bytes > (long long)free_b) {
      // does not fit now: it stays at the head until memory is freed
      S->queue.insert(S->queue.begin(), q.id);
      return;
    }
    try {
      make_resident(S, q, now);
    } catch (const Status& e) {
      S->err = "request " + std::to_string(q.id) + ": " + e.msg;
      fail(S, q, e.code, now);
      continue;
    }
    S->used += q.bytes;
    S->stats.peak_device_bytes = std::max(S->stats.peak_device_bytes, S->used);
    S->stats.admitted++;
    S->resident.push_back(q.id);
    S->set_changed = true;
  }
}

void retire(kfbi_server* S, double now) {
  std::vector<int> keep;
  for (int id : S->resident) {
    Req& q = *S->reqs[id];
    if (q.state == KFBI_REQ_FAILED) {
      S->set_changed = true;
      continue;
    }
    if (q.steps_done < q.r.steps) {
      keep.push_back(id);
      continue;
    }
    const int planes = q.r.equation == KFBI_SCHRODINGER ? 2 : 1;
    const size_t grid = (size_t)q.D->n1 * q.D->n1 * planes;
    ensure_stage(S, grid);
    kfbi_status s = kfbi_state_get_u(q.S, S->d_stage, S->st);
    if (s != KFBI_OK) throw Status{s, kfbi_last_error(q.D)};
    KFBI_CUDA(cudaMemcpyAsync(q.r.u_out, S->d_stage, grid * sizeof(double), cudaMemcpyDeviceToHost,
                              S->st));
    KFBI_CUDA(cudaStreamSynchronize(S->st));
    S->stats.d2h_bytes += (long long)(grid * sizeof(double));
    release(S, q);
    q.state = KFBI_REQ_DONE;
    q.finished = S->wall ? S->clock_now() : now;
    q.finish_tick = S->stats.ticks;
    S->stats.completed++;
    S->set_changed = true;
  }
  S->resident.swap(keep);
}

// One lockstep step of every resident request.
kfbi_status step_resident(kfbi_server* S, double now) {
  const int n = (int)S->resident.size();
  if (n == 0) return KFBI_OK;
  std::vector<kfbi_domain*> doms(n);
  std::vector<kfbi_state*> states(n);
  std::vector<const void*> g(n);
  std::vector<const double*> src(n);
  std::vector<double> scale(n, 1.0);
  for (int i = 0; i < n; ++i) {
    Req& q = *S->reqs[S->resident[i]];
    doms[i] = q.D;
    states[i] = q.S;
    g[i] = q.d_g + (size_t)q.steps_done * q.gstride;
    src[i] = q.d_src;
    if (q.r.equation == KFBI_HEAT) scale[i] = q.coef[q.steps_done];
  }
  if (S->set_changed) {
    batch_bind(S->B, doms.data(), n);
    S->set_changed = false;
  }
  std::vector<kfbi_solve_info> infos(n);
  const auto t = Clock::now();
  kfbi_status s = batch_step(S->B, states.data(), g.data(), src.data(), scale.data(), infos.data(),
                             S->st);
  S->stats.busy_seconds += std::chrono::duration<double>(Clock::now() - t).count();
  S->stats.ticks++;
  S->stats.resident_ticks += n;
  if (s != KFBI_OK && s != KFBI_ERR_NOT_CONVERGED && s != KFBI_ERR_NONFINITE) {
    S->err = std::string("batch step failed: ") + kfbi_batch_last_error(S->B);
    for (int id : S->resident) fail(S, *S->reqs[id], s, now);
    S->resident.clear();
    S->set_changed = true;
    return s;
  }
  for (int i = 0; i < n; ++i) {
    Req& q = *S->reqs[S->resident[i]];
    q.steps_done++;
    q.max_iters = std::max(q.max_iters, infos[i].iters);
    if (std::isfinite(infos[i].rel_residual)) q.max_res = std::max(q.max_res, infos[i].rel_residual);
    S->stats.grid_point_steps += (double)q.D->M * (double)q.D->M;
    if (!infos[i].converged) {
      const bool nonfinite = !std::isfinite(infos[i].rel_residual);
      S->err = "request " + std::to_string(q.id) +
               (nonfinite ? ": non-finite density residual" : ": GMRES reached gmres_maxit");
      fail(S, q, nonfinite ? KFBI_ERR_NONFINITE : KFBI_ERR_NOT_CONVERGED, now);
    }
  }
  return KFBI_OK;
}

kfbi_status tick_impl(kfbi_server* S, double now, int* n_resident) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->published_now = now;
  }
  S->cv.notify_all();
  const auto ta = Clock::now();
  admit(S, now);
  S->stats.admit_seconds += std::chrono::duration<double>(Clock::now() - ta).count();
  if (n_resident) *n_resident = (int)S->resident.size();
  kfbi_status s = step_resident(S, now);
  if (s != KFBI_OK) return s;
  retire(S, now);
  return KFBI_OK;
}

kfbi_status check_request(const kfbi_server* S, const kfbi_request* r, std::string& why) {
  if (!r) return why = "request is NULL", KFBI_ERR_ARG;
  if (r->domain.precision != KFBI_MIXED_TF32)
    return why = "served requests run on KFBI_MIXED_TF32 domains", KFBI_ERR_ARG;
  if (r->domain.gmres_restart != S->desc.gmres_restart)
    return why = "the request's gmres_restart must equal the server's", KFBI_ERR_ARG;
  if (r->domain.gmres_maxit < 1 || !(r->domain.gmres_tol > 0.0))
    return why = "GMRES parameters out of range", KFBI_ERR_ARG;
  if (r->equation < KFBI_HEAT || r->equation > KFBI_SCHRODINGER)
    return why = "unknown equation", KFBI_ERR_ARG;
  if (r->steps < 1 || !(r->dt > 0.0) || !(r->arrival >= 0.0))
    return why = "steps >= 1, dt > 0 and arrival >= 0 are required", KFBI_ERR_ARG;
  if (!r->u0 || !r->lap_u0 || !r->g || !r->u_out)
    return why = "u0, lap_u0, g and u_out are required", KFBI_ERR_ARG;
  if (r->equation == KFBI_WAVE && (!r->u1 || !r->lap_u1 || !(r->theta > 0.0)))
    return why = "wave requests need u1, lap_u1 and theta > 0", KFBI_ERR_ARG;
  if (r->equation == KFBI_SCHRODINGER && !r->potential)
    return why = "Schroedinger requests need the potential", KFBI_ERR_ARG;
  return KFBI_OK;
}

}  // namespace

extern "C" {

kfbi_status kfbi_server_create(const kfbi_server_desc* desc, void* stream, kfbi_server** out) {
  if (!out) return KFBI_ERR_ARG;
  *out = nullptr;
  if (!desc || desc->max_resident < 1 || desc->max_resident > 4096 || desc->hbm_budget_bytes < 0 ||
      desc->hbm_reserve_bytes < 0 || desc->gmres_restart < 1 || desc->gmres_restart > 64 ||
      desc->plan_threads < 0 || desc->plan_threads > 64) {
    set_global_error("kfbi_server_create: max_resident 1..4096, budgets >= 0, gmres_restart 1..64, "
                     "plan_threads 0..64");
    return KFBI_ERR_ARG;
  }
  kfbi_server* S = new (std::nothrow) kfbi_server();
  if (!S) return KFBI_ERR_OOM;
  S->desc = *desc;
  S->st = (cudaStream_t)stream;
  S->t0 = Clock::now();
  kfbi_status s = guarded(nullptr, [&]() -> kfbi_status {
    S->B = batch_new();
    size_t free_b = 0, total_b = 0;
    KFBI_CUDA(cudaMemGetInfo(&free_b, &total_b));
    S->budget = desc->hbm_budget_bytes > 0
                    ? desc->hbm_budget_bytes
                    : std::max<long long>(0, (long long)free_b - desc->hbm_reserve_bytes);
    return KFBI_OK;
  });
  if (s != KFBI_OK) {
    kfbi_server_destroy(S);
    return s;
  }
  for (int t = 0; t < desc->plan_threads; ++t) S->workers.emplace_back(worker_loop, S);
  *out = S;
  return KFBI_OK;
}

void kfbi_server_destroy(kfbi_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (std::thread& t : S->workers) t.join();
  cudaDeviceSynchronize();
  for (int id : S->resident) release(S, *S->reqs[id]);
  if (S->B) kfbi_batch_destroy(S->B);
  if (S->d_stage) cudaFree(S->d_stage);
  delete S;
}

kfbi_status kfbi_server_submit(kfbi_server* S, const kfbi_request* req, int* id) {
  if (!S) return KFBI_ERR_ARG;
  std::string why;
  kfbi_status s = check_request(S, req, why);
  if (s != KFBI_OK) {
    S->err = why;
    return s;
  }
  std::unique_ptr<Req> q(new (std::nothrow) Req());
  if (!q) return KFBI_ERR_OOM;
  q->r = *req;
  q->id = (int)S->reqs.size();
  q->job = std::make_shared<PlanJob>();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto pos = std::upper_bound(S->queue.begin(), S->queue.end(), q->id, [&](int a, int b) {
      const double ta = a == q->id ? req->arrival : S->reqs[a]->r.arrival;
      const double tb = b == q->id ? req->arrival : S->reqs[b]->r.arrival;
      return ta < tb;
    });
    S->queue.insert(pos, q->id);
    S->reqs.push_back(std::move(q));
  }
  S->cv.notify_all();
  if (id) *id = (int)S->reqs.size() - 1;
  return KFBI_OK;
}

kfbi_status kfbi_server_tick(kfbi_server* S, double now, int* n_resident) {
  if (!S) return KFBI_ERR_ARG;
  S->err.clear();
  return guarded(nullptr, [&]() -> kfbi_status {
    return tick_impl(S, now < 0.0 ? S->clock_now() : now, n_resident);
  });
}

kfbi_status kfbi_server_run(kfbi_server* S, double time_limit) {
  if (!S) return KFBI_ERR_ARG;
  S->err.clear();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->t0 = Clock::now();
    S->wall = true;
  }
  S->cv.notify_all();
  kfbi_status s = guarded(nullptr, [&]() -> kfbi_status {
    for (;;) {
      if (S->queue.empty() && S->resident.empty()) return KFBI_OK;
      const double now = S->clock_now();
      if (time_limit > 0.0 && now > time_limit) {
        S->err = "kfbi_server_run: time limit reached";
        return KFBI_ERR_TIMEOUT;
      }
      if (S->resident.empty()) {
        const double next = S->reqs[S->queue.front()]->r.arrival;
        if (next > now) {
          std::this_thread::sleep_for(std::chrono::duration<double>(std::min(next - now, 0.01)));
          continue;
        }
      }
      kfbi_status t = tick_impl(S, now, nullptr);
      if (t != KFBI_OK) return t;
    }
  });
  S->wall = false;
  return s;
}

kfbi_status kfbi_server_request_info(const kfbi_server* S, int id, kfbi_request_info* info) {
  if (!S || !info || id < 0 || id >= (int)S->reqs.size()) return KFBI_ERR_ARG;
  const Req& q = *S->reqs[id];
  info->state = q.state;
  info->status = q.status;
  info->arrival = q.r.arrival;
  info->admitted = q.admitted;
  info->finished = q.finished;
  info->admit_tick = q.admit_tick;
  info->finish_tick = q.finish_tick;
  info->steps_done = q.steps_done;
  info->max_iters = q.max_iters;
  info->max_rel_residual = q.max_res;
  info->device_bytes = q.bytes;
  return KFBI_OK;
}

kfbi_status kfbi_server_get_stats(const kfbi_server* S, kfbi_server_stats* stats) {
  if (!S || !stats) return KFBI_ERR_ARG;
  *stats = S->stats;
  return KFBI_OK;
}

const char* kfbi_server_last_error(const kfbi_server* S) { return S ? S->err.c_str() : ""; }

}  // extern "C"
