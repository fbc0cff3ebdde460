// Served stream: a request server with continuous batching on one device.
//
// Requests are independent time-stepping problems (heat, wave, Schroedinger;
// any grid size and interface curve).  The server keeps every admitted
// request's domain tables, time-level fields, Krylov workspace, boundary
// data and source on the device until the request completes, and advances
// resident requests together: each tick of a lane is one lockstep batch step
// (grouped tcgen05 passes over all instances' tiles, one CUDA graph per
// GMRES iteration) of the lane's requests.  Between ticks, completed
// requests are retired (result copied to the caller's host buffer, device
// memory freed) and arrived requests are admitted first come first served
// while a slot is free and their exact device bytes fit the budget and the
// free device memory.
//
// Lanes: requests are split by padded grid size (up to 512, up to 1024,
// larger) into up to three lanes, each with its own batch and stream.  On
// the wall clock (kfbi_server_run) every lane has its own host thread, so a
// small request steps at its lane's pace instead of waiting for the
// largest grid in every tick, and the device interleaves the lanes' kernels.
//
// Host plan building (geometry, cut edges, coefficient tables: Procedure 1,
// Sec. 3.3) is the expensive host part of admission; worker threads start it
// as soon as a request has arrived, while the device is busy.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "tc_internal.h"

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
  int lane = 0;
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

struct Lane {
  int id = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  kfbi_batch* B = nullptr;
  std::vector<int> queue;     // not yet admitted, ordered by (arrival, id); server mutex
  std::vector<int> resident;  // in admission order; touched by the lane's thread only
  bool set_changed = false;
  double* d_stage = nullptr;  // staging for initial grids and results
  size_t stage_cap = 0;       // doubles
  int ticks = 0;
};

using Clock = std::chrono::steady_clock;

}  // namespace

struct kfbi_server {
  kfbi_server_desc desc{};
  int device = 0;
  std::vector<std::unique_ptr<Lane>> lanes;
  std::vector<std::unique_ptr<Req>> reqs;
  long long budget = 0, used = 0;
  int n_resident = 0;
  kfbi_server_stats stats{};
  Clock::time_point t0;
  bool wall = false;  // run(): workers read the wall clock
  // one mutex for the queues, plan jobs, byte and slot accounting and stats
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

// The earliest arrived request, over all lanes, whose plan nobody has
// started (server mutex held).
Req* next_plan_job(kfbi_server* S, double now) {
  Req* best = nullptr;
  for (auto& L : S->lanes)
    for (int id : L->queue) {
      Req& q = *S->reqs[id];
      if (q.r.arrival > now) break;  // each queue is ordered by arrival
      if (q.job->stage == 0) {
        if (!best || q.r.arrival < best->r.arrival) best = &q;
        break;
      }
    }
  return best;
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

void ensure_stage(Lane& L, size_t doubles) {
  if (doubles <= L.stage_cap) return;
  if (L.d_stage) KFBI_CUDA(cudaFree(L.d_stage));
  L.d_stage = nullptr;
  L.stage_cap = 0;
  KFBI_CUDA(cudaMalloc(&L.d_stage, doubles * sizeof(double)));
  L.stage_cap = doubles;
}

// Free a request's device memory (no lock held: may synchronise the device).
void release_device(Req& q) {
  if (q.S) kfbi_state_destroy(q.S);
  if (q.D) kfbi_destroy_domain(q.D);
  if (q.d_g) cudaFree(q.d_g);
  if (q.d_src) cudaFree(q.d_src);
  q.S = nullptr;
  q.D = nullptr;
  q.d_g = nullptr;
  q.d_src = nullptr;
  q.job.reset();
}

// Mark a request failed; a resident one returns its bytes and slot.
void fail(kfbi_server* S, Lane& L, Req& q, kfbi_status s, double now, bool resident) {
  release_device(q);
  std::lock_guard<std::mutex> lk(S->mu);
  if (resident) {
    S->used -= q.bytes;
    S->n_resident--;
  }
  q.state = KFBI_REQ_FAILED;
  q.status = s;
  q.finished = now;
  q.finish_tick = L.ticks;
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

long long upload(double* dst, const void* src, size_t n, cudaStream_t st) {
  KFBI_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, st));
  return (long long)(n * sizeof(double));
}

// Make request q resident (domain, state, data, initial fields) on lane L.
void make_resident(Lane& L, Req& q, long long& h2d) {
  const Plan& P = q.job->plan;
  const kfbi_request& r = q.r;
  const int planes = r.equation == KFBI_SCHRODINGER ? 2 : 1;
  const size_t grid = (size_t)P.n1 * P.n1;
  q.D = domain_from_plan(P, L.st);
  kfbi_status s = kfbi_state_create(q.D, r.equation, &q.S);
  if (s != KFBI_OK) throw Status{s, kfbi_last_error(q.D)};
  q.gstride = (size_t)planes * P.nb;
  KFBI_CUDA(cudaMalloc(&q.d_g, (size_t)r.steps * q.gstride * sizeof(double)));
  h2d += upload(q.d_g, r.g, (size_t)r.steps * q.gstride, L.st);
  const double* grid_src = r.equation == KFBI_HEAT ? r.src_profile
                           : r.equation == KFBI_SCHRODINGER ? r.potential : nullptr;
  if (grid_src) {
    KFBI_CUDA(cudaMalloc(&q.d_src, grid * sizeof(double)));
    h2d += upload(q.d_src, grid_src, grid, L.st);
  }
  if (r.equation == KFBI_HEAT) {
    q.coef.assign(r.steps, 1.0);
    if (r.src_coef) q.coef.assign(r.src_coef, r.src_coef + r.steps);
  }
  // initial fields through the lane's staging buffer
  const int nfields = r.equation == KFBI_WAVE ? 4 : (r.equation == KFBI_HEAT && r.src_init ? 3 : 2);
  ensure_stage(L, nfields * planes * grid);
  double* f0 = L.d_stage;
  double* f1 = f0 + planes * grid;
  double* f2 = f1 + planes * grid;
  double* f3 = f2 + planes * grid;
  h2d += upload(f0, r.u0, planes * grid, L.st);
  h2d += upload(f1, r.lap_u0, planes * grid, L.st);
  if (r.equation == KFBI_HEAT) {
    if (r.src_init) h2d += upload(f2, r.src_init, grid, L.st);
    s = kfbi_state_init_heat(q.S, r.dt, f0, f1, r.src_init ? f2 : nullptr, L.st);
  } else if (r.equation == KFBI_WAVE) {
    h2d += upload(f2, r.u1, grid, L.st);
    h2d += upload(f3, r.lap_u1, grid, L.st);
    s = kfbi_state_init_wave(q.S, r.dt, r.theta, f0, f1, f2, f3, L.st);
  } else {
    s = kfbi_state_init_schrodinger(q.S, r.dt, f0, f1, L.st);
  }
  if (s != KFBI_OK) throw Status{s, kfbi_last_error(q.D)};
  KFBI_CUDA(cudaStreamSynchronize(L.st));
  q.bytes = kfbi_domain_device_bytes(q.D) + kfbi_state_device_bytes(q.S) + data_bytes(r, P);
}

// First come first served admission into lane L at time now.
void admit(kfbi_server* S, Lane& L, double now) {
  for (;;) {
    Req* qp = nullptr;
    long long need = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (L.queue.empty()) return;
      Req& q = *S->reqs[L.queue.front()];
      if (q.r.arrival > now) return;
      if (S->n_resident >= S->desc.max_resident) return;
      if (q.job->stage == 0) {
        // nobody took it yet: build here
        q.job->stage = 1;
        lk.unlock();
        build_job(q.job.get(), q.r.domain);
        lk.lock();
        q.job->stage = 2;
        S->cv.notify_all();
      } else if (q.job->stage == 1) {
        // a worker is building it: wait only when the lane would idle
        if (!L.resident.empty()) return;
        S->cv.wait(lk, [&] { return q.job->stage == 2; });
      }
      L.queue.erase(L.queue.begin());
      qp = &q;
      if (q.job->status == KFBI_OK) {
        const Plan& P = q.job->plan;
        need = kfbi::domain_bytes_for(P) +
               state_bytes_for(((P.n1 + 127) / 128) * 128, P.nb, q.r.equation, true) +
               data_bytes(q.r, P);
        if (need <= S->budget) {
          size_t free_b = 0, total_b = 0;
          if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
          if (S->used + need > S->budget || need + S->desc.hbm_reserve_bytes > (long long)free_b) {
            // does not fit now: it stays at the head until memory is freed
            L.queue.insert(L.queue.begin(), q.id);
            return;
          }
          S->used += need;  // reserved before the allocations
          S->n_resident++;
        }
      }
    }
    Req& q = *qp;
    if (q.job->status != KFBI_OK) {
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->err = "request " + std::to_string(q.id) + ": " + q.job->err;
      }
      fail(S, L, q, q.job->status, now, false);
      continue;
    }
    if (need > S->budget) {
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->err = "request " + std::to_string(q.id) + " needs more device memory than the budget";
      }
      fail(S, L, q, KFBI_ERR_OOM, now, false);
      continue;
    }
    long long h2d = 0;
    try {
      make_resident(L, q, h2d);
    } catch (const Status& e) {
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->err = "request " + std::to_string(q.id) + ": " + e.msg;
        S->used -= need;
        S->n_resident--;
      }
      q.bytes = 0;
      fail(S, L, q, e.code, now, false);
      continue;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->used += q.bytes - need;  // the plan's count is exact; keep the books right regardless
    S->stats.peak_device_bytes = std::max(S->stats.peak_device_bytes, S->used);
    S->stats.admitted++;
    S->stats.h2d_bytes += h2d;
    q.state = KFBI_REQ_RESIDENT;
    q.admitted = now;
    q.admit_tick = L.ticks;
    L.resident.push_back(q.id);
    L.set_changed = true;
  }
}

void retire(kfbi_server* S, Lane& L, double now) {
  std::vector<int> keep;
  for (int id : L.resident) {
    Req& q = *S->reqs[id];
    if (q.state == KFBI_REQ_FAILED) {
      L.set_changed = true;
      continue;
    }
    if (q.steps_done < q.r.steps) {
      keep.push_back(id);
      continue;
    }
    const int planes = q.r.equation == KFBI_SCHRODINGER ? 2 : 1;
    const size_t grid = (size_t)q.D->n1 * q.D->n1 * planes;
    ensure_stage(L, grid);
    kfbi_status s = kfbi_state_get_u(q.S, L.d_stage, L.st);
    if (s != KFBI_OK) throw Status{s, kfbi_last_error(q.D)};
    KFBI_CUDA(cudaMemcpyAsync(q.r.u_out, L.d_stage, grid * sizeof(double), cudaMemcpyDeviceToHost,
                              L.st));
    KFBI_CUDA(cudaStreamSynchronize(L.st));
    release_device(q);
    const double fin = S->wall ? S->clock_now() : now;
    std::lock_guard<std::mutex> lk(S->mu);
    S->stats.d2h_bytes += (long long)(grid * sizeof(double));
    S->used -= q.bytes;
    S->n_resident--;
    q.state = KFBI_REQ_DONE;
    q.finished = fin;
    q.finish_tick = L.ticks;
    S->stats.completed++;
    L.set_changed = true;
  }
  L.resident.swap(keep);
}

// One lockstep step of every request resident in lane L.
kfbi_status step_resident(kfbi_server* S, Lane& L, double now) {
  const int n = (int)L.resident.size();
  if (n == 0) return KFBI_OK;
  std::vector<kfbi_domain*> doms(n);
  std::vector<kfbi_state*> states(n);
  std::vector<const void*> g(n);
  std::vector<const double*> src(n);
  std::vector<double> scale(n, 1.0);
  for (int i = 0; i < n; ++i) {
    Req& q = *S->reqs[L.resident[i]];
    doms[i] = q.D;
    states[i] = q.S;
    g[i] = q.d_g + (size_t)q.steps_done * q.gstride;
    src[i] = q.d_src;
    if (q.r.equation == KFBI_HEAT) scale[i] = q.coef[q.steps_done];
  }
  if (L.set_changed) {
    batch_bind(L.B, doms.data(), n);
    L.set_changed = false;
  }
  std::vector<kfbi_solve_info> infos(n);
  const auto t = Clock::now();
  kfbi_status s = batch_step(L.B, states.data(), g.data(), src.data(), scale.data(), infos.data(),
                             L.st);
  const double busy = std::chrono::duration<double>(Clock::now() - t).count();
  L.ticks++;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stats.busy_seconds += busy;
    S->stats.ticks++;
    S->stats.resident_ticks += n;
  }
  if (s != KFBI_OK && s != KFBI_ERR_NOT_CONVERGED && s != KFBI_ERR_NONFINITE) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->err = std::string("batch step failed: ") + kfbi_batch_last_error(L.B);
    }
    for (int id : L.resident) fail(S, L, *S->reqs[id], s, now, true);
    L.resident.clear();
    L.set_changed = true;
    return s;
  }
  double gps = 0.0;
  for (int i = 0; i < n; ++i) {
    Req& q = *S->reqs[L.resident[i]];
    q.steps_done++;
    q.max_iters = std::max(q.max_iters, infos[i].iters);
    if (std::isfinite(infos[i].rel_residual)) q.max_res = std::max(q.max_res, infos[i].rel_residual);
    gps += (double)q.D->M * (double)q.D->M;
    if (!infos[i].converged) {
      const bool nonfinite = !std::isfinite(infos[i].rel_residual);
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->err = "request " + std::to_string(q.id) +
                 (nonfinite ? ": non-finite density residual" : ": GMRES reached gmres_maxit");
      }
      fail(S, L, q, nonfinite ? KFBI_ERR_NONFINITE : KFBI_ERR_NOT_CONVERGED, now, true);
    }
  }
  std::lock_guard<std::mutex> lk(S->mu);
  S->stats.grid_point_steps += gps;
  return KFBI_OK;
}

void publish(kfbi_server* S, double now) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->published_now = now;
  }
  S->cv.notify_all();
}

// Admission, one step and retirement of one lane; stepped receives the
// requests that stepped.
kfbi_status tick_lane(kfbi_server* S, Lane& L, double now, int& stepped) {
  const auto ta = Clock::now();
  admit(S, L, now);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stats.admit_seconds += std::chrono::duration<double>(Clock::now() - ta).count();
  }
  stepped = (int)L.resident.size();
  kfbi_status s = step_resident(S, L, now);
  if (s != KFBI_OK) return s;
  retire(S, L, now);
  return KFBI_OK;
}

bool lane_idle(kfbi_server* S, Lane& L) {
  std::lock_guard<std::mutex> lk(S->mu);
  return L.queue.empty() && L.resident.empty();
}

// The wall-clock loop of one lane (its own host thread when there are
// several lanes).
kfbi_status lane_loop(kfbi_server* S, Lane& L, double time_limit) {
  for (;;) {
    if (lane_idle(S, L)) return KFBI_OK;
    const double now = S->clock_now();
    if (time_limit > 0.0 && now > time_limit) {
      std::lock_guard<std::mutex> lk(S->mu);
      S->err = "kfbi_server_run: time limit reached";
      return KFBI_ERR_TIMEOUT;
    }
    if (L.resident.empty()) {
      double next;
      {
        std::lock_guard<std::mutex> lk(S->mu);
        next = S->reqs[L.queue.front()]->r.arrival;
      }
      if (next > now) {
        std::this_thread::sleep_for(std::chrono::duration<double>(std::min(next - now, 0.01)));
        continue;
      }
    }
    int stepped = 0;
    kfbi_status t = tick_lane(S, L, now, stepped);
    if (t != KFBI_OK) return t;
  }
}

int lane_of(const kfbi_server* S, const kfbi_domain_desc& d) {
  const int Mp = ((d.M - 1 + 127) / 128) * 128;
  const int cls = Mp <= 512 ? 0 : (Mp <= 1024 ? 1 : 2);
  return std::min(cls, (int)S->lanes.size() - 1);
}

kfbi_status check_request(const kfbi_server* S, const kfbi_request* r, std::string& why) {
  if (!r) return why = "request is NULL", KFBI_ERR_ARG;
  if (r->domain.precision != KFBI_MIXED_TF32 && r->domain.precision != KFBI_MIXED_FFT32)
    return why = "served requests run on KFBI_MIXED_TF32 or KFBI_MIXED_FFT32 domains", KFBI_ERR_ARG;
  if (r->domain.precision == KFBI_MIXED_FFT32 && !fft_supported(r->domain.M))
    return why = "no FFT pass for this grid size (KFBI_MIXED_FFT32 needs M = 32 N1)",
           KFBI_ERR_UNSUPPORTED;
  if (r->domain.gmres_restart != S->desc.gmres_restart)
    return why = "the request's gmres_restart must equal the server's", KFBI_ERR_ARG;
  if (r->domain.gmres_maxit < 1 || !(r->domain.gmres_tol > 0.0))
    return why = "GMRES parameters out of range", KFBI_ERR_ARG;
  if (r->domain.solver != KFBI_GMRES)
    return why = "served requests are solved by GMRES", KFBI_ERR_ARG;
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
      desc->plan_threads < 0 || desc->plan_threads > 64 || desc->lanes < 0 || desc->lanes > 3) {
    set_global_error("kfbi_server_create: max_resident 1..4096, budgets >= 0, gmres_restart 1..64, "
                     "plan_threads 0..64, lanes 0..3");
    return KFBI_ERR_ARG;
  }
  kfbi_server* S = new (std::nothrow) kfbi_server();
  if (!S) return KFBI_ERR_OOM;
  S->desc = *desc;
  S->t0 = Clock::now();
  const int nl = std::max(1, desc->lanes);
  kfbi_status s = guarded(nullptr, [&]() -> kfbi_status {
    KFBI_CUDA(cudaGetDevice(&S->device));
    for (int l = 0; l < nl; ++l) {
      std::unique_ptr<Lane> L(new Lane());
      L->id = l;
      if (nl == 1) {
        L->st = (cudaStream_t)stream;
      } else {
        KFBI_CUDA(cudaStreamCreateWithFlags(&L->st, cudaStreamNonBlocking));
        L->own_stream = true;
      }
      L->B = batch_new();
      S->lanes.push_back(std::move(L));
    }
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
  for (auto& L : S->lanes) {
    for (int id : L->resident) release_device(*S->reqs[id]);
    if (L->B) kfbi_batch_destroy(L->B);
    if (L->d_stage) cudaFree(L->d_stage);
    if (L->own_stream) cudaStreamDestroy(L->st);
  }
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
  q->job = std::make_shared<PlanJob>();
  q->lane = lane_of(S, req->domain);
  int qid;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    qid = (int)S->reqs.size();
    q->id = qid;
    std::vector<int>& queue = S->lanes[q->lane]->queue;
    auto pos = std::upper_bound(queue.begin(), queue.end(), req->arrival, [&](double t, int b) {
      return t < S->reqs[b]->r.arrival;
    });
    queue.insert(pos, qid);
    S->reqs.push_back(std::move(q));
  }
  S->cv.notify_all();
  if (id) *id = qid;
  return KFBI_OK;
}

kfbi_status kfbi_server_tick(kfbi_server* S, double now, int* n_resident) {
  if (!S) return KFBI_ERR_ARG;
  S->err.clear();
  return guarded(nullptr, [&]() -> kfbi_status {
    const double t = now < 0.0 ? S->clock_now() : now;
    publish(S, t);
    int total = 0;
    for (auto& L : S->lanes) {
      int stepped = 0;
      kfbi_status s = tick_lane(S, *L, t, stepped);
      total += stepped;
      if (s != KFBI_OK) return s;
    }
    if (n_resident) *n_resident = total;
    return KFBI_OK;
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
  const int nl = (int)S->lanes.size();
  std::vector<kfbi_status> st(nl, KFBI_OK);
  auto body = [&](int l) {
    st[l] = guarded(nullptr, [&]() -> kfbi_status {
      KFBI_CUDA(cudaSetDevice(S->device));
      return lane_loop(S, *S->lanes[l], time_limit);
    });
  };
  if (nl == 1) {
    body(0);
  } else {
    std::vector<std::thread> th;
    for (int l = 0; l < nl; ++l) th.emplace_back(body, l);
    for (auto& t : th) t.join();
  }
  S->wall = false;
  for (kfbi_status s : st)
    if (s != KFBI_OK) return s;
  return KFBI_OK;
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
