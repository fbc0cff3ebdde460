// Time steppers (Sec. 3.1 and Procedure 3 of Sec. 3.3, arXiv 2404.14864).
//
// Each step solves Delta u - kappa u = -F in Omega, u = g on Gamma through
// the Dirichlet BIE: b = g - u+[0, f-tilde], GMRES for phi (initial guess
// 2 phi^n - phi^(n-1), the previous density at the second step), then one
// interface solve with (f-tilde, phi) whose grid
// values in Omega are u^{n+1}.  The right-hand side F is carried as its own
// variable (Eq. 3.4 for heat; the recurrence after Eq. 3.7 for the
// theta-scheme; u* = 2u^{n+1} - u** for the Strang step, which is the
// backward-Euler identity Delta u^{n+1} = kappa (u^{n+1} - u**)).
// All grid kernels are elementwise over the padded planes, in float64.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace kfbi {
namespace stp {

// Grid kernels walk the padded plane; (r, c) inside [0, n1)^2 map to the
// caller's (n1 x n1) index r*n1 + c.
#define GRID_LOOP(Mp)                                                              \
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;                 \
       idx < (size_t)(Mp) * (Mp); idx += (size_t)gridDim.x * blockDim.x)

__global__ void k_heat_init(double* F, double* u, const double* u0, const double* lap0,
                            const double* src, int n1, int Mp, double two_dt) {
  KFBI_PDL_ENTRY();
  GRID_LOOP(Mp) {
    const int r = (int)(idx / Mp), c = (int)(idx % Mp);
    double f = 0.0, uu = 0.0;
    if (r < n1 && c < n1) {
      const size_t s = (size_t)r * n1 + c;
      uu = u0[s];
      f = two_dt * uu + lap0[s] + (src ? src[s] : 0.0);
    }
    F[idx] = f;
    u[idx] = uu;
  }
}

__global__ void k_wave_init(double* F, double* Fprev, double* u, const double* u0,
                            const double* lap0, const double* u1, const double* lap1, int n1,
                            int Mp, double kappa, double c1) {
  KFBI_PDL_ENTRY();
  GRID_LOOP(Mp) {
    const int r = (int)(idx / Mp), c = (int)(idx % Mp);
    double f = 0.0, fp = 0.0, uu = 0.0;
    if (r < n1 && c < n1) {
      const size_t s = (size_t)r * n1 + c;
      uu = u1[s];
      fp = kappa * u1[s] - lap1[s];
      f = kappa * (2.0 * u1[s] - u0[s]) + c1 * lap1[s] + lap0[s];
    }
    F[idx] = f;
    Fprev[idx] = fp;
    u[idx] = uu;
  }
}

// u* = u0 - i (dt/2) lap u0 (Step 1 of the Strang step), u = u0.
__global__ void k_schr_init(double* ustar, double* u, const double* u0, const double* lap0,
                            int n1, int Mp, double half_dt) {
  KFBI_PDL_ENTRY();
  const size_t plane = (size_t)Mp * Mp;
  GRID_LOOP(Mp) {
    const int r = (int)(idx / Mp), c = (int)(idx % Mp);
    double ur = 0, ui = 0, sr = 0, si = 0;
    if (r < n1 && c < n1) {
      const size_t s = (size_t)r * n1 + c;
      ur = u0[2 * s];
      ui = u0[2 * s + 1];
      // -i (dt/2) (lr + i li) = (dt/2) li - i (dt/2) lr
      sr = ur + half_dt * lap0[2 * s + 1];
      si = ui - half_dt * lap0[2 * s];
    }
    u[idx] = ur;
    u[plane + idx] = ui;
    ustar[idx] = sr;
    ustar[plane + idx] = si;
  }
}

// f-tilde = -F on Omega, 0 outside (Eq. 3.25 with f = -F).
__global__ void k_make_ft(double* ft, const double* F, const uint8_t* mask, int Mp) {
  KFBI_PDL_ENTRY();
  GRID_LOOP(Mp) { ft[idx] = mask[idx] ? -F[idx] : 0.0; }
}

// Pointwise Crank-Nicolson step of Eq. 3.10,
// u + i (dt/2)(v + w|u|^2) u = u* - i (dt/2)(v + w|u*|^2) u*.  Its root keeps
// the modulus (with |u| = |u*| both sides carry the same real factor
// a = (dt/2)(v + w|u*|^2), and |1 + i a| = |1 - i a|), so the root the
// paper's Newton iteration converges to from u* is
// u** = (1 - i a)/(1 + i a) u*, in closed form; for w = 0 it is the linear
// Cayley factor.  Then f-tilde = -kappa u** on Omega with kappa = i kim
// (Eq. 3.12: Delta u - kappa u = -kappa u**).
__global__ void k_schr_bstep(double* uss, double* ft, const double* ustar, const double* v,
                             const uint8_t* mask, int n1, int Mp, double half_dt, double w,
                             double kim) {
  KFBI_PDL_ENTRY();
  const size_t plane = (size_t)Mp * Mp;
  GRID_LOOP(Mp) {
    const int r = (int)(idx / Mp), c = (int)(idx % Mp);
    double xr = 0, xi = 0;
    if (r < n1 && c < n1) {
      const double sr = ustar[idx], si = ustar[plane + idx];
      const double a = half_dt * (v[(size_t)r * n1 + c] + w * (sr * sr + si * si));
      const double den = 1.0 / (1.0 + a * a);
      const double pr = (1.0 - a * a) * den, pi = -2.0 * a * den;
      xr = pr * sr - pi * si;
      xi = pr * si + pi * sr;
    }
    uss[idx] = xr;
    uss[plane + idx] = xi;
    // -kappa u** = -i kim (xr + i xi) = kim xi - i kim xr
    const bool in = mask[idx] != 0;
    ft[idx] = in ? kim * xi : 0.0;
    ft[plane + idx] = in ? -kim * xr : 0.0;
  }
}

// b = g - u+[0, f-tilde], complex interleaved; g is real unless C.
__global__ void k_make_b(double* b, const double* g, const double* ub, int nb, int C) {
  KFBI_PDL_ENTRY();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  const double gr = C ? g[2 * k] : g[k], gi = C ? g[2 * k + 1] : 0.0;
  b[2 * k] = gr - ub[2 * k];
  b[2 * k + 1] = gi - ub[2 * k + 1];
}

// Heat: u = U; F^{n+2} = (4/dt) U - F^{n+1} + src.
__global__ void k_heat_update(double* u, double* F, const double* U, const double* src, int n1,
                              int Mp, double four_dt) {
  KFBI_PDL_ENTRY();
  GRID_LOOP(Mp) {
    const int r = (int)(idx / Mp), c = (int)(idx % Mp);
    const double uu = U[idx];
    double f = four_dt * uu - F[idx];
    if (src && r < n1 && c < n1) f += src[(size_t)r * n1 + c];
    u[idx] = uu;
    F[idx] = f;
  }
}

// Wave: F^{n+2} = (kappa/theta) U - ((1-2theta)/theta) F^{n+1} - F^n.
__global__ void k_wave_update(double* u, double* F, double* Fprev, const double* U, int Mp,
                              double k_theta, double c1) {
  KFBI_PDL_ENTRY();
  GRID_LOOP(Mp) {
    const double uu = U[idx], f = F[idx];
    const double fn = k_theta * uu - c1 * f - Fprev[idx];
    Fprev[idx] = f;
    F[idx] = fn;
    u[idx] = uu;
  }
}

// Strang: u = U; next u* = 2 U - u**.
__global__ void k_schr_update(double* u, double* ustar, const double* U, const double* uss,
                              int Mp) {
  KFBI_PDL_ENTRY();
  const size_t plane = (size_t)Mp * Mp;
  GRID_LOOP(Mp) {
    for (int p = 0; p < 2; ++p) {
      const size_t q = p * plane + idx;
      u[q] = U[q];
      ustar[q] = 2.0 * U[q] - uss[q];
    }
  }
}

__global__ void k_copy_phi(const double* src, double* dst, int nb, int C) {
  KFBI_PDL_ENTRY();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  if (C) {
    dst[2 * k] = src[2 * k];
    dst[2 * k + 1] = src[2 * k + 1];
  } else {
    dst[k] = src[2 * k];
  }
}

}  // namespace stp

using namespace stp;

// One BIE solve of the step: b = g - u+[0, ft], GMRES for phi, then the grid
// solution of Eq. 3.30 with (ft, phi) in D->d_U.  b and the final grid use
// the accurate operator (FP64-level on either domain precision).
// Superposition of the refined solve: U = W phi (in U) + Y f-tilde.
__global__ void k_add_grid(double* __restrict__ U, const double* __restrict__ uf, size_t n) {
  KFBI_PDL_ENTRY();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    U[i] += uf[i];
}

// History update and extrapolation of the initial density (complex
// interleaved, 2 nb doubles): mode 1: x = 2 x - x_prev and x_prev = old x;
// mode 0: x_prev = x; mode -1: nothing (a for the cached A phi).
__global__ void k_extrap(double* __restrict__ x, double* __restrict__ xp, double* __restrict__ a,
                         double* __restrict__ ap, int nb, int mode_x, int mode_a) {
  KFBI_PDL_ENTRY();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nb) return;
  for (int c = 0; c < 2; ++c) {
    const size_t i = 2 * (size_t)e + c;
    const double t = x[i];
    if (mode_x == 1) x[i] = 2.0 * t - xp[i];
    xp[i] = t;
    if (mode_a >= 0) {
      const double u = a[i];
      if (mode_a == 1) a[i] = 2.0 * u - ap[i];
      ap[i] = u;
    }
  }
}

static kfbi_status solve_step(kfbi_domain* D, kfbi_state* S, const double* g, bool gC,
                              kfbi_solve_info* info, cudaStream_t st) {
  // Neumann states: every application below is psi -> d_n u+ and the final
  // grid is u = Y f - V psi (Eq. 3.20)
  NeumannScope ns(D, S->neumann);
  const int nb = D->nb;
  const size_t pl = (size_t)S->planes * D->Mp * D->Mp;
  apply_accurate(D, S->kre, S->kim, D->d_zero_nb, 2, S->d_ft, S->d_ub, 2, st);
  // mixed domains keep Y f-tilde so that the final grid is a sum (the
  // discrete solution is linear in (f-tilde, phi))
  if (S->d_uf)
    KFBI_CUDA(cudaMemcpyAsync(S->d_uf, D->d_U, pl * sizeof(double), cudaMemcpyDeviceToDevice, st));
  KFBI_LAUNCH_P(KFBI_PROF_GRID, k_make_b, (nb + 255) / 256, 256, 0, st, S->d_b, g, S->d_ub, nb, gC ? 1 : 0);
  KFBI_CHECK_LAUNCH();
  kfbi_solve_info loc{};
  bool grid_wx = false;
  // initial density: the previous one, or, once two converged densities
  // exist, their linear extrapolation in time 2 phi^n - phi^(n-1) (on mixed
  // domains the cached A phi is extrapolated with it, the operator being
  // linear); the density entering this step becomes the history
  bool have_ax = S->d_ax && S->ax_valid && !S->phi_zero;
  if (!S->phi_zero) {
    const int mphi = S->hist ? 1 : 0;
    int max_ = -1;
    if (S->d_ax && S->ax_valid) max_ = (S->hist && S->ax_prev_valid) ? 1 : 0;
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_extrap, (nb + 255) / 256, 256, 0, st, S->d_phi, S->d_phi_prev,
                  S->d_ax, S->d_ax_prev, nb, mphi, max_);
    KFBI_CHECK_LAUNCH();
    S->ax_prev_valid = max_ >= 0;
    if (mphi == 1 && max_ != 1) have_ax = false;  // A x0 unknown: GMRES applies it
    S->hist = true;
  }
  S->ax_valid = false;
  kfbi_status s = gmres_solve(D, S->kre, S->kim, S->d_b, S->d_phi, S->phi_zero, &loc, st,
                              have_ax ? S->d_ax : nullptr, S->d_ax, &grid_wx);
  S->phi_zero = false;
  S->ax_valid = grid_wx;
  loc.applications += grid_wx ? 1 : 2;
  if (info) *info = loc;
  if (s != KFBI_OK) return s;
  if (grid_wx) {
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_add_grid, grid_for(pl, 256), 256, 0, st, D->d_U, S->d_uf, pl);
    KFBI_CHECK_LAUNCH();
  } else {
    apply_accurate(D, S->kre, S->kim, S->d_phi, 2, S->d_ft, nullptr, 2, st);
  }
  return KFBI_OK;
}

}  // namespace kfbi

using namespace kfbi;

namespace {
struct StateBlobHeader {
  char magic[8];  // "KFBIST2\0" (2: the header carries w)
  int eq, planes, Mp, nb;
  int initialised, phi_zero, neumann, hist, ax_valid, ax_prev_valid, has_ax;
  double dt, theta, kre, kim, w;
};

// (device pointer, doubles) of every array the blob carries, in order
std::vector<std::pair<double*, size_t>> state_arrays(kfbi_state* S) {
  const size_t plane = (size_t)S->planes * S->dom->Mp * S->dom->Mp;
  const size_t nb2 = 2 * (size_t)S->dom->nb;
  std::vector<std::pair<double*, size_t>> a = {{S->d_u, plane}, {S->d_F, plane},
                                               {S->d_phi, nb2}, {S->d_phi_prev, nb2}};
  if (S->d_Fprev) a.push_back({S->d_Fprev, plane});
  if (S->d_ax) {
    a.push_back({S->d_ax, nb2});
    a.push_back({S->d_ax_prev, nb2});
  }
  return a;
}
}  // namespace

extern "C" {

kfbi_status kfbi_state_create(kfbi_domain* dom, int equation, kfbi_state** out) {
  if (!dom || !out) return KFBI_ERR_ARG;
  *out = nullptr;
  if (equation < KFBI_HEAT || equation > KFBI_SCHRODINGER) {
    dom->err = "unknown equation";
    return KFBI_ERR_ARG;
  }
  kfbi_state* S = new (std::nothrow) kfbi_state();
  if (!S) return KFBI_ERR_OOM;
  S->dom = dom;
  S->eq = equation;
  S->planes = equation == KFBI_SCHRODINGER ? 2 : 1;
  kfbi_status s = guarded(dom, [&]() -> kfbi_status {
    const size_t plane = (size_t)dom->Mp * dom->Mp * S->planes;
    const size_t nb2 = 2 * (size_t)dom->nb;
    auto alloc = [&](double** p, size_t n) {
      KFBI_CUDA(cudaMalloc(p, n * sizeof(double)));
      S->bytes += (long long)(n * sizeof(double));
    };
    alloc(&S->d_u, plane);
    alloc(&S->d_F, plane);
    alloc(&S->d_ft, plane);
    if (equation == KFBI_WAVE) alloc(&S->d_Fprev, plane);
    if (equation == KFBI_SCHRODINGER) alloc(&S->d_aux, plane);
    alloc(&S->d_phi, nb2);
    alloc(&S->d_b, nb2);
    alloc(&S->d_ub, nb2);
    alloc(&S->d_phi_prev, nb2);
    if (dom->tc) {
      alloc(&S->d_uf, plane);
      alloc(&S->d_ax, nb2);
      alloc(&S->d_ax_prev, nb2);
    }
    KFBI_CUDA(cudaMemset(S->d_phi, 0, nb2 * sizeof(double)));
    return KFBI_OK;
  });
  if (s != KFBI_OK) {
    kfbi_state_destroy(S);
    return s;
  }
  *out = S;
  return KFBI_OK;
}

long long kfbi_state_device_bytes(const kfbi_state* st) { return st ? st->bytes : -1; }

void kfbi_state_destroy(kfbi_state* S) {
  if (!S) return;
  cudaDeviceSynchronize();
  double* ptrs[] = {S->d_u,   S->d_F, S->d_Fprev, S->d_ft, S->d_aux,       S->d_phi,
                    S->d_b,   S->d_ub, S->d_uf,   S->d_ax, S->d_phi_prev, S->d_ax_prev};
  for (double* p : ptrs)
    if (p) cudaFree(p);
  delete S;
}

static kfbi_status check_state(kfbi_state* S, int eq) {
  if (!S || !S->dom) return KFBI_ERR_ARG;
  if (S->eq != eq) {
    S->dom->err = "state was created for another equation";
    return KFBI_ERR_ARG;
  }
  return KFBI_OK;
}

kfbi_status kfbi_state_init_heat(kfbi_state* S, double dt, const double* u0, const double* lap0,
                                 const double* src, void* stream) {
  kfbi_status c = check_state(S, KFBI_HEAT);
  if (c != KFBI_OK) return c;
  kfbi_domain* D = S->dom;
  if (!(dt > 0.0) || !u0 || !lap0) {
    D->err = "dt > 0 and u0, lap_u0 are required";
    return KFBI_ERR_ARG;
  }
  return guarded(D, [&]() -> kfbi_status {
    cudaStream_t st = (cudaStream_t)stream;
    S->dt = dt;
    S->kre = 2.0 / dt;
    S->kim = 0.0;
    const size_t plane = (size_t)D->Mp * D->Mp;
    KFBI_LAUNCH(k_heat_init, grid_for(plane, 256), 256, 0, st, S->d_F, S->d_u, u0, lap0, src,
                D->n1, D->Mp, 2.0 / dt);
    KFBI_CHECK_LAUNCH();
    KFBI_CUDA(cudaMemsetAsync(S->d_phi, 0, 2 * (size_t)D->nb * sizeof(double), st));
    S->phi_zero = true;
    S->ax_valid = false;
    S->hist = false;
    S->ax_prev_valid = false;
    S->initialised = true;
    return KFBI_OK;
  });
}

kfbi_status kfbi_state_init_wave(kfbi_state* S, double dt, double theta, const double* u0,
                                 const double* lap0, const double* u1, const double* lap1,
                                 void* stream) {
  kfbi_status c = check_state(S, KFBI_WAVE);
  if (c != KFBI_OK) return c;
  kfbi_domain* D = S->dom;
  if (!(dt > 0.0) || !(theta > 0.0) || !u0 || !lap0 || !u1 || !lap1) {
    D->err = "dt > 0, theta > 0 and u0, lap_u0, u1, lap_u1 are required";
    return KFBI_ERR_ARG;
  }
  return guarded(D, [&]() -> kfbi_status {
    cudaStream_t st = (cudaStream_t)stream;
    S->dt = dt;
    S->theta = theta;
    S->kre = 1.0 / (theta * dt * dt);
    S->kim = 0.0;
    const size_t plane = (size_t)D->Mp * D->Mp;
    KFBI_LAUNCH(k_wave_init, grid_for(plane, 256), 256, 0, st, S->d_F, S->d_Fprev, S->d_u, u0,
                lap0, u1, lap1, D->n1, D->Mp, S->kre, (1.0 - 2.0 * theta) / theta);
    KFBI_CHECK_LAUNCH();
    KFBI_CUDA(cudaMemsetAsync(S->d_phi, 0, 2 * (size_t)D->nb * sizeof(double), st));
    S->phi_zero = true;
    S->ax_valid = false;
    S->hist = false;
    S->ax_prev_valid = false;
    S->initialised = true;
    return KFBI_OK;
  });
}

kfbi_status kfbi_state_init_schrodinger(kfbi_state* S, double dt, const void* u0,
                                        const void* lap0, void* stream) {
  kfbi_status c = check_state(S, KFBI_SCHRODINGER);
  if (c != KFBI_OK) return c;
  kfbi_domain* D = S->dom;
  if (!(dt > 0.0) || !u0 || !lap0) {
    D->err = "dt > 0 and u0, lap_u0 are required";
    return KFBI_ERR_ARG;
  }
  return guarded(D, [&]() -> kfbi_status {
    cudaStream_t st = (cudaStream_t)stream;
    S->dt = dt;
    S->kre = 0.0;
    S->kim = 2.0 / dt;
    const size_t plane = (size_t)D->Mp * D->Mp;
    KFBI_LAUNCH(k_schr_init, grid_for(plane, 256), 256, 0, st, S->d_F, S->d_u,
                (const double*)u0, (const double*)lap0, D->n1, D->Mp, 0.5 * dt);
    KFBI_CHECK_LAUNCH();
    KFBI_CUDA(cudaMemsetAsync(S->d_phi, 0, 2 * (size_t)D->nb * sizeof(double), st));
    S->phi_zero = true;
    S->ax_valid = false;
    S->hist = false;
    S->ax_prev_valid = false;
    S->initialised = true;
    return KFBI_OK;
  });
}

kfbi_status kfbi_step_heat(kfbi_domain* dom, kfbi_state* S, const double* g_next,
                           const double* src_sum_next, kfbi_solve_info* info, void* stream) {
  kfbi_status c = check_state(S, KFBI_HEAT);
  if (c != KFBI_OK) return c;
  if (!dom || dom != S->dom || !g_next || !S->initialised) {
    if (dom) dom->err = "step needs the state's domain, g_next and an initialised state";
    return KFBI_ERR_ARG;
  }
  return guarded(dom, [&]() -> kfbi_status {
    cudaStream_t st = (cudaStream_t)stream;
    const size_t plane = (size_t)dom->Mp * dom->Mp;
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_make_ft, grid_for(plane, 256), 256, 0, st, S->d_ft, S->d_F, dom->d_mask, dom->Mp);
    KFBI_CHECK_LAUNCH();
    kfbi_status s = solve_step(dom, S, g_next, false, info, st);
    if (s != KFBI_OK) return s;
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_heat_update, grid_for(plane, 256), 256, 0, st, S->d_u, S->d_F, dom->d_U,
                src_sum_next, dom->n1, dom->Mp, 4.0 / S->dt);
    KFBI_CHECK_LAUNCH();
    KFBI_CUDA(cudaStreamSynchronize(st));
    return KFBI_OK;
  });
}

kfbi_status kfbi_step_wave(kfbi_domain* dom, kfbi_state* S, const double* g_next,
                           kfbi_solve_info* info, void* stream) {
  kfbi_status c = check_state(S, KFBI_WAVE);
  if (c != KFBI_OK) return c;
  if (!dom || dom != S->dom || !g_next || !S->initialised) {
    if (dom) dom->err = "step needs the state's domain, g_next and an initialised state";
    return KFBI_ERR_ARG;
  }
  return guarded(dom, [&]() -> kfbi_status {
    cudaStream_t st = (cudaStream_t)stream;
    const size_t plane = (size_t)dom->Mp * dom->Mp;
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_make_ft, grid_for(plane, 256), 256, 0, st, S->d_ft, S->d_F, dom->d_mask, dom->Mp);
    KFBI_CHECK_LAUNCH();
    kfbi_status s = solve_step(dom, S, g_next, false, info, st);
    if (s != KFBI_OK) return s;
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_wave_update, grid_for(plane, 256), 256, 0, st, S->d_u, S->d_F, S->d_Fprev,
                dom->d_U, dom->Mp, S->kre / S->theta, (1.0 - 2.0 * S->theta) / S->theta);
    KFBI_CHECK_LAUNCH();
    KFBI_CUDA(cudaStreamSynchronize(st));
    return KFBI_OK;
  });
}

kfbi_status kfbi_step_schrodinger(kfbi_domain* dom, kfbi_state* S, const double* v, double w,
                                  const void* g_next, kfbi_solve_info* info, void* stream) {
  kfbi_status c = check_state(S, KFBI_SCHRODINGER);
  if (c != KFBI_OK) return c;
  if (!dom || dom != S->dom || !g_next || !v || !S->initialised) {
    if (dom) dom->err = "step needs the state's domain, v, g_next and an initialised state";
    return KFBI_ERR_ARG;
  }
  if (!std::isfinite(w)) {
    dom->err = "w must be finite";
    return KFBI_ERR_ARG;
  }
  return guarded(dom, [&]() -> kfbi_status {
    cudaStream_t st = (cudaStream_t)stream;
    const size_t plane = (size_t)dom->Mp * dom->Mp;
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_schr_bstep, grid_for(plane, 256), 256, 0, st, S->d_aux, S->d_ft, S->d_F, v,
                dom->d_mask, dom->n1, dom->Mp, 0.5 * S->dt, w, S->kim);
    KFBI_CHECK_LAUNCH();
    kfbi_status s = solve_step(dom, S, (const double*)g_next, true, info, st);
    if (s != KFBI_OK) return s;
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_schr_update, grid_for(plane, 256), 256, 0, st, S->d_u, S->d_F, dom->d_U,
                S->d_aux, dom->Mp);
    KFBI_CHECK_LAUNCH();
    KFBI_CUDA(cudaStreamSynchronize(st));
    return KFBI_OK;
  });
}

kfbi_status kfbi_state_set_w(kfbi_state* S, double w) {
  if (!S || !S->dom) return KFBI_ERR_ARG;
  if (S->eq != KFBI_SCHRODINGER || !std::isfinite(w)) {
    S->dom->err = "w needs a Schroedinger state and a finite value";
    return KFBI_ERR_ARG;
  }
  S->w = w;
  return KFBI_OK;
}

kfbi_status kfbi_state_set_neumann(kfbi_state* S, int neumann) {
  if (!S || !S->dom) return KFBI_ERR_ARG;
  return guarded(S->dom, [&]() -> kfbi_status {
    S->neumann = neumann != 0;
    // the density changes meaning: start the next solve from zero
    KFBI_CUDA(cudaMemset(S->d_phi, 0, 2 * (size_t)S->dom->nb * sizeof(double)));
    S->phi_zero = true;
    S->ax_valid = false;
    S->hist = false;
    S->ax_prev_valid = false;
    return KFBI_OK;
  });
}

kfbi_status kfbi_state_get_u(kfbi_state* S, void* u_out, void* stream) {
  if (!S || !S->dom || !u_out) return KFBI_ERR_ARG;
  return guarded(S->dom, [&]() -> kfbi_status {
    unpad(S->dom, S->d_u, (double*)u_out, S->planes == 2, (cudaStream_t)stream);
    return KFBI_OK;
  });
}

// ---- checkpoint: the state's time-level data as one host blob -------------


long long kfbi_state_blob_bytes(const kfbi_state* S) {
  if (!S || !S->dom) return -1;
  size_t n = sizeof(StateBlobHeader);
  for (auto& a : state_arrays(const_cast<kfbi_state*>(S))) n += a.second * sizeof(double);
  return (long long)n;
}

kfbi_status kfbi_state_export(kfbi_state* S, void* host_buf, long long bytes) {
  if (!S || !S->dom || !host_buf) return KFBI_ERR_ARG;
  if (bytes < kfbi_state_blob_bytes(S)) {
    S->dom->err = "state blob buffer too small (kfbi_state_blob_bytes)";
    return KFBI_ERR_ARG;
  }
  return guarded(S->dom, [&]() -> kfbi_status {
    StateBlobHeader h{};
    std::memcpy(h.magic, "KFBIST2", 8);
    h.eq = S->eq;
    h.planes = S->planes;
    h.Mp = S->dom->Mp;
    h.nb = S->dom->nb;
    h.initialised = S->initialised;
    h.phi_zero = S->phi_zero;
    h.neumann = S->neumann;
    h.hist = S->hist;
    h.ax_valid = S->ax_valid;
    h.ax_prev_valid = S->ax_prev_valid;
    h.has_ax = S->d_ax != nullptr;
    h.dt = S->dt;
    h.theta = S->theta;
    h.kre = S->kre;
    h.kim = S->kim;
    h.w = S->w;
    char* out = (char*)host_buf;
    std::memcpy(out, &h, sizeof(h));
    out += sizeof(h);
    KFBI_CUDA(cudaDeviceSynchronize());
    for (auto& a : state_arrays(S)) {
      KFBI_CUDA(cudaMemcpy(out, a.first, a.second * sizeof(double), cudaMemcpyDeviceToHost));
      out += a.second * sizeof(double);
    }
    return KFBI_OK;
  });
}

kfbi_status kfbi_state_import(kfbi_state* S, const void* host_buf, long long bytes) {
  if (!S || !S->dom || !host_buf) return KFBI_ERR_ARG;
  if (bytes < (long long)sizeof(StateBlobHeader)) {
    S->dom->err = "state blob too short";
    return KFBI_ERR_ARG;
  }
  StateBlobHeader h;
  std::memcpy(&h, host_buf, sizeof(h));
  if (std::memcmp(h.magic, "KFBIST2", 8) != 0 || h.eq != S->eq || h.planes != S->planes ||
      h.Mp != S->dom->Mp || h.nb != S->dom->nb || h.has_ax != (S->d_ax != nullptr) ||
      bytes < kfbi_state_blob_bytes(S)) {
    S->dom->err = "state blob does not match this state (equation, grid, boundary nodes or "
                  "domain precision)";
    return KFBI_ERR_ARG;
  }
  return guarded(S->dom, [&]() -> kfbi_status {
    const char* in = (const char*)host_buf + sizeof(h);
    KFBI_CUDA(cudaDeviceSynchronize());
    for (auto& a : state_arrays(S)) {
      KFBI_CUDA(cudaMemcpy(a.first, in, a.second * sizeof(double), cudaMemcpyHostToDevice));
      in += a.second * sizeof(double);
    }
    S->initialised = h.initialised != 0;
    S->phi_zero = h.phi_zero != 0;
    S->neumann = h.neumann != 0;
    S->hist = h.hist != 0;
    S->ax_valid = h.ax_valid != 0;
    S->ax_prev_valid = h.ax_prev_valid != 0;
    S->dt = h.dt;
    S->theta = h.theta;
    S->kre = h.kre;
    S->kim = h.kim;
    S->w = h.w;
    return KFBI_OK;
  });
}

kfbi_status kfbi_state_get_phi(kfbi_state* S, void* phi_out, void* stream) {
  if (!S || !S->dom || !phi_out) return KFBI_ERR_ARG;
  return guarded(S->dom, [&]() -> kfbi_status {
    const int nb = S->dom->nb;
    KFBI_LAUNCH(k_copy_phi, (nb + 255) / 256, 256, 0, (cudaStream_t)stream, S->d_phi,
                (double*)phi_out, nb, S->planes == 2 ? 1 : 0);
    KFBI_CHECK_LAUNCH();
    return KFBI_OK;
  });
}

}  // extern "C"

namespace kfbi {

long long state_bytes_for(int Mp, int nb, int equation, bool mixed) {
  const int planes = equation == KFBI_SCHRODINGER ? 2 : 1;
  const size_t plane = (size_t)Mp * Mp * planes;
  const int fields = 3 + (equation != KFBI_HEAT ? 1 : 0) + (mixed ? 1 : 0);
  const int vectors = 4 + (mixed ? 2 : 0);  // phi, b, ub, phi_prev (+ ax, ax_prev)
  return (long long)((fields * plane + vectors * 2 * (size_t)nb) * sizeof(double));
}

}  // namespace kfbi
