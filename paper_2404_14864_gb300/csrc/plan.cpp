// Host-side setup of a KFBI domain: geometry (Procedure 1 of Sec. 3.3,
// arXiv 2404.14864) and the coefficient tables that reduce Procedure 2's
// jump / correction / extraction steps to fixed-weight gathers.
//
// Every jump the method needs is linear in the density values phi at six
// consecutive boundary nodes, in kappa*phi and in f at one or two grid
// nodes.  Expanding Eq. 3.35 (second row read as = psi = 0 for the
// Dirichlet BIE) and the 3x3 system of Sec. 3.2.5 in the tangent/normal
// frame gives, with r1 = phi_ss - (t . t') phi_s, r2 = (t' x t) phi_s,
// R3 = f + kappa phi:
//   [u_x] = tau1 phi_s,  [u_y] = tau2 phi_s,
//   [u_xx] = r1 (tau1^2 - tau2^2) + 2 r2 tau1 tau2 + R3 tau2^2,
//   [u_yy] = r1 (tau2^2 - tau1^2) - 2 r2 tau1 tau2 + R3 tau1^2,
//   [u_xy] = 2 r1 tau1 tau2 + r2 (tau2^2 - tau1^2) - R3 tau1 tau2,
// which is the unique solution of the 3x3 system (its determinant is -1).
// The correction term of each cut arm (Sec. 3.2.4) and the jump-corrected
// extraction of Eq. 3.36 are then fixed linear combinations, stored per arm
// and per boundary node.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace kfbi {

static const double kTwoPi = 6.283185307179586476925286766559;

void Curve::z(double t, double& x, double& y) const {
  if (kind == KFBI_CURVE_POLAR) {
    double r = p[0] + p[1] * std::sin(p[2] * t + p[3]);
    x = cx + r * std::cos(t);
    y = cy + r * std::sin(t);
  } else {
    double u = p[0] * std::cos(t), v = p[1] * std::sin(t);
    x = cx + (ca * u - sa * v);
    y = cy + (sa * u + ca * v);
  }
}

void Curve::dz(double t, double& x, double& y) const {
  if (kind == KFBI_CURVE_POLAR) {
    double r = p[0] + p[1] * std::sin(p[2] * t + p[3]);
    double dr = p[1] * p[2] * std::cos(p[2] * t + p[3]);
    double c = std::cos(t), s = std::sin(t);
    x = dr * c - r * s;
    y = dr * s + r * c;
  } else {
    double u = -p[0] * std::sin(t), v = p[1] * std::cos(t);
    x = ca * u - sa * v;
    y = sa * u + ca * v;
  }
}

void Curve::d2z(double t, double& x, double& y) const {
  if (kind == KFBI_CURVE_POLAR) {
    double r = p[0] + p[1] * std::sin(p[2] * t + p[3]);
    double dr = p[1] * p[2] * std::cos(p[2] * t + p[3]);
    double d2r = -p[1] * p[2] * p[2] * std::sin(p[2] * t + p[3]);
    double c = std::cos(t), s = std::sin(t);
    x = d2r * c - 2.0 * dr * s - r * c;
    y = d2r * s + 2.0 * dr * c - r * s;
  } else {
    double u = -p[0] * std::cos(t), v = -p[1] * std::sin(t);
    x = ca * u - sa * v;
    y = sa * u + ca * v;
  }
}

double Curve::level(double x, double y) const {
  if (kind == KFBI_CURVE_POLAR) {
    double dx = x - cx, dy = y - cy;
    return std::hypot(dx, dy) - (p[0] + p[1] * std::sin(p[2] * std::atan2(dy, dx) + p[3]));
  }
  double dx = x - cx, dy = y - cy;
  double u = ca * dx + sa * dy, v = -sa * dx + ca * dy;
  double a = u / p[0], b = v / p[1];
  return a * a + b * b - 1.0;
}

double Curve::param_of(double x, double y) const {
  double t;
  if (kind == KFBI_CURVE_POLAR) {
    t = std::atan2(y - cy, x - cx);
  } else {
    double dx = x - cx, dy = y - cy;
    double u = ca * dx + sa * dy, v = -sa * dx + ca * dy;
    t = std::atan2(v / p[1], u / p[0]);
  }
  return t < 0.0 ? t + kTwoPi : t;
}

void fd_weights(double z, const double* x, int n, int nd, double* c) {
  const int w = nd + 1;
  std::memset(c, 0, sizeof(double) * n * w);
  double c1 = 1.0, c4 = x[0] - z;
  c[0] = 1.0;
  for (int i = 1; i < n; ++i) {
    int mn = std::min(i, nd);
    double c2 = 1.0, c5 = c4;
    c4 = x[i] - z;
    for (int j = 0; j < i; ++j) {
      double c3 = x[i] - x[j];
      c2 *= c3;
      if (j == i - 1) {
        for (int k = mn; k >= 1; --k)
          c[i * w + k] = c1 * (k * c[(i - 1) * w + k - 1] - c5 * c[(i - 1) * w + k]) / c2;
        c[i * w] = -c1 * c5 * c[(i - 1) * w] / c2;
      }
      for (int k = mn; k >= 1; --k) c[j * w + k] = (c4 * c[j * w + k] - k * c[j * w + k - 1]) / c3;
      c[j * w] = c4 * c[j * w] / c3;
    }
    c1 = c2;
  }
}

namespace {

// Root of the level function along p -> q by bisection until the bracket
// cannot shrink in float64; returns the fraction along the segment.
double bisect_edge(const Curve& cv, double px, double py, double qx, double qy, bool p_inside) {
  double t_in = p_inside ? 0.0 : 1.0, t_out = p_inside ? 1.0 : 0.0;
  for (int it = 0; it < 200; ++it) {
    double tm = 0.5 * (t_in + t_out);
    if (tm == t_in || tm == t_out) break;
    if (cv.level(px + tm * (qx - px), py + tm * (qy - py)) < 0.0)
      t_in = tm;
    else
      t_out = tm;
  }
  return 0.5 * (t_in + t_out);
}

// Geometry of the curve at parameter t: unit tangent and its arc-length
// derivative, speed sigma = |z'| and d sigma / dt.
struct Frame {
  double t1, t2, t1p, t2p, sigma, sigma_t;
};

Frame frame_at(const Curve& cv, double t) {
  double dx, dy, ddx, ddy;
  cv.dz(t, dx, dy);
  cv.d2z(t, ddx, ddy);
  Frame f;
  f.sigma = std::hypot(dx, dy);
  f.sigma_t = (dx * ddx + dy * ddy) / f.sigma;
  f.t1 = dx / f.sigma;
  f.t2 = dy / f.sigma;
  f.t1p = (ddx / f.sigma - dx * f.sigma_t / (f.sigma * f.sigma)) / f.sigma;
  f.t2p = (ddy / f.sigma - dy * f.sigma_t / (f.sigma * f.sigma)) / f.sigma;
  return f;
}

// Arc-length weights of the six-point density stencil (local nodes -2..3)
// at local coordinate s: value W0, first and second arc-length derivatives.
void density_weights(double s, const Frame& fr, double dtheta, double W0[6], double As[6],
                     double Ass[6]) {
  static const double xs[6] = {-2.0, -1.0, 0.0, 1.0, 2.0, 3.0};
  double c[18];
  fd_weights(s, xs, 6, 2, c);
  for (int m = 0; m < 6; ++m) {
    double w0 = c[m * 3], w1 = c[m * 3 + 1] / dtheta, w2 = c[m * 3 + 2] / (dtheta * dtheta);
    W0[m] = w0;
    As[m] = w1 / fr.sigma;
    Ass[m] = (w2 - w1 * fr.sigma_t / fr.sigma) / (fr.sigma * fr.sigma);
  }
}

// Solve A x = b (n x n, row-major, destroyed) by Gaussian elimination with
// partial pivoting.  Returns false if a pivot vanishes.
bool gepp(double* A, double* b, int n) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int r = k + 1; r < n; ++r)
      if (std::fabs(A[r * n + k]) > std::fabs(A[piv * n + k])) piv = r;
    if (A[piv * n + k] == 0.0) return false;
    if (piv != k) {
      for (int c = 0; c < n; ++c) std::swap(A[k * n + c], A[piv * n + c]);
      std::swap(b[k], b[piv]);
    }
    for (int r = k + 1; r < n; ++r) {
      double f = A[r * n + k] / A[k * n + k];
      for (int c = k; c < n; ++c) A[r * n + c] -= f * A[k * n + c];
      b[r] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int c = k + 1; c < n; ++c) s -= A[k * n + c] * b[c];
    b[k] = s / A[k * n + k];
  }
  return true;
}

}  // namespace

kfbi_status build_plan(const kfbi_domain_desc& desc, Plan& P, std::string& err) {
  if (desc.M < 8 || desc.M > 4096 || desc.n_boundary < 16 || desc.n_boundary > 16384 ||
      !(desc.box_hi > desc.box_lo)) {
    err = "domain sizes out of range (8 <= M <= 4096, 16 <= n_boundary <= 16384, lo < hi)";
    return KFBI_ERR_ARG;
  }
  if (desc.curve_kind != KFBI_CURVE_POLAR && desc.curve_kind != KFBI_CURVE_ELLIPSE) {
    err = "unknown curve kind";
    return KFBI_ERR_ARG;
  }
  if (desc.curve_kind == KFBI_CURVE_ELLIPSE && !(desc.params[0] > 0 && desc.params[1] > 0)) {
    err = "ellipse semi-axes must be positive";
    return KFBI_ERR_ARG;
  }
  P.desc = desc;
  P.M = desc.M;
  P.nb = desc.n_boundary;
  P.n1 = P.M - 1;
  P.lo = desc.box_lo;
  P.hi = desc.box_hi;
  P.h = (P.hi - P.lo) / P.M;
  P.dtheta = kTwoPi / P.nb;
  Curve& cv = P.curve;
  cv.kind = desc.curve_kind;
  cv.cx = desc.cx;
  cv.cy = desc.cy;
  for (int q = 0; q < 6; ++q) cv.p[q] = desc.params[q];
  if (cv.kind == KFBI_CURVE_ELLIPSE) {
    cv.ca = std::cos(cv.p[2]);
    cv.sa = std::sin(cv.p[2]);
  }
  const int M = P.M, n1 = P.n1, nb = P.nb;
  const double h = P.h;
  std::vector<double> xg(M + 1);
  for (int i = 0; i <= M; ++i) xg[i] = P.lo + h * (double)i;

  // (a) boundary nodes
  P.zx.resize(nb);
  P.zy.resize(nb);
  for (int k = 0; k < nb; ++k) cv.z(P.dtheta * (double)k, P.zx[k], P.zy[k]);

  // (c) inside mask and the distance-to-box checks
  P.inside.assign((size_t)(M + 1) * (M + 1), 0);
  for (int j = 0; j <= M; ++j)
    for (int i = 0; i <= M; ++i) P.inside[(size_t)j * (M + 1) + i] = cv.level(xg[i], xg[j]) < 0.0;
  for (int j = 0; j <= M; ++j)
    for (int i = 0; i <= M; ++i)
      if (P.in(i, j) && (i < 2 || j < 2 || i > M - 2 || j > M - 2)) {
        err = "interface closer than 2h to the box boundary";
        return KFBI_ERR_GEOMETRY;
      }
  const double lim_lo = P.lo + 2.0 * h, lim_hi = P.hi - 2.0 * h;
  for (int k = 0; k < nb; ++k)
    if (P.zx[k] < lim_lo || P.zx[k] > lim_hi || P.zy[k] < lim_lo || P.zy[k] > lim_hi) {
      err = "boundary node closer than 2h to the box boundary";
      return KFBI_ERR_GEOMETRY;
    }

  // (d) cut edges: horizontal (row-major over j, i) then vertical
  for (int j = 0; j <= M; ++j)
    for (int i = 0; i < M; ++i)
      if (P.in(i, j) != P.in(i + 1, j)) {
        double t = bisect_edge(cv, xg[i], xg[j], xg[i + 1], xg[j], P.in(i, j));
        double c = xg[i] + t * h;
        P.e_i.push_back(i);
        P.e_j.push_back(j);
        P.e_dir.push_back(0);
        P.e_coord.push_back(c);
        P.e_theta.push_back(cv.param_of(c, xg[j]));
      }
  for (int j = 0; j < M; ++j)
    for (int i = 0; i <= M; ++i)
      if (P.in(i, j) != P.in(i, j + 1)) {
        double t = bisect_edge(cv, xg[i], xg[j], xg[i], xg[j + 1], P.in(i, j));
        double c = xg[j] + t * h;
        P.e_i.push_back(i);
        P.e_j.push_back(j);
        P.e_dir.push_back(1);
        P.e_coord.push_back(c);
        P.e_theta.push_back(cv.param_of(xg[i], c));
      }

  // irregular nodes: interior nodes with a neighbour on the other side
  std::vector<int> irr_of((size_t)n1 * n1, -1);
  for (int j = 1; j < M; ++j)
    for (int i = 1; i < M; ++i) {
      bool s = P.in(i, j);
      if (P.in(i + 1, j) != s || P.in(i - 1, j) != s || P.in(i, j + 1) != s || P.in(i, j - 1) != s) {
        irr_of[(size_t)(j - 1) * n1 + (i - 1)] = (int)P.irr.size();
        P.irr.push_back((j - 1) * n1 + (i - 1));
      }
    }

  // correction arms: two per cut edge, grouped by node
  struct Arm {
    int node, k0;
    double alpha[6], beta[6], delta[6];
    int fidx[2];
    double fcoef[2];
  };
  std::vector<Arm> arms;
  arms.reserve(2 * P.e_i.size());
  const double inv_h2 = 1.0 / (h * h);
  for (int e = 0; e < P.n_edges(); ++e) {
    const int i = P.e_i[e], j = P.e_j[e], dir = P.e_dir[e];
    const double c = P.e_coord[e], th = P.e_theta[e];
    const int qi = dir == 0 ? i + 1 : i, qj = dir == 0 ? j : j + 1;
    Frame fr = frame_at(cv, th);
    double q = th / P.dtheta;
    int k0 = (int)std::floor(q);
    if (k0 > nb - 1) k0 = nb - 1;
    double s = q - (double)k0;
    double W0[6], As[6], Ass[6];
    density_weights(s, fr, P.dtheta, W0, As, Ass);
    const double ct = fr.t1p * fr.t1 + fr.t2p * fr.t2;
    const double cn = fr.t1p * fr.t2 - fr.t2p * fr.t1;
    // along the cut direction d: td = t.e_d, nd = n.e_d with n = (t2, -t1)
    double td, nd, Pw, Qw, Nw;
    if (dir == 0) {
      td = fr.t1; nd = fr.t2; Pw = fr.t1 * fr.t1 - fr.t2 * fr.t2; Qw = fr.t1 * fr.t2; Nw = fr.t2 * fr.t2;
    } else {
      td = fr.t2; nd = -fr.t1; Pw = fr.t2 * fr.t2 - fr.t1 * fr.t1; Qw = -fr.t1 * fr.t2; Nw = fr.t1 * fr.t1;
    }
    // f at the intersection: linear extrapolation along the grid line from
    // the Omega-side endpoint pin and the next node inward.
    const bool p_in = P.in(i, j);
    const int pi = p_in ? i : qi, pj = p_in ? j : qj;
    const int step = p_in ? -1 : 1;
    const int p2i = dir == 0 ? pi + step : pi, p2j = dir == 0 ? pj : pj + step;
    const double delta = std::fabs(c - (dir == 0 ? xg[pi] : xg[pj]));
    const bool p2_in = P.in(p2i, p2j);
    for (int side = 0; side < 2; ++side) {
      const int ni = side == 0 ? i : qi, nj = side == 0 ? j : qj;
      const int mi = side == 0 ? qi : i, mj = side == 0 ? qj : j;
      const double d = (dir == 0 ? xg[mi] : xg[mj]) - c;
      const double sc = (P.in(ni, nj) ? -1.0 : 1.0) * inv_h2;
      Arm a;
      a.node = irr_of[(size_t)(nj - 1) * n1 + (ni - 1)];
      if (a.node < 0) {
        err = "cut-edge endpoint is not an interior irregular node";
        return KFBI_ERR_GEOMETRY;
      }
      a.k0 = ((k0 - 2) % nb + nb) % nb;
      const double hd2 = 0.5 * d * d;
      for (int m = 0; m < 6; ++m) {
        a.alpha[m] = sc * (W0[m] + d * td * As[m] +
                           hd2 * ((Ass[m] - ct * As[m]) * Pw + 2.0 * cn * As[m] * Qw));
        a.beta[m] = sc * hd2 * Nw * W0[m];
        // psi part: [u] = 0, [u_d] = nd psi, and in the (t, n) frame
        // H_tt = -cn psi, H_tn = psi_s - ct psi, H_nn = cn psi, so
        // [u_dd] = -cn Pw psi + 2 Qw (psi_s - ct psi)
        a.delta[m] = sc * (d * nd * W0[m] +
                           hd2 * (-cn * Pw * W0[m] + 2.0 * Qw * (As[m] - ct * W0[m])));
      }
      const double gam = sc * hd2 * Nw;
      a.fidx[0] = (pj - 1) * n1 + (pi - 1);
      if (p2_in) {
        a.fidx[1] = (p2j - 1) * n1 + (p2i - 1);
        a.fcoef[0] = gam * (1.0 + delta / h);
        a.fcoef[1] = -gam * (delta / h);
      } else {
        a.fidx[1] = a.fidx[0];
        a.fcoef[0] = gam;
        a.fcoef[1] = 0.0;
      }
      arms.push_back(a);
    }
  }
  std::stable_sort(arms.begin(), arms.end(), [](const Arm& x, const Arm& y) { return x.node < y.node; });
  const int na = (int)arms.size();
  P.arm_start.assign(P.n_irr() + 1, 0);
  P.arm_node.resize(na);
  P.arm_k0.resize(na);
  P.arm_alpha.resize((size_t)na * 6);
  P.arm_beta.resize((size_t)na * 6);
  P.arm_delta.resize((size_t)na * 6);
  P.arm_fidx.resize((size_t)na * 2);
  P.arm_fcoef.resize((size_t)na * 2);
  for (int a = 0; a < na; ++a) {
    P.arm_node[a] = arms[a].node;
    P.arm_k0[a] = arms[a].k0;
    P.arm_start[arms[a].node + 1]++;
    for (int m = 0; m < 6; ++m) {
      P.arm_alpha[(size_t)a * 6 + m] = arms[a].alpha[m];
      P.arm_beta[(size_t)a * 6 + m] = arms[a].beta[m];
      P.arm_delta[(size_t)a * 6 + m] = arms[a].delta[m];
    }
    for (int q2 = 0; q2 < 2; ++q2) {
      P.arm_fidx[(size_t)a * 2 + q2] = arms[a].fidx[q2];
      P.arm_fcoef[(size_t)a * 2 + q2] = arms[a].fcoef[q2];
    }
  }
  for (int n = 0; n < P.n_irr(); ++n) P.arm_start[n + 1] += P.arm_start[n];

  // extraction tables (Eq. 3.36) per boundary node
  P.node_gidx.resize((size_t)nb * 6);
  P.node_w.resize((size_t)nb * 6);
  P.node_a.resize((size_t)nb * 6);
  P.node_b.resize((size_t)nb * 6);
  P.node_fidx.resize(nb);
  P.node_fcoef.resize(nb);
  P.node_wn.resize((size_t)nb * 6);
  P.node_e.resize((size_t)nb * 6);
  P.node_fcoef_n.resize(nb);
  for (int k = 0; k < nb; ++k) {
    const double zx = P.zx[k], zy = P.zy[k];
    const int i0 = (int)std::floor((zx - P.lo) / h + 0.5);
    const int j0 = (int)std::floor((zy - P.lo) / h + 0.5);
    const int sx = (zx - xg[i0] >= 0.0) ? 1 : -1;
    const int sy = (zy - xg[j0] >= 0.0) ? 1 : -1;
    const int si[6] = {i0, i0 + 1, i0 - 1, i0, i0, i0 + sx};
    const int sj[6] = {j0, j0, j0, j0 + 1, j0 - 1, j0 + sy};
    double A[36], rhs[6] = {1, 0, 0, 0, 0, 0};
    double xi[6], eta[6];
    int best = -1;
    double bestd = 0.0;
    for (int m = 0; m < 6; ++m) {
      if (si[m] < 1 || si[m] > M - 1 || sj[m] < 1 || sj[m] > M - 1) {
        err = "extraction stencil leaves the interior grid";
        return KFBI_ERR_GEOMETRY;
      }
      P.node_gidx[(size_t)k * 6 + m] = (sj[m] - 1) * n1 + (si[m] - 1);
      xi[m] = xg[si[m]] - zx;
      eta[m] = xg[sj[m]] - zy;
      // transposed, column-scaled Taylor matrix: A[c][m] = T[m][c] * D_c
      const double row[6] = {1.0, xi[m] / h, eta[m] / h, 0.5 * xi[m] * xi[m] / (h * h),
                             xi[m] * eta[m] / (h * h), 0.5 * eta[m] * eta[m] / (h * h)};
      for (int cc = 0; cc < 6; ++cc) A[cc * 6 + m] = row[cc];
      if (P.in(si[m], sj[m])) {
        double dd = (xg[si[m]] - zx) * (xg[si[m]] - zx) + (xg[sj[m]] - zy) * (xg[sj[m]] - zy);
        if (best < 0 || dd < bestd) {
          best = m;
          bestd = dd;
        }
      }
    }
    if (best < 0) {
      err = "extraction stencil has no point in Omega";
      return KFBI_ERR_GEOMETRY;
    }
    // normal-derivative weights: the same system with right-hand side
    // (t2 e_1 - t1 e_2) / h (the 1/h undoes the column scaling)
    Frame fr = frame_at(cv, P.dtheta * (double)k);
    const double t1 = fr.t1, t2 = fr.t2;
    double An[36], rn[6] = {0.0, t2 / h, -t1 / h, 0.0, 0.0, 0.0};
    std::memcpy(An, A, sizeof(A));
    if (!gepp(A, rhs, 6) || !gepp(An, rn, 6)) {
      err = "singular extraction system";
      return KFBI_ERR_GEOMETRY;
    }
    double G[6] = {0, 0, 0, 0, 0, 0}, Gn[6] = {0, 0, 0, 0, 0, 0};
    for (int m = 0; m < 6; ++m) {
      P.node_w[(size_t)k * 6 + m] = rhs[m];
      P.node_wn[(size_t)k * 6 + m] = rn[m];
      if (!P.in(si[m], sj[m])) {
        const double tay[6] = {1.0, xi[m], eta[m], 0.5 * xi[m] * xi[m], xi[m] * eta[m],
                               0.5 * eta[m] * eta[m]};
        for (int c2 = 0; c2 < 6; ++c2) {
          G[c2] += rhs[m] * tay[c2];
          Gn[c2] += rn[m] * tay[c2];
        }
      }
    }
    double W0[6], As[6], Ass[6];
    density_weights(0.0, fr, P.dtheta, W0, As, Ass);
    const double ct = fr.t1p * t1 + fr.t2p * t2;
    const double cn = fr.t1p * t2 - fr.t2p * t1;
    const double Mss = G[3] * (t1 * t1 - t2 * t2) + G[5] * (t2 * t2 - t1 * t1) + 2.0 * G[4] * t1 * t2;
    const double Mtn = 2.0 * G[3] * t1 * t2 - 2.0 * G[5] * t1 * t2 + G[4] * (t2 * t2 - t1 * t1);
    const double cR3 = G[3] * t2 * t2 + G[5] * t1 * t1 - G[4] * t1 * t2;
    const double cphis = G[1] * t1 + G[2] * t2 - ct * Mss + cn * Mtn;
    for (int m = 0; m < 6; ++m) {
      P.node_a[(size_t)k * 6 + m] = G[0] * W0[m] + cphis * As[m] + Mss * Ass[m];
      P.node_b[(size_t)k * 6 + m] = cR3 * W0[m];
    }
    P.node_fidx[k] = (sj[best] - 1) * n1 + (si[best] - 1);
    P.node_fcoef[k] = cR3;
    // d_n u+ with Phi = 0, Psi = psi: jumps [u_x] = t2 psi, [u_y] = -t1 psi
    // and, in the (t, n) frame, H_tt = -cn psi, H_tn = psi_s - ct psi,
    // H_nn = f + cn psi, projected through the Omega^c rows (Gn)
    const double Ktt = Gn[3] * t1 * t1 + Gn[4] * t1 * t2 + Gn[5] * t2 * t2;
    const double Ktn = 2.0 * (Gn[3] - Gn[5]) * t1 * t2 + Gn[4] * (t2 * t2 - t1 * t1);
    const double Knn = Gn[3] * t2 * t2 - Gn[4] * t1 * t2 + Gn[5] * t1 * t1;
    const double cpsi = Gn[1] * t2 - Gn[2] * t1 - cn * Ktt - ct * Ktn + cn * Knn;
    for (int m = 0; m < 6; ++m) P.node_e[(size_t)k * 6 + m] = cpsi * W0[m] + Ktn * As[m];
    P.node_fcoef_n[k] = Knn;
  }
  return KFBI_OK;
}

}  // namespace kfbi
