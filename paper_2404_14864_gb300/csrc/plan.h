// Host-side setup of a KFBI domain (Procedure 1 of Sec. 3.3, arXiv 2404.14864)
// and the coefficient tables that turn Procedure 2 into three gather kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "kfbi.h"

namespace kfbi {

// Analytic interface curve, counter-clockwise.
struct Curve {
  int kind = KFBI_CURVE_POLAR;
  double cx = 0, cy = 0;
  double p[6] = {0, 0, 0, 0, 0, 0};
  double ca = 1, sa = 0;  // ellipse rotation

  void z(double t, double& x, double& y) const;
  void dz(double t, double& x, double& y) const;
  void d2z(double t, double& x, double& y) const;
  double level(double x, double y) const;     // < 0 inside
  double param_of(double x, double y) const;  // curve parameter in [0, 2 pi)
};

struct Plan {
  kfbi_domain_desc desc{};
  int M = 0, nb = 0, n1 = 0;  // n1 = M - 1 unknowns per side
  double lo = 0, hi = 0, h = 0, dtheta = 0;
  Curve curve;

  std::vector<uint8_t> inside;  // (M+1)^2, [j*(M+1)+i]
  std::vector<double> zx, zy;   // boundary nodes

  // cut edges
  std::vector<int> e_i, e_j, e_dir;
  std::vector<double> e_coord, e_theta;

  // irregular nodes (interior index, ascending) and their correction arms
  std::vector<int> irr;        // (j-1)*n1 + (i-1)
  std::vector<int> arm_start;  // n_irr + 1 (arms of node n: [arm_start[n], arm_start[n+1]) )
  std::vector<int> arm_node, arm_k0;  // k0 = first density node of the stencil
  std::vector<double> arm_alpha, arm_beta;  // [a*6 + m]
  std::vector<int> arm_fidx;                // [a*2 + q], interior index
  std::vector<double> arm_fcoef;            // [a*2 + q]
  // Neumann data (Psi = psi, Phi = 0): correction weights of psi at the
  // arm's six density nodes (no kappa term: [u] = 0)
  std::vector<double> arm_delta;  // [a*6 + m]

  // boundary-node extraction tables
  std::vector<int> node_gidx;     // [k*6 + m]
  std::vector<double> node_w;     // [k*6 + m]
  std::vector<double> node_a, node_b;  // [k*6 + j], density nodes k-2+j
  std::vector<int> node_fidx;     // [k]
  std::vector<double> node_fcoef; // [k]
  // interior normal derivative d_n u+ (Neumann BIE, Eq. 3.19): stencil
  // weights, psi weights at density nodes k-2+j, f coefficient
  std::vector<double> node_wn, node_e;  // [k*6 + m], [k*6 + j]
  std::vector<double> node_fcoef_n;     // [k]

  int n_irr() const { return (int)irr.size(); }
  int n_arms() const { return (int)arm_node.size(); }
  int n_edges() const { return (int)e_i.size(); }
  bool in(int i, int j) const { return inside[(size_t)j * (M + 1) + i] != 0; }
};

// Build the plan; returns KFBI_OK or an error with a message in err.
kfbi_status build_plan(const kfbi_domain_desc& desc, Plan& plan, std::string& err);

// Weights of the polynomial interpolant through nodes x[0..n-1] for the
// derivatives 0..nd at z (Fornberg's recursion, Math. Comp. 51, 1988).
// c[i*(nd+1) + d] = weight of node i for derivative d.
void fd_weights(double z, const double* x, int n, int nd, double* c);

}  // namespace kfbi
