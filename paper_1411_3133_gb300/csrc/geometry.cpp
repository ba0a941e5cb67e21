// Channel geometry in FP64 from the closed forms printed in the paper.
//
//  * Cylindrical coordinates (Sec. III): g = diag(1, r^2, 1); the only
//    non-vanishing Christoffel symbols are Gamma^r_thth = -r and
//    Gamma^th_rth = Gamma^th_thr = 1/r.
//  * Ellipsoidal coordinates with a = c = 1 (Sec. IV): the six metric
//    components printed there; at theta = 0 they reduce to
//    g = diag(1, b^2 r^2 cos^2 phi, r^2). The Christoffel symbols printed there
//    (Gamma^r_thth = -r cos^2 phi, Gamma^r_phph = -r, Gamma^th_rth =
//    Gamma^ph_rph = 1/r, Gamma^th_thph = -tan phi, Gamma^ph_thth = sin phi cos
//    phi) depend on neither b nor theta.
//  * Lattice map (Sec. III, IV): Delta r = Delta theta = Delta x3 = Delta t = h
//    and the rescaled spacings of Sec. IV.B. With scaled coordinates
//    y^i = x^i / s_i, s = (1, dtheta_scale, d3_scale), a tensor picks up
//    g'_ij = g_ij s_i s_j and Gamma'^i_jk = Gamma^i_jk s_j s_k / s_i, so every
//    lattice spacing is h. Lattice velocities are per time step and
//    Delta t = h, so the update uses h * Gamma'.
//  * Body force: constant covariant streamwise component, F^i = g'^{i theta} G.
#include "geometry.h"

#include <cmath>
#include <cstdio>

namespace lbgm {

std::string validate_geometry(lb_metric metric, const lb_geometry_desc& g) {
  char buf[256];
  if (metric != LB_METRIC_FLAT && metric != LB_METRIC_CYLINDRICAL && metric != LB_METRIC_ELLIPSOIDAL &&
      metric != LB_METRIC_ELLIPSOIDAL_THETA)
    return "unknown metric";
  const bool ell = metric == LB_METRIC_ELLIPSOIDAL || metric == LB_METRIC_ELLIPSOIDAL_THETA;
  if (!(g.r_outer > g.r_inner)) return "need r_outer > r_inner";
  if (metric != LB_METRIC_FLAT && !(g.r_inner > 0.0)) return "need r_inner > 0";
  if (g.wall != LB_WALL_BOUNCEBACK && g.wall != LB_WALL_EQUILIBRIUM) return "unknown wall condition";
  const bool eq = g.wall == LB_WALL_EQUILIBRIUM;
  if (eq) {
    if (g.nr < 3) return "need nr >= 3 (two wall nodes and a fluid node)";
  } else if (g.nr < 7) {
    return "need nr >= 7 (walls with |c| = 3 populations)";
  }
  if (g.ntheta < 1 || g.n3 < 1) return "need ntheta >= 1 and n3 >= 1";
  if (!g.periodic3 && g.n3 < (eq ? 3 : 7))
    return eq ? "need n3 >= 3 when the third axis has walls" : "need n3 >= 7 when the third axis has walls";
  if (!(g.dtheta_scale > 0.0) || !(g.d3_scale > 0.0)) return "need positive dtheta_scale, d3_scale";
  if (ell) {
    if (!(g.b > 0.0)) return "need b > 0";
    const double h = lattice_h(g);
    const double phmax = (eq && !g.periodic3 ? 0.5 * (g.n3 - 1) : 0.5 * g.n3) * h * g.d3_scale;
    if (!(phmax < 0.5 * M_PI)) {
      std::snprintf(buf, sizeof buf, "phi range +-%.4g reaches the pole (|phi| must stay < pi/2)",
                    phmax);
      return buf;
    }
  }
  const double cells = double(g.nr) * g.ntheta * g.n3;
  if (cells * 41.0 >= 2147483647.0) return "too many nodes per instance (41 N must fit in int32)";
  return "";
}

double curvature_radius(lb_metric metric, const lb_geometry_desc& g) {
  if (metric == LB_METRIC_CYLINDRICAL) return g.r_inner;
  if (metric == LB_METRIC_ELLIPSOIDAL || metric == LB_METRIC_ELLIPSOIDAL_THETA) return g.r_inner * g.b * g.b;
  return 0.0;
}

namespace {

// One row of the theta-resolved ellipsoid at physical (r, theta, phi): the
// six printed Sec. IV metric components, scaled by the lattice map and
// inverted; the frozen channel's Christoffel symbols (they depend on neither
// b nor theta); the observables' weights of the node.
void theta_row(const lb_geometry_desc& gd, double r, double th, double ph, double* row) {
  const double h = lattice_h(gd);
  const double s[3] = {1.0, gd.dtheta_scale, gd.d3_scale};
  const double b2 = gd.b * gd.b;
  const double ct = std::cos(th), st = std::sin(th), cp = std::cos(ph), sp = std::sin(ph);
  const double q = ct * ct + b2 * st * st;  // cos^2 th + b^2 sin^2 th
  double g[3][3];
  g[0][0] = sp * sp + cp * cp * q;
  g[1][1] = r * r * cp * cp * (st * st + b2 * ct * ct);
  g[2][2] = r * r * (cp * cp + sp * sp * q);
  g[0][1] = g[1][0] = r * (b2 - 1.0) * cp * cp * ct * st;
  g[0][2] = g[2][0] = r * (1.0 - b2) * st * st * cp * sp;
  g[1][2] = g[2][1] = r * r * (1.0 - b2) * cp * sp * ct * st;
  double gs[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) gs[i][j] = g[i][j] * s[i] * s[j];
  // inverse by cofactors
  const double c00 = gs[1][1] * gs[2][2] - gs[1][2] * gs[2][1];
  const double c01 = gs[1][2] * gs[2][0] - gs[1][0] * gs[2][2];
  const double c02 = gs[1][0] * gs[2][1] - gs[1][1] * gs[2][0];
  const double det = gs[0][0] * c00 + gs[0][1] * c01 + gs[0][2] * c02;
  double inv[3][3];
  inv[0][0] = c00 / det;
  inv[1][0] = c01 / det;
  inv[2][0] = c02 / det;
  inv[0][1] = (gs[0][2] * gs[2][1] - gs[0][1] * gs[2][2]) / det;
  inv[1][1] = (gs[0][0] * gs[2][2] - gs[0][2] * gs[2][0]) / det;
  inv[2][1] = (gs[0][1] * gs[2][0] - gs[0][0] * gs[2][1]) / det;
  inv[0][2] = (gs[0][1] * gs[1][2] - gs[0][2] * gs[1][1]) / det;
  inv[1][2] = (gs[0][2] * gs[1][0] - gs[0][0] * gs[1][2]) / det;
  inv[2][2] = (gs[0][0] * gs[1][1] - gs[0][1] * gs[1][0]) / det;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) row[GEO_DELTA + i * 3 + j] = inv[i][j] - (i == j ? 1.0 : 0.0);
  double G[3][3][3] = {};
  G[0][1][1] = -r * cp * cp;
  G[0][2][2] = -r;
  G[1][0][1] = G[1][1][0] = 1.0 / r;
  G[2][0][2] = G[2][2][0] = 1.0 / r;
  G[1][1][2] = G[1][2][1] = -sp / cp;
  G[2][1][1] = sp * cp;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) row[GEO_GAMMA + (i * 3 + j) * 3 + k] = h * G[i][j][k] * s[j] * s[k] / s[i];
  for (int i = 0; i < 3; ++i) row[GEO_FDIR + i] = inv[i][1];
  row[GEO_SQRTG] = std::sqrt(det);
  row[GEO_SPEED] = std::sqrt(gs[1][1]);
  row[GEO_WA] = std::sqrt(g[0][0] * g[2][2] - g[0][2] * g[0][2]);
  row[GEO_WOMEGA] = std::sqrt(g[1][1]);
  row[GEO_RPHYS] = r;
}

}  // namespace

std::vector<double> evaluate_geometry(lb_metric metric, const lb_geometry_desc& gd) {
  if (metric == LB_METRIC_ELLIPSOIDAL_THETA) {
    std::vector<double> out(geometry_rows(metric, gd) * LB_GEO_STRIDE, 0.0);
    for (int ir = 0; ir < gd.nr; ++ir)
      for (int it = 0; it < gd.ntheta; ++it)
        for (int i3 = 0; i3 < gd.n3; ++i3)
          theta_row(gd, node_r(gd, ir), node_theta(gd, it), node_x3(gd, i3),
                    &out[((size_t(ir) * gd.ntheta + it) * gd.n3 + i3) * LB_GEO_STRIDE]);
    return out;
  }
  const int nr = gd.nr, n3 = gd.n3;
  const double h = lattice_h(gd);
  const double s[3] = {1.0, gd.dtheta_scale, gd.d3_scale};
  std::vector<double> out(size_t(nr) * n3 * LB_GEO_STRIDE, 0.0);
  for (int ir = 0; ir < nr; ++ir) {
    const double r = node_r(gd, ir);
    for (int i3 = 0; i3 < n3; ++i3) {
      const double x3 = node_x3(gd, i3);  // z or phi
      const NodeMetric nm = node_metric(metric, gd, r, x3);  // physical, diagonal at theta = 0
      double G[3][3][3] = {};                                  // physical Gamma^i_jk
      if (metric == LB_METRIC_CYLINDRICAL) {
        G[0][1][1] = -r;
        G[1][0][1] = G[1][1][0] = 1.0 / r;
      } else if (metric == LB_METRIC_ELLIPSOIDAL) {
        const double cp = std::cos(x3), sp = std::sin(x3);
        G[0][1][1] = -r * cp * cp;
        G[0][2][2] = -r;
        G[1][0][1] = G[1][1][0] = 1.0 / r;
        G[2][0][2] = G[2][2][0] = 1.0 / r;
        G[1][1][2] = G[1][2][1] = -sp / cp;
        G[2][1][1] = sp * cp;
      }
      double* row = &out[(size_t(ir) * n3 + i3) * LB_GEO_STRIDE];
      double gs[3];
      scaled_metric(nm, gd, gs);
      for (int i = 0; i < 3; ++i) row[GEO_DELTA + i * 3 + i] = 1.0 / gs[i] - 1.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          for (int k = 0; k < 3; ++k)
            row[GEO_GAMMA + (i * 3 + j) * 3 + k] = h * G[i][j][k] * s[j] * s[k] / s[i];
      row[GEO_FDIR + 1] = 1.0 / gs[1];
      observable_weights(metric, gd, ir, i3, &row[GEO_SQRTG]);  // sqrt g', speed, wA, wOmega
      row[GEO_RPHYS] = r;
    }
  }
  return out;
}

void curved_poiseuille(const lb_geometry_desc& gd, double tau, double G, double* A, double* B,
                       double* C) {
  // nu (v'' + v'/r - v/r^2) = -G_phys / r with G_phys = G / h and nu_phys =
  // nu h in units where lattice speeds equal physical speeds; the particular
  // solution is A r ln r with A = -G / (2 nu h^2).
  const double cs2 = 1.0 - std::sqrt(0.4);
  const double nu = (tau - 0.5) * cs2;
  const double h = lattice_h(gd);
  const double a = -G / (2.0 * nu * h * h);
  const double ri = gd.r_inner, ro = gd.r_outer;
  // B r + C / r = -a r ln r at r_i and r_o
  const double m00 = ri, m01 = 1.0 / ri, m10 = ro, m11 = 1.0 / ro;
  const double b0 = -a * ri * std::log(ri), b1 = -a * ro * std::log(ro);
  const double det = m00 * m11 - m01 * m10;
  *A = a;
  *B = (b0 * m11 - m01 * b1) / det;
  *C = (m00 * b1 - b0 * m10) / det;
}

}  // namespace lbgm
