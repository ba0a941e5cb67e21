// Host-side FP64 geometry of a channel: metric, Christoffel symbols, lattice
// scaling (Sec. III and IV of the paper), evaluated once per context.
#pragma once

#include <cmath>
#include <string>
#include <vector>

#include "../../include/lbgm.h"

namespace lbgm {

// Field offsets inside one LB_GEO_STRIDE row (see lb_geometry_eval).
enum GeoField {
  GEO_DELTA = 0,    // 9
  GEO_GAMMA = 9,    // 27
  GEO_FDIR = 36,    // 3
  GEO_SQRTG = 39,
  GEO_SPEED = 40,
  GEO_WA = 41,
  GEO_WOMEGA = 42,
  GEO_RPHYS = 43,
};

// Validate a descriptor; returns an empty string when valid.
std::string validate_geometry(lb_metric metric, const lb_geometry_desc& g);

// geometry_rows rows of LB_GEO_STRIDE doubles (row = i_r * n3 + i_3, or
// (i_r * ntheta + i_theta) * n3 + i_3 for LB_METRIC_ELLIPSOIDAL_THETA).
std::vector<double> evaluate_geometry(lb_metric metric, const lb_geometry_desc& g);

// Functions compiled for the host and, inside CUDA translation units, for the
// device too, so that the host's geometry table and device code that needs
// the same numbers share one formula.
#if defined(__CUDACC__)
#define LBGM_HD __host__ __device__
#else
#define LBGM_HD
#endif

// Lattice spacing h: d / nr (bounce-back walls) or d / (nr - 1) (wall nodes).
inline LBGM_HD double lattice_h(const lb_geometry_desc& g) {
  return (g.r_outer - g.r_inner) / (g.wall == LB_WALL_EQUILIBRIUM ? g.nr - 1 : g.nr);
}
// Physical radius of node i_r: nodes at r_i + (i_r + 1/2) h between
// bounce-back walls, at r_i + i_r h with the end nodes on equilibrium walls.
inline LBGM_HD double node_r(const lb_geometry_desc& g, int ir) {
  return g.r_inner + (g.wall == LB_WALL_EQUILIBRIUM ? ir : ir + 0.5) * lattice_h(g);
}
// x3 coordinate (z or phi) of node i_3, centred on the channel's mid-plane.
inline LBGM_HD double node_x3(const lb_geometry_desc& g, int i3) {
  const bool on_walls = g.wall == LB_WALL_EQUILIBRIUM && !g.periodic3;
  return (on_walls ? i3 - 0.5 * (g.n3 - 1) : i3 + 0.5 - 0.5 * g.n3) * lattice_h(g) * g.d3_scale;
}

// theta of node i_theta of a theta-resolved channel, centred on theta = 0.
inline LBGM_HD double node_theta(const lb_geometry_desc& g, int it) {
  return (it + 0.5 - 0.5 * g.ntheta) * lattice_h(g) * g.dtheta_scale;
}

// Geometry rows of a descriptor: nr * n3, or nr * ntheta * n3 when the metric
// is evaluated at each theta node.
inline size_t geometry_rows(lb_metric metric, const lb_geometry_desc& g) {
  return size_t(g.nr) * g.n3 * (metric == LB_METRIC_ELLIPSOIDAL_THETA ? size_t(g.ntheta) : 1);
}

// Physical metric of a node at theta = 0 (diagonal there: g_rr, g_thth,
// g_33) and the weights of the observables: the cross-section's area element
// wA (1 for the cylinder's dr dz, r for the ellipsoid's r dr dphi) and the
// vorticity weight wOm = sqrt(g_thth) (Sec. III and IV formulas for <v_theta>
// and <omega^theta>).
struct NodeMetric {
  double g[3];
  double wA, wOm;
};
inline LBGM_HD NodeMetric node_metric(lb_metric metric, const lb_geometry_desc& gd, double r, double x3) {
  NodeMetric m{{1.0, 1.0, 1.0}, 1.0, 1.0};
  if (metric == LB_METRIC_CYLINDRICAL) {
    m.g[1] = r * r;
    m.wOm = r;
  } else if (metric == LB_METRIC_ELLIPSOIDAL) {
    const double cp = cos(x3);
    m.g[1] = gd.b * gd.b * r * r * cp * cp;
    m.g[2] = r * r;
    m.wA = r;
    m.wOm = gd.b * r * cp;
  }
  return m;
}
// The metric in the scaled lattice coordinates y^i = x^i / s_i, s = (1,
// dtheta_scale, d3_scale) (Sec. IV.B spacings): g'_ii = g_ii s_i^2.
inline LBGM_HD void scaled_metric(const NodeMetric& m, const lb_geometry_desc& gd, double gs[3]) {
  const double s[3] = {1.0, gd.dtheta_scale, gd.d3_scale};
  for (int i = 0; i < 3; ++i) gs[i] = m.g[i] * (s[i] * s[i]);
}
// The four per-row weights of the observables: sqrt g', sqrt g'_thth (the
// physical streamwise speed per unit u^theta), wA, wOm.
inline LBGM_HD void observable_weights(lb_metric metric, const lb_geometry_desc& gd, int ir, int i3,
                                       double w[4]) {
  const NodeMetric m = node_metric(metric, gd, node_r(gd, ir), node_x3(gd, i3));
  double gs[3];
  scaled_metric(m, gd, gs);
  w[0] = sqrt(gs[0] * gs[1] * gs[2]);
  w[1] = sqrt(gs[1]);
  w[2] = m.wA;
  w[3] = m.wOm;
}

// Streamwise curvature radius of the inner wall (r_i, r_i b^2; 0 for FLAT).
double curvature_radius(lb_metric metric, const lb_geometry_desc& g);

// Laminar curved-channel Poiseuille speed v(r) = A r ln r + B r + C / r for
// force G per step (cylinder, Sec. III), coefficients in physical r.
void curved_poiseuille(const lb_geometry_desc& g, double tau, double G, double* A,
                       double* B, double* C);

}  // namespace lbgm
