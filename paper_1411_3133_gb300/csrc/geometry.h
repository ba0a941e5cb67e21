// Host-side FP64 geometry of a channel: metric, Christoffel symbols, lattice
// scaling (Sec. III and IV of the paper), evaluated once per context.
#pragma once

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

// nr * n3 rows of LB_GEO_STRIDE doubles (row = i_r * n3 + i_3).
std::vector<double> evaluate_geometry(lb_metric metric, const lb_geometry_desc& g);

// Lattice spacing h: d / nr (bounce-back walls) or d / (nr - 1) (wall nodes).
double lattice_h(const lb_geometry_desc& g);
// Physical radius of node i_r and the x3 coordinate of node i_3 (z or phi).
double node_r(const lb_geometry_desc& g, int ir);
double node_x3(const lb_geometry_desc& g, int i3);

// Streamwise curvature radius of the inner wall (r_i, r_i b^2; 0 for FLAT).
double curvature_radius(lb_metric metric, const lb_geometry_desc& g);

// Laminar curved-channel Poiseuille speed v(r) = A r ln r + B r + C / r for
// force G per step (cylinder, Sec. III), coefficients in physical r.
void curved_poiseuille(const lb_geometry_desc& g, double tau, double G, double* A,
                       double* B, double* C);

}  // namespace lbgm
