// Device building blocks of the lattice Boltzmann update in generalized
// metrics (Sec. II of the paper): pull streaming with full bounce-back along
// the path, moments, equilibrium, non-equilibrium stress, forcing term, BGK.
//
// Arithmetic is organised per velocity pair (c, -c): every term is either even
// or odd in c, so each pair costs one evaluation of the even part E and of
// the odd part O, and f(+c) uses E + O while f(-c) uses E - O.
#pragma once

#include <cstdint>
#include <type_traits>

#include "lattice.cuh"

namespace lbgm {

enum MetricKind { KFLAT = 0, KCYL = 1, KELL = 2 };

// ---------------------------------------------------------------------------
// launch geometry
// ---------------------------------------------------------------------------
// Division by a runtime-invariant unsigned integer (round-up multiply-shift).
struct FastDiv {
  uint32_t d, mul, shift;
  __host__ static FastDiv make(uint32_t d_) {
    FastDiv f{d_, 0u, 0u};
    if (d_ == 1) return f;
    uint32_t l = 0;
    while ((1ull << l) < d_) ++l;
    f.shift = l - 1;
    f.mul = uint32_t(((1ull << (32 + l)) + d_ - 1) / d_ - (1ull << 32));
    return f;
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    if (d == 1) return n;
    uint32_t t = __umulhi(n, mul);
    return (t + ((n - t) >> 1)) >> shift;
  }
};

struct Dims {
  int nr, nt, n3;
  int ncell;       // nr * nt * n3 (one instance)
  int periodic3;   // 0: walls on x3
  int batch;
  int geo_rows3;   // n3 for the ellipsoid's (r, x3) rows, 1 otherwise
  FastDiv div_ncell, div_n3, div_nt;
};

// Geometry rows in the compute precision. A row is i_r * geo_rows3 + i_3 (or
// i_r). Only the components that are non-zero for the metric kind are read:
// every other Delta^ij, Gamma^i_jk and g^{i theta} is zero at theta = 0.
template <typename Real>
struct GeoDev {
  const Real* dtt;    // Delta^{theta theta}
  const Real* dpp;    // Delta^{33}
  const Real* g_rtt;  // h Gamma^r_{theta theta}
  const Real* g_rpp;  // h Gamma^r_{33}
  const Real* g_trt;  // h Gamma^theta_{r theta}
  const Real* g_prp;  // h Gamma^3_{r 3}
  const Real* g_ttp;  // h Gamma^theta_{theta 3}
  const Real* g_ptt;  // h Gamma^3_{theta theta}
  const Real* fth;    // g^{theta theta}
};

template <typename Real>
struct InstParams {
  Real omega;  // 1 / tau
  Real kappa;  // 1 - 1/(2 tau) (improved forcing) or 0 (old forcing)
  Real G;      // covariant streamwise force per step
  Real pad;
};

struct CellPos {
  int b, cell, ir, it, i3;
};

__device__ __forceinline__ CellPos locate(const Dims& d, uint32_t t) {
  CellPos p;
  p.b = int(d.div_ncell.div(t));
  p.cell = int(t) - p.b * d.ncell;
  uint32_t row = d.div_n3.div(uint32_t(p.cell));
  p.i3 = p.cell - int(row) * d.n3;
  p.ir = int(d.div_nt.div(row));
  p.it = int(row) - p.ir * d.nt;
  return p;
}

// ---------------------------------------------------------------------------
// compile-time loops
// ---------------------------------------------------------------------------
template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

template <int P>
struct Pair {
  static constexpr int x = PAIRS[P].x, y = PAIRS[P].y, z = PAIRS[P].z;
  static constexpr double w = PAIRS[P].w;
  static constexpr int s = (x != 0 ? (x < 0 ? -x : x) : (y != 0 ? (y < 0 ? -y : y) : (z < 0 ? -z : z)));
};

// ---------------------------------------------------------------------------
// pull streaming
// ---------------------------------------------------------------------------
// periodic wrap of v in [-3, n + 3) onto [0, n)
__device__ __forceinline__ int wrap_small(int v, int n) {
  if (n >= 3) {
    v += (v < 0) ? n : 0;
    v -= (v >= n) ? n : 0;
    return v;
  }
  v %= n;
  return v < 0 ? v + n : v;
}

// Node offsets of the sources of one node far from every wall:
// source of population c is x - c (periodic in theta, and in x3 if periodic).
struct Neighbours {
  int rrow[7];  // (i_r - c) * nt for c = -3..3 (index c + 3)
  int tcol[7];  // wrap(i_t - c)
  int zcol[7];  // i_3 - c, wrapped if periodic
};

__device__ __forceinline__ void make_neighbours(const CellPos& p, const Dims& d, Neighbours& n) {
#pragma unroll
  for (int c = -3; c <= 3; ++c) {
    n.rrow[c + 3] = (p.ir - c) * d.nt;
    n.tcol[c + 3] = wrap_small(p.it - c, d.nt);
    int z = p.i3 - c;
    n.zcol[c + 3] = d.periodic3 ? wrap_small(z, d.n3) : z;
  }
}

template <int CX, int CY, int CZ>
__device__ __forceinline__ int src_far(const Neighbours& n, const Dims& d) {
  return (n.rrow[CX + 3] + n.tcol[CY + 3]) * d.n3 + n.zcol[CZ + 3];
}

// Source of population c arriving at a node near a wall. The population's
// path is a straight line x + q * sigma (sigma = c / s, q in lattice units
// along each non-zero axis); a wall reverses the whole velocity, so the path
// folds back and forth on the interval of the line inside the walls. In
// half-node units Q = 2 q the walls are odd integers lo < 0 < hi. Going back
// one time step means moving 2 s towards negative Q; each fold flips the
// population to its opposite.
template <int CX, int CY, int CZ, int S>
__device__ __forceinline__ int src_wall(const CellPos& p, const Dims& d, bool& flip) {
  constexpr int sx = (CX > 0) - (CX < 0), sy = (CY > 0) - (CY < 0), sz = (CZ > 0) - (CZ < 0);
  int lo = -(1 << 30), hi = (1 << 30);
  if constexpr (sx != 0) {
    const int l_ = sx > 0 ? -1 - 2 * p.ir : 2 * p.ir + 1 - 2 * d.nr;
    const int h_ = sx > 0 ? 2 * d.nr - 1 - 2 * p.ir : 2 * p.ir + 1;
    lo = max(lo, l_);
    hi = min(hi, h_);
  }
  if constexpr (sz != 0) {
    if (!d.periodic3) {
      const int l_ = sz > 0 ? -1 - 2 * p.i3 : 2 * p.i3 + 1 - 2 * d.n3;
      const int h_ = sz > 0 ? 2 * d.n3 - 1 - 2 * p.i3 : 2 * p.i3 + 1;
      lo = max(lo, l_);
      hi = min(hi, h_);
    }
  }
  constexpr int D = 2 * S;
  int Qe;
  flip = false;
  if (-D >= lo) {
    Qe = -D;
  } else {
    int v = D + lo;  // distance left after the first fold (odd, < D)
    const int L = hi - lo;
    int k = 0;
    while (v > L) {  // at most D / 2 iterations
      v -= L;
      ++k;
    }
    flip = (k & 1) == 0;  // k + 1 folds
    Qe = (k & 1) ? hi - v : lo + v;
  }
  const int q = Qe / 2;
  const int yr = p.ir + q * sx;
  const int yt = wrap_small(p.it + q * sy, d.nt);
  int yz = p.i3 + q * sz;
  if (d.periodic3) yz = wrap_small(yz, d.n3);
  return (yr * d.nt + yt) * d.n3 + yz;
}

__device__ __forceinline__ bool near_wall(const CellPos& p, const Dims& d) {
  return p.ir < 3 || p.ir > d.nr - 4 || (!d.periodic3 && (p.i3 < 3 || p.i3 > d.n3 - 4));
}

// Streamed populations of a node near a wall: every moving population from
// its (possibly folded) source, read from the post-collision state fin.
template <typename Real>
__device__ __forceinline__ void gather_wall(const Real* __restrict__ fin, const CellPos& p,
                                            const Dims& d, Real (&f)[Q]) {
  const int N = d.ncell;
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    using C = Pair<P>;
    bool fp, fm;
    const int sp = src_wall<C::x, C::y, C::z, C::s>(p, d, fp);
    const int sm = src_wall<-C::x, -C::y, -C::z, C::s>(p, d, fm);
    f[2 * P + 1] = __ldg(fin + (fp ? 2 * P + 2 : 2 * P + 1) * N + sp);
    f[2 * P + 2] = __ldg(fin + (fm ? 2 * P + 1 : 2 * P + 2) * N + sm);
  });
}

// Load the 41 streamed populations of node p from the post-collision state
// fin (one instance's block: population l of cell c at fin[l * ncell + c]).
template <typename Real>
__device__ __forceinline__ void gather(const Real* __restrict__ fin, const CellPos& p,
                                       const Dims& d, Real (&f)[Q]) {
  const int N = d.ncell;
  f[0] = __ldg(fin + p.cell);
  if (!near_wall(p, d)) {
    Neighbours nb;
    make_neighbours(p, d, nb);
    static_for<0, NPAIR>([&](auto P_) {
      constexpr int P = decltype(P_)::value;
      using C = Pair<P>;
      const int sp = src_far<C::x, C::y, C::z>(nb, d);
      const int sm = src_far<-C::x, -C::y, -C::z>(nb, d);
      f[2 * P + 1] = __ldg(fin + (2 * P + 1) * N + sp);
      f[2 * P + 2] = __ldg(fin + (2 * P + 2) * N + sm);
    });
  } else {
    gather_wall(fin, p, d, f);
  }
}

// ---------------------------------------------------------------------------
// moments and collision
// ---------------------------------------------------------------------------
template <typename Real>
struct Moments {
  Real rho, jx, jy, jz;
  Real sxx, syy, szz, sxy, sxz, syz;  // sum_l c^i c^j f_l
};

template <typename Real>
__device__ __forceinline__ Moments<Real> moments(const Real (&f)[Q]) {
  Moments<Real> m;
  m.rho = f[0];
  m.jx = m.jy = m.jz = Real(0);
  m.sxx = m.syy = m.szz = m.sxy = m.sxz = m.syz = Real(0);
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    using C = Pair<P>;
    const Real s = f[2 * P + 1] + f[2 * P + 2];
    const Real df = f[2 * P + 1] - f[2 * P + 2];
    m.rho += s;
    if constexpr (C::x != 0) m.jx += Real(C::x) * df;
    if constexpr (C::y != 0) m.jy += Real(C::y) * df;
    if constexpr (C::z != 0) m.jz += Real(C::z) * df;
    if constexpr (C::x != 0) m.sxx += Real(C::x * C::x) * s;
    if constexpr (C::y != 0) m.syy += Real(C::y * C::y) * s;
    if constexpr (C::z != 0) m.szz += Real(C::z * C::z) * s;
    if constexpr (C::x * C::y != 0) m.sxy += Real(C::x * C::y) * s;
    if constexpr (C::x * C::z != 0) m.sxz += Real(C::x * C::z) * s;
    if constexpr (C::y * C::z != 0) m.syz += Real(C::y * C::z) * s;
  });
  return m;
}

// Geometry of one node, read for the metric kind K.
template <typename Real, int K>
struct NodeGeo {
  Real dtt = Real(0), dpp = Real(0);
  Real g_rtt = Real(0), g_rpp = Real(0), g_trt = Real(0), g_prp = Real(0), g_ttp = Real(0),
       g_ptt = Real(0);
  Real fth = Real(1);

  __device__ __forceinline__ void load(const GeoDev<Real>& g, int row) {
    fth = __ldg(g.fth + row);
    if constexpr (K == KCYL || K == KELL) {
      dtt = __ldg(g.dtt + row);
      g_rtt = __ldg(g.g_rtt + row);
      g_trt = __ldg(g.g_trt + row);
    }
    if constexpr (K == KELL) {
      dpp = __ldg(g.dpp + row);
      g_rpp = __ldg(g.g_rpp + row);
      g_prp = __ldg(g.g_prp + row);
      g_ttp = __ldg(g.g_ttp + row);
      g_ptt = __ldg(g.g_ptt + row);
    }
  }
};

// Per-node coefficients of the equilibrium and of the forcing term.
//   f^eq(+-c) = w (E +- O), forcing(+-c) = w (Fe +- Fo), with
//   E  = e0 + eA c.Delta.c + eB (u.c)^2
//   O  = u.c (oA + eB c.Delta.c + oC (u.c)^2) - Vs.c
//   Fe = fA (u.c)(F.c) - fB (u.F)
//   Fo = (F.c)(t0 + (c.A2s.c) / (2 cs^2)) - F.(A2s c)
// where, from Sec. II,
//   a2 = rho (cs^2 Delta + u u),  tr a2 = rho (cs^2 tr Delta + |u|^2),
//   V^k = a3^{iik} = rho (cs^2 (tr Delta u^k + 2 (Delta u)^k) + |u|^2 u^k),
//   A2 = a2 + kappa Pi,  Pi = sum c c f - rho (cs^2 g^-1 + u u)
//   (sum c c f^eq = rho cs^2 g^ij + rho u^i u^j by the lattice's 4th-moment
//   identity), A2s = A2 / cs^4, F^i = F_ext^i - Gamma^i_jk c^j c^k.
template <typename Real>
struct Coef {
  Real rho, ux, uy, uz;
  Real e0, eA, eB, oA, oC;
  Real vx, vy, vz;  // Vs = V / (2 cs^4)
  Real fA, fB, t0;
  Real axx, ayy, azz, axy, axz, ayz;  // A2s
  Real fext_t;                         // F^theta_ext
};

template <typename Real, int K>
__device__ __forceinline__ Coef<Real> coefficients(const Moments<Real>& m, const NodeGeo<Real, K>& g,
                                                   Real kappa, Real G) {
  constexpr Real cs2 = Real(CS2);
  constexpr Real inv_cs2 = Real(1.0 / CS2);
  constexpr Real inv_cs4 = Real(1.0 / (CS2 * CS2));
  Coef<Real> c;
  const Real rho = m.rho;
  const Real irho = Real(1) / rho;
  const Real ux = m.jx * irho, uy = m.jy * irho, uz = m.jz * irho;
  c.rho = rho;
  c.ux = ux;
  c.uy = uy;
  c.uz = uz;
  const Real uu = ux * ux + uy * uy + uz * uz;
  const Real trD = g.dtt + g.dpp;
  const Real tra2 = rho * (cs2 * trD + uu);
  c.e0 = rho - Real(0.5) * inv_cs2 * tra2;
  c.eA = rho * Real(0.5 * (1.0 / CS2));
  c.eB = rho * Real(0.5 / (CS2 * CS2));
  c.oA = rho * inv_cs2;
  c.oC = rho * Real(1.0 / (6.0 * CS2 * CS2 * CS2));
  // V / (2 cs^4), Delta diagonal (dtt on theta, dpp on x3)
  const Real vs = Real(0.5 / (CS2 * CS2)) * rho;
  c.vx = vs * (cs2 * (trD * ux) + uu * ux);
  c.vy = vs * (cs2 * (trD * uy + Real(2) * g.dtt * uy) + uu * uy);
  c.vz = vs * (cs2 * (trD * uz + Real(2) * g.dpp * uz) + uu * uz);
  c.fA = rho * inv_cs4;
  c.fB = rho * inv_cs2;
  // A2 = (1 - kappa) rho (cs^2 Delta + u u) + kappa (S - rho cs^2 delta)
  const Real k1 = Real(1) - kappa;
  const Real rc = rho * cs2;
  Real axx = k1 * (rho * ux * ux) + kappa * (m.sxx - rc);
  Real ayy = k1 * (rho * (cs2 * g.dtt + uy * uy)) + kappa * (m.syy - rc);
  Real azz = k1 * (rho * (cs2 * g.dpp + uz * uz)) + kappa * (m.szz - rc);
  Real axy = k1 * (rho * ux * uy) + kappa * m.sxy;
  Real axz = k1 * (rho * ux * uz) + kappa * m.sxz;
  Real ayz = k1 * (rho * uy * uz) + kappa * m.syz;
  const Real trA2 = axx + ayy + azz;
  c.t0 = c.fB - Real(0.5) * inv_cs4 * trA2;
  c.axx = axx * inv_cs4;
  c.ayy = ayy * inv_cs4;
  c.azz = azz * inv_cs4;
  c.axy = axy * inv_cs4;
  c.axz = axz * inv_cs4;
  c.ayz = ayz * inv_cs4;
  c.fext_t = G * g.fth;
  return c;
}

// BGK collision with the forcing term for the pair (c, -c), in place.
template <typename Real, int K, int P>
__device__ __forceinline__ void collide_pair(Real& fp, Real& fm, const Coef<Real>& k,
                                             const NodeGeo<Real, K>& g, Real omega) {
  using C = Pair<P>;
  constexpr int cx = C::x, cy = C::y, cz = C::z;
  constexpr Real w = Real(C::w);
  constexpr Real half_inv_cs2 = Real(0.5 / CS2);
  // u.c and c.Delta.c
  Real uc = Real(0);
  if constexpr (cx != 0) uc += Real(cx) * k.ux;
  if constexpr (cy != 0) uc += Real(cy) * k.uy;
  if constexpr (cz != 0) uc += Real(cz) * k.uz;
  Real cDc = Real(0);
  if constexpr (cy != 0) cDc += Real(cy * cy) * g.dtt;
  if constexpr (cz != 0 && K == KELL) cDc += Real(cz * cz) * g.dpp;
  Real vc = Real(0);
  if constexpr (cx != 0) vc += Real(cx) * k.vx;
  if constexpr (cy != 0) vc += Real(cy) * k.vy;
  if constexpr (cz != 0) vc += Real(cz) * k.vz;
  const Real uc2 = uc * uc;
  const Real E = k.e0 + k.eA * cDc + k.eB * uc2;
  const Real O = uc * (k.oA + k.eB * cDc + k.oC * uc2) - vc;
  // F = F_ext - Gamma(c, c) (even in c)
  Real Fr = Real(0), Ft = k.fext_t, Fz = Real(0);
  if constexpr (K == KCYL || K == KELL) {
    if constexpr (cy != 0) Fr -= Real(cy * cy) * g.g_rtt;
    if constexpr (cx * cy != 0) Ft -= Real(2 * cx * cy) * g.g_trt;
  }
  if constexpr (K == KELL) {
    if constexpr (cz != 0) Fr -= Real(cz * cz) * g.g_rpp;
    if constexpr (cy * cz != 0) Ft -= Real(2 * cy * cz) * g.g_ttp;
    if constexpr (cx * cz != 0) Fz -= Real(2 * cx * cz) * g.g_prp;
    if constexpr (cy != 0) Fz -= Real(cy * cy) * g.g_ptt;
  }
  Real Fc = Real(cy) * Ft;
  if constexpr (cx != 0) Fc += Real(cx) * Fr;
  if constexpr (cz != 0) Fc += Real(cz) * Fz;
  Real uF = k.ux * Fr + k.uy * Ft;
  if constexpr (K == KELL) uF += k.uz * Fz;
  // A2s c
  Real ax = Real(0), ay = Real(0), az = Real(0);
  if constexpr (cx != 0) { ax += Real(cx) * k.axx; ay += Real(cx) * k.axy; az += Real(cx) * k.axz; }
  if constexpr (cy != 0) { ax += Real(cy) * k.axy; ay += Real(cy) * k.ayy; az += Real(cy) * k.ayz; }
  if constexpr (cz != 0) { ax += Real(cz) * k.axz; ay += Real(cz) * k.ayz; az += Real(cz) * k.azz; }
  Real cAc = Real(0);
  if constexpr (cx != 0) cAc += Real(cx) * ax;
  if constexpr (cy != 0) cAc += Real(cy) * ay;
  if constexpr (cz != 0) cAc += Real(cz) * az;
  Real FAc = Fr * ax + Ft * ay;
  if constexpr (K == KELL) FAc += Fz * az;
  const Real Fe = k.fA * uc * Fc - k.fB * uF;
  const Real Fo = Fc * (k.t0 + half_inv_cs2 * cAc) - FAc;
  // BGK: f* = f + omega (f^eq - f) + forcing
  const Real eqp = w * (E + O), eqm = w * (E - O);
  const Real frp = w * (Fe + Fo), frm = w * (Fe - Fo);
  fp = fp + omega * (eqp - fp) + frp;
  fm = fm + omega * (eqm - fm) + frm;
}

template <typename Real, int K>
__device__ __forceinline__ void collide(Real (&f)[Q], const Coef<Real>& k, const NodeGeo<Real, K>& g,
                                        Real omega) {
  constexpr Real w0 = Real(W_REST);
  // rest velocity: f^eq = w0 e0, forcing = -w0 fB (u . F_ext)
  const Real eq0 = w0 * k.e0;
  const Real fr0 = -w0 * k.fB * (k.uy * k.fext_t);
  f[0] = f[0] + omega * (eq0 - f[0]) + fr0;
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    collide_pair<Real, K, P>(f[2 * P + 1], f[2 * P + 2], k, g, omega);
  });
}

// f^eq(rho, u) for all 41 velocities (initial state, Sec. II).
template <typename Real, int K>
__device__ __forceinline__ void equilibrium(Real rho, Real ux, Real uy, Real uz,
                                            const NodeGeo<Real, K>& g, Real (&f)[Q]) {
  Moments<Real> m;
  m.rho = rho;
  m.jx = rho * ux;
  m.jy = rho * uy;
  m.jz = rho * uz;
  // kappa = 0: the second moment is not used
  m.sxx = m.syy = m.szz = m.sxy = m.sxz = m.syz = Real(0);
  Coef<Real> k = coefficients<Real, K>(m, g, Real(0), Real(0));
  k.ux = ux;
  k.uy = uy;
  k.uz = uz;
  f[0] = Real(W_REST) * k.e0;
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    using C = Pair<P>;
    constexpr Real w = Real(C::w);
    Real uc = Real(C::x) * ux + Real(C::y) * uy + Real(C::z) * uz;
    Real cDc = Real(C::y * C::y) * g.dtt + Real(C::z * C::z) * g.dpp;
    Real vc = Real(C::x) * k.vx + Real(C::y) * k.vy + Real(C::z) * k.vz;
    const Real E = k.e0 + k.eA * cDc + k.eB * uc * uc;
    const Real O = uc * (k.oA + k.eB * cDc + k.oC * uc * uc) - vc;
    f[2 * P + 1] = w * (E + O);
    f[2 * P + 2] = w * (E - O);
  });
}

}  // namespace lbgm
