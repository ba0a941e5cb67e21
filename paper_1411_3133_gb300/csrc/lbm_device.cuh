// Device building blocks of the lattice Boltzmann update in generalized
// metrics (Sec. II of the paper): pull streaming with full bounce-back along
// the path, moments, equilibrium, non-equilibrium stress, forcing term, BGK.
//
// Arithmetic is organised per velocity pair (c, -c): every term is either even
// or odd in c, so each pair costs one evaluation of the even part E and of
// the odd part O, and f(+c) uses E + O while f(-c) uses E - O.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

#include "lattice.cuh"

namespace lbgm {

// KELT: the theta-resolved double-curved channel -- the ellipsoidal metric
// of each theta node (full Delta^ij, body force with r and phi components),
// the frozen channel's Christoffel symbols, one geometry row per node.
enum MetricKind { KFLAT = 0, KCYL = 1, KELL = 2, KELT = 3 };

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
  int geo_rows3;   // geometry rows per i_r: n3 for the ellipsoid's (r, x3)
                   // rows, nt n3 for the theta-resolved one, 1 otherwise
  FastDiv div_ncell, div_n3, div_nt;
  // 2-byte storage: reference populations over the nr * geo_rows3 geometry
  // rows, per instance (ref_index; NULL for FP32 / FP64 storage)
  const float* ref;
  int wall_eq;     // 1: equilibrium (Dirichlet) walls on the end nodes
  // 2-byte storage: the stream table of each instance (stream_index; NULL
  // for FP32 / FP64 storage) over nr * st_rows3 stream rows
  const float4* st;
  int st_rows3;    // n3 (ellipsoid), 1 (periodic x3), 7 (walls on x3)
  int geo_theta;   // 1: geometry rows (and observable weights) per node
};

// Index of reference population l of geometry row r in an instance's table:
// row-major [r][l] where rows are i_r only (cylinder, flat: a warp shares
// the row, and the offsets of a node's 41 entries are compile-time
// constants), population-major [l][r] for the ellipsoid's (i_r, i_3) rows
// (consecutive nodes read consecutive rows).
template <int K>
__device__ __forceinline__ uint32_t ref_index(const Dims& d, int l, int row) {
  if constexpr (K == KELL) return uint32_t(l) * uint32_t(d.nr) * uint32_t(d.geo_rows3) + uint32_t(row);
  else return uint32_t(row) * 41u + uint32_t(l);
}

// Geometry row of node (i_r, i_3): i_r * n3 + i_3 for the ellipsoid, i_r
// otherwise.
template <int K>
__device__ __forceinline__ int geo_row(const Dims& d, int ir, int i3) {
  if constexpr (K == KELL) return ir * d.geo_rows3 + i3;
  else return ir;
}

// Geometry row of node p for metric kind K: i_r (flat, cylinder), (i_r, i_3)
// (ellipsoid), the node itself (theta-resolved ellipsoid).
template <int K>
__device__ __forceinline__ int geo_row_node(const Dims& d, int ir, int it, int i3) {
  if constexpr (K == KELL) return ir * d.geo_rows3 + i3;
  else if constexpr (K == KELT) return ir * d.geo_rows3 + it * d.n3 + i3;
  else return ir;
}

// Reference table of instance b (see Dims::ref).
__device__ __forceinline__ const float* ref_of(const Dims& d, int b) {
  return d.ref ? d.ref + size_t(b) * 41 * size_t(d.nr) * size_t(d.geo_rows3) : nullptr;
}

// Stream rows of 2-byte storage. Which stored population (and whose
// geometry row's reference) a node receives in streaming depends on its
// position only through i_r and, with walls on x3, through its distance to
// them; theta is periodic and the references do not depend on it. A stream
// row groups the nodes that receive alike: (i_r, i_3) for the ellipsoid
// (its references vary along x3), i_r for a periodic x3, and (i_r, class of
// i_3) with classes 0, 1, 2 (first layers), 3 (inside), 4, 5, 6 (last
// layers) for walls on x3.
template <int K>
__device__ __forceinline__ int stream_row(const Dims& d, int ir, int i3) {
  if constexpr (K == KELL) return ir * d.geo_rows3 + i3;
  if (d.st_rows3 == 1) return ir;
  const int c = i3 < 3 ? i3 : (i3 > d.n3 - 4 ? i3 - d.n3 + 7 : 3);
  return ir * 7 + c;
}

// Stream table of instance b: 13 float4 per stream row, stored [k][row]
// (consecutive rows are consecutive float4, so a warp of consecutive i_3
// reads coalesced). Entry k of row s (f_l = w_l g_l + rho_l: g the stored
// deviation, rho_l the reference population of the stored value a node of
// row s receives as population l, t_l = ((1 - omega) rho_l - r_l) / w_l with
// r_l the node's own reference):
//   k = 0: sum rho_l, sum c^x rho_l, sum c^y rho_l, sum c^z rho_l
//   k = 1: sum c^x c^x rho_l, c^y c^y, c^z c^z, c^x c^y
//   k = 2: sum c^x c^z rho_l, sum c^y c^z rho_l, t_0, 0
//   k = 3 + j, j = 0..9: (t_+ + t_-) / 2 and (t_+ - t_-) / 2 of pair 2 j,
//           then of pair 2 j + 1 (t_+ of population 2 P + 1, t_- of 2 P + 2)
constexpr int ST_K = 13;
__device__ __forceinline__ const float4* stream_of(const Dims& d, int b) {
  return d.st + size_t(b) * ST_K * size_t(d.nr) * size_t(d.st_rows3);
}

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
  // theta-resolved ellipsoid only: Delta^rr, Delta^{r theta}, Delta^{r 3},
  // Delta^{theta 3}, g^{r theta}, g^{3 theta} at ext + j * ext_stride
  const Real* ext;
  uint32_t ext_stride;
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

// Position of node `cell` of instance b.
__device__ __forceinline__ CellPos locate_cell(const Dims& d, int b, uint32_t cell) {
  CellPos p;
  p.b = b;
  p.cell = int(cell);
  uint32_t row = d.div_n3.div(cell);
  p.i3 = p.cell - int(row) * d.n3;
  p.ir = int(d.div_nt.div(row));
  p.it = int(row) - p.ir * d.nt;
  return p;
}

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

template <int L>
struct WeightOf {
  static constexpr double w = L == 0 ? W_REST : PAIRS[(L - 1) / 2].w;
};

// ---------------------------------------------------------------------------
// population storage
// ---------------------------------------------------------------------------
// Codec<S, R> reads populations stored as S into the compute type R and back.
// For the reduced-precision formats the stored value is the scaled deviation
// (f_l - r_l) / w_l from a reference population r_l of the storing node's
// geometry row (a table entry, passed as a pointer), so every stored number
// is small whatever its weight: f_l = w_l s_l + r_l. With r_l = w_l this is
// the deviation from the rest state of unit density.
template <class S, class R>
struct Codec {
  static constexpr bool uses_ref = false;
  template <int L>
  __device__ static __forceinline__ R dec(S v, const float*) { return R(v); }
  template <int L>
  __device__ static __forceinline__ S enc(R f, const float*) { return S(f); }
};
template <>
struct Codec<__half, float> {
  static constexpr bool uses_ref = true;
  template <int L>
  __device__ static __forceinline__ float dec(__half v, const float* ref) {
    constexpr float w = float(WeightOf<L>::w);
    return fmaf(w, __half2float(v), __ldg(ref));
  }
  template <int L>
  __device__ static __forceinline__ __half enc(float f, const float* ref) {
    constexpr float iw = float(1.0 / WeightOf<L>::w);
    return __float2half_rn((f - __ldg(ref)) * iw);
  }
};
template <>
struct Codec<__nv_bfloat16, float> {
  static constexpr bool uses_ref = true;
  template <int L>
  __device__ static __forceinline__ float dec(__nv_bfloat16 v, const float* ref) {
    constexpr float w = float(WeightOf<L>::w);
    return fmaf(w, __bfloat162float(v), __ldg(ref));
  }
  template <int L>
  __device__ static __forceinline__ __nv_bfloat16 enc(float f, const float* ref) {
    constexpr float iw = float(1.0 / WeightOf<L>::w);
    return __float2bfloat16_rn((f - __ldg(ref)) * iw);
  }
};

// The stored number itself (2-byte storage: the deviation g) in FP32 and
// back, round to nearest.
__device__ __forceinline__ float raw_dec(__half v) { return __half2float(v); }
__device__ __forceinline__ float raw_dec(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class S>
__device__ __forceinline__ S raw_enc(float x);
template <>
__device__ __forceinline__ __half raw_enc<__half>(float x) { return __float2half_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 raw_enc<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

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
__device__ __forceinline__ int src_wall(const CellPos& p, const Dims& d, bool& flip, int& src_ir, int& src_i3) {
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
  src_ir = yr;
  src_i3 = yz;
  return (yr * d.nt + yt) * d.n3 + yz;
}

__device__ __forceinline__ bool near_wall(const CellPos& p, const Dims& d) {
  return p.ir < 3 || p.ir > d.nr - 4 || (!d.periodic3 && (p.i3 < 3 || p.i3 > d.n3 - 4));
}

// Visit the sources of the 41 streamed populations of node p: fn(L, src,
// sl, row) with L a std::integral_constant (the population received), src
// the address in fin (one instance's block: population l of cell c at
// fin[l * ncell + c]) of the post-collision value it is streamed from, sl
// the population index stored there (L, or its opposite after a fold) and
// row the geometry row of the node that stored it (sl and row select the
// reference population of 2-byte storage). Near a wall every moving
// population comes from its (possibly folded) source; opposite velocities
// share their weight. Offsets are
// 32-bit: an instance block holds fewer than 2^32 bytes (checked when the
// context is created).
template <int K, class S, class Fn>
__device__ __forceinline__ void for_each_source_far(const S* __restrict__ fin, const CellPos& p, const Dims& d,
                                                    Fn&& fn) {
  const uint32_t N = uint32_t(d.ncell);
  Neighbours nb;
  make_neighbours(p, d, nb);
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    using C = Pair<P>;
    const uint32_t sp = uint32_t(src_far<C::x, C::y, C::z>(nb, d));
    const uint32_t sm = uint32_t(src_far<-C::x, -C::y, -C::z>(nb, d));
    fn(std::integral_constant<int, 2 * P + 1>{}, fin + ((2 * P + 1) * N + sp), 2 * P + 1,
       geo_row<K>(d, p.ir - C::x, nb.zcol[C::z + 3]));
    fn(std::integral_constant<int, 2 * P + 2>{}, fin + ((2 * P + 2) * N + sm), 2 * P + 2,
       geo_row<K>(d, p.ir + C::x, nb.zcol[-C::z + 3]));
  });
}

// Equilibrium walls: the source x - c with walled axes clamped onto the
// wall layer (periodic axes wrapped); no flip.
template <int K, class S, class Fn>
__device__ __forceinline__ void for_each_source_clamped(const S* __restrict__ fin, const CellPos& p,
                                                        const Dims& d, Fn&& fn) {
  const uint32_t N = uint32_t(d.ncell);
  auto src = [&](int cx, int cy, int cz, int& yr, int& yz) {
    yr = min(max(p.ir - cx, 0), d.nr - 1);
    const int yt = wrap_small(p.it - cy, d.nt);
    yz = p.i3 - cz;
    yz = d.periodic3 ? wrap_small(yz, d.n3) : min(max(yz, 0), d.n3 - 1);
    return uint32_t((yr * d.nt + yt) * d.n3 + yz);
  };
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    using C = Pair<P>;
    int rp, zp, rm, zm;
    const uint32_t sp = src(C::x, C::y, C::z, rp, zp);
    const uint32_t sm = src(-C::x, -C::y, -C::z, rm, zm);
    fn(std::integral_constant<int, 2 * P + 1>{}, fin + ((2 * P + 1) * N + sp), 2 * P + 1, geo_row<K>(d, rp, zp));
    fn(std::integral_constant<int, 2 * P + 2>{}, fin + ((2 * P + 2) * N + sm), 2 * P + 2, geo_row<K>(d, rm, zm));
  });
}

template <int K, class S, class Fn>
__device__ __forceinline__ void for_each_source_wall(const S* __restrict__ fin, const CellPos& p, const Dims& d,
                                                     Fn&& fn) {
  if (d.wall_eq) {
    for_each_source_clamped<K>(fin, p, d, fn);
    return;
  }
  const uint32_t N = uint32_t(d.ncell);
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    using C = Pair<P>;
    bool fp, fm;
    int rp, zp, rm, zm;
    const uint32_t sp = uint32_t(src_wall<C::x, C::y, C::z, C::s>(p, d, fp, rp, zp));
    const uint32_t sm = uint32_t(src_wall<-C::x, -C::y, -C::z, C::s>(p, d, fm, rm, zm));
    const int lp = fp ? 2 * P + 2 : 2 * P + 1, lm = fm ? 2 * P + 1 : 2 * P + 2;
    fn(std::integral_constant<int, 2 * P + 1>{}, fin + (lp * N + sp), lp, geo_row<K>(d, rp, zp));
    fn(std::integral_constant<int, 2 * P + 2>{}, fin + (lm * N + sm), lm, geo_row<K>(d, rm, zm));
  });
}

// WALLS selects the code paths compiled in: 0 far from every wall only, 1
// near a wall only, 2 both (the node decides).
template <int K, class S, int WALLS = 2, class Fn>
__device__ __forceinline__ void for_each_source(const S* __restrict__ fin, const CellPos& p, const Dims& d,
                                                Fn&& fn) {
  fn(std::integral_constant<int, 0>{}, fin + uint32_t(p.cell), 0, geo_row<K>(d, p.ir, p.i3));
  if constexpr (WALLS == 0) {
    for_each_source_far<K>(fin, p, d, fn);
  } else if constexpr (WALLS == 1) {
    for_each_source_wall<K>(fin, p, d, fn);
  } else {
    if (!near_wall(p, d))
      for_each_source_far<K>(fin, p, d, fn);
    else
      for_each_source_wall<K>(fin, p, d, fn);
  }
}

// Sources for a node J = 0, 1, 2 layers from the wall on side SIDE (0: low,
// 1: high) of axis AX (0: r, 2: x3), at least 3 layers from the walls of
// the other axis (or with that axis periodic), the walled axis at least 7
// nodes long: only that wall can lie on a population's one-step path, so the
// wall rule of src_wall reduces to constants. A population whose backward
// path (along -c, length s = |c|_inf) meets the wall 2 J + 1 half-nodes away
// folds once: its source is x + (s - 1 - 2 J) sigma (sigma = c / s) and it
// arrives flipped; every other population comes from x - c as away from
// walls.
template <int AX, int SIDE, int J, int CX, int CY, int CZ, int S>
struct LayerFold {
  static constexpr int sx = (CX > 0) - (CX < 0), sy = (CY > 0) - (CY < 0), sz = (CZ > 0) - (CZ < 0);
  static constexpr int sa = AX == 0 ? sx : sz;
  static constexpr bool hit = ((SIDE == 0 && sa > 0) || (SIDE == 1 && sa < 0)) && (2 * S > 1 + 2 * J);
  static constexpr int q = hit ? S - 1 - 2 * J : -S;
  static constexpr int dx = q * sx, dy = q * sy, dz = q * sz;  // source - node
};

template <int K, int AX, int SIDE, int J, class S, class Fn>
__device__ __forceinline__ void for_each_source_layer(const S* __restrict__ fin, const CellPos& p,
                                                      const Dims& d, Fn&& fn) {
  const uint32_t N = uint32_t(d.ncell);
  Neighbours nb;
  make_neighbours(p, d, nb);
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    using C = Pair<P>;
    using Fp = LayerFold<AX, SIDE, J, C::x, C::y, C::z, C::s>;
    using Fm = LayerFold<AX, SIDE, J, -C::x, -C::y, -C::z, C::s>;
    const uint32_t sp = uint32_t((nb.rrow[3 - Fp::dx] + nb.tcol[3 - Fp::dy]) * d.n3 + nb.zcol[3 - Fp::dz]);
    const uint32_t sm = uint32_t((nb.rrow[3 - Fm::dx] + nb.tcol[3 - Fm::dy]) * d.n3 + nb.zcol[3 - Fm::dz]);
    constexpr int lp = Fp::hit ? 2 * P + 2 : 2 * P + 1, lm = Fm::hit ? 2 * P + 1 : 2 * P + 2;
    fn(std::integral_constant<int, 2 * P + 1>{}, fin + (lp * N + sp), lp,
       geo_row<K>(d, p.ir + Fp::dx, nb.zcol[3 - Fp::dz]));
    fn(std::integral_constant<int, 2 * P + 2>{}, fin + (lm * N + sm), lm,
       geo_row<K>(d, p.ir + Fm::dx, nb.zcol[3 - Fm::dz]));
  });
}

// Decoding visitor: f[L] from the stored value at src, with the reference
// row table ref (instance base; NULL for FP32 / FP64 storage).
template <int K, class S, class R>
struct DecodeInto {
  R (&f)[Q];
  const float* ref;
  const Dims& d;
  template <class LC>
  __device__ __forceinline__ void operator()(LC, const S* src, int sl, int row) const {
    constexpr int L = LC::value;
    if constexpr (Codec<S, R>::uses_ref)
      f[L] = Codec<S, R>::template dec<L>(__ldg(src), ref + ref_index<K>(d, sl, row));
    else
      f[L] = Codec<S, R>::template dec<L>(__ldg(src), nullptr);
  }
};

// Raw visitor of 2-byte storage: f[L] holds the stored deviation g itself
// (the step works on deviations; see collide_store).
template <class S>
struct RawInto {
  float (&f)[Q];
  template <class LC>
  __device__ __forceinline__ void operator()(LC, const S* src, int, int) const {
    f[LC::value] = raw_dec(__ldg(src));
  }
};

// Streamed populations of a node within 3 layers of a wall of axis AX (0:
// an r-wall, with x3 periodic or the node at least 3 layers from the
// x3-walls, nr >= 7; 2: an x3-wall, the node at least 3 layers from the
// r-walls, n3 >= 7), through the per-layer constant folds, into the visitor
// put (DecodeInto or RawInto).
template <int K, int AX, class S, class Put>
__device__ __forceinline__ void gather_edge_v(const S* __restrict__ fin, const CellPos& p, const Dims& d,
                                              const Put& put) {
  put(std::integral_constant<int, 0>{}, fin + uint32_t(p.cell), 0, geo_row<K>(d, p.ir, p.i3));
  const int i = AX == 0 ? p.ir : p.i3, n = AX == 0 ? d.nr : d.n3;
  const int side = i < 3 ? 0 : 1;
  const int j = side == 0 ? i : n - 1 - i;
  switch (side * 3 + j) {
    case 0: for_each_source_layer<K, AX, 0, 0>(fin, p, d, put); break;
    case 1: for_each_source_layer<K, AX, 0, 1>(fin, p, d, put); break;
    case 2: for_each_source_layer<K, AX, 0, 2>(fin, p, d, put); break;
    case 3: for_each_source_layer<K, AX, 1, 0>(fin, p, d, put); break;
    case 4: for_each_source_layer<K, AX, 1, 1>(fin, p, d, put); break;
    default: for_each_source_layer<K, AX, 1, 2>(fin, p, d, put); break;
  }
}

// The visitor of a gather: decoded populations f, or with RAW (2-byte
// storage only) the stored deviations.
template <int K, class S, class R, bool RAW>
struct GatherPut {
  using type = DecodeInto<K, S, R>;
  __device__ static __forceinline__ type make(R (&f)[Q], const float* ref, const Dims& d) { return {f, ref, d}; }
};
template <int K, class S>
struct GatherPut<K, S, float, true> {
  using type = RawInto<S>;
  __device__ static __forceinline__ type make(float (&f)[Q], const float*, const Dims&) { return {f}; }
};

template <int K, class S, class R, bool RAW = false, int AX = 0>
__device__ __forceinline__ void gather_edge(const S* __restrict__ fin, const float* ref, const CellPos& p,
                                            const Dims& d, R (&f)[Q]) {
  gather_edge_v<K, AX>(fin, p, d, GatherPut<K, S, R, RAW>::make(f, ref, d));
}

// Load the 41 streamed populations of node p from the post-collision state
// (instance block fin, reference table ref). WALLS selects the paths
// compiled in: 0 far from every wall; 1 the general wall rule; 2 the node
// decides among far, the r-layer folds and the general rule; 3 the r-layer
// folds alone (gather_edge, AX 0); 4 the x3-layer folds alone (AX 2).
// WALLS = 2: near an r-wall with bounce-back walls, at least 3 nodes away
// from any x3 wall, only the r-wall can lie on a population's path, and the
// compile-time folds of gather_edge replace the general wall rule (the same
// sources, fewer instructions).
// RAW (2-byte storage only): f receives the stored deviations g instead of
// the decoded populations.
template <int K, class S, class R, int WALLS = 2, bool RAW = false>
__device__ __forceinline__ void gather(const S* __restrict__ fin, const float* ref, const CellPos& p,
                                       const Dims& d, R (&f)[Q]) {
  if constexpr (WALLS == 3 || WALLS == 4) {
    gather_edge<K, S, R, RAW, WALLS == 3 ? 0 : 2>(fin, ref, p, d, f);
    return;
  }
  if constexpr (WALLS == 2) {
    const bool x3_clear = d.periodic3 || (p.i3 >= 3 && p.i3 <= d.n3 - 4);
    if (!d.wall_eq && d.nr >= 7 && x3_clear && (p.ir < 3 || p.ir > d.nr - 4)) {
      gather_edge<K, S, R, RAW>(fin, ref, p, d, f);
      return;
    }
  }
  for_each_source<K, S, WALLS>(fin, p, d, GatherPut<K, S, R, RAW>::make(f, ref, d));
}

// Store the 41 post-collision deviations g of node p (2-byte storage).
template <class S>
__device__ __forceinline__ void store_raw(S* __restrict__ out, const CellPos& p, const Dims& d,
                                          const float (&g)[Q]) {
  const uint32_t N = uint32_t(d.ncell), cell = uint32_t(p.cell);
  static_for<0, Q>([&](auto L_) {
    constexpr int L = decltype(L_)::value;
    out[uint32_t(L) * N + cell] = raw_enc<S>(g[L]);
  });
}

// Store the 41 post-collision populations of node p into the instance block
// `out` (32-bit offsets, as for_each_source).
template <int K, class S, class R>
__device__ __forceinline__ void store_node(S* __restrict__ out, const float* ref, const CellPos& p, const Dims& d,
                                           const R (&f)[Q]) {
  using Cd = Codec<S, R>;
  const uint32_t N = uint32_t(d.ncell), cell = uint32_t(p.cell);
  const int row = geo_row<K>(d, p.ir, p.i3);
  static_for<0, Q>([&](auto L_) {
    constexpr int L = decltype(L_)::value;
    if constexpr (Cd::uses_ref)
      out[uint32_t(L) * N + cell] = Cd::template enc<L>(f[L], ref + ref_index<K>(d, L, row));
    else
      out[uint32_t(L) * N + cell] = Cd::template enc<L>(f[L], nullptr);
  });
}

// ---------------------------------------------------------------------------
// arithmetic types
// ---------------------------------------------------------------------------
// The update is written once for an arithmetic type V: double, float, or PF2
// -- two nodes per thread in packed FP32x2 instructions (FFMA2/FADD2/FMUL2 of
// sm_100 and later), one node per lane, each lane rounded exactly like the
// scalar float instruction. Multiplications by the lattice's integer
// velocity components are spelled out with compile-time helpers (mac, dot3)
// so that no multiplication by 0 or +-1 is issued for any type.
// Every multiply-add is an explicit fmav and the library is compiled with
// -fmad=false, so the compiler fuses no other product into an add: every
// kernel that inlines these functions (plain, TMA, work-list) rounds alike.
struct PF2 {
  float2 v;
  PF2() = default;
  __device__ __forceinline__ PF2(float2 a) : v(a) {}
  __device__ __forceinline__ PF2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit PF2(double c) : v(make_float2(float(c), float(c))) {}
};
__device__ __forceinline__ PF2 operator+(PF2 a, PF2 b) { return PF2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ PF2 operator*(PF2 a, PF2 b) { return PF2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ PF2 operator-(PF2 a, PF2 b) {
  return PF2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v));
}
__device__ __forceinline__ PF2 fmav(PF2 a, PF2 b, PF2 c) { return PF2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ float fmav(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmav(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ PF2 rcpv(PF2 a) { return PF2(__frcp_rn(a.v.x), __frcp_rn(a.v.y)); }
__device__ __forceinline__ float rcpv(float a) { return 1.0f / a; }
__device__ __forceinline__ double rcpv(double a) { return 1.0 / a; }
__device__ __forceinline__ bool finite_v(PF2 a) { return fabsf(a.v.x) < 1e30f && fabsf(a.v.y) < 1e30f; }
__device__ __forceinline__ bool finite_v(float a) { return fabsf(a) < 1e30f; }
__device__ __forceinline__ bool finite_v(double a) { return fabs(a) < 1e300; }

// acc + C x, compile-time integer C
template <int C, class V>
__device__ __forceinline__ V mac(const V& acc, const V& x) {
  if constexpr (C == 0) return acc;
  else if constexpr (C == 1) return acc + x;
  else if constexpr (C == -1) return acc - x;
  else return fmav(V(double(C)), x, acc);
}
// C x, compile-time integer C != 0
template <int C, class V>
__device__ __forceinline__ V mulc(const V& x) {
  static_assert(C != 0, "mulc by zero");
  if constexpr (C == 1) return x;
  else return V(double(C)) * x;
}
// cx ax + cy ay + cz az; the first non-zero component of every pair's
// representative velocity is positive
template <int CX, int CY, int CZ, class V>
__device__ __forceinline__ V dot3(const V& ax, const V& ay, const V& az) {
  if constexpr (CX != 0) return mac<CZ>(mac<CY>(mulc<CX>(ax), ay), az);
  else if constexpr (CY != 0) return mac<CZ>(mulc<CY>(ay), az);
  else return mulc<CZ>(az);
}

// ---------------------------------------------------------------------------
// moments and collision
// ---------------------------------------------------------------------------
template <typename V>
struct Moments {
  V rho, jx, jy, jz;
  V sxx, syy, szz, sxy, sxz, syz;  // sum_l c^i c^j f_l
};

template <typename V>
__device__ __forceinline__ Moments<V> moments(const V (&f)[Q]) {
  Moments<V> m;
  const V z = V(0.0);
  m.rho = f[0];
  m.jx = m.jy = m.jz = z;
  m.sxx = m.syy = m.szz = m.sxy = m.sxz = m.syz = z;
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    using C = Pair<P>;
    const V s = f[2 * P + 1] + f[2 * P + 2];
    const V df = f[2 * P + 1] - f[2 * P + 2];
    m.rho = m.rho + s;
    m.jx = mac<C::x>(m.jx, df);
    m.jy = mac<C::y>(m.jy, df);
    m.jz = mac<C::z>(m.jz, df);
    m.sxx = mac<C::x * C::x>(m.sxx, s);
    m.syy = mac<C::y * C::y>(m.syy, s);
    m.szz = mac<C::z * C::z>(m.szz, s);
    m.sxy = mac<C::x * C::y>(m.sxy, s);
    m.sxz = mac<C::x * C::z>(m.sxz, s);
    m.syz = mac<C::y * C::z>(m.syz, s);
  });
  return m;
}

// acc + (C w_P) x: a lattice-integer coefficient times pair P's weight
template <int C, int P, class V>
__device__ __forceinline__ V macw(const V& acc, const V& x) {
  if constexpr (C == 0) return acc;
  else return fmav(V(double(C) * Pair<P>::w), x, acc);
}

// Moments of the streamed populations f_l = w_l g_l + rho_l from the stored
// deviations g of 2-byte storage: the streamed references' moments (stream
// table entries a, b, c) start the sums, and every weight is folded into the
// multiply-add that accumulates it.
template <typename V>
__device__ __forceinline__ Moments<V> moments_dev(const V (&g)[Q], const float4& a, const float4& b,
                                                  const float4& c) {
  Moments<V> m;
  m.rho = fmav(V(W_REST), g[0], V(a.x));
  m.jx = V(a.y);
  m.jy = V(a.z);
  m.jz = V(a.w);
  m.sxx = V(b.x);
  m.syy = V(b.y);
  m.szz = V(b.z);
  m.sxy = V(b.w);
  m.sxz = V(c.x);
  m.syz = V(c.y);
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    using C = Pair<P>;
    const V s = g[2 * P + 1] + g[2 * P + 2];
    const V df = g[2 * P + 1] - g[2 * P + 2];
    m.rho = macw<1, P>(m.rho, s);
    m.jx = macw<C::x, P>(m.jx, df);
    m.jy = macw<C::y, P>(m.jy, df);
    m.jz = macw<C::z, P>(m.jz, df);
    m.sxx = macw<C::x * C::x, P>(m.sxx, s);
    m.syy = macw<C::y * C::y, P>(m.syy, s);
    m.szz = macw<C::z * C::z, P>(m.szz, s);
    m.sxy = macw<C::x * C::y, P>(m.sxy, s);
    m.sxz = macw<C::x * C::z, P>(m.sxz, s);
    m.syz = macw<C::y * C::z, P>(m.syz, s);
  });
  return m;
}

// Geometry of one node, read for the metric kind K. The Christoffel symbols
// are kept with a minus sign (F^i = F_ext^i - Gamma^i_jk c^j c^k).
template <typename V, int K>
struct NodeGeo {
  V dtt = V(0.0), dpp = V(0.0);
  V n_rtt = V(0.0), n_rpp = V(0.0), n_trt = V(0.0), n_prp = V(0.0), n_ttp = V(0.0), n_ptt = V(0.0);
  V fth = V(1.0);
};

// The theta-resolved ellipsoid adds the off-diagonal and r r components of
// Delta and the r and x3 components of the body force direction.
template <typename V>
struct NodeGeo<V, KELT> : NodeGeo<V, KELL> {
  V drr = V(0.0), drt = V(0.0), drp = V(0.0), dtp = V(0.0);
  V fr = V(0.0), fp = V(0.0);
};

template <typename Real, int K>
__device__ __forceinline__ NodeGeo<Real, K> load_geo(const GeoDev<Real>& g, int row) {
  NodeGeo<Real, K> n;
  n.fth = __ldg(g.fth + row);
  if constexpr (K == KCYL || K == KELL || K == KELT) {
    n.dtt = __ldg(g.dtt + row);
    n.n_rtt = -__ldg(g.g_rtt + row);
    n.n_trt = -__ldg(g.g_trt + row);
  }
  if constexpr (K == KELL || K == KELT) {
    n.dpp = __ldg(g.dpp + row);
    n.n_rpp = -__ldg(g.g_rpp + row);
    n.n_prp = -__ldg(g.g_prp + row);
    n.n_ttp = -__ldg(g.g_ttp + row);
    n.n_ptt = -__ldg(g.g_ptt + row);
  }
  if constexpr (K == KELT) {
    const Real* e = g.ext + row;
    n.drr = __ldg(e);
    n.drt = __ldg(e + g.ext_stride);
    n.drp = __ldg(e + 2 * g.ext_stride);
    n.dtp = __ldg(e + 3 * g.ext_stride);
    n.fr = __ldg(e + 4 * g.ext_stride);
    n.fp = __ldg(e + 5 * g.ext_stride);
  }
  return n;
}

// two nodes' rows into the lanes of a PF2 geometry
template <int K>
__device__ __forceinline__ NodeGeo<PF2, K> load_geo2(const GeoDev<float>& g, int row0, int row1) {
  const NodeGeo<float, K> a = load_geo<float, K>(g, row0);
  const NodeGeo<float, K> b = row1 == row0 ? a : load_geo<float, K>(g, row1);
  NodeGeo<PF2, K> n;
  n.dtt = PF2(a.dtt, b.dtt);
  n.dpp = PF2(a.dpp, b.dpp);
  n.n_rtt = PF2(a.n_rtt, b.n_rtt);
  n.n_rpp = PF2(a.n_rpp, b.n_rpp);
  n.n_trt = PF2(a.n_trt, b.n_trt);
  n.n_prp = PF2(a.n_prp, b.n_prp);
  n.n_ttp = PF2(a.n_ttp, b.n_ttp);
  n.n_ptt = PF2(a.n_ptt, b.n_ptt);
  n.fth = PF2(a.fth, b.fth);
  return n;
}

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
// Stored with signs chosen so that every term is one multiply-add:
// nv = -Vs, nfB = -fB, na = -A2s, and eAt = eA Delta^thth etc.
template <typename V>
struct Coef {
  V ux, uy, uz;
  V e0, eB, oA, oC;
  V eAt, eAp, eBt, eBp;     // eA dtt, eA dpp, eB dtt, eB dpp
  V nvx, nvy, nvz;
  V fA, nfB, t0;
  V naxx, nayy, nazz, naxy, naxz, nayz;
  V fext_t;
  // theta-resolved ellipsoid: eA and eB times Delta^rr, Delta^{r theta},
  // Delta^{r 3}, Delta^{theta 3}; the body force's r and x3 components
  V eArr, eArt, eArp, eAtp, eBrr, eBrt, eBrp, eBtp;
  V fext_r, fext_p;
};

template <typename V, int K>
__device__ __forceinline__ Coef<V> coefficients(const Moments<V>& m, const NodeGeo<V, K>& g, const V& kappa,
                                                const V& G) {
  const V cs2 = V(CS2);
  const V inv_cs2 = V(1.0 / CS2);
  const V inv_cs4 = V(1.0 / (CS2 * CS2));
  Coef<V> c;
  const V rho = m.rho;
  const V irho = rcpv(rho);
  const V ux = m.jx * irho, uy = m.jy * irho, uz = m.jz * irho;
  c.ux = ux;
  c.uy = uy;
  c.uz = uz;
  const V uu = fmav(uz, uz, fmav(uy, uy, ux * ux));
  V trD = g.dtt + g.dpp;
  if constexpr (K == KELT) trD = trD + g.drr;
  const V tra2 = rho * fmav(cs2, trD, uu);
  c.e0 = fmav(V(-0.5 / CS2), tra2, rho);
  const V eA = rho * V(0.5 / CS2);
  c.eB = rho * V(0.5 / (CS2 * CS2));
  c.eAt = eA * g.dtt;
  c.eAp = eA * g.dpp;
  c.eBt = c.eB * g.dtt;
  c.eBp = c.eB * g.dpp;
  c.oA = rho * inv_cs2;
  c.oC = rho * V(1.0 / (6.0 * CS2 * CS2 * CS2));
  // -V / (2 cs^4), Delta diagonal (dtt on theta, dpp on x3)
  const V nvs = V(-0.5 / (CS2 * CS2)) * rho;
  const V trDc = cs2 * trD;
  if constexpr (K == KELT) {
    // full Delta: V^k / rho = cs^2 (tr Delta u^k + 2 (Delta u)^k) + |u|^2 u^k
    const V c2 = V(2.0 * CS2);
    const V dux = fmav(g.drr, ux, fmav(g.drt, uy, g.drp * uz));
    const V duy = fmav(g.drt, ux, fmav(g.dtt, uy, g.dtp * uz));
    const V duz = fmav(g.drp, ux, fmav(g.dtp, uy, g.dpp * uz));
    c.nvx = nvs * fmav(c2, dux, fmav(trDc, ux, uu * ux));
    c.nvy = nvs * fmav(c2, duy, fmav(trDc, uy, uu * uy));
    c.nvz = nvs * fmav(c2, duz, fmav(trDc, uz, uu * uz));
    c.eArr = eA * g.drr;
    c.eArt = eA * g.drt;
    c.eArp = eA * g.drp;
    c.eAtp = eA * g.dtp;
    c.eBrr = c.eB * g.drr;
    c.eBrt = c.eB * g.drt;
    c.eBrp = c.eB * g.drp;
    c.eBtp = c.eB * g.dtp;
  } else {
    c.nvx = nvs * (fmav(trDc, ux, uu * ux));
    c.nvy = nvs * (fmav(fmav(V(2.0 * CS2), g.dtt, trDc), uy, uu * uy));
    c.nvz = nvs * (fmav(fmav(V(2.0 * CS2), g.dpp, trDc), uz, uu * uz));
  }
  c.fA = rho * inv_cs4;
  c.nfB = rho * V(-1.0 / CS2);
  // A2 = (1 - kappa) rho (cs^2 Delta + u u) + kappa (S - rho cs^2 delta)
  const V k1 = V(1.0) - kappa;
  const V rc = rho * cs2;
  const V rk = rho * k1;
  V axx, axy, axz, ayz;
  if constexpr (K == KELT) {
    axx = fmav(rk, fmav(cs2, g.drr, ux * ux), kappa * (m.sxx - rc));
    axy = fmav(rk, fmav(cs2, g.drt, ux * uy), kappa * m.sxy);
    axz = fmav(rk, fmav(cs2, g.drp, ux * uz), kappa * m.sxz);
    ayz = fmav(rk, fmav(cs2, g.dtp, uy * uz), kappa * m.syz);
  } else {
    axx = fmav(rk, ux * ux, kappa * (m.sxx - rc));
    axy = fmav(rk, ux * uy, kappa * m.sxy);
    axz = fmav(rk, ux * uz, kappa * m.sxz);
    ayz = fmav(rk, uy * uz, kappa * m.syz);
  }
  const V ayy = fmav(rk, fmav(cs2, g.dtt, uy * uy), kappa * (m.syy - rc));
  const V azz = fmav(rk, fmav(cs2, g.dpp, uz * uz), kappa * (m.szz - rc));
  const V trA2 = axx + ayy + azz;
  c.t0 = fmav(V(-0.5 / (CS2 * CS2)), trA2, rho * inv_cs2);
  const V nic4 = V(-1.0 / (CS2 * CS2));
  c.naxx = axx * nic4;
  c.nayy = ayy * nic4;
  c.nazz = azz * nic4;
  c.naxy = axy * nic4;
  c.naxz = axz * nic4;
  c.nayz = ayz * nic4;
  c.fext_t = G * g.fth;
  if constexpr (K == KELT) {
    c.fext_r = G * g.fr;
    c.fext_p = G * g.fp;
  }
  return c;
}

// E += eA c.Delta.c and X += eB c.Delta.c for velocity (cx, cy, cz): the
// diagonal theta and x3 terms of every curved metric, and the theta-resolved
// ellipsoid's r r and off-diagonal terms.
template <int K, int cx, int cy, int cz, class V>
__device__ __forceinline__ void add_cdc(V& E, V& X, const Coef<V>& k) {
  constexpr bool curv = K != KFLAT;
  constexpr bool ell = K == KELL || K == KELT;
  if constexpr (curv && cy != 0) {
    E = mac<cy * cy>(E, k.eAt);
    X = mac<cy * cy>(X, k.eBt);
  }
  if constexpr (ell && cz != 0) {
    E = mac<cz * cz>(E, k.eAp);
    X = mac<cz * cz>(X, k.eBp);
  }
  if constexpr (K == KELT) {
    if constexpr (cx != 0) {
      E = mac<cx * cx>(E, k.eArr);
      X = mac<cx * cx>(X, k.eBrr);
    }
    if constexpr (cx * cy != 0) {
      E = mac<2 * cx * cy>(E, k.eArt);
      X = mac<2 * cx * cy>(X, k.eBrt);
    }
    if constexpr (cx * cz != 0) {
      E = mac<2 * cx * cz>(E, k.eArp);
      X = mac<2 * cx * cz>(X, k.eBrp);
    }
    if constexpr (cy * cz != 0) {
      E = mac<2 * cy * cz>(E, k.eAtp);
      X = mac<2 * cy * cz>(X, k.eBtp);
    }
  }
}

// BGK collision with the forcing term for the pair (c, -c), in place:
//   f* = (1 - omega) f + omega f^eq + F
//      = (1 - omega) f + w (omega E + Fe) +- w (omega O + Fo)
//
// DEV (2-byte storage): fp, fm are the stored deviations g = (f - r) / w and
// the result is the post-collision deviation
//   g* = (1 - omega) g + (omega E + Fe + te) +- (omega O + Fo + to)
// with te, to the even and odd parts of t = ((1 - omega) rho - r) / w from the
// stream table; te and to start the sums of Fe and Fo, so they cost no
// instruction, and the weight multiply of the pair drops out.
template <typename V, int K, int P, bool DEV = false>
__device__ __forceinline__ void collide_pair(V& fp, V& fm, const Coef<V>& k, const NodeGeo<V, K>& g,
                                             const V& omega, const V& om1, const V& te = V(0.0),
                                             const V& to = V(0.0)) {
  using C = Pair<P>;
  constexpr int cx = C::x, cy = C::y, cz = C::z;
  constexpr bool curv = K != KFLAT;
  constexpr bool ell = K == KELL || K == KELT;
  constexpr bool gen = K == KELT;
  const V uc = dot3<cx, cy, cz>(k.ux, k.uy, k.uz);
  const V uc2 = uc * uc;
  V E = fmav(k.eB, uc2, k.e0);
  V X = fmav(k.oC, uc2, k.oA);
  add_cdc<K, cx, cy, cz>(E, X, k);
  const V O = fmav(uc, X, dot3<cx, cy, cz>(k.nvx, k.nvy, k.nvz));
  // F = F_ext - Gamma(c, c), even in c; which components exist is known here
  // (the theta-resolved ellipsoid's body force has all three)
  constexpr bool hasFr = gen || (curv && (cy != 0 || (ell && cz != 0)));
  constexpr bool hasFz = gen || (ell && (cx * cz != 0 || cy != 0));
  V Fr = V(0.0), Fz = V(0.0);
  if constexpr (gen) {
    Fr = k.fext_r;
    if constexpr (cy != 0) Fr = mac<cy * cy>(Fr, g.n_rtt);
    if constexpr (cz != 0) Fr = mac<cz * cz>(Fr, g.n_rpp);
    Fz = k.fext_p;
    if constexpr (cy != 0) Fz = mac<cy * cy>(Fz, g.n_ptt);
    if constexpr (cx * cz != 0) Fz = mac<2 * cx * cz>(Fz, g.n_prp);
  } else {
    if constexpr (curv && cy != 0) Fr = mulc<cy * cy>(g.n_rtt);
    if constexpr (ell && cz != 0) Fr = (cy != 0) ? mac<cz * cz>(Fr, g.n_rpp) : mulc<cz * cz>(g.n_rpp);
    if constexpr (ell && cx * cz != 0 && cy != 0) Fz = mac<2 * cx * cz>(mulc<cy * cy>(g.n_ptt), g.n_prp);
    else if constexpr (ell && cx * cz != 0) Fz = mulc<2 * cx * cz>(g.n_prp);
    else if constexpr (ell && cy != 0) Fz = mulc<cy * cy>(g.n_ptt);
  }
  V Ft = k.fext_t;
  if constexpr (curv && cx * cy != 0) Ft = mac<2 * cx * cy>(Ft, g.n_trt);
  if constexpr (ell && cy * cz != 0) Ft = mac<2 * cy * cz>(Ft, g.n_ttp);
  // F.c and u.F
  constexpr bool hasFc = cy != 0 || (cx != 0 && hasFr) || (cz != 0 && hasFz);
  V Fc = V(0.0);
  if constexpr (hasFc) {
    constexpr int ax_ = hasFr ? cx : 0, az_ = hasFz ? cz : 0;
    Fc = dot3<ax_, cy, az_>(Fr, Ft, Fz);
  }
  V uF = k.uy * Ft;
  if constexpr (hasFr) uF = fmav(k.ux, Fr, uF);
  if constexpr (hasFz) uF = fmav(k.uz, Fz, uF);
  // -A2s c, its quadratic form, and F.(-A2s c)
  const V nax = dot3<cx, cy, cz>(k.naxx, k.naxy, k.naxz);
  const V nay = dot3<cx, cy, cz>(k.naxy, k.nayy, k.nayz);
  const V naz = dot3<cx, cy, cz>(k.naxz, k.nayz, k.nazz);
  V FnA;
  if constexpr (DEV) FnA = fmav(Ft, nay, to);
  else FnA = Ft * nay;
  if constexpr (hasFr) FnA = fmav(Fr, nax, FnA);
  if constexpr (hasFz) FnA = fmav(Fz, naz, FnA);
  // Fe = fA uc Fc - fB uF,  Fo = Fc (t0 + cAc / (2 cs^2)) - F.A2s c
  V Fe;
  if constexpr (DEV) Fe = fmav(k.nfB, uF, te);
  else Fe = k.nfB * uF;
  V Fo = FnA;
  if constexpr (hasFc) {
    Fe = fmav(k.fA * uc, Fc, Fe);
    const V ncAc = dot3<cx, cy, cz>(nax, nay, naz);
    Fo = fmav(Fc, fmav(V(-0.5 / CS2), ncAc, k.t0), FnA);
  }
  if constexpr (DEV) {
    const V B = fmav(omega, O, Fo);
    const V a = fmav(omega, E, Fe);
    fp = fmav(om1, fp, a + B);
    fm = fmav(om1, fm, a - B);
  } else {
    const V w = V(C::w);
    const V Bw = fmav(omega, O, Fo) * w;
    const V a = fmav(omega, E, Fe);
    fp = fmav(om1, fp, fmav(a, w, Bw));
    fm = fmav(om1, fm, fmav(a, w, -Bw));
  }
}

template <typename V, int K>
__device__ __forceinline__ void collide(V (&f)[Q], const Coef<V>& k, const NodeGeo<V, K>& g, const V& omega) {
  const V om1 = V(1.0) - omega;
  // rest velocity: f^eq = w0 e0, forcing = -w0 fB (u . F_ext)
  V uF0 = k.uy * k.fext_t;
  if constexpr (K == KELT) uF0 = fmav(k.ux, k.fext_r, fmav(k.uz, k.fext_p, uF0));
  f[0] = fmav(om1, f[0], fmav(omega, k.e0, k.nfB * uF0) * V(W_REST));
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    collide_pair<V, K, P>(f[2 * P + 1], f[2 * P + 2], k, g, omega, om1);
  });
}

// A node's stream-table row: entry k of the table in global memory (st the
// k = 0 entry, stride the table's rows), or of a block's shared-memory copy
// of one row.
struct TabGlobal {
  const float4* __restrict__ st;
  uint32_t stride;
  __device__ __forceinline__ float4 at(int k) const { return __ldg(st + k * stride); }
};
struct TabShared {
  const float4* st;
  __device__ __forceinline__ float4 at(int k) const { return st[k]; }
};

// A node's stream-table row staged in shared memory by its own thread
// (stage_table): entry k at st[k * stride], stride the block's threads.
struct TabStaged {
  const float4* st;
  int stride;
  __device__ __forceinline__ float4 at(int k) const { return st[k * stride]; }
};

// Copy the ST_K entries of stream-table row `row` (table st0 of rows
// `stride` apart) into this thread's shared-memory slots dst[k * step] by
// cp.async (16-byte copies that hold no registers while in flight), so
// their latency runs under the node's gather. The caller waits with
// stage_wait before reading them.
__device__ __forceinline__ void stage_table(float4* dst, int step, const float4* __restrict__ st0, uint32_t stride) {
#pragma unroll
  for (int k = 0; k < ST_K; ++k) {
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(dst + k * step));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(st0 + k * stride) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// BGK collision with forcing on the stored deviations g of 2-byte storage,
// in place (collide_pair with DEV), with the node's stream-table row tab.
template <int K, class Tab>
__device__ __forceinline__ void collide_dev(float (&g)[Q], const Coef<float>& k, const NodeGeo<float, K>& geo,
                                            float omega, const Tab& tab, float t0) {
  const float om1 = 1.0f - omega;
  g[0] = fmaf(om1, g[0], fmaf(omega, k.e0, fmaf(k.nfB, k.uy * k.fext_t, t0)));
  // each table entry is requested one pair group ahead of its use, so a
  // global load overlaps the arithmetic of the group before
  float4 t = tab.at(3);
  static_for<0, NPAIR / 2>([&](auto J_) {
    constexpr int J = decltype(J_)::value;
    float4 tn = t;
    if constexpr (J + 1 < NPAIR / 2) tn = tab.at(4 + J);
    collide_pair<float, K, 2 * J, true>(g[4 * J + 1], g[4 * J + 2], k, geo, omega, om1, t.x, t.y);
    collide_pair<float, K, 2 * J + 1, true>(g[4 * J + 3], g[4 * J + 4], k, geo, omega, om1, t.z, t.w);
    t = tn;
  });
}

// f^eq(rho, u) for all 41 velocities (initial state, Sec. II).
template <typename V, int K>
__device__ __forceinline__ void equilibrium(const V& rho, const V& ux, const V& uy, const V& uz,
                                            const NodeGeo<V, K>& g, V (&f)[Q]) {
  Moments<V> m;
  m.rho = rho;
  m.jx = rho * ux;
  m.jy = rho * uy;
  m.jz = rho * uz;
  m.sxx = m.syy = m.szz = m.sxy = m.sxz = m.syz = V(0.0);  // unused with kappa = 0
  Coef<V> k = coefficients<V, K>(m, g, V(0.0), V(0.0));
  k.ux = ux;
  k.uy = uy;
  k.uz = uz;
  f[0] = k.e0 * V(W_REST);
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    using C = Pair<P>;
    constexpr int cx = C::x, cy = C::y, cz = C::z;
    const V uc = dot3<cx, cy, cz>(ux, uy, uz);
    const V uc2 = uc * uc;
    V E = fmav(k.eB, uc2, k.e0);
    V X = fmav(k.oC, uc2, k.oA);
    if constexpr (cy != 0) {
      E = mac<cy * cy>(E, k.eAt);
      X = mac<cy * cy>(X, k.eBt);
    }
    if constexpr (cz != 0) {
      E = mac<cz * cz>(E, k.eAp);
      X = mac<cz * cz>(X, k.eBp);
    }
    if constexpr (K == KELT) {
      if constexpr (cx != 0) {
        E = mac<cx * cx>(E, k.eArr);
        X = mac<cx * cx>(X, k.eBrr);
      }
      if constexpr (cx * cy != 0) {
        E = mac<2 * cx * cy>(E, k.eArt);
        X = mac<2 * cx * cy>(X, k.eBrt);
      }
      if constexpr (cx * cz != 0) {
        E = mac<2 * cx * cz>(E, k.eArp);
        X = mac<2 * cx * cz>(X, k.eBrp);
      }
      if constexpr (cy * cz != 0) {
        E = mac<2 * cy * cz>(E, k.eAtp);
        X = mac<2 * cy * cz>(X, k.eBtp);
      }
    }
    const V O = fmav(uc, X, dot3<cx, cy, cz>(k.nvx, k.nvy, k.nvz));
    f[2 * P + 1] = (E + O) * V(C::w);
    f[2 * P + 2] = (E - O) * V(C::w);
  });
}

}  // namespace lbgm
