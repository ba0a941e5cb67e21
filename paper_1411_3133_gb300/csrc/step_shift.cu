// Fused step with the half-force velocity variant (lb_params.old_forcing =
// 2): not the paper's printed scheme, which evaluates f^eq and the forcing
// term at the streamed velocity u = sum c f / rho' (Sec. II). Here they are
// evaluated at u_s = u + M(u_s) / (2 rho'), M the forcing term's first
// moment, taken by two fixed-point iterations from u
//   u_1 = u + M(u) / (2 rho'),   u_s = u + M(u_1) / (2 rho'),
// and the forcing term is scaled by 1 - 1/(2 tau): the usual second-order
// treatment of a body force in a discrete-time BGK update. Without it the
// streamed radial velocity of a curved channel's rest state (half the
// per-step Christoffel momentum source) feeds the mass source
// -2 rho' u^i Gamma^j_ij at every step.
//
// M comes from its closed form (Hermite orthogonality of the forcing term):
//   M^m = rho' F_ext^m - rho' cs^2 (Gamma^m_jj + 2 Gamma^j_jm)
//         - 2 A2^ml Gamma^j_jl - A2^lj Gamma^m_lj,
//   A2(u) = (1 - kappa) rho' (cs^2 Delta + u u) + kappa (S - rho' cs^2 delta),
// S = sum c c f (the improved forcing's a2^eq - sigma, Sec. II; kappa = 0 for
// the old forcing is not combined with the variant). With u_s in hand, the
// coefficients of f^eq and of the forcing term are those of the literal
// step for the moments (rho', rho' u_s, S), and the forcing coefficients are
// scaled. Only the plain one-node-per-thread kernel carries the variant; the
// per-instance switch is InstParams::pad (1: variant, 0: literal), so one
// context may mix both.
#include "step_launch.cuh"

namespace lbgm {
namespace {

template <typename V, int K>
__device__ __forceinline__ Coef<V> shifted_coefficients(const Moments<V>& m, const NodeGeo<V, K>& g,
                                                        const InstParams<V>& ip) {
  const V cs2 = V(CS2);
  const V rho = m.rho;
  const V irho = rcpv(rho);
  const V ux0 = m.jx * irho, uy0 = m.jy * irho, uz0 = m.jz * irho;
  // lattice Christoffel symbols (NodeGeo keeps them negated) and contractions
  const V G_rtt = -g.n_rtt, G_rpp = -g.n_rpp, G_trt = -g.n_trt, G_prp = -g.n_prp;
  const V G_ttp = -g.n_ttp, G_ptt = -g.n_ptt;
  const V gam_r = G_trt + G_prp;  // Gamma^j_jr
  const V gam_p = G_ttp;          // Gamma^j_j3
  const V fext_t = ip.G * g.fth;
  const V k1 = V(1.0) - ip.kappa;
  const V rc = rho * cs2;
  V ux = ux0, uy = uy0, uz = uz0;
#pragma unroll 1
  for (int it = 0; it < 2; ++it) {
    const V rk = rho * k1;
    const V axx = fmav(rk, ux * ux, ip.kappa * (m.sxx - rc));
    const V ayy = fmav(rk, fmav(cs2, g.dtt, uy * uy), ip.kappa * (m.syy - rc));
    const V azz = fmav(rk, fmav(cs2, g.dpp, uz * uz), ip.kappa * (m.szz - rc));
    const V axy = fmav(rk, ux * uy, ip.kappa * m.sxy);
    const V axz = fmav(rk, ux * uz, ip.kappa * m.sxz);
    const V ayz = fmav(rk, uy * uz, ip.kappa * m.syz);
    // M^r, M^theta, M^3 (only the components non-zero at theta = 0)
    const V Mr = -rc * (G_rtt + G_rpp + V(2.0) * gam_r) - V(2.0) * fmav(axx, gam_r, axz * gam_p) -
                 fmav(ayy, G_rtt, azz * G_rpp);
    const V Mt = rho * fext_t - V(2.0) * fmav(axy, gam_r, ayz * gam_p) - V(2.0) * fmav(axy, G_trt, ayz * G_ttp);
    const V Mp = -rc * (G_ptt + V(2.0) * gam_p) - V(2.0) * fmav(axz, gam_r, azz * gam_p) -
                 fmav(V(2.0) * axz, G_prp, ayy * G_ptt);
    const V h = V(0.5) * irho;
    ux = fmav(h, Mr, ux0);
    uy = fmav(h, Mt, uy0);
    uz = fmav(h, Mp, uz0);
  }
  Moments<V> ms = m;
  ms.jx = rho * ux;
  ms.jy = rho * uy;
  ms.jz = rho * uz;
  Coef<V> k = coefficients<V, K>(ms, g, ip.kappa, ip.G);
  const V s = fmav(V(-0.5), ip.omega, V(1.0));  // 1 - 1/(2 tau)
  k.fA = k.fA * s;
  k.nfB = k.nfB * s;
  k.t0 = k.t0 * s;
  k.naxx = k.naxx * s;
  k.nayy = k.nayy * s;
  k.nazz = k.nazz * s;
  k.naxy = k.naxy * s;
  k.naxz = k.naxz * s;
  k.nayz = k.nayz * s;
  return k;
}

// One node: pull streaming + walls, then the collision of its instance's
// variant (the same wall-node rule and store as the literal step).
template <typename S, typename Real, int K>
__global__ void __launch_bounds__(KBounds<S, Real, K>::maxt, KBounds<S, Real, K>::minb)
    k_step_shift(const S* __restrict__ fin, S* __restrict__ fout, GeoDev<Real> geo,
                 const InstParams<Real>* __restrict__ inst, Dims d, int* __restrict__ flag) {
  const uint32_t cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= uint32_t(d.ncell)) return;
  const int b = int(blockIdx.y);
  const CellPos p = locate_cell(d, b, cell);
  const size_t base = size_t(b) * Q * uint32_t(d.ncell);
  const float* ref = ref_of(d, b);
  const InstParams<Real>& ip = inst[b];
  Real f[Q];
  gather<K, S, Real, 2>(fin + base, ref, p, d, f);
  const Moments<Real> m = moments(f);
  if (!finite_v(m.rho)) {
    if (*flag == 0) atomicExch(flag, 1);
  }
  const int row = geo_row_node<K>(d, p.ir, p.it, p.i3);
  const NodeGeo<Real, K> g = load_geo<Real, K>(geo, row);
  if (d.wall_eq && (p.ir == 0 || p.ir == d.nr - 1 || (!d.periodic3 && (p.i3 == 0 || p.i3 == d.n3 - 1)))) {
    equilibrium<Real, K>(m.rho, Real(0.0), Real(0.0), Real(0.0), g, f);
    store_node<K>(fout + base, ref, p, d, f);
    return;
  }
  const Coef<Real> k = ip.pad != Real(0) ? shifted_coefficients<Real, K>(m, g, ip)
                                         : coefficients<Real, K>(m, g, ip.kappa, ip.G);
  collide<Real, K>(f, k, g, ip.omega);
  store_node<K>(fout + base, ref, p, d, f);
}

template <class S, class R>
cudaError_t launch_shift_t(int K, const S* fin, S* fout, const GeoDev<R>& geo, const InstParams<R>* inst,
                           const Dims& d, int* flag, int threads, cudaStream_t s) {
  if (d.batch < 1 || d.batch > 65535) return cudaErrorInvalidValue;
  threads = threads < StepBounds<S, R>::maxt ? threads : StepBounds<S, R>::maxt;
  const dim3 blocks((uint32_t(d.ncell) + threads - 1) / threads, uint32_t(d.batch));
  switch (K) {
    case KFLAT: k_step_shift<S, R, KFLAT><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    case KCYL: k_step_shift<S, R, KCYL><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    case KELL: k_step_shift<S, R, KELL><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_shift_f64(int K, const double* fin, double* fout, const GeoDev<double>& geo,
                                  const InstParams<double>* inst, const Dims& d, int* flag, int threads,
                                  cudaStream_t s) {
  return launch_shift_t<double, double>(K, fin, fout, geo, inst, d, flag, threads, s);
}

cudaError_t launch_step_shift_f32(int K, const float* fin, float* fout, const GeoDev<float>& geo,
                                  const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                                  cudaStream_t s) {
  return launch_shift_t<float, float>(K, fin, fout, geo, inst, d, flag, threads, s);
}

}  // namespace lbgm
