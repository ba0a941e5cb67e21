// Kernels of the lattice Boltzmann path. One thread per lattice node; nodes
// are numbered with x3 fastest so that a warp shares (instance, i_r, i_theta)
// and the wall branch along r is warp-uniform.
#pragma once

#include "lbm_device.cuh"

namespace lbgm {

// Fused time step (Eq. LB) of one node p of one instance whose state blocks
// start at fin and fout: pull streaming + walls, moments, equilibrium,
// non-equilibrium stress, forcing, BGK, store. flag is set to 1 when the
// node's density is not finite.
template <typename S, typename Real, int K>
__device__ __forceinline__ void step_node(const S* __restrict__ fin, S* __restrict__ fout,
                                          const GeoDev<Real>& geo, const InstParams<Real>& ip, const Dims& d,
                                          const CellPos& p, int* __restrict__ flag) {
  Real f[Q];
  gather(fin, p, d, f);
  const Moments<Real> m = moments(f);
  if (!finite_v(m.rho)) {  // NaN or Inf
    if (*flag == 0) atomicExch(flag, 1);
  }
  const int row = K == KELL ? p.ir * d.geo_rows3 + p.i3 : p.ir;
  const NodeGeo<Real, K> g = load_geo<Real, K>(geo, row);
  const Coef<Real> k = coefficients<Real, K>(m, g, ip.kappa, ip.G);
  collide<Real, K>(f, k, g, ip.omega);
  store_node(fout + p.cell, d.ncell, f);
}

// Uniform batch: fin/fout are whole states (batch blocks of Q * ncell).
template <typename S, typename Real, int K>
__global__ void __launch_bounds__(256) k_step(const S* __restrict__ fin, S* __restrict__ fout,
                                              GeoDev<Real> geo, const InstParams<Real>* __restrict__ inst,
                                              Dims d, int* __restrict__ flag) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= uint32_t(d.batch) * uint32_t(d.ncell)) return;
  const CellPos p = locate(d, t);
  const size_t base = size_t(p.b) * Q * d.ncell;
  step_node<S, Real, K>(fin + base, fout + base, geo, inst[p.b], d, p, flag);
}

// One instance of a batch whose instances differ in geometry and size: its
// dimensions (batch 1), geometry tables, parameters, two state blocks and
// the flag that records a non-finite density.
template <typename S, typename Real>
struct ListInst {
  Dims d;
  GeoDev<Real> geo;
  const InstParams<Real>* ip;
  const S* f0;
  S* f1;
  int* flag;
};

// Work-list step over instances of one metric kind. Work item j updates the
// nodes [work[j].y, work[j].y + blockDim.x) of instance work[j].x; blocks
// take items j = blockIdx.x, blockIdx.x + gridDim.x, ... (a persistent grid
// when gridDim.x < nwork). `parity` 0 reads f0 and writes f1, 1 the reverse.
// The instance record is staged once per item in shared memory.
template <typename S, typename Real, int K>
__global__ void __launch_bounds__(256) k_step_list(const ListInst<S, Real>* __restrict__ insts,
                                                   const int2* __restrict__ work, int nwork, int parity) {
  constexpr int kWords = sizeof(ListInst<S, Real>) / 4;
  static_assert(sizeof(ListInst<S, Real>) % 4 == 0, "record must be whole words");
  static_assert(kWords <= 64, "the smallest block (64 threads) copies the record");
  __shared__ union {
    ListInst<S, Real> rec;
    uint32_t w[kWords];
  } sh;
  for (int j = blockIdx.x; j < nwork; j += gridDim.x) {
    const int2 w = work[j];
    __syncthreads();  // the previous item's readers are done
    if (threadIdx.x < kWords)
      sh.w[threadIdx.x] = reinterpret_cast<const uint32_t*>(insts + w.x)[threadIdx.x];
    __syncthreads();
    const ListInst<S, Real>& I = sh.rec;
    const uint32_t t = uint32_t(w.y) + threadIdx.x;
    if (t < uint32_t(I.d.ncell)) {
      const Dims d = I.d;
      const CellPos p = locate(d, t);
      const S* fin = parity ? I.f1 : I.f0;
      S* fout = const_cast<S*>(parity ? I.f0 : I.f1);
      step_node<S, Real, K>(fin, fout, I.geo, *I.ip, d, p, I.flag);
    }
  }
}

// rho' and u of the streamed populations (moments only).
template <typename S, typename Real, int K>
__global__ void __launch_bounds__(256) k_macros(const S* __restrict__ fin, double* __restrict__ rho,
                                                double* __restrict__ u, Dims d) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= uint32_t(d.batch) * uint32_t(d.ncell)) return;
  const CellPos p = locate(d, t);
  Real f[Q];
  gather(fin + size_t(p.b) * Q * d.ncell, p, d, f);
  const Moments<Real> m = moments(f);
  const double r = double(m.rho);
  if (rho) rho[t] = r;
  if (u) {
    const size_t ub = size_t(p.b) * 3 * d.ncell + p.cell;
    u[ub] = double(m.jx / m.rho);
    u[ub + d.ncell] = double(m.jy / m.rho);
    u[ub + 2 * size_t(d.ncell)] = double(m.jz / m.rho);
  }
}

// SplitMix64: output number k (from 0) of the generator seeded with `seed`.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct InitInst {
  unsigned long long seed;
  double amp;
};

// Initial state f = f^eq(rho', u): either from caller fields (rho_in, u_in
// non-NULL) or rho' = 1/sqrt(g), u = base(b, i_r) + noise.
template <typename S, typename Real, int K>
__global__ void __launch_bounds__(256) k_init(S* __restrict__ f, GeoDev<Real> geo,
                                              const double* __restrict__ sqrtg,
                                              const double* __restrict__ base_uth,
                                              const InitInst* __restrict__ ini,
                                              const double* __restrict__ rho_in,
                                              const double* __restrict__ u_in, Dims d) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= uint32_t(d.batch) * uint32_t(d.ncell)) return;
  const CellPos p = locate(d, t);
  double rho, u[3];
  if (rho_in) {
    rho = rho_in[t];
    const size_t ub = size_t(p.b) * 3 * d.ncell + p.cell;
    u[0] = u_in[ub];
    u[1] = u_in[ub + d.ncell];
    u[2] = u_in[ub + 2 * size_t(d.ncell)];
  } else {
    rho = 1.0 / sqrtg[p.ir * d.n3 + p.i3];
    u[0] = 0.0;
    u[1] = base_uth ? base_uth[size_t(p.b) * d.nr + p.ir] : 0.0;
    u[2] = 0.0;
    const InitInst in = ini[p.b];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const uint64_t s = splitmix64_at(in.seed, 3ull * uint64_t(p.cell) + uint64_t(i));
      const double U = double(s >> 11) * 0x1.0p-53;
      u[i] += in.amp * (2.0 * U - 1.0);
    }
  }
  const int row = K == KELL ? p.ir * d.geo_rows3 + p.i3 : p.ir;
  const NodeGeo<Real, K> g = load_geo<Real, K>(geo, row);
  Real fe[Q];
  equilibrium<Real, K>(Real(rho), Real(u[0]), Real(u[1]), Real(u[2]), g, fe);
  store_node(f + size_t(p.b) * Q * d.ncell + p.cell, d.ncell, fe);
}

}  // namespace lbgm
