// Kernels of the lattice Boltzmann path. One thread per lattice node; nodes
// are numbered with x3 fastest so that a warp shares (instance, i_r, i_theta)
// and the wall branch along r is warp-uniform.
#pragma once

#include "lbm_device.cuh"

namespace lbgm {

// Collision half of the fused step (Eq. LB) for node p whose streamed
// populations are in f: moments, equilibrium, non-equilibrium stress,
// forcing, BGK, store into the instance block fout. flag is set to 1 when
// the node's density is not finite.
// Nodes on an equilibrium wall (the end nodes of the walled axes) leave the
// step as f^eq(rho', 0) of their own density and metric (Sec. III).
//
// 2-byte storage (Codec uses_ref): f holds the stored deviations g of the
// streamed populations (gather with RAW), and the collision runs on them
// through the stream table of the node's row: moments from the table's
// reference moments plus the weighted deviations, post-collision
// deviations from collide_dev. Only equilibrium-wall nodes, which store
// f^eq, encode against the reference table.
// With `staged` (2-byte storage) the node's stream-table row is already in
// shared memory (stage_table; the caller has waited for it), else it is
// read from global memory.
template <typename S, typename Real, int K>
__device__ __forceinline__ void collide_store(Real (&f)[Q], S* __restrict__ fout, const float* ref,
                                              const GeoDev<Real>& geo, const InstParams<Real>& ip, const Dims& d,
                                              const CellPos& p, int* __restrict__ flag,
                                              const TabStaged* staged = nullptr) {
  if constexpr (Codec<S, Real>::uses_ref) {
    const uint32_t stride = uint32_t(d.nr) * uint32_t(d.st_rows3);
    const float4* st = stream_of(d, p.b) + stream_row<K>(d, p.ir, p.i3);
    const float4 ta = staged ? staged->at(0) : __ldg(st);
    const float4 tb = staged ? staged->at(1) : __ldg(st + stride);
    const float4 tc = staged ? staged->at(2) : __ldg(st + 2 * stride);
    const Moments<float> m = moments_dev(f, ta, tb, tc);
    if (!finite_v(m.rho)) {
      if (*flag == 0) atomicExch(flag, 1);
    }
    const int row = geo_row_node<K>(d, p.ir, p.it, p.i3);
    const NodeGeo<float, K> g = load_geo<float, K>(geo, row);
    if (d.wall_eq && (p.ir == 0 || p.ir == d.nr - 1 || (!d.periodic3 && (p.i3 == 0 || p.i3 == d.n3 - 1)))) {
      equilibrium<float, K>(m.rho, 0.0f, 0.0f, 0.0f, g, f);
      store_node<K>(fout, ref, p, d, f);
      return;
    }
    const Coef<float> k = coefficients<float, K>(m, g, ip.kappa, ip.G);
    if (staged)
      collide_dev<K>(f, k, g, ip.omega, *staged, tc.z);
    else
      collide_dev<K>(f, k, g, ip.omega, TabGlobal{st, stride}, tc.z);
    store_raw<S>(fout, p, d, f);
    return;
  }
  const Moments<Real> m = moments(f);
  if (!finite_v(m.rho)) {  // NaN or Inf
    if (*flag == 0) atomicExch(flag, 1);
  }
  const int row = geo_row_node<K>(d, p.ir, p.it, p.i3);
  const NodeGeo<Real, K> g = load_geo<Real, K>(geo, row);
  if (d.wall_eq && (p.ir == 0 || p.ir == d.nr - 1 || (!d.periodic3 && (p.i3 == 0 || p.i3 == d.n3 - 1)))) {
    equilibrium<Real, K>(m.rho, Real(0.0), Real(0.0), Real(0.0), g, f);
    store_node<K>(fout, ref, p, d, f);
    return;
  }
  const Coef<Real> k = coefficients<Real, K>(m, g, ip.kappa, ip.G);
  collide<Real, K>(f, k, g, ip.omega);
  store_node<K>(fout, ref, p, d, f);
}

// Fused time step of one node p of one instance whose state blocks start at
// fin and fout (reference table ref): pull streaming + walls, then
// collide_store.
// 2-byte storage of the ellipsoid, whose stream rows are (i_r, i_3) -- one
// per node: the node's stream-table row is staged into shared memory before
// the gather (stage_table), so its latency runs under the gather's and no
// register holds it meanwhile (the four-wall 24 x 64x4x256 ellipsoid in
// FP16 storage 9.0 -> 10.3 GLUPS with 5 blocks per SM). Where a block's
// nodes share one row (flat, cylinder) the table reads are broadcasts from
// L1 and staging measured slower (128 mixed channels 12.1 -> 10.6).
#ifndef LBGM_STAGE_TABLE
#define LBGM_STAGE_TABLE 1
#endif
template <typename S, typename Real, int K, int WALLS = 2>
__device__ __forceinline__ void step_node(const S* __restrict__ fin, S* __restrict__ fout, const float* ref,
                                          const GeoDev<Real>& geo, const InstParams<Real>& ip, const Dims& d,
                                          const CellPos& p, int* __restrict__ flag) {
  Real f[Q];
  if constexpr (Codec<S, Real>::uses_ref && K == KELL && LBGM_STAGE_TABLE) {
    __shared__ float4 s_tab[ST_K * 128];  // the 2-byte kernels' blocks hold at most 128 threads
    const TabStaged tab{s_tab + threadIdx.x, int(blockDim.x)};
    stage_table(s_tab + threadIdx.x, int(blockDim.x), stream_of(d, p.b) + stream_row<K>(d, p.ir, p.i3),
                uint32_t(d.nr) * uint32_t(d.st_rows3));
    gather<K, S, Real, WALLS, true>(fin, ref, p, d, f);
    stage_wait();
    collide_store<S, Real, K>(f, fout, ref, geo, ip, d, p, flag, &tab);
  } else {
    gather<K, S, Real, WALLS, Codec<S, Real>::uses_ref>(fin, ref, p, d, f);
    collide_store<S, Real, K>(f, fout, ref, geo, ip, d, p, flag);
  }
}

// Launch bounds of k_step per storage / compute type. FP32 arithmetic: at
// most 128 threads per block and 6 (FP32 storage) or 4 (2-byte storage,
// whose stream-table reads and conversions need registers) resident blocks
// per SM, i.e. a register cap that trades a few spilled values for more
// resident warps (the FP32 kernel is bound by latency and issue as much as
// by HBM; measured best of 5..8; the 2-byte kernels measured 4 > 5 > 6).
// FP64 keeps its registers (bound by the FP64 units). LBGM_STEP32_MAXT /
// LBGM_STEP32_MINB / LBGM_STEP16_MINB override the FP32 values for tuning
// builds.
#ifndef LBGM_STEP32_MAXT
#define LBGM_STEP32_MAXT 128
#endif
#ifndef LBGM_STEP32_MINB
#define LBGM_STEP32_MINB 6
#endif
#ifndef LBGM_STEP16_MINB
#define LBGM_STEP16_MINB 4
#endif
template <class S, class Real>
struct StepBounds {
  static constexpr int maxt = LBGM_STEP32_MAXT;
  static constexpr int minb = sizeof(S) == 2 ? LBGM_STEP16_MINB : LBGM_STEP32_MINB;
};
// step_node's staged stream-table rows hold 128 threads' worth
static_assert(StepBounds<__half, float>::maxt <= 128 && StepBounds<__nv_bfloat16, float>::maxt <= 128,
              "2-byte blocks of at most 128 threads");
template <>
struct StepBounds<double, double> {
  static constexpr int maxt = 256, minb = 1;
};
// Per metric kind: one block fewer per SM for the ellipsoid with FP32
// storage, whose (i_r, i_3) geometry rows and extra Christoffel terms need
// more registers; one more for the ellipsoid with 2-byte storage, whose
// staged stream-table rows free the registers of the table prefetch
// (LBGM_STEP16_KELL_MINB; measured 5 > 4).
#ifndef LBGM_STEP16_KELL_MINB
#define LBGM_STEP16_KELL_MINB 5
#endif
template <class S, class Real, int K>
struct KBounds {
  static constexpr int maxt = StepBounds<S, Real>::maxt;
  static constexpr int minb = sizeof(S) == 2 && K == KELL ? LBGM_STEP16_KELL_MINB
                              : (K == KELL || K == KELT) && sizeof(S) != 2 && StepBounds<S, Real>::minb > 1
                                  ? StepBounds<S, Real>::minb - 1
                                  : StepBounds<S, Real>::minb;
};
// Uniform batch: fin/fout are whole states (batch blocks of Q * ncell);
// block (x, y) updates nodes [x blockDim, (x + 1) blockDim) of instance y, so
// the instance's block base is uniform across the thread block.
template <typename S, typename Real, int K>
__global__ void __launch_bounds__(KBounds<S, Real, K>::maxt, KBounds<S, Real, K>::minb)
    k_step(const S* __restrict__ fin, S* __restrict__ fout, GeoDev<Real> geo,
           const InstParams<Real>* __restrict__ inst, Dims d, int* __restrict__ flag) {
  const uint32_t cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= uint32_t(d.ncell)) return;
  const int b = int(blockIdx.y);
  const CellPos p = locate_cell(d, b, cell);
  const size_t base = size_t(b) * Q * uint32_t(d.ncell);
  step_node<S, Real, K>(fin + base, fout + base, ref_of(d, b), geo, inst[b], d, p, flag);
}

// The same update split by region for channels periodic in x3, where only
// the three node layers next to each r-wall need the wall rule: k_step_bulk
// covers the contiguous interior layers 3 .. nr - 4 with the far-from-wall
// gather alone, k_step_edge the 6 wall layers with the per-layer constant
// folds (gather_edge), so neither kernel carries the other's code.
template <typename S, typename Real, int K>
__global__ void __launch_bounds__(KBounds<S, Real, K>::maxt, KBounds<S, Real, K>::minb)
    k_step_bulk(const S* __restrict__ fin, S* __restrict__ fout, GeoDev<Real> geo,
                const InstParams<Real>* __restrict__ inst, Dims d, int* __restrict__ flag) {
  const uint32_t layer = uint32_t(d.nt) * uint32_t(d.n3);
  const uint32_t cell = 3u * layer + blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= uint32_t(d.nr - 3) * layer) return;
  const int b = int(blockIdx.y);
  const CellPos p = locate_cell(d, b, cell);
  const size_t base = size_t(b) * Q * uint32_t(d.ncell);
  step_node<S, Real, K, 0>(fin + base, fout + base, ref_of(d, b), geo, inst[b], d, p, flag);
}

// 2-byte storage for metrics whose geometry and stream rows are i_r alone
// (flat, cylinder), with blocks that never straddle an i_r layer (nt n3 a
// multiple of blockDim.x): the block's nodes share one geometry row, one
// stream-table row and one instance, which three threads copy into shared
// memory while the gather's loads are in flight; the collision then reads
// them from shared memory instead of waiting on dependent global loads
// inside the arithmetic (long-scoreboard stalls per issue 2.6 -> 1.7 on the
// 24 x 64x4x256 cylinder sweep, 15.4 -> 16.8 GLUPS at equal occupancy). Same
// arithmetic as collide_store: bitwise-equal states. The gather fills f (stored deviations) for node p; live is false
// for the threads past the end of the range, which only take part in the
// block barrier.
template <typename S, int K, class Gather>
__device__ __forceinline__ void step_row_shared(S* __restrict__ fout, GeoDev<float> geo,
                                                const InstParams<float>* __restrict__ inst, const Dims& d,
                                                const CellPos& p, bool live, int* __restrict__ flag,
                                                Gather&& gather_into) {
  static_assert(Codec<S, float>::uses_ref && K != KELL, "2-byte storage, rows of i_r alone");
  __shared__ float4 s_tab[ST_K];
  __shared__ __align__(16) unsigned char s_geo_raw[sizeof(NodeGeo<float, K>)];
  __shared__ InstParams<float> s_ip;
  auto& s_geo = *reinterpret_cast<NodeGeo<float, K>*>(s_geo_raw);
  const uint32_t stride = uint32_t(d.nr) * uint32_t(d.st_rows3);
  float4 tv;
  if (threadIdx.x < ST_K) tv = __ldg(stream_of(d, p.b) + p.ir + threadIdx.x * stride);
  float f[Q];
  gather_into(f);
  if (threadIdx.x < ST_K) s_tab[threadIdx.x] = tv;
  if (threadIdx.x == 32) s_geo = load_geo<float, K>(geo, p.ir);
  if (threadIdx.x == 33) s_ip = inst[p.b];
  __syncthreads();
  if (!live) return;
  const Moments<float> m = moments_dev(f, s_tab[0], s_tab[1], s_tab[2]);
  if (!finite_v(m.rho)) {
    if (*flag == 0) atomicExch(flag, 1);
  }
  const NodeGeo<float, K> g = s_geo;
  const InstParams<float> ip = s_ip;
  const Coef<float> k = coefficients<float, K>(m, g, ip.kappa, ip.G);
  collide_dev<K>(f, k, g, ip.omega, TabShared{s_tab}, s_tab[2].z);
  store_raw<S>(fout, p, d, f);
}

// Interior kernel of the region split with step_row_shared: 6 resident
// blocks per SM (80 registers, 28 bytes spilled for the cylinder; the row
// in shared memory frees the registers the stream-table prefetch held).
// Measured on the 24 x 64x4x256 cylinder sweep, FP16 storage, with the
// wall-layer kernel at 5: 19.0 GLUPS; at 5 / 4 / 3 blocks 18.8 / 16.9 /
// 14.9. LBGM_ROWSM_MINB overrides it for tuning builds.
#ifndef LBGM_ROWSM_MINB
#define LBGM_ROWSM_MINB 6
#endif
template <typename S, int K>
__global__ void __launch_bounds__(KBounds<S, float, K>::maxt, LBGM_ROWSM_MINB)
    k_step_bulk_rowsm(const S* __restrict__ fin, S* __restrict__ fout, GeoDev<float> geo,
                      const InstParams<float>* __restrict__ inst, Dims d, int* __restrict__ flag) {
  const uint32_t layer = uint32_t(d.nt) * uint32_t(d.n3);
  const uint32_t cell0 = 3u * layer + blockIdx.x * blockDim.x;
  const uint32_t cell = cell0 + threadIdx.x;
  const bool live = cell < uint32_t(d.nr - 3) * layer;
  const int b = int(blockIdx.y);
  const CellPos p = locate_cell(d, b, live ? cell : cell0);
  const size_t base = size_t(b) * Q * uint32_t(d.ncell);
  step_row_shared<S, K>(fout + base, geo, inst, d, p, live, flag,
                        [&](float (&f)[Q]) { gather<K, S, float, 0, true>(fin + base, nullptr, p, d, f); });
}

// Wall-layer kernel of the region split with step_row_shared: 5 resident
// blocks per SM (96 registers; +0.5 % on the step against 4).
// LBGM_EDGE_ROWSM_MINB overrides it for tuning builds.
#ifndef LBGM_EDGE_ROWSM_MINB
#define LBGM_EDGE_ROWSM_MINB 5
#endif
template <typename S, int K>
__global__ void __launch_bounds__(KBounds<S, float, K>::maxt, LBGM_EDGE_ROWSM_MINB)
    k_step_edge_rowsm(const S* __restrict__ fin, S* __restrict__ fout, GeoDev<float> geo,
                      const InstParams<float>* __restrict__ inst, Dims d, int* __restrict__ flag) {
  const uint32_t layer = uint32_t(d.nt) * uint32_t(d.n3);
  const uint32_t e0 = blockIdx.x * blockDim.x;
  const uint32_t e = e0 + threadIdx.x;
  const bool live = e < 6u * layer;
  const uint32_t ee = live ? e : e0;
  const uint32_t cell = ee < 3u * layer ? ee : ee + uint32_t(d.nr - 6) * layer;
  const int b = int(blockIdx.y);
  const CellPos p = locate_cell(d, b, cell);
  const size_t base = size_t(b) * Q * uint32_t(d.ncell);
  step_row_shared<S, K>(fout + base, geo, inst, d, p, live, flag,
                        [&](float (&f)[Q]) { gather_edge<K, S, float, true>(fin + base, nullptr, p, d, f); });
}

// Wall-layer kernel: 4 resident blocks per SM whatever the storage (no
// spills with the six fold variants' address arithmetic; it runs beside the
// interior kernel, which keeps the SMs' other slots; measured +1 % on the
// whole FP32 step against the interior kernel's cap).
template <typename S, typename Real, int K>
__global__ void __launch_bounds__(KBounds<S, Real, K>::maxt, KBounds<S, Real, K>::minb < 4 ? KBounds<S, Real, K>::minb : 4)
    k_step_edge(const S* __restrict__ fin, S* __restrict__ fout, GeoDev<Real> geo,
                const InstParams<Real>* __restrict__ inst, Dims d, int* __restrict__ flag) {
  const uint32_t layer = uint32_t(d.nt) * uint32_t(d.n3);
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 6u * layer) return;
  const uint32_t cell = e < 3u * layer ? e : e + uint32_t(d.nr - 6) * layer;
  const int b = int(blockIdx.y);
  const CellPos p = locate_cell(d, b, cell);
  const size_t base = size_t(b) * Q * uint32_t(d.ncell);
  const float* ref = ref_of(d, b);
  Real f[Q];
  gather_edge<K, S, Real, Codec<S, Real>::uses_ref>(fin + base, ref, p, d, f);
  collide_store<S, Real, K>(f, fout + base, ref, geo, inst[b], d, p, flag);
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

// Work-list step over instances of one metric kind. Work item j = (instance,
// first, count) covers `count` nodes of one instance: at most blockDim.x,
// one per thread, or with MULTI a tile of several blocks' worth (thread t
// takes nodes t, t + blockDim.x, ...; a separate instantiation, because the
// loop costs the one-block tiles ~5 % on the four-wall ellipsoid): with
// WALLS = 0 the interior nodes first .. first + count - 1 (no wall within 3
// nodes: the far-from-wall gather alone); otherwise the wall nodes
// cells[first .. first + count - 1] of one class, each in its own
// instantiation -- WALLS = 3: within 3 layers of an r-wall only (the r
// folds), 4: of an x3-wall only (the x3 folds), 1: the rest (corners,
// equilibrium walls, short axes: the general wall rule). Splitting them
// keeps each kernel's code small (instruction fetch is what binds a kernel
// carrying every wall variant).
// Blocks take items j = blockIdx.x, blockIdx.x + gridDim.x, ... (a
// persistent grid when gridDim.x < nwork). `parity` 0 reads f0 and writes f1,
// 1 the reverse. The instance record is staged once per item in shared
// memory.
template <typename S, typename Real, int K, int WALLS, bool MULTI>
__global__ void __launch_bounds__(KBounds<S, Real, K>::maxt, KBounds<S, Real, K>::minb)
    k_step_list(const ListInst<S, Real>* __restrict__ insts, const int4* __restrict__ work, int nwork,
                const int* __restrict__ cells, int parity) {
  constexpr int kWords = sizeof(ListInst<S, Real>) / 4;
  static_assert(sizeof(ListInst<S, Real>) % 4 == 0, "record must be whole words");
  static_assert(kWords <= 64, "the smallest block (64 threads) copies the record");
  static_assert(KBounds<S, Real, K>::maxt >= 64, "blocks of 64 threads must be allowed");
  __shared__ union {
    ListInst<S, Real> rec;
    uint32_t w[kWords];
  } sh;
  for (int j = blockIdx.x; j < nwork; j += gridDim.x) {
    const int4 w = work[j];
    __syncthreads();  // the previous item's readers are done
    if (threadIdx.x < kWords)
      sh.w[threadIdx.x] = reinterpret_cast<const uint32_t*>(insts + w.x)[threadIdx.x];
    __syncthreads();
    const ListInst<S, Real>& I = sh.rec;
    auto node = [&](int i) {
      const uint32_t t = WALLS == 0 ? uint32_t(w.y + i) : uint32_t(cells[w.y + i]);
      const Dims d = I.d;
      const CellPos p = locate(d, t);
      const S* fin = parity ? I.f1 : I.f0;
      S* fout = const_cast<S*>(parity ? I.f0 : I.f1);
      step_node<S, Real, K, WALLS>(fin, fout, d.ref, I.geo, *I.ip, d, p, I.flag);
    };
    if constexpr (MULTI) {
      for (int i = int(threadIdx.x); i < w.z; i += int(blockDim.x)) node(i);
    } else {
      if (int(threadIdx.x) < w.z) node(int(threadIdx.x));
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
  gather<K>(fin + size_t(p.b) * Q * d.ncell, ref_of(d, p.b), p, d, f);
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
    rho = 1.0 / sqrtg[d.geo_theta ? p.cell : p.ir * d.n3 + p.i3];
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
  const int row = geo_row_node<K>(d, p.ir, p.it, p.i3);
  const NodeGeo<Real, K> g = load_geo<Real, K>(geo, row);
  Real fe[Q];
  equilibrium<Real, K>(Real(rho), Real(u[0]), Real(u[1]), Real(u[2]), g, fe);
  store_node<K>(f + size_t(p.b) * Q * d.ncell, ref_of(d, p.b), p, d, fe);
}

// Reference populations of 2-byte storage (Codec): for instance b and
// geometry row r, mode 0: r_l = w_l (the rest state of unit density);
// mode 1: the equilibrium f^eq(rho', u) of the row's initial state: with
// caller fields (rho_in, u_in non-NULL) their mean over the row's nodes,
// else rho' = 1/sqrt(g) and u = (0, base(b, i_r), 0) (rest where base is
// NULL). Written at ref_index<K> of instance b's table.
template <int K>
__global__ void __launch_bounds__(256) k_ref_table(float* __restrict__ ref, GeoDev<float> geo,
                                                   const double* __restrict__ sqrtg,
                                                   const double* __restrict__ base_uth,
                                                   const double* __restrict__ rho_in,
                                                   const double* __restrict__ u_in, Dims d, int mode) {
  const uint32_t nrows = uint32_t(d.nr) * uint32_t(d.geo_rows3);
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= uint32_t(d.batch) * nrows) return;
  const uint32_t b = t / nrows, row = t - b * nrows;
  const int ir = int(row) / d.geo_rows3, i3 = int(row) - ir * d.geo_rows3;
  float fe[Q];
  if (mode == 0) {
    static_for<0, Q>([&](auto L_) {
      constexpr int L = decltype(L_)::value;
      fe[L] = float(WeightOf<L>::w);
    });
  } else if (rho_in) {
    // mean over the row's nodes: all (i_theta, i_3) of layer i_r, or all
    // i_theta of (i_r, i_3) for the ellipsoid's rows
    double rs = 0.0, us[3] = {0.0, 0.0, 0.0};
    const int n3s = d.geo_rows3 > 1 ? 1 : d.n3;
    int cnt = 0;
    for (int it = 0; it < d.nt; ++it)
      for (int k3 = 0; k3 < n3s; ++k3) {
        const size_t cell = (size_t(ir) * d.nt + it) * d.n3 + (d.geo_rows3 > 1 ? i3 : k3);
        rs += rho_in[size_t(b) * d.ncell + cell];
        const size_t ub = size_t(b) * 3 * d.ncell + cell;
        us[0] += u_in[ub];
        us[1] += u_in[ub + d.ncell];
        us[2] += u_in[ub + 2 * size_t(d.ncell)];
        ++cnt;
      }
    const NodeGeo<float, K> g = load_geo<float, K>(geo, int(row));
    equilibrium<float, K>(float(rs / cnt), float(us[0] / cnt), float(us[1] / cnt), float(us[2] / cnt), g, fe);
  } else {
    const double rho = 1.0 / sqrtg[ir * d.n3 + i3];
    const double uth = base_uth ? base_uth[size_t(b) * d.nr + ir] : 0.0;
    const NodeGeo<float, K> g = load_geo<float, K>(geo, int(row));
    equilibrium<float, K>(float(rho), 0.0f, float(uth), 0.0f, g, fe);
  }
  float* rb = ref + size_t(b) * Q * nrows;
#pragma unroll
  for (int l = 0; l < Q; ++l) rb[ref_index<K>(d, l, int(row))] = fe[l];
}

// Stream table of 2-byte storage (stream_of): one thread per instance and
// stream row. The sources of a representative node of the row (theta = 0;
// i_3 the row's own, or any inside / the class's layer for walls on x3) give,
// for every population l, the stored population index and geometry row whose
// reference rho_l it receives -- from the same source functions as the step
// (for_each_source; the compile-time edge folds select the same sources).
// fin is any state block of the context: its addresses are formed, never read.
template <int K, class S>
__global__ void __launch_bounds__(128) k_stream_table(float4* __restrict__ st, const float* __restrict__ ref,
                                                      const InstParams<float>* __restrict__ inst, const S* fin,
                                                      Dims d) {
  const uint32_t nrows = uint32_t(d.nr) * uint32_t(d.st_rows3);
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= uint32_t(d.batch) * nrows) return;
  const int b = int(t / nrows), srow = int(t - uint32_t(b) * nrows);
  CellPos p;
  p.b = b;
  p.it = 0;
  if constexpr (K == KELL) {
    p.ir = srow / d.geo_rows3;
    p.i3 = srow - p.ir * d.geo_rows3;
  } else if (d.st_rows3 == 1) {
    p.ir = srow;
    p.i3 = 0;
  } else {
    p.ir = srow / 7;
    const int c = srow - p.ir * 7;
    p.i3 = c < 3 ? c : (c == 3 ? 3 : d.n3 - 7 + c);
  }
  p.cell = (p.ir * d.nt + p.it) * d.n3 + p.i3;
  const float* rb = ref + size_t(b) * Q * size_t(d.nr) * size_t(d.geo_rows3);
  double rho_l[Q];
  for_each_source<K, S>(fin, p, d, [&](auto L_, const S*, int sl, int row) {
    constexpr int L = decltype(L_)::value;
    rho_l[L] = double(rb[ref_index<K>(d, sl, row)]);
  });
  const float om1 = 1.0f - inst[b].omega;  // as the step computes it
  const int own = geo_row<K>(d, p.ir, p.i3);
  double tl[Q];
  double m[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  static_for<0, Q>([&](auto L_) {
    constexpr int L = decltype(L_)::value;
    constexpr int cx = L == 0 ? 0 : ((L - 1) % 2 == 0 ? 1 : -1) * PAIRS[L == 0 ? 0 : (L - 1) / 2].x;
    constexpr int cy = L == 0 ? 0 : ((L - 1) % 2 == 0 ? 1 : -1) * PAIRS[L == 0 ? 0 : (L - 1) / 2].y;
    constexpr int cz = L == 0 ? 0 : ((L - 1) % 2 == 0 ? 1 : -1) * PAIRS[L == 0 ? 0 : (L - 1) / 2].z;
    const double r = rho_l[L];
    m[0] += r;
    m[1] += cx * r;
    m[2] += cy * r;
    m[3] += cz * r;
    m[4] += cx * cx * r;
    m[5] += cy * cy * r;
    m[6] += cz * cz * r;
    m[7] += cx * cy * r;
    m[8] += cx * cz * r;
    m[9] += cy * cz * r;
    tl[L] = (double(om1) * r - double(rb[ref_index<K>(d, L, own)])) / WeightOf<L>::w;
  });
  float4* out = st + size_t(b) * ST_K * nrows + uint32_t(srow);
  out[0] = make_float4(float(m[0]), float(m[1]), float(m[2]), float(m[3]));
  out[nrows] = make_float4(float(m[4]), float(m[5]), float(m[6]), float(m[7]));
  out[2 * nrows] = make_float4(float(m[8]), float(m[9]), float(tl[0]), 0.0f);
#pragma unroll
  for (int j = 0; j < NPAIR / 2; ++j) {
    const double tp0 = tl[4 * j + 1], tm0 = tl[4 * j + 2], tp1 = tl[4 * j + 3], tm1 = tl[4 * j + 4];
    out[(3 + j) * nrows] = make_float4(float(0.5 * (tp0 + tm0)), float(0.5 * (tp0 - tm0)),
                                       float(0.5 * (tp1 + tm1)), float(0.5 * (tp1 - tm1)));
  }
}

}  // namespace lbgm
