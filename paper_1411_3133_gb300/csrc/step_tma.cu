// Fused time step, FP32, with the pull gather staged through shared memory by
// TMA (cp.async.bulk.tensor) in a two-stage mbarrier pipeline.
//
// A tile is one (instance, i_r, i_theta) row of NX = n3 nodes. For every
// population l the tile needs one row of the previous state: the row
// (i_r - c_r, i_theta - c_theta) of population l, all x3 -- the x3 shift and
// its periodic wrap are applied when reading shared memory, so every TMA box
// starts at x3 = 0 (16-byte aligned) and no halo is needed. One thread per
// node; warp 0 issues the 41 box loads of the tile two ahead into the stage
// every warp has finished reading, so the copies overlap the collision.
// Rows within 3 nodes of an r-wall, and nodes near x3-walls, gather from
// global memory with the folded bounce-back path instead.
//
// Every wait on an mbarrier is bounded (mbarrier.cuh); on expiry the kernel
// sets bit 1 of the status flag, waits (bounded) for its copies still in
// flight, and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "kernels.cuh"
#include "launch.h"
#include "mbarrier.cuh"

namespace lbgm {
namespace {

__device__ __forceinline__ void tma_load_row(float* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                             int t, int r, int pl) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(t), "r"(r), "r"(pl), "r"(smem_addr(bar))
      : "memory");
}

struct TileRow {
  int b, ir, it;
};

__device__ __forceinline__ TileRow tile_row(int tile, const Dims& d) {
  TileRow tr;
  const int rows = d.nr * d.nt;
  tr.b = tile / rows;
  const int rr = tile - tr.b * rows;
  tr.ir = rr / d.nt;
  tr.it = rr - tr.ir * d.nt;
  return tr;
}


// The 41 box loads of one tile into a stage, issued by the lanes of one warp
// (population l by lane l % 32); the barrier expects all their bytes.
// Population l comes from row (i_r - c_r, i_theta - c_theta); rows outside
// [0, nr) are zero-filled by the TMA unit and never read.
template <int NX>
__device__ __forceinline__ void issue_tile(const CUtensorMap* map, float* stage, uint64_t* bar, int tile,
                                           const Dims& d, const int4* vel, int lane) {
  const TileRow tr = tile_row(tile, d);
  if (lane == 0) mbar_expect_tx(bar, uint32_t(Q * NX * sizeof(float)));
  __syncwarp();
  for (int l = lane; l < Q; l += 32) {
    const int4 c = vel[l];
    tma_load_row(stage + l * NX, map, bar, 0, wrap_small(tr.it - c.y, d.nt), tr.ir - c.x, tr.b * Q + l);
  }
}

// Warps of a CTA run decoupled: each waits for the stage's data (full
// barrier), gathers from it, and signals it has finished reading (empty
// barrier, one arrival per warp). Warp 0 refills a stage once every warp has
// read it; no CTA-wide barrier is taken inside the tile loop.
template <int K, int NX>
__global__ void __launch_bounds__(NX, 512 / NX) k_step_tma(const __grid_constant__ CUtensorMap map,
                                                 const float* __restrict__ fin, float* __restrict__ fout,
                                                 GeoDev<float> geo, const InstParams<float>* __restrict__ inst,
                                                 Dims d, int* __restrict__ flag) {
  constexpr int NW = NX / 32;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* stages = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * Q * NX * sizeof(float));
  uint64_t* empty = full + 2;
  int4* vel = reinterpret_cast<int4*>(full + 4);
  const int x = threadIdx.x, lane = x & 31, warp = x >> 5;
  const int ntiles = d.batch * d.nr * d.nt;
  const int G = gridDim.x;
  if (x == 0) vel[0] = make_int4(0, 0, 0, 0);
  static_for<0, NPAIR>([&](auto P_) {
    constexpr int P = decltype(P_)::value;
    using C = Pair<P>;
    if (x == 2 * P + 1) vel[x] = make_int4(C::x, C::y, C::z, 0);
    if (x == 2 * P + 2) vel[x] = make_int4(-C::x, -C::y, -C::z, 0);
  });
  if (x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], NW);
    mbar_init(&empty[1], NW);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) {
    if (int(blockIdx.x) < ntiles) issue_tile<NX>(&map, stages, &full[0], blockIdx.x, d, vel, lane);
    if (int(blockIdx.x) + G < ntiles)
      issue_tile<NX>(&map, stages + Q * NX, &full[1], blockIdx.x + G, d, vel, lane);
  }
  // x3 index of the source of a shift c3 (periodic wrap; NX = n3 is a power of two)
  int xs[7];
#pragma unroll
  for (int c = -3; c <= 3; ++c) xs[c + 3] = (x - c) & (NX - 1);

  int k = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += G, ++k) {
    const int s = k & 1;
    const uint32_t par = uint32_t((k >> 1) & 1);
    if (!mbar_wait_bounded(&full[s], par)) {
      if (lane == 0) atomicOr(flag, 2);
      if (warp == 0 && lane == 0 && tile + G < ntiles)  // copies into the other stage may be in flight
        mbar_wait_bounded(&full[s ^ 1], uint32_t(((k + 1) >> 1) & 1));
      return;
    }
    const TileRow tr = tile_row(tile, d);
    CellPos p;
    p.b = tr.b;
    p.ir = tr.ir;
    p.it = tr.it;
    p.i3 = x;
    p.cell = (tr.ir * d.nt + tr.it) * NX + x;
    const float* st = stages + s * Q * NX;
    float f[Q];
    if (!near_wall(p, d)) {
      f[0] = st[x];
      static_for<0, NPAIR>([&](auto P_) {
        constexpr int P = decltype(P_)::value;
        using C = Pair<P>;
        f[2 * P + 1] = st[(2 * P + 1) * NX + xs[C::z + 3]];
        f[2 * P + 2] = st[(2 * P + 2) * NX + xs[-C::z + 3]];
      });
    } else {
      gather<K>(fin + size_t(p.b) * Q * d.ncell, static_cast<const float*>(nullptr), p, d, f);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (warp == 0 && tile + 2 * G < ntiles) {
      if (!mbar_wait_bounded(&empty[s], par)) {
        if (lane == 0) {
          atomicOr(flag, 2);
          if (tile + G < ntiles) mbar_wait_bounded(&full[s ^ 1], uint32_t(((k + 1) >> 1) & 1));
        }
        return;
      }
      fence_proxy_async_smem();
      issue_tile<NX>(&map, stages + s * Q * NX, &full[s], tile + 2 * G, d, vel, lane);
    }
    const Moments<float> m = moments(f);
    if (!finite_v(m.rho)) {
      if (*flag == 0) atomicOr(flag, 1);
    }
    const int row = geo_row_node<K>(d, p.ir, p.it, p.i3);
    const NodeGeo<float, K> g = load_geo<float, K>(geo, row);
    const InstParams<float> ip = inst[p.b];
    const Coef<float> kc = coefficients<float, K>(m, g, ip.kappa, ip.G);
    collide<float, K>(f, kc, g, ip.omega);
    float* out = fout + size_t(p.b) * Q * d.ncell + p.cell;
#pragma unroll
    for (int l = 0; l < Q; ++l) out[size_t(l) * d.ncell] = f[l];
  }
}

template <int NX>
cudaError_t launch_nx(int K, const void* map, const float* fin, float* fout, const GeoDev<float>& geo,
                      const InstParams<float>* inst, const Dims& d, int* flag, cudaStream_t s) {
  const size_t smem = 2 * Q * NX * sizeof(float) + 4 * sizeof(uint64_t) + Q * sizeof(int4);
  static int configured[3] = {0, 0, 0};
  static int blocks_per_sm[3] = {1, 1, 1};
  static int sms = 0;
  auto kern = K == KFLAT ? k_step_tma<KFLAT, NX> : K == KCYL ? k_step_tma<KCYL, NX> : k_step_tma<KELL, NX>;
  if (!configured[K]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[K], kern, NX, smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    configured[K] = 1;
  }
  const int ntiles = d.batch * d.nr * d.nt;
  int grid = sms * (blocks_per_sm[K] > 0 ? blocks_per_sm[K] : 1);
  if (grid > ntiles) grid = ntiles;
  kern<<<grid, NX, smem, s>>>(*static_cast<const CUtensorMap*>(map), fin, fout, geo, inst, d, flag);
  return cudaGetLastError();
}

}  // namespace

bool tma_step_supported(const Dims& d) { return d.n3 == 128 || d.n3 == 256; }

size_t tensor_map_bytes() { return sizeof(CUtensorMap); }

cudaError_t make_state_tensor_map(void* map_out, const float* base, const Dims& d) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[4] = {cuuint64_t(d.n3), cuuint64_t(d.nt), cuuint64_t(d.nr), cuuint64_t(d.batch) * Q};
  const cuuint64_t strides[3] = {cuuint64_t(d.n3) * 4, cuuint64_t(d.n3) * d.nt * 4,
                                 cuuint64_t(d.n3) * d.nt * d.nr * 4};
  const cuuint32_t box[4] = {cuuint32_t(d.n3), 1, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode(static_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                      const_cast<float*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_step_tma_f32(int K, const void* map, const float* fin, float* fout,
                                const GeoDev<float>& geo, const InstParams<float>* inst, const Dims& d,
                                int* flag, cudaStream_t s) {
  if (d.n3 == 256) return launch_nx<256>(K, map, fin, fout, geo, inst, d, flag, s);
  if (d.n3 == 128) return launch_nx<128>(K, map, fin, fout, geo, inst, d, flag, s);
  return cudaErrorInvalidValue;
}

}  // namespace lbgm
