// Launcher of the fused step kernel for one storage/compute type pair; each
// step_*.cu translation unit instantiates one pair so that the large unrolled
// kernel bodies compile in parallel.
#pragma once

#include "kernels.cuh"
#include "launch.h"

namespace lbgm {

template <class S, class R>
cudaError_t launch_step_t(int K, const S* fin, S* fout, const GeoDev<R>& geo, const InstParams<R>* inst,
                          const Dims& d, int* flag, int threads, cudaStream_t s) {
  if (d.batch < 1 || d.batch > 65535) return cudaErrorInvalidValue;
  threads = threads < StepBounds<S, R>::maxt ? threads : StepBounds<S, R>::maxt;
  const dim3 blocks((uint32_t(d.ncell) + threads - 1) / threads, uint32_t(d.batch));
  switch (K) {
    case KFLAT: k_step<S, R, KFLAT><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    case KCYL: k_step<S, R, KCYL><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    case KELL: k_step<S, R, KELL><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    case KELT:  // the theta-resolved ellipsoid: FP64 / FP32 storage, this kernel only
      if constexpr (!Codec<S, R>::uses_ref) {
        k_step<S, R, KELT><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag);
        break;
      }
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// The region split of 2-byte storage for the flat and cylindrical metrics
// (geometry and stream rows of i_r alone) with blocks that never straddle an
// i_r layer: the kernels that keep the block's row in shared memory
// (step_row_shared); false for the other storage types and metrics.
template <class S, class R, int K>
bool launch_split_rowsm(dim3 gb, dim3 ge, int threads, cudaStream_t s, cudaStream_t se, const S* fin, S* fout,
                        const GeoDev<R>& geo, const InstParams<R>* inst, const Dims& d, int* flag) {
  if constexpr (Codec<S, R>::uses_ref && K != KELL) {
    k_step_bulk_rowsm<S, K><<<gb, threads, 0, s>>>(fin, fout, geo, inst, d, flag);
    k_step_edge_rowsm<S, K><<<ge, threads, 0, se>>>(fin, fout, geo, inst, d, flag);
    return true;
  }
  return false;
}

// Region-split step (periodic x3 only): the interior on stream s, then the
// 6 wall layers on stream se (the caller orders the two streams around the
// step). Launched second, the small wall-layer kernel takes SMs as interior
// blocks retire (measured 0.6 % faster than the reverse order).
template <class S, class R>
cudaError_t launch_step_split_t(int K, const S* fin, S* fout, const GeoDev<R>& geo, const InstParams<R>* inst,
                                const Dims& d, int* flag, int threads, cudaStream_t s, cudaStream_t se) {
  if (d.batch < 1 || d.batch > 65535 || !d.periodic3 || d.nr < 7) return cudaErrorInvalidValue;
  threads = threads < StepBounds<S, R>::maxt ? threads : StepBounds<S, R>::maxt;
  const uint32_t layer = uint32_t(d.nt) * uint32_t(d.n3);
  const dim3 ge((6u * layer + threads - 1) / threads, uint32_t(d.batch));
  const dim3 gb((uint32_t(d.nr - 6) * layer + threads - 1) / threads, uint32_t(d.batch));
  const bool rowsm = layer % uint32_t(threads) == 0;
  switch (K) {
    case KFLAT:
      if (rowsm && launch_split_rowsm<S, R, KFLAT>(gb, ge, threads, s, se, fin, fout, geo, inst, d, flag)) break;
      k_step_bulk<S, R, KFLAT><<<gb, threads, 0, s>>>(fin, fout, geo, inst, d, flag);
      k_step_edge<S, R, KFLAT><<<ge, threads, 0, se>>>(fin, fout, geo, inst, d, flag);
      break;
    case KCYL:
      if (rowsm && launch_split_rowsm<S, R, KCYL>(gb, ge, threads, s, se, fin, fout, geo, inst, d, flag)) break;
      k_step_bulk<S, R, KCYL><<<gb, threads, 0, s>>>(fin, fout, geo, inst, d, flag);
      k_step_edge<S, R, KCYL><<<ge, threads, 0, se>>>(fin, fout, geo, inst, d, flag);
      break;
    case KELL:
      k_step_bulk<S, R, KELL><<<gb, threads, 0, s>>>(fin, fout, geo, inst, d, flag);
      k_step_edge<S, R, KELL><<<ge, threads, 0, se>>>(fin, fout, geo, inst, d, flag);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// grid 0: one block per work item; otherwise `grid` persistent blocks.
// walls bits 0-1: the list's class -- 0 interior tiles (cells NULL), 1
// r-layer wall nodes (compile-time folds along r), 2 x3-layer wall nodes
// (folds along x3), 3 every other wall node (the general wall rule), the
// last three over `cells`; bit 2: interior tiles of more than one block's
// worth of nodes.
template <class S, class R>
cudaError_t launch_step_list_t(int K, int walls, const void* insts, const int4* work, int nwork, const int* cells,
                               int threads, int grid, int parity, cudaStream_t s) {
  if (nwork == 0) return cudaSuccess;
  const auto* I = static_cast<const ListInst<S, R>*>(insts);
  const int g = grid > 0 && grid < nwork ? grid : nwork;
  const int sel = (walls & 3) == 0 ? (walls & 4 ? 4 : 0) : walls & 3;
#define LB_LIST(KK)                                                                                       \
  (sel == 0   ? (k_step_list<S, R, KK, 0, false><<<g, threads, 0, s>>>(I, work, nwork, cells, parity), 0) \
   : sel == 4 ? (k_step_list<S, R, KK, 0, true><<<g, threads, 0, s>>>(I, work, nwork, cells, parity), 0)  \
   : sel == 1 ? (k_step_list<S, R, KK, 3, false><<<g, threads, 0, s>>>(I, work, nwork, cells, parity), 0) \
   : sel == 2 ? (k_step_list<S, R, KK, 4, false><<<g, threads, 0, s>>>(I, work, nwork, cells, parity), 0) \
              : (k_step_list<S, R, KK, 1, false><<<g, threads, 0, s>>>(I, work, nwork, cells, parity), 0))
  switch (K) {
    case KFLAT: LB_LIST(KFLAT); break;
    case KCYL: LB_LIST(KCYL); break;
    case KELL: LB_LIST(KELL); break;
    default: return cudaErrorInvalidValue;
  }
#undef LB_LIST
  return cudaGetLastError();
}

// Largest block of the work-list kernel (its launch bounds).
template <class S, class R>
int step_list_max_threads_t() {
  return StepBounds<S, R>::maxt;
}

// Resident blocks per SM of the work-list kernel at `threads` per block.
template <class S, class R>
cudaError_t step_list_occupancy_t(int K, int threads, int* blocks_per_sm) {
  switch (K) {
    case KFLAT:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_step_list<S, R, KFLAT, 0, false>, threads,
                                                           0);
    case KCYL:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_step_list<S, R, KCYL, 0, false>, threads,
                                                           0);
    case KELL:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_step_list<S, R, KELL, 0, false>, threads,
                                                           0);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace lbgm
