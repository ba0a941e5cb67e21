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
  const uint32_t total = uint32_t(d.batch) * uint32_t(d.ncell);
  const uint32_t blocks = (total + threads - 1) / threads;
  switch (K) {
    case KFLAT: k_step<S, R, KFLAT><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    case KCYL: k_step<S, R, KCYL><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    case KELL: k_step<S, R, KELL><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbgm
