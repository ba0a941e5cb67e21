// Fused time-step kernel, float populations and arithmetic: instantiations for
// the flat, cylindrical and ellipsoidal metrics and their launcher.
#include "kernels.cuh"
#include "launch.h"

namespace lbgm {

cudaError_t launch_step_f32(int K, const float* fin, float* fout, const GeoDev<float>& geo,
                            const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                            cudaStream_t s) {
  const uint32_t total = uint32_t(d.batch) * uint32_t(d.ncell);
  const uint32_t blocks = (total + threads - 1) / threads;
  switch (K) {
    case KFLAT: k_step<float, KFLAT><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    case KCYL: k_step<float, KCYL><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    case KELL: k_step<float, KELL><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbgm
