// Fused time-step kernel, double populations and arithmetic: instantiations for
// the flat, cylindrical and ellipsoidal metrics and their launcher.
#include "kernels.cuh"
#include "launch.h"

namespace lbgm {

cudaError_t launch_step_f64(int K, const double* fin, double* fout, const GeoDev<double>& geo,
                            const InstParams<double>* inst, const Dims& d, int* flag, int threads,
                            cudaStream_t s) {
  const uint32_t total = uint32_t(d.batch) * uint32_t(d.ncell);
  const uint32_t blocks = (total + threads - 1) / threads;
  switch (K) {
    case KFLAT: k_step<double, KFLAT><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    case KCYL: k_step<double, KCYL><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    case KELL: k_step<double, KELL><<<blocks, threads, 0, s>>>(fin, fout, geo, inst, d, flag); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbgm
