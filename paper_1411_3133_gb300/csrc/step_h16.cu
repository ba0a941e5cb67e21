// Fused time-step kernel, FP16 population deviations, FP32 arithmetic: instantiations for the flat,
// cylindrical and ellipsoidal metrics.
#include "step_launch.cuh"

namespace lbgm {

cudaError_t launch_step_h16(int K, const __half* fin, __half* fout, const GeoDev<float>& geo,
                            const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                            cudaStream_t s) {
  return launch_step_t<__half, float>(K, fin, fout, geo, inst, d, flag, threads, s);
}

}  // namespace lbgm
