// Fused time-step kernel, FP32 populations and arithmetic: instantiations for the flat,
// cylindrical and ellipsoidal metrics.
#include "step_launch.cuh"

namespace lbgm {

cudaError_t launch_step_f32(int K, const float* fin, float* fout, const GeoDev<float>& geo,
                            const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                            cudaStream_t s) {
  return launch_step_t<float, float>(K, fin, fout, geo, inst, d, flag, threads, s);
}

}  // namespace lbgm
