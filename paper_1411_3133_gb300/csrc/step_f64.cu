// Fused time-step kernel, FP64 populations and arithmetic: instantiations for the flat,
// cylindrical and ellipsoidal metrics.
#include "step_launch.cuh"

namespace lbgm {

cudaError_t launch_step_f64(int K, const double* fin, double* fout, const GeoDev<double>& geo,
                            const InstParams<double>* inst, const Dims& d, int* flag, int threads,
                            cudaStream_t s) {
  return launch_step_t<double, double>(K, fin, fout, geo, inst, d, flag, threads, s);
}

}  // namespace lbgm
