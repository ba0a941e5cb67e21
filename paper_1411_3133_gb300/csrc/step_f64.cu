// Fused time-step kernel, FP64 populations and arithmetic: instantiations for the flat,
// cylindrical and ellipsoidal metrics.
#include "step_launch.cuh"

namespace lbgm {

cudaError_t launch_step_f64(int K, const double* fin, double* fout, const GeoDev<double>& geo,
                            const InstParams<double>* inst, const Dims& d, int* flag, int threads,
                            cudaStream_t s) {
  return launch_step_t<double, double>(K, fin, fout, geo, inst, d, flag, threads, s);
}

cudaError_t launch_step_list_f64(int K, int walls, const void* insts, const int4* work, int nwork,
                                 const int* cells, int threads, int grid, int parity, cudaStream_t s) {
  return launch_step_list_t<double, double>(K, walls, insts, work, nwork, cells, threads, grid, parity, s);
}

int step_list_max_threads_f64() { return step_list_max_threads_t<double, double>(); }

cudaError_t step_list_occupancy_f64(int K, int threads, int* blocks_per_sm) {
  return step_list_occupancy_t<double, double>(K, threads, blocks_per_sm);
}

cudaError_t launch_step_split_f64(int K, const double* fin, double* fout, const GeoDev<double>& geo,
                                  const InstParams<double>* inst, const Dims& d, int* flag, int threads,
                                  cudaStream_t s, cudaStream_t se) {
  return launch_step_split_t<double, double>(K, fin, fout, geo, inst, d, flag, threads, s, se);
}

}  // namespace lbgm
