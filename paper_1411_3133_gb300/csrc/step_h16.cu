// Fused time-step kernel, FP16 population deviations, FP32 arithmetic: instantiations for the flat,
// cylindrical and ellipsoidal metrics.
#include "step_launch.cuh"

namespace lbgm {

cudaError_t launch_step_h16(int K, const __half* fin, __half* fout, const GeoDev<float>& geo,
                            const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                            cudaStream_t s) {
  return launch_step_t<__half, float>(K, fin, fout, geo, inst, d, flag, threads, s);
}

cudaError_t launch_step_list_h16(int K, int walls, const void* insts, const int4* work, int nwork,
                                 const int* cells, int threads, int grid, int parity, cudaStream_t s) {
  return launch_step_list_t<__half, float>(K, walls, insts, work, nwork, cells, threads, grid, parity, s);
}

int step_list_max_threads_h16() { return step_list_max_threads_t<__half, float>(); }

cudaError_t step_list_occupancy_h16(int K, int threads, int* blocks_per_sm) {
  return step_list_occupancy_t<__half, float>(K, threads, blocks_per_sm);
}

cudaError_t launch_step_split_h16(int K, const __half* fin, __half* fout, const GeoDev<float>& geo,
                                  const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                                  cudaStream_t s, cudaStream_t se) {
  return launch_step_split_t<__half, float>(K, fin, fout, geo, inst, d, flag, threads, s, se);
}

}  // namespace lbgm
