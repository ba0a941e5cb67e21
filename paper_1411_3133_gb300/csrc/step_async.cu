// Launchers of the prefetching step kernel k_step_async for every storage
// precision.
#include "kernels.cuh"
#include "launch.h"

namespace lbgm {

namespace {

template <class S, class R, int K>
cudaError_t launch_k(const S* fin, S* fout, const GeoDev<R>& geo, const InstParams<R>* inst, const Dims& d,
                     int* flag, int threads, int npt, cudaStream_t s) {
  // two buffers of Q units per thread, and for 2-byte storage as many
  // reference values (k_step_async's `sref`)
  const size_t smem = 2 * size_t(Q) * threads * sizeof(typename AsyncUnit<S>::T) *
                      (Codec<S, R>::uses_ref ? 2 : 1);
  static size_t opted[64] = {};  // per device: largest dynamic shared memory enabled so far
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || smem > opted[dev]) {
    e = cudaFuncSetAttribute(k_step_async<S, R, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) opted[dev] = smem;
  }
  const uint64_t total = uint64_t(d.batch) * uint64_t(d.ncell);
  const uint64_t per_block = uint64_t(threads) * uint64_t(npt);
  const unsigned grid = unsigned((total + per_block - 1) / per_block);
  k_step_async<S, R, K><<<grid, threads, smem, s>>>(fin, fout, geo, inst, d, npt, flag);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_t(int K, const S* fin, S* fout, const GeoDev<R>& geo, const InstParams<R>* inst,
                     const Dims& d, int* flag, int threads, int npt, cudaStream_t s) {
  if (threads < 32 || threads > 256 || threads % 32 || npt < 1) return cudaErrorInvalidValue;
  switch (K) {
    case KFLAT: return launch_k<S, R, KFLAT>(fin, fout, geo, inst, d, flag, threads, npt, s);
    case KCYL: return launch_k<S, R, KCYL>(fin, fout, geo, inst, d, flag, threads, npt, s);
    case KELL: return launch_k<S, R, KELL>(fin, fout, geo, inst, d, flag, threads, npt, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_step_async_f32(int K, const float* fin, float* fout, const GeoDev<float>& geo,
                                  const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                                  int npt, cudaStream_t s) {
  return launch_t<float, float>(K, fin, fout, geo, inst, d, flag, threads, npt, s);
}

cudaError_t launch_step_async_f64(int K, const double* fin, double* fout, const GeoDev<double>& geo,
                                  const InstParams<double>* inst, const Dims& d, int* flag, int threads,
                                  int npt, cudaStream_t s) {
  return launch_t<double, double>(K, fin, fout, geo, inst, d, flag, threads, npt, s);
}

cudaError_t launch_step_async_h16(int K, const __half* fin, __half* fout, const GeoDev<float>& geo,
                                  const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                                  int npt, cudaStream_t s) {
  return launch_t<__half, float>(K, fin, fout, geo, inst, d, flag, threads, npt, s);
}

cudaError_t launch_step_async_b16(int K, const __nv_bfloat16* fin, __nv_bfloat16* fout,
                                  const GeoDev<float>& geo, const InstParams<float>* inst, const Dims& d,
                                  int* flag, int threads, int npt, cudaStream_t s) {
  return launch_t<__nv_bfloat16, float>(K, fin, fout, geo, inst, d, flag, threads, npt, s);
}

}  // namespace lbgm
