// Observables without any device allocation (lb_diagnostics_noalloc).
//
// Some callers cannot call cudaMalloc: a program whose device memory is
// already owned by another allocator (a framework's caching pool that
// reserved the device), or a long-running loop that must not allocate (and
// so must not risk an implicit device synchronisation) after start-up. This
// entry point computes the same observables as lb_diagnostics from fields the
// caller already holds on the device, and keeps its working memory in one
// fixed, file-scope device array instead of allocating.
//
// The array holds LB_NOALLOC_SCRATCH_BYTES bytes on every GPU that loads the
// library, for the life of the process. All calls share it and it keeps the
// last call's contents; every word a call reads is written earlier in that
// same call, so nothing has to be cleared. Two calls whose work overlaps on
// the GPU (different streams, or different host threads) race on it.
//
// Host code cannot use the array's name as a device address: every call
// looks the address up with cudaGetSymbolAddress on the current device, so
// the pointer it passes to the kernels is always that device's copy (also
// after a cudaDeviceReset, which reloads the module).
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/lbgm.h"
#include "geometry.h"
#include "lattice.cuh"
#include "launch.h"

namespace lbgm {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[LB_NOALLOC_SCRATCH_BYTES];

lb_status noalloc_fail(lb_status s, const std::string& m) {
  set_last_error_noctx(m);  // reported by lb_last_error(NULL)
  return s;
}

// Per-row weights for the observables (sqrt g, sqrt g_thth, cross-section
// area weight, vorticity weight), from the same helper as the context's
// geometry table (observable_weights), written straight into the scratch
// array.
__global__ void k_noalloc_weights(lb_metric metric, lb_geometry_desc g, double* w) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= g.nr * g.n3) return;
  const int ir = row / g.n3, i3 = row - ir * g.n3;
  observable_weights(metric, g, ir, i3, w + 4 * row);
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace
}  // namespace lbgm

using namespace lbgm;

extern "C" lb_status lb_diagnostics_noalloc(lb_metric metric, const lb_geometry_desc* geom, int batch,
                                            const double* tau, const double* rho, const double* u,
                                            void* cuda_stream, lb_diag* out) {
  if (!geom || !tau || !rho || !u || !out) return noalloc_fail(LB_ERR_ARG, "null argument");
  const std::string v = validate_geometry(metric, *geom);
  if (!v.empty()) return noalloc_fail(LB_ERR_ARG, v);
  if (metric == LB_METRIC_ELLIPSOIDAL_THETA)
    return noalloc_fail(LB_ERR_ARG, "the theta-resolved ellipsoid has per-node weights: use lb_diagnostics");
  if (batch < 1 || batch > LB_NOALLOC_MAX_BATCH)
    return noalloc_fail(LB_ERR_ARG, "need 1 <= batch <= " + std::to_string(LB_NOALLOC_MAX_BATCH));
  for (int b = 0; b < batch; ++b)
    if (!(tau[b] > 0.5)) return noalloc_fail(LB_ERR_ARG, "need tau > 1/2");

  Dims d{};
  d.nr = geom->nr;
  d.nt = geom->ntheta;
  d.n3 = geom->n3;
  d.ncell = geom->nr * geom->ntheta * geom->n3;
  d.periodic3 = geom->periodic3 ? 1 : 0;
  d.wall_eq = geom->wall == LB_WALL_EQUILIBRIUM ? 1 : 0;
  d.batch = batch;
  const size_t N = size_t(d.ncell);
  const int nblk = int(std::min<size_t>(1024, (N + 255) / 256));
  const size_t nrow64 = size_t(d.nr) * d.n3;
  const size_t off_w = 0;
  const size_t off_rowmean = off_w + align256(nrow64 * 4 * sizeof(double));
  const size_t off_partial = off_rowmean + align256(size_t(batch) * d.nr * d.nt * sizeof(double));
  const size_t off_out = off_partial + align256(size_t(batch) * nblk * DIAG_NQ * sizeof(double));
  const size_t need = off_out + align256(size_t(batch) * DIAG_NQ * sizeof(double));
  if (need > LB_NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(LB_ERR_ARG, "needs " + std::to_string(need) + " bytes of scratch; the fixed limit is " +
                                        std::to_string(LB_NOALLOC_SCRATCH_BYTES));

  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // this device's copy
  if (e != cudaSuccess)
    return noalloc_fail(LB_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  unsigned char* base = static_cast<unsigned char*>(p);
  double* w = reinterpret_cast<double*>(base + off_w);
  double* rowmean = reinterpret_cast<double*>(base + off_rowmean);
  double* partial = reinterpret_cast<double*>(base + off_partial);
  double* sums = reinterpret_cast<double*>(base + off_out);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  k_noalloc_weights<<<int((nrow64 + 255) / 256), 256, 0, s>>>(metric, *geom, w);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_diag(rho, u, rowmean, w, d, partial, nblk, sums, s);
  double h[LB_NOALLOC_MAX_BATCH * DIAG_NQ];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h, sums, size_t(batch) * DIAG_NQ * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return noalloc_fail(LB_ERR_CUDA, std::string("diagnostics: ") + cudaGetErrorString(e));

  const double R = curvature_radius(metric, *geom);
  const double dd = geom->r_outer - geom->r_inner;
  for (int b = 0; b < batch; ++b) {
    const double* q = &h[b * DIAG_NQ];
    lb_diag& o = out[b];
    o.mass_rho_prime = q[0];
    o.mass_physical = q[1];
    o.mean_v_theta = q[2] / q[3];
    const double nu = (tau[b] - 0.5) * CS2;
    o.dean = R > 0.0 ? o.mean_v_theta * (dd / lattice_h(*geom)) / nu * std::sqrt(dd / R) : 0.0;
    o.mean_vorticity = q[4] / q[3];
    o.vortex_amp = std::sqrt(q[5] / double(N));
    o.vortex_amp_x3 = std::sqrt(q[6] / double(N));
    o.max_speed = q[7];
    o.nonfinite = (long long)q[8];
    o.step = -1;
  }
  return LB_OK;
}
