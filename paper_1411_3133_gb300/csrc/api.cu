// C ABI of liblbgm.so (declared in include/lbgm.h): context management,
// parameter validation, geometry upload, and the host side of every entry
// point. All numerical work runs in the kernels of kernels.cuh / aux.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lbgm.h"
#include "ctx.h"
#include "geometry.h"
#include "kernels.cuh"
#include "launch.h"

using namespace lbgm;

namespace {

thread_local std::string g_err;

lb_status fail(lb_ctx* c, lb_status s, const std::string& msg) {
  if (c) {
    c->err = msg;
    if (s == LB_ERR_CUDA || s == LB_ERR_NONFINITE) c->poisoned = true;
  } else {
    g_err = msg;
  }
  return s;
}

lb_status cuda_fail(lb_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(c, LB_ERR_CUDA, m);
}

#define LB_CUDA(ctx, call)                                    \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

void* dalloc(lb_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (c->has_alloc) {
    p = c->alloc.alloc(bytes, c->stream, c->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) c->allocations.emplace_back(p, bytes);
  return p;
}

void free_all(lb_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  for (auto& a : c->allocations) {
    if (c->has_alloc)
      c->alloc.free(a.first, a.second, c->stream, c->alloc.user);
    else
      cudaFree(a.first);
  }
  c->allocations.clear();
}

bool usable(lb_ctx* c, lb_status* s) {
  if (!c) {
    *s = fail(nullptr, LB_ERR_ARG, "null context");
    return false;
  }
  if (c->poisoned) {
    *s = fail(c, LB_ERR_STATE, "context poisoned by an earlier failure: " + c->err);
    return false;
  }
  if (!c->initialized) {
    *s = fail(c, LB_ERR_STATE, "context not initialised (call lb_init first)");
    return false;
  }
  return true;
}

template <typename Real>
void fill_inst(const lb_params* p, int batch, std::vector<InstParams<Real>>& out) {
  out.resize(batch);
  for (int b = 0; b < batch; ++b) {
    out[b].omega = Real(1.0 / p[b].tau);
    out[b].kappa = p[b].old_forcing == 1 ? Real(0) : Real(1.0 - 1.0 / (2.0 * p[b].tau));
    out[b].G = Real(p[b].force_G);
    out[b].pad = p[b].old_forcing == 2 ? Real(1) : Real(0);  // the half-force velocity variant
  }
}

lb_status upload_params(lb_ctx* c, const lb_params* p) {
  for (int b = 0; b < c->batch; ++b) {
    if (!(p[b].tau > 0.5) || !std::isfinite(p[b].tau))
      return fail(c, LB_ERR_ARG, "instance " + std::to_string(b) + ": need tau > 1/2");
    if (!std::isfinite(p[b].force_G) || !std::isfinite(p[b].noise_amp))
      return fail(c, LB_ERR_ARG, "instance " + std::to_string(b) + ": non-finite force or noise");
    if (p[b].old_forcing < 0 || p[b].old_forcing > 2)
      return fail(c, LB_ERR_ARG, "instance " + std::to_string(b) + ": old_forcing must be 0, 1 or 2");
    if (p[b].old_forcing == 2 && c->prec != LB_FP64 && c->prec != LB_FP32)
      return fail(c, LB_ERR_ARG, "instance " + std::to_string(b) +
                                     ": the half-force velocity (old_forcing 2) needs FP64 or FP32 storage");
    if (p[b].old_forcing == 2 && c->K == KELT)
      return fail(c, LB_ERR_ARG, "instance " + std::to_string(b) +
                                     ": the half-force velocity (old_forcing 2) is not built for the "
                                     "theta-resolved ellipsoid");
  }
  c->any_shift = false;
  for (int b = 0; b < c->batch; ++b) c->any_shift = c->any_shift || p[b].old_forcing == 2;
  if (c->prec == LB_FP64) {
    std::vector<InstParams<double>> h;
    fill_inst(p, c->batch, h);
    LB_CUDA(c, cudaMemcpyAsync(c->inst, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice,
                               c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
  } else {
    std::vector<InstParams<float>> h;
    fill_inst(p, c->batch, h);
    LB_CUDA(c, cudaMemcpyAsync(c->inst, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice,
                               c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  c->tau.resize(c->batch);
  for (int b = 0; b < c->batch; ++b) c->tau[b] = p[b].tau;
  return LB_OK;
}

template <typename Real>
void geo_arrays(Real* base, size_t nrows, GeoDev<Real>& g) {
  g.dtt = base;
  g.dpp = base + nrows;
  g.g_rtt = base + 2 * nrows;
  g.g_rpp = base + 3 * nrows;
  g.g_trt = base + 4 * nrows;
  g.g_prp = base + 5 * nrows;
  g.g_ttp = base + 6 * nrows;
  g.g_ptt = base + 7 * nrows;
  g.fth = base + 8 * nrows;
  g.ext = base + 9 * nrows;  // theta-resolved ellipsoid only
  g.ext_stride = uint32_t(nrows);
}

// Device geometry arrays of metric kind K in the compute precision: the 9
// arrays of GeoDev over the kind's rows (i_r; (i_r, i_3); every node for the
// theta-resolved ellipsoid, which adds the 6 arrays of GeoDev::ext).
size_t geo_arrays_count(int K) { return K == KELT ? 15 : 9; }

template <typename Real>
std::vector<Real> geo_host_tables(const std::vector<double>& rows, const lb_geometry_desc& g, int K) {
  const size_t rows3 = K == KELL ? g.n3 : K == KELT ? size_t(g.ntheta) * g.n3 : 1;
  const size_t nrows = size_t(g.nr) * rows3;
  std::vector<Real> t(geo_arrays_count(K) * nrows);
  for (int ir = 0; ir < g.nr; ++ir)
    for (size_t i3 = 0; i3 < rows3; ++i3) {
      // host rows: (i_r, i_3) for the frozen kinds, (i_r, i_theta, i_3) = i3 here for KELT
      const double* r = &rows[(size_t(ir) * (K == KELT ? rows3 : g.n3) + i3) * LB_GEO_STRIDE];
      const size_t k = ir * rows3 + i3;
      if (K == KELT) {
        t[9 * nrows + k] = Real(r[GEO_DELTA + 0]);
        t[10 * nrows + k] = Real(r[GEO_DELTA + 1]);
        t[11 * nrows + k] = Real(r[GEO_DELTA + 2]);
        t[12 * nrows + k] = Real(r[GEO_DELTA + 5]);
        t[13 * nrows + k] = Real(r[GEO_FDIR + 0]);
        t[14 * nrows + k] = Real(r[GEO_FDIR + 2]);
      }
      auto gam = [&](int i, int j, int l) { return r[GEO_GAMMA + (i * 3 + j) * 3 + l]; };
      t[0 * nrows + k] = Real(r[GEO_DELTA + 4]);
      t[1 * nrows + k] = Real(r[GEO_DELTA + 8]);
      t[2 * nrows + k] = Real(gam(0, 1, 1));
      t[3 * nrows + k] = Real(gam(0, 2, 2));
      t[4 * nrows + k] = Real(gam(1, 0, 1));
      t[5 * nrows + k] = Real(gam(2, 0, 2));
      t[6 * nrows + k] = Real(gam(1, 1, 2));
      t[7 * nrows + k] = Real(gam(2, 1, 1));
      t[8 * nrows + k] = Real(r[GEO_FDIR + 1]);
    }
  return t;
}

// The kernels read only the components listed in GeoDev; check that every
// other component of the evaluated geometry is zero for this metric kind.
std::string check_sparsity(const std::vector<double>& rows, const lb_geometry_desc& g, int K) {
  const size_t n = rows.size() / LB_GEO_STRIDE;
  for (size_t k = 0; k < n; ++k) {
    const double* r = &rows[k * LB_GEO_STRIDE];
    for (int i = 0; i < 9; ++i) {
      const bool used = (i == 4 && K != KFLAT) || (i == 8 && (K == KELL || K == KELT)) || K == KELT;
      if (!used && r[GEO_DELTA + i] != 0.0) return "unexpected Delta component";
    }
    if (K == KELT) {  // a symmetric Delta, as the kernels read it
      if (r[GEO_DELTA + 3] != r[GEO_DELTA + 1] || r[GEO_DELTA + 6] != r[GEO_DELTA + 2] ||
          r[GEO_DELTA + 7] != r[GEO_DELTA + 5])
        return "Delta not symmetric";
    }
    for (int idx = 0; idx < 27; ++idx) {
      const int i = idx / 9, j = (idx / 3) % 3, l = idx % 3;
      bool used = false;
      if (K == KCYL || K == KELL || K == KELT)
        used = (i == 0 && j == 1 && l == 1) || (i == 1 && ((j == 0 && l == 1) || (j == 1 && l == 0)));
      if (K == KELL || K == KELT)
        used = used || (i == 0 && j == 2 && l == 2) || (i == 2 && ((j == 0 && l == 2) || (j == 2 && l == 0))) ||
               (i == 1 && ((j == 1 && l == 2) || (j == 2 && l == 1))) || (i == 2 && j == 1 && l == 1);
      if (!used && r[GEO_GAMMA + idx] != 0.0) return "unexpected Christoffel component";
    }
    if (K != KELT && (r[GEO_FDIR] != 0.0 || r[GEO_FDIR + 2] != 0.0)) return "unexpected force direction";
  }
  // the cylinder and flat kernels read rows by i_r only
  if (K == KFLAT || K == KCYL)
    for (int ir = 0; ir < g.nr; ++ir)
      for (int i3 = 1; i3 < g.n3; ++i3)
        for (int f = 0; f < 39; ++f)
          if (rows[(size_t(ir) * g.n3 + i3) * LB_GEO_STRIDE + f] !=
              rows[(size_t(ir) * g.n3) * LB_GEO_STRIDE + f])
            return "geometry varies along x3";
  return "";
}

bool use_tma(const lb_ctx* c) { return c->prec == LB_FP32 && c->tma_ok && c->step_kernel == 2; }


// Region-split step: the wall layers run on the context's second stream,
// concurrently with the interior on the main stream (fork and join by events,
// which a graph capture records as branches).
cudaError_t launch_split(lb_ctx* c, int src, int dst) {
  cudaError_t e = cudaSuccess;
  if (!c->aux) {
    e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  e = cudaEventRecord(c->ev_fork, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->aux, c->ev_fork, 0);
  if (e != cudaSuccess) return e;
  switch (c->prec) {
    case LB_FP64:
      e = launch_step_split_f64(c->K, static_cast<const double*>(c->f[src]), static_cast<double*>(c->f[dst]),
                                c->geo_d, static_cast<const InstParams<double>*>(c->inst), c->dims, c->flag,
                                c->block_threads, c->stream, c->aux);
      break;
    case LB_FP32:
      e = launch_step_split_f32(c->K, static_cast<const float*>(c->f[src]), static_cast<float*>(c->f[dst]),
                                c->geo_f, static_cast<const InstParams<float>*>(c->inst), c->dims, c->flag,
                                c->block_threads, c->stream, c->aux);
      break;
    case LB_FP16_SHIFTED:
      e = launch_step_split_h16(c->K, static_cast<const __half*>(c->f[src]), static_cast<__half*>(c->f[dst]),
                                c->geo_f, static_cast<const InstParams<float>*>(c->inst), c->dims, c->flag,
                                c->block_threads, c->stream, c->aux);
      break;
    default:
      e = launch_step_split_b16(c->K, static_cast<const __nv_bfloat16*>(c->f[src]),
                                static_cast<__nv_bfloat16*>(c->f[dst]), c->geo_f,
                                static_cast<const InstParams<float>*>(c->inst), c->dims, c->flag,
                                c->block_threads, c->stream, c->aux);
      break;
  }
  cudaError_t e2 = cudaEventRecord(c->ev_join, c->aux);  // join even after a failed launch
  if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
  return e != cudaSuccess ? e : e2;
}

// LB_OPT_STEP_KERNEL 0 (auto): the region split where x3 is periodic and the
// arithmetic is FP32 (measured fastest there), the one-kernel step otherwise.
int resolved_kernel(const lb_ctx* c) {
  if (c->any_shift) return 1;  // the half-force variant runs in the plain kernel only
  if (c->K == KELT) return 1;   // the theta-resolved ellipsoid too
  if (c->step_kernel != 0) return c->step_kernel;
  if (c->prec == LB_FP64) return 1;
  return (c->geom.periodic3 && c->geom.wall == LB_WALL_BOUNCEBACK) ? 4 : 5;
}

lb_status launch_step_once(lb_ctx* c) {
  const int src = c->cur, dst = 1 - c->cur;
  const int kern = resolved_kernel(c);
  cudaError_t e;
  if (kern == 4)
    e = launch_split(c, src, dst);
  else if (kern == 5) {
    lb_status st = ctx_tiled_prepare(c);  // a no-op once the tiles are current
    if (st == LB_OK) st = ctx_tiled_launch(c);
    if (st != LB_OK) return st;
    e = cudaSuccess;
  }
  else if (c->any_shift && c->prec == LB_FP64)
    e = launch_step_shift_f64(c->K, static_cast<const double*>(c->f[src]), static_cast<double*>(c->f[dst]),
                              c->geo_d, static_cast<const InstParams<double>*>(c->inst), c->dims, c->flag,
                              c->block_threads, c->stream);
  else if (c->any_shift)
    e = launch_step_shift_f32(c->K, static_cast<const float*>(c->f[src]), static_cast<float*>(c->f[dst]),
                              c->geo_f, static_cast<const InstParams<float>*>(c->inst), c->dims, c->flag,
                              c->block_threads, c->stream);
  else if (use_tma(c))
    e = launch_step_tma_f32(c->K, c->tmap[src], static_cast<const float*>(c->f[src]),
                            static_cast<float*>(c->f[dst]), c->geo_f,
                            static_cast<const InstParams<float>*>(c->inst), c->dims, c->flag, c->stream);
  else if (c->prec == LB_FP64)
    e = launch_step_f64(c->K, static_cast<const double*>(c->f[src]), static_cast<double*>(c->f[dst]),
                        c->geo_d, static_cast<const InstParams<double>*>(c->inst), c->dims, c->flag,
                        c->block_threads, c->stream);
  else if (c->prec == LB_FP32)
    e = launch_step_f32(c->K, static_cast<const float*>(c->f[src]), static_cast<float*>(c->f[dst]),
                        c->geo_f, static_cast<const InstParams<float>*>(c->inst), c->dims, c->flag,
                        c->block_threads, c->stream);
  else if (c->prec == LB_FP16_SHIFTED)
    e = launch_step_h16(c->K, static_cast<const __half*>(c->f[src]), static_cast<__half*>(c->f[dst]),
                        c->geo_f, static_cast<const InstParams<float>*>(c->inst), c->dims, c->flag,
                        c->block_threads, c->stream);
  else
    e = launch_step_b16(c->K, static_cast<const __nv_bfloat16*>(c->f[src]),
                        static_cast<__nv_bfloat16*>(c->f[dst]), c->geo_f,
                        static_cast<const InstParams<float>*>(c->inst), c->dims, c->flag,
                        c->block_threads, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
  c->cur = dst;
  return LB_OK;
}

lb_status check_flag(lb_ctx* c) {
  int h = 0;
  LB_CUDA(c, cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  if (h & 2) return fail(c, LB_ERR_TIMEOUT, "a bounded device wait expired in the step kernel");
  if (h) return fail(c, LB_ERR_NONFINITE, "non-finite density after step " + std::to_string(c->step));
  return LB_OK;
}

lb_status reset_after_init(lb_ctx* c) {
  LB_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  c->step = 0;
  c->initialized = true;
  c->poisoned = false;
  c->err.clear();
  return LB_OK;
}

const void* geo_ptr(lb_ctx* c) {
  return c->prec == LB_FP64 ? static_cast<const void*>(&c->geo_d) : static_cast<const void*>(&c->geo_f);
}

}  // namespace

void lbgm::set_last_error_noctx(const std::string& msg) { g_err = msg; }
lb_status lbgm::ctx_fail(lb_ctx* c, lb_status s, const std::string& msg) { return fail(c, s, msg); }
bool lbgm::ctx_usable(lb_ctx* c, lb_status* s) { return usable(c, s); }

// ---------------------------------------------------------------------------
extern "C" {

int lb_velocity_set(int* cv, double* w) {
  for (int l = 0; l < Q; ++l) {
    if (cv)
      for (int i = 0; i < 3; ++i) cv[l * 3 + i] = vel(l, i);
    if (w) w[l] = weight(l);
  }
  return Q;
}

lb_status lb_geometry_eval(lb_metric metric, const lb_geometry_desc* geom, double* out, size_t out_len) {
  if (!geom || !out) return fail(nullptr, LB_ERR_ARG, "null argument");
  const std::string v = validate_geometry(metric, *geom);
  if (!v.empty()) return fail(nullptr, LB_ERR_ARG, v);
  const size_t need = geometry_rows(metric, *geom) * LB_GEO_STRIDE;
  if (out_len < need) return fail(nullptr, LB_ERR_ARG, "output too small: need " + std::to_string(need));
  const std::vector<double> rows = evaluate_geometry(metric, *geom);
  std::memcpy(out, rows.data(), need * sizeof(double));
  return LB_OK;
}

lb_status lb_force_for_dean(lb_metric metric, const lb_geometry_desc* geom, double tau, double De,
                            double* G_out) {
  if (!geom || !G_out) return fail(nullptr, LB_ERR_ARG, "null argument");
  const std::string v = validate_geometry(metric, *geom);
  if (!v.empty()) return fail(nullptr, LB_ERR_ARG, v);
  if (metric != LB_METRIC_CYLINDRICAL || geom->dtheta_scale != 1.0)
    return fail(nullptr, LB_ERR_ARG, "closed form only for the cylinder with dtheta_scale = 1");
  if (!(tau > 0.5) || !std::isfinite(De)) return fail(nullptr, LB_ERR_ARG, "need tau > 1/2, finite De");
  // De per unit force: mean over the nodes of v(r) for G = 1
  double A, B, C;
  curved_poiseuille(*geom, tau, 1.0, &A, &B, &C);
  double vsum = 0.0;
  for (int i = 0; i < geom->nr; ++i) {
    const double r = node_r(*geom, i);
    vsum += A * r * std::log(r) + B * r + C / r;
  }
  const double vmean = vsum / geom->nr;
  const double nu = (tau - 0.5) * CS2;
  const double d = geom->r_outer - geom->r_inner;
  const double de_per_G = vmean * (d / lattice_h(*geom)) / nu * std::sqrt(d / geom->r_inner);
  *G_out = De / de_per_G;
  return LB_OK;
}

lb_status lb_create_geometry(lb_metric metric, const lb_geometry_desc* geom, int batch, lb_precision prec,
                             void* cuda_stream, const lb_allocator* alloc, lb_ctx** out) {
  if (!geom || !out) return fail(nullptr, LB_ERR_ARG, "null argument");
  *out = nullptr;
  const std::string v = validate_geometry(metric, *geom);
  if (!v.empty()) return fail(nullptr, LB_ERR_ARG, v);
  if (batch < 1) return fail(nullptr, LB_ERR_ARG, "need batch >= 1");
  if (prec != LB_FP64 && prec != LB_FP32 && prec != LB_FP16_SHIFTED && prec != LB_BF16_SHIFTED)
    return fail(nullptr, LB_ERR_ARG, "unknown precision");
  if (metric == LB_METRIC_ELLIPSOIDAL_THETA && prec != LB_FP64 && prec != LB_FP32)
    return fail(nullptr, LB_ERR_ARG, "the theta-resolved ellipsoid needs FP64 or FP32 storage");
  if (alloc && (!alloc->alloc || !alloc->free)) return fail(nullptr, LB_ERR_ARG, "allocator needs alloc and free");
  const double total = double(batch) * geom->nr * geom->ntheta * geom->n3;
  if (total >= 4294967295.0) return fail(nullptr, LB_ERR_ARG, "batch * nodes must fit in uint32");
  if (batch > 65535) return fail(nullptr, LB_ERR_ARG, "need batch <= 65535 (one grid row per instance)");
  const int pop_bytes = prec == LB_FP64 ? 8 : prec == LB_FP32 ? 4 : 2;
  const double inst_bytes = double(Q) * geom->nr * geom->ntheta * geom->n3 * pop_bytes;
  if (inst_bytes >= 4294967296.0)
    return fail(nullptr, LB_ERR_ARG, "one instance's populations must stay below 4 GiB (32-bit offsets)");
  if (std::fabs(SQRT10 * SQRT10 - 10.0) > 1e-14 || std::fabs(SQRT10 - std::sqrt(10.0)) > 1e-15)
    return fail(nullptr, LB_ERR_ARG, "internal constant check failed");

  lb_ctx* c = new lb_ctx();
  c->metric = metric;
  c->geom = *geom;
  c->batch = batch;
  c->prec = prec;
  c->K = metric == LB_METRIC_FLAT ? KFLAT
         : metric == LB_METRIC_CYLINDRICAL ? KCYL
         : metric == LB_METRIC_ELLIPSOIDAL ? KELL
                                           : KELT;
  if (alloc) {
    c->alloc = *alloc;
    c->has_alloc = true;
  }
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, LB_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return fail(nullptr, LB_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    c->own_stream = true;
  }
  auto bail = [&](lb_status s, const std::string& m) {
    std::string msg = m;
    free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return fail(nullptr, s, msg);
  };

  c->host_geo = evaluate_geometry(metric, *geom);
  const std::string sp = check_sparsity(c->host_geo, *geom, c->K);
  if (!sp.empty()) return bail(LB_ERR_ARG, "geometry does not fit the kernel: " + sp);

  Dims& d = c->dims;
  d.nr = geom->nr;
  d.nt = geom->ntheta;
  d.n3 = geom->n3;
  d.ncell = geom->nr * geom->ntheta * geom->n3;
  d.periodic3 = geom->periodic3 ? 1 : 0;
  d.wall_eq = geom->wall == LB_WALL_EQUILIBRIUM ? 1 : 0;
  d.batch = batch;
  d.geo_rows3 = c->K == KELL ? geom->n3 : c->K == KELT ? geom->ntheta * geom->n3 : 1;
  d.geo_theta = c->K == KELT ? 1 : 0;
  d.div_ncell = FastDiv::make(uint32_t(d.ncell));
  d.div_n3 = FastDiv::make(uint32_t(d.n3));
  d.div_nt = FastDiv::make(uint32_t(d.nt));
  c->ncell = size_t(d.ncell);
  c->state_elems = size_t(batch) * Q * c->ncell;
  c->elem_bytes = prec == LB_FP64 ? 8 : prec == LB_FP32 ? 4 : 2;

  const size_t nrows = size_t(geom->nr) * d.geo_rows3;
  const size_t nrow64 = geometry_rows(metric, *geom);
  c->nblk = int(std::min<size_t>(1024, (c->ncell + 255) / 256));
  c->f[0] = dalloc(c, c->state_elems * c->elem_bytes);
  c->f[1] = dalloc(c, c->state_elems * c->elem_bytes);
  c->geo_real = dalloc(c, geo_arrays_count(c->K) * nrows * (prec == LB_FP64 ? sizeof(double) : sizeof(float)));
  c->geo64 = static_cast<double*>(dalloc(c, nrow64 * 4 * sizeof(double)));
  c->sqrtg = static_cast<double*>(dalloc(c, nrow64 * sizeof(double)));
  c->base_uth = static_cast<double*>(dalloc(c, size_t(batch) * geom->nr * sizeof(double)));
  c->ini = static_cast<InitInst*>(dalloc(c, size_t(batch) * sizeof(InitInst)));
  c->inst = dalloc(c, size_t(batch) * sizeof(InstParams<double>));
  c->rho_s = static_cast<double*>(dalloc(c, size_t(batch) * c->ncell * sizeof(double)));
  c->u_s = static_cast<double*>(dalloc(c, size_t(batch) * 3 * c->ncell * sizeof(double)));
  c->rowmean = static_cast<double*>(dalloc(c, size_t(batch) * geom->nr * geom->ntheta * sizeof(double)));
  c->partial = static_cast<double*>(dalloc(c, size_t(batch) * c->nblk * DIAG_NQ * sizeof(double)));
  c->diag_out = static_cast<double*>(dalloc(c, size_t(batch) * DIAG_NQ * sizeof(double)));
  c->flag = static_cast<int*>(dalloc(c, sizeof(int)));
  d.st_rows3 = c->K == KELL ? d.geo_rows3 : (d.periodic3 ? 1 : 7);
  if (c->elem_bytes == 2) {
    c->ref_tab = static_cast<float*>(dalloc(c, size_t(batch) * Q * nrows * sizeof(float)));
    c->st_tab = static_cast<float4*>(
        dalloc(c, size_t(batch) * ST_K * size_t(geom->nr) * size_t(d.st_rows3) * sizeof(float4)));
    if (!c->ref_tab || !c->st_tab) return bail(LB_ERR_CUDA, "device allocation failed");
    d.ref = c->ref_tab;
    d.st = c->st_tab;
  }
  if (!c->f[0] || !c->f[1] || !c->geo_real || !c->geo64 || !c->sqrtg || !c->base_uth || !c->ini ||
      !c->inst || !c->rho_s || !c->u_s || !c->rowmean || !c->partial || !c->diag_out || !c->flag)
    return bail(LB_ERR_CUDA, "device allocation failed");

  // geometry tables
  std::vector<double> g64(nrow64 * 4), sg(nrow64);
  for (size_t k = 0; k < nrow64; ++k) {
    const double* r = &c->host_geo[k * LB_GEO_STRIDE];
    g64[4 * k + 0] = r[GEO_SQRTG];
    g64[4 * k + 1] = r[GEO_SPEED];
    g64[4 * k + 2] = r[GEO_WA];
    g64[4 * k + 3] = r[GEO_WOMEGA];
    sg[k] = r[GEO_SQRTG];
  }
  e = cudaMemcpyAsync(c->geo64, g64.data(), g64.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->sqrtg, sg.data(), sg.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    if (prec == LB_FP64) {  // FP64 tables for the FP64 path, FP32 for the others
      auto t = geo_host_tables<double>(c->host_geo, *geom, c->K);
      e = cudaMemcpyAsync(c->geo_real, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      geo_arrays(static_cast<double*>(c->geo_real), nrows, c->geo_d);
    } else {
      auto t = geo_host_tables<float>(c->host_geo, *geom, c->K);
      e = cudaMemcpyAsync(c->geo_real, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      geo_arrays(static_cast<float*>(c->geo_real), nrows, c->geo_f);
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return bail(LB_ERR_CUDA, std::string("geometry upload: ") + cudaGetErrorString(e));
  if (prec == LB_FP32 && c->K != KELT && geom->wall == LB_WALL_BOUNCEBACK && tma_step_supported(d) &&
      tensor_map_bytes() <= sizeof(c->tmap[0]))
    c->tma_ok = make_state_tensor_map(c->tmap[0], static_cast<const float*>(c->f[0]), d) == cudaSuccess &&
                make_state_tensor_map(c->tmap[1], static_cast<const float*>(c->f[1]), d) == cudaSuccess;
  *out = c;
  return LB_OK;
}

lb_status lb_init(lb_ctx* c, const lb_params* p) {
  if (!c || !p) return fail(c, LB_ERR_ARG, "null argument");
  lb_status s = upload_params(c, p);
  if (s != LB_OK) return s;
  const lb_geometry_desc& g = c->geom;
  std::vector<double> base(size_t(c->batch) * g.nr, 0.0);
  bool any_base = false;
  const bool eqw = g.wall == LB_WALL_EQUILIBRIUM;
  for (int b = 0; b < c->batch; ++b) {
    if (!p[b].init_base_flow) continue;
    any_base = true;
    if (g.dtheta_scale != 1.0 || c->metric == LB_METRIC_ELLIPSOIDAL)
      return fail(c, LB_ERR_ARG, "base flow needs FLAT or CYLINDRICAL with dtheta_scale = 1");
    const double nu = (p[b].tau - 0.5) * CS2;
    for (int i = 0; i < g.nr; ++i) {
      if (c->metric == LB_METRIC_FLAT) {
        // plane Poiseuille between walls at -1/2 and nr - 1/2, or on the
        // wall nodes 0 and nr - 1 (lattice units)
        base[size_t(b) * g.nr + i] = eqw ? p[b].force_G / (2.0 * nu) * i * (g.nr - 1 - i)
                                         : p[b].force_G / (2.0 * nu) * (i + 0.5) * (g.nr - 0.5 - i);
      } else {
        double A, B, C;
        curved_poiseuille(g, p[b].tau, p[b].force_G, &A, &B, &C);
        const double r = node_r(g, i);
        base[size_t(b) * g.nr + i] = (A * r * std::log(r) + B * r + C / r) / r;
      }
    }
  }
  std::vector<InitInst> ini(c->batch);
  for (int b = 0; b < c->batch; ++b) {
    ini[b].seed = p[b].seed;
    ini[b].amp = p[b].noise_amp;
  }
  LB_CUDA(c, cudaMemcpyAsync(c->base_uth, base.data(), base.size() * sizeof(double), cudaMemcpyHostToDevice,
                             c->stream));
  LB_CUDA(c, cudaMemcpyAsync(c->ini, ini.data(), ini.size() * sizeof(InitInst), cudaMemcpyHostToDevice,
                             c->stream));
  c->cur = 0;
  if (c->ref_tab) {
    LB_CUDA(c, launch_ref_table(c->K, c->ref_tab, c->geo_f, c->sqrtg, any_base ? c->base_uth : nullptr, nullptr,
                                nullptr, c->dims, c->ref_mode, c->stream));
    LB_CUDA(c, launch_stream_table(int(c->prec), c->K, c->st_tab, c->ref_tab,
                                   static_cast<const InstParams<float>*>(c->inst), c->f[0], c->dims, c->stream));
  }
  LB_CUDA(c, launch_init(int(c->prec), c->K, c->f[0], geo_ptr(c), c->sqrtg,
                         any_base ? c->base_uth : nullptr, c->ini, nullptr, nullptr, c->dims, c->stream));
  return reset_after_init(c);
}

lb_status lb_init_fields(lb_ctx* c, const lb_params* p, const double* rho, const double* u, int on_device) {
  if (!c || !p || !rho || !u) return fail(c, LB_ERR_ARG, "null argument");
  lb_status s = upload_params(c, p);
  if (s != LB_OK) return s;
  const size_t n = size_t(c->batch) * c->ncell;
  const double* drho = rho;
  const double* du = u;
  if (!on_device) {
    LB_CUDA(c, cudaMemcpyAsync(c->rho_s, rho, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(c, cudaMemcpyAsync(c->u_s, u, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    drho = c->rho_s;
    du = c->u_s;
  }
  c->cur = 0;
  if (c->ref_tab) {
    LB_CUDA(c, launch_ref_table(c->K, c->ref_tab, c->geo_f, c->sqrtg, nullptr, drho, du, c->dims, c->ref_mode,
                                c->stream));
    LB_CUDA(c, launch_stream_table(int(c->prec), c->K, c->st_tab, c->ref_tab,
                                   static_cast<const InstParams<float>*>(c->inst), c->f[0], c->dims, c->stream));
  }
  LB_CUDA(c, launch_init(int(c->prec), c->K, c->f[0], geo_ptr(c), c->sqrtg, nullptr, c->ini,
                         drho, du, c->dims, c->stream));
  return reset_after_init(c);
}

lb_status lb_step(lb_ctx* c, long long n) {
  lb_status s;
  if (!usable(c, &s)) return s;
  if (n < 0) return fail(c, LB_ERR_ARG, "need n >= 0");
  if (c->use_graph && c->check_every == 0 && n >= 3) {
    if (c->cur != 0) {  // the captured pair starts from buffer 0
      s = launch_step_once(c);
      if (s != LB_OK) return s;
      ++c->step;
      --n;
    }
    if (resolved_kernel(c) == 5) {  // tiles are uploaded outside the capture
      s = ctx_tiled_prepare(c);
      if (s != LB_OK) return s;
    }
    // the captured kernels depend on the resolved step kernel and on whether
    // an instance uses the half-force variant (both can change with lb_init)
    const int gk = 2 * resolved_kernel(c) + (c->any_shift ? 1 : 0);
    if (!c->graph || c->graph_threads != c->block_threads || c->graph_kernel != gk) {
      if (c->graph) cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
      cudaGraph_t g = nullptr;
      LB_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      lb_status s1 = launch_step_once(c);
      lb_status s2 = s1 == LB_OK ? launch_step_once(c) : s1;
      cudaError_t e = cudaStreamEndCapture(c->stream, &g);
      if (s2 != LB_OK) return s2;
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&c->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
      c->graph_threads = c->block_threads;
      c->graph_kernel = gk;
    }
    for (long long i = 0; i + 1 < n; i += 2) {
      LB_CUDA(c, cudaGraphLaunch(c->graph, c->stream));
      c->step += 2;
    }
    n &= 1;
  }
  for (long long i = 0; i < n; ++i) {
    s = launch_step_once(c);
    if (s != LB_OK) return s;
    ++c->step;
    if (c->check_every > 0 && (c->step % c->check_every) == 0) {
      s = check_flag(c);
      if (s != LB_OK) return s;
    }
  }
  return LB_OK;
}

lb_status lb_macros(lb_ctx* c, double* rho, double* u, int on_device) {
  lb_status s;
  if (!usable(c, &s)) return s;
  const size_t n = size_t(c->batch) * c->ncell;
  double* drho = on_device ? rho : (rho ? c->rho_s : nullptr);
  double* du = on_device ? u : (u ? c->u_s : nullptr);
  LB_CUDA(c, launch_macros(int(c->prec), c->K, c->f[c->cur], drho, du, c->dims, c->stream));
  if (!on_device) {
    if (rho) LB_CUDA(c, cudaMemcpyAsync(rho, c->rho_s, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (u) LB_CUDA(c, cudaMemcpyAsync(u, c->u_s, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return LB_OK;
}

lb_status lb_diagnostics(lb_ctx* c, lb_diag* out) {
  lb_status s;
  if (!usable(c, &s)) return s;
  if (!out) return fail(c, LB_ERR_ARG, "null argument");
  LB_CUDA(c, launch_macros(int(c->prec), c->K, c->f[c->cur], c->rho_s, c->u_s, c->dims, c->stream));
  LB_CUDA(c, launch_diag(c->rho_s, c->u_s, c->rowmean, c->geo64, c->dims, c->partial, c->nblk, c->diag_out,
                         c->stream));
  std::vector<double> h(size_t(c->batch) * DIAG_NQ);
  LB_CUDA(c, cudaMemcpyAsync(h.data(), c->diag_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  const lb_geometry_desc& g = c->geom;
  const double R = curvature_radius(c->metric, g);
  const double d = g.r_outer - g.r_inner;
  const double width = d / lattice_h(g);  // channel width in lattice units
  const double N = double(c->ncell);
  for (int b = 0; b < c->batch; ++b) {
    const double* q = &h[size_t(b) * DIAG_NQ];
    lb_diag& o = out[b];
    o.mass_rho_prime = q[0];
    o.mass_physical = q[1];
    o.mean_v_theta = q[2] / q[3];
    const double nu = (c->tau[b] - 0.5) * CS2;
    o.dean = R > 0.0 ? o.mean_v_theta * width / nu * std::sqrt(d / R) : 0.0;
    o.mean_vorticity = q[4] / q[3];
    o.vortex_amp = std::sqrt(q[5] / N);
    o.vortex_amp_x3 = std::sqrt(q[6] / N);
    o.max_speed = q[7];
    o.nonfinite = (long long)q[8];
    o.step = c->step;
  }
  return LB_OK;
}

lb_status lb_velocity_change(lb_ctx* c, double* u_prev, double* change, double* umax) {
  lb_status s;
  if (!usable(c, &s)) return s;
  if (!u_prev || !change) return fail(c, LB_ERR_ARG, "null argument");
  // partial maxima reuse the observables' partial buffer (batch * nblk * DIAG_NQ >= batch * nblk * 2)
  LB_CUDA(c, launch_macros(int(c->prec), c->K, c->f[c->cur], nullptr, c->u_s, c->dims, c->stream));
  LB_CUDA(c, launch_residual(c->u_s, u_prev, c->dims, c->partial, c->nblk, c->diag_out, c->stream));
  std::vector<double> h(2 * size_t(c->batch));
  LB_CUDA(c, cudaMemcpyAsync(h.data(), c->diag_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int b = 0; b < c->batch; ++b) {
    change[b] = h[2 * b];
    if (umax) umax[b] = h[2 * b + 1];
  }
  return LB_OK;
}

lb_status lb_get_populations(lb_ctx* c, double* f, int on_device) {
  lb_status s;
  if (!usable(c, &s)) return s;
  if (!f) return fail(c, LB_ERR_ARG, "null argument");
  const size_t n = c->state_elems;
  if (c->prec == LB_FP64) {
    LB_CUDA(c, cudaMemcpyAsync(f, c->f[c->cur], n * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  } else {
    double* dst = f;
    if (!on_device) {
      if (!c->dbl_stage) c->dbl_stage = static_cast<double*>(dalloc(c, n * sizeof(double)));
      if (!c->dbl_stage) return fail(c, LB_ERR_CUDA, "staging allocation failed");
      dst = c->dbl_stage;
    }
    LB_CUDA(c, launch_convert(int(c->prec), 1, c->f[c->cur], dst, n, c->dims, c->stream));
    if (!on_device)
      LB_CUDA(c, cudaMemcpyAsync(f, dst, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  return LB_OK;
}

lb_status lb_capture_reference(lb_ctx* c) {
  lb_status s;
  if (!usable(c, &s)) return s;
  if (!c->ref_tab) return fail(c, LB_ERR_ARG, "only the 2-byte storage formats have a reference");
  const size_t n = c->state_elems;
  if (!c->dbl_stage) c->dbl_stage = static_cast<double*>(dalloc(c, n * sizeof(double)));
  if (!c->dbl_stage) return fail(c, LB_ERR_CUDA, "staging allocation failed");
  // decode with the old table, average, re-encode with the new one
  LB_CUDA(c, launch_convert(int(c->prec), 1, c->f[c->cur], c->dbl_stage, n, c->dims, c->stream));
  LB_CUDA(c, launch_ref_from_state(c->dbl_stage, c->ref_tab, c->dims, c->stream));
  LB_CUDA(c, launch_stream_table(int(c->prec), c->K, c->st_tab, c->ref_tab,
                                 static_cast<const InstParams<float>*>(c->inst), c->f[0], c->dims, c->stream));
  LB_CUDA(c, launch_convert(int(c->prec), 0, c->f[c->cur], c->dbl_stage, n, c->dims, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  return LB_OK;
}

lb_status lb_set_populations(lb_ctx* c, const double* f, int on_device) {
  if (!c || !f) return fail(c, LB_ERR_ARG, "null argument");
  if (c->tau.empty()) return fail(c, LB_ERR_STATE, "call lb_init once first (parameters)");
  const size_t n = c->state_elems;
  c->cur = 0;
  if (c->prec == LB_FP64) {
    LB_CUDA(c, cudaMemcpyAsync(c->f[0], f, n * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  } else {
    const double* src = f;
    if (!on_device) {
      if (!c->dbl_stage) c->dbl_stage = static_cast<double*>(dalloc(c, n * sizeof(double)));
      if (!c->dbl_stage) return fail(c, LB_ERR_CUDA, "staging allocation failed");
      LB_CUDA(c, cudaMemcpyAsync(c->dbl_stage, f, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      src = c->dbl_stage;
    }
    LB_CUDA(c, launch_convert(int(c->prec), 0, c->f[0], const_cast<double*>(src), n, c->dims, c->stream));
  }
  const long long keep = c->step;
  lb_status s = reset_after_init(c);
  c->step = keep;
  return s;
}

size_t lb_state_bytes(const lb_ctx* c) { return c ? c->state_elems * c->elem_bytes : 0; }

lb_status lb_get_state(lb_ctx* c, void* buf, size_t bytes, int on_device) {
  lb_status s;
  if (!usable(c, &s)) return s;
  if (!buf || bytes != lb_state_bytes(c)) return fail(c, LB_ERR_ARG, "buffer size must be lb_state_bytes()");
  LB_CUDA(c, cudaMemcpyAsync(buf, c->f[c->cur], bytes,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  LB_CUDA(c, cudaStreamSynchronize(c->stream));
  return LB_OK;
}

lb_status lb_set_state(lb_ctx* c, const void* buf, size_t bytes, int on_device) {
  if (!c || !buf) return fail(c, LB_ERR_ARG, "null argument");
  if (bytes != lb_state_bytes(c)) return fail(c, LB_ERR_ARG, "buffer size must be lb_state_bytes()");
  if (c->tau.empty()) return fail(c, LB_ERR_STATE, "call lb_init once first (parameters)");
  c->cur = 0;
  LB_CUDA(c, cudaMemcpyAsync(c->f[0], buf, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->stream));
  const long long keep = c->step;
  lb_status s = reset_after_init(c);
  c->step = keep;
  return s;
}

lb_status lb_set_option(lb_ctx* c, int option, long long value) {
  if (!c) return fail(nullptr, LB_ERR_ARG, "null context");
  switch (option) {
    case LB_OPT_CHECK_EVERY:
      if (value < 0) return fail(c, LB_ERR_ARG, "need k >= 0");
      c->check_every = value;
      return LB_OK;
    case LB_OPT_BLOCK_THREADS:
      if (value < 64 || value > 256 || value % 32) return fail(c, LB_ERR_ARG, "need 64..256, multiple of 32");
      c->block_threads = int(value);
      return LB_OK;
    case LB_OPT_USE_GRAPH:
      c->use_graph = value ? 1 : 0;
      return LB_OK;
    case LB_OPT_STEP_KERNEL:
      if (value < 0 || value > 5 || value == 3)
        return fail(c, LB_ERR_ARG, "need 0 (auto), 1 (plain), 2 (TMA), 4 (region split) or 5 (tiled)");
      if (c->K == KELT && value > 1)
        return fail(c, LB_ERR_ARG, "the theta-resolved ellipsoid runs the plain step kernel only");
      if (value == 4 && (!c->geom.periodic3 || c->geom.wall != LB_WALL_BOUNCEBACK))
        return fail(c, LB_ERR_ARG, "the region-split step kernel needs a periodic x3 axis and bounce-back walls");
      if (value == 2 && !c->tma_ok)
        return fail(c, LB_ERR_ARG, "the TMA step kernel needs FP32 and n3 in {128, 256}");
      c->step_kernel = int(value);
      return LB_OK;
    case LB_OPT_STORAGE_REFERENCE:
      if (value < 0 || value > 1) return fail(c, LB_ERR_ARG, "need 0 (weights) or 1 (initial rows)");
      if (c->elem_bytes != 2) return fail(c, LB_ERR_ARG, "only the 2-byte storage formats have a reference");
      if (int(value) != c->ref_mode) c->initialized = false;  // the stored deviations change meaning
      c->ref_mode = int(value);
      return LB_OK;
    default:
      return fail(c, LB_ERR_ARG, "unknown option");
  }
}

long long lb_step_count(const lb_ctx* c) { return c ? c->step : -1; }

lb_status lb_autotune(lb_ctx* c, int steps_per_trial, lb_tune* best, lb_tune* trials, int max_trials,
                      int* n_trials) {
  lb_status s;
  if (!usable(c, &s)) return s;
  if (steps_per_trial < 1) return fail(c, LB_ERR_ARG, "need steps_per_trial >= 1");
  if (max_trials < 0 || (max_trials > 0 && !trials)) return fail(c, LB_ERR_ARG, "bad trials buffer");
  std::vector<lb_tune> cand;
  if (c->prec == LB_FP64)
    for (int t : {64, 128, 192, 256}) cand.push_back({t, 1, 0, 0.0});
  else
    for (int t : {64, 96, 128}) cand.push_back({t, 1, 0, 0.0});
  if (!c->any_shift && c->K != KELT) {  // the half-force variant and KELT have the plain kernel only
    if (c->geom.periodic3 && c->geom.wall == LB_WALL_BOUNCEBACK)
      for (int t : {64, 96, 128}) cand.push_back({t, 4, 0, 0.0});
    for (int t : {64, 96, 128}) cand.push_back({t, 5, 0, 0.0});
    if (c->tma_ok) cand.push_back({0, 2, 0, 0.0});  // the TMA kernel fixes its own block shape
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LB_CUDA(c, cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(c, e, "cudaEventCreate");
  }
  const int keep_threads = c->block_threads;
  lb_status st = LB_OK;
  for (lb_tune& k : cand) {
    c->block_threads = k.block_threads > 0 ? k.block_threads : keep_threads;
    c->step_kernel = k.schedule;
    for (int i = 0; i <= steps_per_trial && st == LB_OK; ++i) {  // step 0 is the untimed warm-up
      if (i == 1 && (e = cudaEventRecord(e0, c->stream)) != cudaSuccess) st = cuda_fail(c, e, "cudaEventRecord");
      if (st == LB_OK) st = launch_step_once(c);
      if (st == LB_OK) ++c->step;
    }
    if (st == LB_OK && (e = cudaEventRecord(e1, c->stream)) != cudaSuccess) st = cuda_fail(c, e, "cudaEventRecord");
    if (st == LB_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) st = cuda_fail(c, e, "cudaEventSynchronize");
    float ms = 0.f;
    if (st == LB_OK && (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
      st = cuda_fail(c, e, "cudaEventElapsedTime");
    if (st != LB_OK) break;
    k.ms_per_step = double(ms) / steps_per_trial;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LB_OK) return st;
  size_t ib = 0;
  for (size_t i = 1; i < cand.size(); ++i)
    if (cand[i].ms_per_step < cand[ib].ms_per_step) ib = i;
  if (cand[ib].block_threads == 0) cand[ib].block_threads = keep_threads;
  for (lb_tune& k : cand) {
    if (k.block_threads == 0) k.block_threads = keep_threads;
  }
  c->block_threads = cand[ib].block_threads;
  c->step_kernel = cand[ib].schedule;
  if (best) *best = cand[ib];
  const int n = int(cand.size());
  for (int i = 0; i < n && i < max_trials; ++i) trials[i] = cand[i];
  if (n_trials) *n_trials = n;
  if (c->check_every > 0) return check_flag(c);
  return LB_OK;
}

void lb_destroy(lb_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  lb_batch_destroy(c->tiles);
  if (c->aux) {
    cudaStreamSynchronize(c->aux);
    cudaStreamDestroy(c->aux);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  free_all(c);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* lb_last_error(const lb_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

}  // extern "C"
