// Host-side state of one context (lb_ctx of include/lbgm.h), shared by the
// translation units that implement the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/lbgm.h"
#include "kernels.cuh"

struct lb_ctx {
  lb_metric metric;
  lb_geometry_desc geom;
  int batch = 0;
  lb_precision prec;
  int K = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  lb_allocator alloc{};
  bool has_alloc = false;
  std::vector<std::pair<void*, size_t>> allocations;

  lbgm::Dims dims{};
  size_t ncell = 0;         // per instance
  size_t state_elems = 0;   // batch * Q * ncell
  size_t elem_bytes = 0;
  void* f[2] = {nullptr, nullptr};
  int cur = 0;

  void* geo_real = nullptr;        // 9 arrays of nrows in the compute precision
  lbgm::GeoDev<double> geo_d{};
  lbgm::GeoDev<float> geo_f{};
  double* geo64 = nullptr;         // [nr * n3][4]: sqrtg, speed, wA, wOmega
  double* sqrtg = nullptr;         // [nr * n3]
  double* base_uth = nullptr;      // [batch * nr]
  lbgm::InitInst* ini = nullptr;         // [batch]
  void* inst = nullptr;            // InstParams<Real>[batch]
  double* rho_s = nullptr;         // macros scratch [batch * N]
  double* u_s = nullptr;           // [batch * 3 * N]
  double* rowmean = nullptr;       // [batch * nr * nt]
  double* partial = nullptr;       // [batch * nblk * DIAG_NQ]
  double* diag_out = nullptr;      // [batch * DIAG_NQ]
  double* dbl_stage = nullptr;     // conversion staging (FP32 populations), lazily allocated
  float* ref_tab = nullptr;        // 2-byte storage: reference populations [batch][Q][rows]
  float4* st_tab = nullptr;        // 2-byte storage: stream table [batch][ST_K][stream rows]
  int ref_mode = 1;                // LB_OPT_STORAGE_REFERENCE
  int* flag = nullptr;
  int nblk = 0;

  std::vector<double> tau;          // per instance, host copy
  std::vector<double> host_geo;     // lb_geometry_eval rows
  long long step = 0;
  bool initialized = false;
  bool poisoned = false;
  std::string err;

  long long check_every = 0;
  int block_threads = 128;
  int use_graph = 0;
  cudaGraphExec_t graph = nullptr;   // two steps, buffer 0 -> 1 -> 0
  int graph_threads = 0;
  int graph_kernel = -1;             // 2 x resolved step kernel + any_shift of the captured graph
  int step_kernel = 0;               // LB_OPT_STEP_KERNEL
  bool any_shift = false;            // an instance uses the half-force velocity (old_forcing 2)
  lb_batch* tiles = nullptr;         // private single-member batch of the tiled step
  cudaStream_t aux = nullptr;        // second stream of the region-split step
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool tma_ok = false;               // tensor maps built for both buffers
  alignas(64) unsigned char tmap[2][128];
};

namespace lbgm {

// Record an error on the context (or the thread's last error when c is
// NULL); CUDA and non-finite errors poison the context.
lb_status ctx_fail(lb_ctx* c, lb_status s, const std::string& msg);
// False (with *s set) unless c is non-NULL, initialised and not poisoned.
bool ctx_usable(lb_ctx* c, lb_status* s);
// Tiled step (LB_OPT_STEP_KERNEL 5): prepare the tiles (outside captures),
// then launch one step of them.
lb_status ctx_tiled_prepare(lb_ctx* c);
lb_status ctx_tiled_launch(lb_ctx* c);

}  // namespace lbgm
