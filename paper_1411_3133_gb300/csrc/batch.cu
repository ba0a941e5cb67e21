// Batches of contexts of different geometry (lb_batch_* of include/lbgm.h).
//
// Every instance of every member becomes one ListInst record; instances are
// grouped by metric kind and each group gets four work lists: tiles of
// interior nodes (instance, first node, count) and, per wall-node class,
// tiles of wall nodes (instance, first index into a list of wall-node
// indices, count) -- nodes near an r-wall only, near an x3-wall only, and
// the rest (corners, equilibrium walls, short axes). One batch step is one
// k_step_list launch per non-empty list; the lists after the first run on
// forked streams, so the wall-node kernels (bound by instruction fetch)
// overlap the interior kernels (bound by memory).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/lbgm.h"
#include "ctx.h"
#include "launch.h"

using namespace lbgm;

namespace {

constexpr int kMaxGroups = 3;  // flat, cylinder, ellipsoid
constexpr int kLists = 4;                  // interior tiles, three wall-node classes
constexpr int kMaxLanes = kLists * kMaxGroups;

struct Group {
  int K = 0;
  int ninst = 0;
  int nwork[kLists] = {};        // interior tiles, wall-node tiles per class
  size_t inst_off = 0;           // byte offset of the ListInst records in dmem
  size_t work_off[kLists] = {};  // byte offsets of the int4 tiles in dmem
  size_t cells_off = 0;         // byte offset of the wall-node indices in dmem
  int blocks_per_sm = 0;        // occupancy of the interior kernel at the built block size
};

// Wall-node class of node (i_r, i_3) near a wall (lists 1..3): 1 within 3
// layers of an r-wall only, 2 of an x3-wall only -- each with one
// compile-time fold per layer, which needs bounce-back walls and the walled
// axis at least 7 nodes long -- and 3 the rest (the general wall rule).
int wall_class(const Dims& d, int ir, int i3) {
  const bool near_r = ir < 3 || ir > d.nr - 4;
  const bool near_3 = !d.periodic3 && (i3 < 3 || i3 > d.n3 - 4);
  if (d.wall_eq) return 3;
  if (near_r && !near_3 && d.nr >= 7) return 1;
  if (near_3 && !near_r && d.n3 >= 7) return 2;
  return 3;
}

// Tiles of one instance (group-local index li): runs of interior nodes (no
// wall within 3 nodes) as (li, first node, count), counts <= tile, into
// lists[0]; the wall nodes' indices appended to cells[c - 1] by class c and
// tiled as (li, first index into cells[c - 1], count), counts <= wall_tile,
// into lists[c].
void instance_tiles(const Dims& d, int li, int tile, int wall_tile, std::vector<int4> (&lists)[kLists],
                    std::vector<int> (&cells)[kLists - 1]) {
  const int nr = d.nr, nt = d.nt, n3 = d.n3;
  auto inner_r = [&](int ir) { return ir >= 3 && ir <= nr - 4; };
  auto inner_3 = [&](int i3) { return d.periodic3 || (i3 >= 3 && i3 <= n3 - 4); };
  int run_start = -1;
  auto close_run = [&](int end) {
    for (int a = run_start; a < end; a += tile) lists[0].push_back(make_int4(li, a, std::min(tile, end - a), 0));
    run_start = -1;
  };
  size_t w0[kLists - 1];
  for (int c = 0; c < kLists - 1; ++c) w0[c] = cells[c].size();
  for (int ir = 0; ir < nr; ++ir)
    for (int it = 0; it < nt; ++it)
      for (int i3 = 0; i3 < n3; ++i3) {
        const int cell = (ir * nt + it) * n3 + i3;
        if (inner_r(ir) && inner_3(i3)) {
          if (run_start < 0) run_start = cell;
        } else {
          if (run_start >= 0) close_run(cell);
          cells[wall_class(d, ir, i3) - 1].push_back(cell);
        }
      }
  if (run_start >= 0) close_run(nr * nt * n3);
  for (int c = 0; c < kLists - 1; ++c)
    for (size_t a = w0[c]; a < cells[c].size(); a += size_t(wall_tile))
      lists[c + 1].push_back(
          make_int4(li, int(a), int(std::min(size_t(wall_tile), cells[c].size() - a)), 0));
}

}  // namespace

struct lb_batch {
  std::vector<lb_ctx*> m;
  lb_precision prec = LB_FP32;
  cudaStream_t stream = nullptr;
  int device = 0;
  int nsm = 0;
  long long nodes = 0;

  // work list, valid while built
  bool built = false;
  int built_threads = 0;
  int built_tile_blocks = 0;
  std::vector<int> base_cur;  // member buffer parity when the records were written
  int parity = 0;             // batch steps since then, mod 2
  Group g[kMaxGroups];
  int ngroups = 0;
  void* dmem = nullptr;
  size_t dmem_bytes = 0;

  cudaStream_t aux[kMaxLanes - 1] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kMaxLanes - 1] = {};

  int threads = 128;
  int tile_blocks = 1;  // LB_OPT_TILE_BLOCKS: nodes per tile = tile_blocks x threads
  int schedule = 0;
  int use_graph = 0;
  long long check_every = 0;
  cudaGraphExec_t graph = nullptr;  // two batch steps, parity 0 then 1
  int graph_threads = 0;
  int graph_tile_blocks = 0;
  int graph_schedule = -1;

  long long step = 0;
  bool poisoned = false;
  std::string err;
};

namespace {

lb_status bfail(lb_batch* b, lb_status s, const std::string& msg) {
  if (!b) return ctx_fail(nullptr, s, msg);
  b->err = msg;
  if (s == LB_ERR_CUDA) b->poisoned = true;
  return s;
}

lb_status bcuda(lb_batch* b, cudaError_t e, const char* what) {
  return bfail(b, LB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LB_BCUDA(b, call)                                \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return bcuda(b, e_, #call);   \
  } while (0)

void drop_graph(lb_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

template <class S, class R>
ListInst<S, R> record(const lb_ctx* c, int bi, int cur, const GeoDev<R>& geo) {
  ListInst<S, R> r{};
  r.d = c->dims;
  r.d.batch = 1;
  if (c->dims.ref) r.d.ref = c->dims.ref + size_t(bi) * Q * size_t(c->dims.nr) * size_t(c->dims.geo_rows3);
  if (c->dims.st) r.d.st = c->dims.st + size_t(bi) * ST_K * size_t(c->dims.nr) * size_t(c->dims.st_rows3);
  r.geo = geo;
  r.ip = static_cast<const InstParams<R>*>(c->inst) + bi;
  const size_t off = size_t(bi) * Q * c->ncell;
  r.f0 = static_cast<const S*>(c->f[cur]) + off;
  r.f1 = static_cast<S*>(c->f[1 - cur]) + off;
  r.flag = c->flag;
  return r;
}

template <class S, class R>
void append_records(const lb_batch* b, int K, std::vector<unsigned char>& bytes, int* ninst,
                    const GeoDev<R> lb_ctx::*geo_member) {
  for (const lb_ctx* c : b->m) {
    if (c->K != K) continue;
    for (int bi = 0; bi < c->batch; ++bi) {
      const ListInst<S, R> r = record<S, R>(c, bi, c->cur, c->*geo_member);
      const unsigned char* p = reinterpret_cast<const unsigned char*>(&r);
      bytes.insert(bytes.end(), p, p + sizeof(r));
      ++*ninst;
    }
  }
}

int max_threads(lb_precision p) {
  switch (p) {
    case LB_FP64: return step_list_max_threads_f64();
    case LB_FP32: return step_list_max_threads_f32();
    case LB_FP16_SHIFTED: return step_list_max_threads_h16();
    default: return step_list_max_threads_b16();
  }
}

cudaError_t occupancy(lb_precision p, int K, int threads, int* out) {
  switch (p) {
    case LB_FP64: return step_list_occupancy_f64(K, threads, out);
    case LB_FP32: return step_list_occupancy_f32(K, threads, out);
    case LB_FP16_SHIFTED: return step_list_occupancy_h16(K, threads, out);
    default: return step_list_occupancy_b16(K, threads, out);
  }
}

// Write the instance records (with the members' current buffer parity) and
// the tile lists for block size b->threads (tiles of b->tile_blocks blocks'
// worth of nodes), and upload them.
lb_status build(lb_batch* b) {
  drop_graph(b);
  b->built = false;
  std::vector<unsigned char> recs;
  std::vector<int4> tiles[kMaxGroups][kLists];
  std::vector<int> cells[kMaxGroups];
  b->ngroups = 0;
  for (int K : {int(KCYL), int(KELL), int(KFLAT)}) {
    Group gr;
    gr.K = K;
    const size_t before = recs.size();
    switch (b->prec) {
      case LB_FP64: append_records<double, double>(b, K, recs, &gr.ninst, &lb_ctx::geo_d); break;
      case LB_FP32: append_records<float, float>(b, K, recs, &gr.ninst, &lb_ctx::geo_f); break;
      case LB_FP16_SHIFTED: append_records<__half, float>(b, K, recs, &gr.ninst, &lb_ctx::geo_f); break;
      default: append_records<__nv_bfloat16, float>(b, K, recs, &gr.ninst, &lb_ctx::geo_f); break;
    }
    if (gr.ninst == 0) continue;
    gr.inst_off = before;
    // tiles, instance-major; instance ids are local to the group
    const int gi = b->ngroups;
    int local = 0;
    std::vector<int> cls[kLists - 1];
    for (const lb_ctx* c : b->m) {
      if (c->K != K) continue;
      for (int bi = 0; bi < c->batch; ++bi, ++local)
        instance_tiles(c->dims, local, b->threads * b->tile_blocks, b->threads, tiles[gi], cls);
    }
    // one index list per group: the classes one after the other
    for (int c = 0; c < kLists - 1; ++c) {
      const int shift = int(cells[gi].size());
      for (int4& t : tiles[gi][c + 1]) t.y += shift;
      cells[gi].insert(cells[gi].end(), cls[c].begin(), cls[c].end());
    }
    for (int m = 0; m < kLists; ++m) gr.nwork[m] = int(tiles[gi][m].size());
    cudaError_t e = occupancy(b->prec, K, b->threads, &gr.blocks_per_sm);
    if (e != cudaSuccess) return bcuda(b, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    b->g[b->ngroups++] = gr;
  }
  // layout: records | per group: interior tiles, wall tiles, wall-node indices
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t off = al(recs.size());
  for (int i = 0; i < b->ngroups; ++i) {
    for (int m = 0; m < kLists; ++m) {
      b->g[i].work_off[m] = off;
      off = al(off + tiles[i][m].size() * sizeof(int4));
    }
    b->g[i].cells_off = off;
    off = al(off + cells[i].size() * sizeof(int));
  }
  const size_t need = off;
  if (need > b->dmem_bytes) {
    if (b->dmem) cudaFree(b->dmem);
    b->dmem = nullptr;
    b->dmem_bytes = 0;
    LB_BCUDA(b, cudaMalloc(&b->dmem, need));
    b->dmem_bytes = need;
  }
  unsigned char* base = static_cast<unsigned char*>(b->dmem);
  LB_BCUDA(b, cudaMemcpyAsync(base, recs.data(), recs.size(), cudaMemcpyHostToDevice, b->stream));
  for (int i = 0; i < b->ngroups; ++i) {
    for (int m = 0; m < kLists; ++m)
      if (!tiles[i][m].empty())
        LB_BCUDA(b, cudaMemcpyAsync(base + b->g[i].work_off[m], tiles[i][m].data(),
                                    tiles[i][m].size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
    if (!cells[i].empty())
      LB_BCUDA(b, cudaMemcpyAsync(base + b->g[i].cells_off, cells[i].data(), cells[i].size() * sizeof(int),
                                  cudaMemcpyHostToDevice, b->stream));
  }
  LB_BCUDA(b, cudaStreamSynchronize(b->stream));  // the host vectors go out of scope
  b->base_cur.resize(b->m.size());
  for (size_t i = 0; i < b->m.size(); ++i) b->base_cur[i] = b->m[i]->cur;
  b->parity = 0;
  b->built_threads = b->threads;
  b->built_tile_blocks = b->tile_blocks;
  b->built = true;
  return LB_OK;
}

// The records hold f0 = the buffer each member read when they were written;
// they stay valid while every member has taken exactly the batch's steps.
bool records_current(const lb_batch* b) {
  if (!b->built || b->built_threads != b->threads || b->built_tile_blocks != b->tile_blocks) return false;
  for (size_t i = 0; i < b->m.size(); ++i)
    if (b->m[i]->cur != (b->base_cur[i] ^ b->parity)) return false;
  return true;
}

// One work list of one group (m = 0: interior tiles, 1..3: wall-node tiles
// of class m) on stream s.
cudaError_t launch_lane(const lb_batch* b, const Group& gr, int m, cudaStream_t s) {
  const unsigned char* base = static_cast<const unsigned char*>(b->dmem);
  const void* insts = base + gr.inst_off;
  const int* cells = reinterpret_cast<const int*>(base + gr.cells_off);
  const int grid = b->schedule == 1 ? std::max(1, gr.blocks_per_sm) * b->nsm : 0;
  const int4* work = reinterpret_cast<const int4*>(base + gr.work_off[m]);
  const int sel = m | (m == 0 && b->built_tile_blocks > 1 ? 4 : 0);  // list class; multi-block tiles
  switch (b->prec) {
    case LB_FP64:
      return launch_step_list_f64(gr.K, sel, insts, work, gr.nwork[m], cells, b->threads, grid, b->parity, s);
    case LB_FP32:
      return launch_step_list_f32(gr.K, sel, insts, work, gr.nwork[m], cells, b->threads, grid, b->parity, s);
    case LB_FP16_SHIFTED:
      return launch_step_list_h16(gr.K, sel, insts, work, gr.nwork[m], cells, b->threads, grid, b->parity, s);
    default:
      return launch_step_list_b16(gr.K, sel, insts, work, gr.nwork[m], cells, b->threads, grid, b->parity, s);
  }
}

// One batch step. Every non-empty work list is a lane of its own: they read
// the same buffer and write disjoint nodes, so they run side by side -- the
// wall-node kernels, bound by instruction fetch, beside the interior
// kernels, bound by memory. The first lane (an interior list) goes on the
// batch stream first; the others are forked after it, interior lists before
// wall-node lists, and joined back (measured: +9 % on 24 four-wall
// double-curved channels; launching the wall-node lists first was slower).
lb_status step_once(lb_batch* b) {
  int lg[kMaxLanes], lm[kMaxLanes], n = 0;
  for (int m = 0; m < kLists; ++m) {
    for (int i = 0; i < b->ngroups; ++i)
      if (b->g[i].nwork[m] > 0) {
        lg[n] = i;
        lm[n] = m;
        ++n;
      }
  }
  if (n > 1) LB_BCUDA(b, cudaEventRecord(b->ev_fork, b->stream));
  if (n > 0) LB_BCUDA(b, launch_lane(b, b->g[lg[0]], lm[0], b->stream));
  for (int k = 1; k < n; ++k) {
    LB_BCUDA(b, cudaStreamWaitEvent(b->aux[k - 1], b->ev_fork, 0));
    LB_BCUDA(b, launch_lane(b, b->g[lg[k]], lm[k], b->aux[k - 1]));
    LB_BCUDA(b, cudaEventRecord(b->ev_join[k - 1], b->aux[k - 1]));
  }
  for (int k = 1; k < n; ++k) LB_BCUDA(b, cudaStreamWaitEvent(b->stream, b->ev_join[k - 1], 0));
  b->parity ^= 1;
  return LB_OK;
}

void advance_members(lb_batch* b, long long n) {
  for (lb_ctx* c : b->m) {
    c->step += n;
    if (n & 1) c->cur ^= 1;
  }
  b->step += n;
}

lb_status check_members(lb_batch* b) {
  for (size_t i = 0; i < b->m.size(); ++i) {
    lb_ctx* c = b->m[i];
    int h = 0;
    LB_BCUDA(b, cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    LB_BCUDA(b, cudaStreamSynchronize(b->stream));
    if (h) {
      const std::string m = "non-finite density in batch member " + std::to_string(i) + " after step " +
                            std::to_string(c->step);
      ctx_fail(c, LB_ERR_NONFINITE, m);
      return bfail(b, LB_ERR_NONFINITE, m);
    }
  }
  return LB_OK;
}

lb_status ready(lb_batch* b) {
  if (!b) return bfail(nullptr, LB_ERR_ARG, "null batch");
  if (b->poisoned) return bfail(b, LB_ERR_STATE, "batch poisoned by an earlier failure: " + b->err);
  for (size_t i = 0; i < b->m.size(); ++i) {
    lb_status s;
    if (!ctx_usable(b->m[i], &s))
      return bfail(b, LB_ERR_STATE, "member " + std::to_string(i) + ": " + b->m[i]->err);
    if (b->m[i]->K == KELT)
      return bfail(b, LB_ERR_ARG, "member " + std::to_string(i) +
                                      " is a theta-resolved ellipsoid, which only the plain step kernel carries");
    if (b->m[i]->any_shift)
      return bfail(b, LB_ERR_ARG, "member " + std::to_string(i) +
                                      " uses the half-force velocity (old_forcing 2), which only the plain "
                                      "step kernel carries");
  }
  return LB_OK;
}

// n steps; trials of the autotuner pass graph = false.
lb_status run(lb_batch* b, long long n, bool graph) {
  if (!records_current(b)) {
    lb_status s = build(b);
    if (s != LB_OK) return s;
  }
  if (graph && b->use_graph && b->check_every == 0 && n >= 3) {
    if (b->parity != 0) {  // the captured pair starts at parity 0
      lb_status s = step_once(b);
      if (s != LB_OK) return s;
      advance_members(b, 1);
      --n;
    }
    if (!b->graph || b->graph_threads != b->threads || b->graph_schedule != b->schedule ||
        b->graph_tile_blocks != b->tile_blocks) {
      drop_graph(b);
      cudaGraph_t g = nullptr;
      LB_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      lb_status s1 = step_once(b);
      lb_status s2 = s1 == LB_OK ? step_once(b) : s1;
      cudaError_t e = cudaStreamEndCapture(b->stream, &g);
      if (s2 != LB_OK) return s2;
      if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
      b->graph_threads = b->threads;
      b->graph_tile_blocks = b->tile_blocks;
      b->graph_schedule = b->schedule;
    }
    const long long pairs = n / 2;
    for (long long i = 0; i < pairs; ++i) LB_BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
    advance_members(b, 2 * pairs);
    n &= 1;
  }
  for (long long i = 0; i < n; ++i) {
    lb_status s = step_once(b);
    if (s != LB_OK) return s;
    advance_members(b, 1);
    if (b->check_every > 0 && (b->step % b->check_every) == 0) {
      s = check_members(b);
      if (s != LB_OK) return s;
    }
  }
  return LB_OK;
}

}  // namespace

// A context stepped through its own single-member batch (interior and
// wall-node tiles in separate kernels): build the tiles for the context's
// current buffer and block size, outside any stream capture.
lb_status lbgm::ctx_tiled_prepare(lb_ctx* c) {
  if (!c->tiles) {
    lb_ctx* one[1] = {c};
    lb_status s = lb_batch_create(one, 1, &c->tiles);
    if (s != LB_OK) return ctx_fail(c, s, std::string("tiled step: ") + lb_last_error(nullptr));
  }
  lb_batch* b = c->tiles;
  b->threads = std::min(c->block_threads, max_threads(b->prec));
  if (!records_current(b)) {
    lb_status s = build(b);
    if (s != LB_OK) return ctx_fail(c, s, "tiled step: " + b->err);
  }
  return LB_OK;
}

// One step's launches; the caller flips the context's buffer and counts the
// step (the batch's parity follows, so its records stay current).
lb_status lbgm::ctx_tiled_launch(lb_ctx* c) {
  lb_batch* b = c->tiles;
  if (!b || !records_current(b) || b->threads != std::min(c->block_threads, max_threads(b->prec)))
    return ctx_fail(c, LB_ERR_STATE, "tiled step used without preparation");
  lb_status s = step_once(b);
  if (s != LB_OK) return ctx_fail(c, s, "tiled step: " + b->err);
  return LB_OK;
}

extern "C" {

lb_status lb_batch_create(lb_ctx* const* members, int count, lb_batch** out) {
  if (!members || !out) return bfail(nullptr, LB_ERR_ARG, "null argument");
  *out = nullptr;
  if (count < 1) return bfail(nullptr, LB_ERR_ARG, "need count >= 1");
  lb_batch* b = new lb_batch();
  auto bail = [&](lb_status s, const std::string& m) {
    lb_batch_destroy(b);
    return bfail(nullptr, s, m);
  };
  long long nodes = 0;
  for (int i = 0; i < count; ++i) {
    lb_ctx* c = members[i];
    if (!c) return bail(LB_ERR_ARG, "member " + std::to_string(i) + " is NULL");
    for (int j = 0; j < i; ++j)
      if (members[j] == c) return bail(LB_ERR_ARG, "member " + std::to_string(i) + " appears twice");
    if (i > 0 && (c->prec != b->prec || c->device != b->device || c->stream != b->stream))
      return bail(LB_ERR_ARG, "member " + std::to_string(i) + " differs in precision, device or stream");
    if (i == 0) {
      b->prec = c->prec;
      b->device = c->device;
      b->stream = c->stream;
    }
    b->m.push_back(c);
    nodes += (long long)c->batch * (long long)c->ncell;
  }
  b->nodes = nodes;
  int cur_dev = 0;
  cudaError_t e = cudaGetDevice(&cur_dev);
  if (e == cudaSuccess && cur_dev != b->device) e = cudaErrorInvalidDevice;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  for (int i = 0; i < kMaxLanes - 1 && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->aux[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) return bail(LB_ERR_CUDA, std::string("batch setup: ") + cudaGetErrorString(e));
  *out = b;
  return LB_OK;
}

lb_status lb_batch_step(lb_batch* b, long long n) {
  lb_status s = ready(b);
  if (s != LB_OK) return s;
  if (n < 0) return bfail(b, LB_ERR_ARG, "need n >= 0");
  return run(b, n, true);
}

lb_status lb_batch_set_option(lb_batch* b, int option, long long value) {
  if (!b) return bfail(nullptr, LB_ERR_ARG, "null batch");
  switch (option) {
    case LB_OPT_CHECK_EVERY:
      if (value < 0) return bfail(b, LB_ERR_ARG, "need k >= 0");
      b->check_every = value;
      return LB_OK;
    case LB_OPT_BLOCK_THREADS:
      if (value < 64 || value > 256 || value % 32) return bfail(b, LB_ERR_ARG, "need 64..256, multiple of 32");
      // tiles are block-sized: the work-list kernel's bound (128 with FP32
      // arithmetic) caps the block
      b->threads = std::min(int(value), max_threads(b->prec));
      return LB_OK;
    case LB_OPT_USE_GRAPH:
      b->use_graph = value ? 1 : 0;
      return LB_OK;
    case LB_OPT_SCHEDULE:
      if (value < 0 || value > 1) return bfail(b, LB_ERR_ARG, "need 0 (tile per block) or 1 (persistent)");
      b->schedule = int(value);
      return LB_OK;
    case LB_OPT_TILE_BLOCKS:
      if (value != 1 && value != 2 && value != 4) return bfail(b, LB_ERR_ARG, "need 1, 2 or 4 blocks per tile");
      b->tile_blocks = int(value);
      return LB_OK;
    default:
      return bfail(b, LB_ERR_ARG, "option not available for batches");
  }
}

lb_status lb_batch_autotune(lb_batch* b, int steps_per_trial, lb_tune* best, lb_tune* trials, int max_trials,
                            int* n_trials) {
  lb_status s = ready(b);
  if (s != LB_OK) return s;
  if (steps_per_trial < 1) return bfail(b, LB_ERR_ARG, "need steps_per_trial >= 1");
  if (max_trials < 0 || (max_trials > 0 && !trials)) return bfail(b, LB_ERR_ARG, "bad trials buffer");
  std::vector<lb_tune> cand;
  for (int t : {64, 96, 128, 192, 256})
    if (t <= max_threads(b->prec))
      for (int sc : {0, 1})
        for (int tb : {1, 2, 4}) cand.push_back({t, sc, t * tb, 0.0});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LB_BCUDA(b, cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return bcuda(b, e, "cudaEventCreate");
  }
  const long long keep_check = b->check_every;
  b->check_every = 0;
  for (lb_tune& k : cand) {
    b->threads = k.block_threads;
    b->schedule = k.schedule;
    b->tile_blocks = k.tile_nodes / k.block_threads;
    s = run(b, 1, false);  // rebuilds the tiles for this block size; untimed
    if (s != LB_OK) break;
    if ((e = cudaEventRecord(e0, b->stream)) != cudaSuccess) {
      s = bcuda(b, e, "cudaEventRecord");
      break;
    }
    s = run(b, steps_per_trial, false);
    if (s != LB_OK) break;
    float ms = 0.f;
    e = cudaEventRecord(e1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      s = bcuda(b, e, "timing a trial");
      break;
    }
    k.ms_per_step = double(ms) / steps_per_trial;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->check_every = keep_check;
  if (s != LB_OK) return s;
  size_t ib = 0;
  for (size_t i = 1; i < cand.size(); ++i)
    if (cand[i].ms_per_step < cand[ib].ms_per_step) ib = i;
  b->threads = cand[ib].block_threads;
  b->schedule = cand[ib].schedule;
  b->tile_blocks = cand[ib].tile_nodes / cand[ib].block_threads;
  if (best) *best = cand[ib];
  const int n = int(cand.size());
  for (int i = 0; i < n && i < max_trials; ++i) trials[i] = cand[i];
  if (n_trials) *n_trials = n;
  if (keep_check > 0) return check_members(b);
  return LB_OK;
}

long long lb_batch_nodes(const lb_batch* b) { return b ? b->nodes : -1; }

long long lb_batch_step_count(const lb_batch* b) { return b ? b->step : -1; }

void lb_batch_destroy(lb_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  if (b->dmem) cudaFree(b->dmem);
  for (int i = 0; i < kMaxLanes - 1; ++i) {
    if (b->aux[i]) cudaStreamDestroy(b->aux[i]);
    if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  delete b;
}

const char* lb_batch_last_error(const lb_batch* b) { return b ? b->err.c_str() : lb_last_error(nullptr); }

}  // extern "C"
