// tgv_ensemble.cu - many TGV instances of uneven size advanced together.
//
// One persistent launch per RK stage covers every instance: the grid-sized
// set of CTAs walks a flattened list of work items (instance, x tile, y tile,
// z chunk) in a fixed round-robin order and runs the same per-tile stage body
// as the single-instance kernel on each.  The per-instance constants and
// buffer pointers travel in the launch's parameter block (no device
// allocation).  A CUDA graph holds `steps_per_graph` steps (three launches
// each) and is replayed; an autotuner picks the tile shape and the z-chunk
// length by timing first-stage launches, which read Q_a and only write the
// scratch buffers Q_b and Qt.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "tgv_modes.cuh"

namespace tgv {

constexpr int ZC_CANDIDATES[] = {16, 24, 32, 48, 64, 96};

struct InstanceIn {
  tgv_config cfg;
  void *q_a, *q_b, *qt;
  double dt;
};

// Fill the table for a tile and a target z-chunk length; instances are laid
// out largest first so the round-robin hands out the biggest items early.
static void build_table(EnsTable& T, const std::vector<InstanceIn>& in, int tile, int zc_target) {
  const int tx = tile_tx(in[0].cfg.compute, tile), ty = tile_ty(in[0].cfg.compute, tile);
  std::vector<int> order(in.size());
  for (size_t i = 0; i < in.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return in[x].cfg.n > in[y].cfg.n; });
  std::memset(&T, 0, sizeof(T));
  T.count = (int)in.size();
  int off = 0;
  for (int r = 0; r < T.count; ++r) {
    const InstanceIn& s = in[order[r]];
    EnsInstance& I = T.inst[r];
    I.P = make_problem(s.cfg);
    I.q_a = s.q_a;
    I.q_b = s.q_b;
    I.qt = s.qt;
    I.dt = s.dt;
    const int n = s.cfg.n;
    I.tiles_x = (n + tx - 1) / tx;
    I.tiles_y = (n + ty - 1) / ty;
    I.zchunk = std::min(n, zc_target);
    I.chunks = (n + I.zchunk - 1) / I.zchunk;
    I.item_off = off;
    off += I.tiles_x * I.tiles_y * I.chunks;
  }
  T.total_items = off;
}

}  // namespace tgv

using namespace tgv;

struct tgv_ensemble {
  EnsTable table;
  std::vector<InstanceIn> in;
  int mode = 0, tile = 0, zc_target = 0, grid = 0, steps_per_graph = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static int32_t ens_check(const tgv_config* cfgs, int32_t count, void* const* q_a, void* const* q_b,
                         void* const* qt, const double* dts) {
  if (!cfgs || !q_a || !q_b || !qt || !dts || count < 1 || count > ENS_MAX) return TGV_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    const tgv_config& c = cfgs[i];
    const int32_t s = tgv_check_config(&c);
    if (s != TGV_OK) return s;
    if (c.q_storage != cfgs[0].q_storage || c.qt_storage != cfgs[0].qt_storage ||
        c.compute != cfgs[0].compute || c.accumulate != cfgs[0].accumulate)
      return TGV_ERR_ARG;  // one precision mode per ensemble
    if (c.split_form != TGV_SPLIT_BLAISDELL && c.split_form != TGV_SPLIT_DIVERGENCE)
      return TGV_ERR_UNSUPPORTED;
    if (!q_a[i] || !q_b[i] || !qt[i] || q_a[i] == q_b[i]) return TGV_ERR_ARG;
    if (!std::isfinite(dts[i]) || !(dts[i] > 0.0)) return TGV_ERR_ARG;
    if (!(c.flags & TGV_FLAG_ALLOW_UNSTABLE_DT) && dts[i] > tgv_dt_max(&c)) return TGV_ERR_UNSTABLE_DT;
  }
  return TGV_OK;
}

// Time `reps` first-stage launches of a candidate (reads Q_a only).
static float ens_time(const EnsFn fn, const EnsTable& T, int grid, int reps, cudaStream_t st,
                      cudaEvent_t e0, cudaEvent_t e1) {
  if (fn(T, grid, RK_A[0], RK_B[0], 0, 1, 0, st) != cudaSuccess) return -1.f;
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps; ++r)
    if (fn(T, grid, RK_A[0], RK_B[0], 0, 1, 0, st) != cudaSuccess) return -1.f;
  cudaEventRecord(e1, st);
  if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms;
}

extern "C" {

int32_t tgv_ensemble_create(const tgv_config* cfgs, int32_t count, void* const* q_a,
                            void* const* q_b, void* const* qt, const double* dts,
                            int32_t steps_per_graph, void* stream, tgv_ensemble** out) {
  if (!out) return TGV_ERR_ARG;
  *out = nullptr;
  int32_t s = ens_check(cfgs, count, q_a, q_b, qt, dts);
  if (s != TGV_OK) return s;
  if (steps_per_graph < 2 || (steps_per_graph & 1)) return TGV_ERR_ARG;
  tgv_ensemble* E = new (std::nothrow) tgv_ensemble;
  if (!E) return TGV_ERR_CUDA;
  E->in.resize(count);
  for (int i = 0; i < count; ++i) E->in[i] = InstanceIn{cfgs[i], q_a[i], q_b[i], qt[i], dts[i]};
  E->steps_per_graph = steps_per_graph;
  E->mode = find_mode(cfgs[0]);
  const ModeLaunchers& L = mode_launchers(E->mode);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete E;
    return TGV_ERR_CUDA;
  }

  // ---- autotune (tile, z-chunk) unless the first config pins them
  const int pin_tile = cfgs[0].tile, pin_zc = cfgs[0].zchunk;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    delete E;
    return TGV_ERR_CUDA;
  }
  float best = -1.f;
  for (int t = 0; t < NUM_TILES; ++t) {
    if (pin_tile > 0 && t != pin_tile - 1) continue;
    const int occ = L.ens_occ[t]();
    if (occ <= 0) continue;
    for (int zc : ZC_CANDIDATES) {
      if (pin_zc > 0 && zc != pin_zc) continue;
      EnsTable T;
      build_table(T, E->in, t, zc);
      const int grid = std::min(T.total_items, occ * sms);
      const float ms = ens_time(L.ens[t], T, grid, 3, st, e0, e1);
      if (ms > 0.f && (best < 0.f || ms < best)) {
        best = ms;
        E->tile = t;
        E->zc_target = zc;
        E->grid = grid;
      }
    }
    if (pin_zc > 0 && best < 0.f) {  // a pinned z-chunk outside the candidate list
      EnsTable T;
      build_table(T, E->in, t, pin_zc);
      const int grid = std::min(T.total_items, occ * sms);
      const float ms = ens_time(L.ens[t], T, grid, 1, st, e0, e1);
      if (ms > 0.f) { best = ms; E->tile = t; E->zc_target = pin_zc; E->grid = grid; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0.f) {
    delete E;
    return TGV_ERR_CUDA;
  }
  build_table(E->table, E->in, E->tile, E->zc_target);

  // ---- capture steps_per_graph steps (3 launches each) on a private stream
  cudaStream_t cap = nullptr;
  if (cudaStreamSynchronize(st) != cudaSuccess ||
      cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete E;
    return TGV_ERR_CUDA;
  }
  bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  for (int m = 0; ok && m < steps_per_graph; ++m)
    for (int i = 0; ok && i < 3; ++i)
      ok = L.ens[E->tile](E->table, E->grid, RK_A[i], RK_B[i], i != 0, i != 2, (3 * m + i) & 1,
                          cap) == cudaSuccess;
  cudaGraph_t g = nullptr;
  const bool ended = cudaStreamEndCapture(cap, &g) == cudaSuccess;
  ok = ok && ended && g;
  if (ok) ok = cudaGraphInstantiate(&E->exec, g, 0) == cudaSuccess;
  E->graph = g;
  cudaStreamDestroy(cap);
  if (!ok) {
    if (E->exec) cudaGraphExecDestroy(E->exec);
    if (E->graph) cudaGraphDestroy(E->graph);
    delete E;
    return TGV_ERR_CUDA;
  }
  *out = E;
  return TGV_OK;
}

int32_t tgv_ensemble_run(tgv_ensemble* E, int32_t replays, void* stream) {
  if (!E || replays < 0) return TGV_ERR_ARG;
  NvtxRange range("tgv ensemble replays");
  for (int r = 0; r < replays; ++r)
    if (cudaGraphLaunch(E->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess)
      return TGV_ERR_CUDA;
  return TGV_OK;
}

int32_t tgv_ensemble_info(const tgv_ensemble* E, int32_t* tile, int32_t* zchunk_target,
                          int32_t* grid, int32_t* items, int32_t* steps_per_graph) {
  if (!E) return TGV_ERR_ARG;
  if (tile) *tile = E->tile + 1;
  if (zchunk_target) *zchunk_target = E->zc_target;
  if (grid) *grid = E->grid;
  if (items) *items = E->table.total_items;
  if (steps_per_graph) *steps_per_graph = E->steps_per_graph;
  return TGV_OK;
}

int32_t tgv_ensemble_destroy(tgv_ensemble* E) {
  if (!E) return TGV_ERR_ARG;
  if (E->exec) cudaGraphExecDestroy(E->exec);
  if (E->graph) cudaGraphDestroy(E->graph);
  delete E;
  return TGV_OK;
}

}  // extern "C"
