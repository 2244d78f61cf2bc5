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

constexpr int ENS_MAX = 64;

struct EnsInstance {
  Problem P;
  void* q_a;
  void* q_b;
  void* qt;
  double dt;
  int tiles_x, tiles_y, chunks, zchunk;
  int item_off;  // first work item of this instance
};

struct EnsTable {
  int count;
  int total_items;
  EnsInstance inst[ENS_MAX];
};

template <int TX, int TY>
__global__ void __launch_bounds__(Geo<TX, TY, 2>::NT, 1)
ensemble_stage_kernel(const EnsTable T, const double a, const double b, const int read_qt,
                      const int write_qt, const int parity) {
  for (int item = blockIdx.x; item < T.total_items; item += gridDim.x) {
    int ii = 0;
    while (ii + 1 < T.count && T.inst[ii + 1].item_off <= item) ++ii;
    const EnsInstance& I = T.inst[ii];
    const int local = item - I.item_off;
    const int bx = local % I.tiles_x;
    const int rest = local / I.tiles_x;
    const int by = rest % I.tiles_y;
    const int bz = rest / I.tiles_y;
    StageArgs S;
    S.q_in = parity ? I.q_b : I.q_a;
    S.q_out = parity ? I.q_a : I.q_b;
    S.qt = I.qt;
    S.r_out = nullptr;
    S.diag_part = nullptr;
    S.a = a;
    S.b = b;
    S.dt = I.dt;
    S.read_qt = read_qt;
    S.write_qt = write_qt;
    S.scaled_qt = 1;  // as rk_step: Qt is internal scratch kept divided by dt
    S.bdt = b * I.dt;
    S.zchunk = I.zchunk;
    S.zg = 0;  // the periodic box
    S.nzl = 0;
    S.fs_q = S.fs_t = 0;
    stage_tile<float, float, float, float, TX, TY, 2, EPI_RK, false>(I.P, S, bx * TX, by * TY,
                                                                      bz * I.zchunk, 0);
    __syncthreads();  // the next item reuses the shared-memory ring
  }
}

using EnsFn = cudaError_t (*)(const EnsTable&, int grid, double a, double b, int read_qt,
                              int write_qt, int parity, cudaStream_t);

template <int TX, int TY>
static cudaError_t ens_launch(const EnsTable& T, int grid, double a, double b, int read_qt,
                              int write_qt, int parity, cudaStream_t st) {
  auto kern = ensemble_stage_kernel<TX, TY>;
  const size_t smem = stage_smem_bytes<float, float, float, TX, TY, 2>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, dim3(TX / 2, TY), smem, st>>>(T, a, b, read_qt, write_qt, parity);
  return cudaGetLastError();
}

template <int TX, int TY>
static int ens_occupancy() {
  auto kern = ensemble_stage_kernel<TX, TY>;
  const size_t smem = stage_smem_bytes<float, float, float, TX, TY, 2>();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, (TX / 2) * TY, smem) != cudaSuccess)
    return 0;
  return nb;
}

static const EnsFn ENS_FN[NUM_TILES] = {ens_launch<TILE_TX[0], TILE_TY[0]>,
                                        ens_launch<TILE_TX[1], TILE_TY[1]>,
                                        ens_launch<TILE_TX[2], TILE_TY[2]>};
static int (*const ENS_OCC[NUM_TILES])() = {ens_occupancy<TILE_TX[0], TILE_TY[0]>,
                                           ens_occupancy<TILE_TX[1], TILE_TY[1]>,
                                           ens_occupancy<TILE_TX[2], TILE_TY[2]>};

constexpr int ZC_CANDIDATES[] = {16, 24, 32, 48, 64, 96};

struct InstanceIn {
  tgv_config cfg;
  void *q_a, *q_b, *qt;
  double dt;
};

// Fill the table for a tile and a target z-chunk length; instances are laid
// out largest first so the round-robin hands out the biggest items early.
static void build_table(EnsTable& T, const std::vector<InstanceIn>& in, int tile, int zc_target) {
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
    I.tiles_x = (n + TILE_TX[tile] - 1) / TILE_TX[tile];
    I.tiles_y = (n + TILE_TY[tile] - 1) / TILE_TY[tile];
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
  int tile = 0, zc_target = 0, grid = 0, steps_per_graph = 0;
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
    if (!(c.q_storage == TGV_F32 && c.qt_storage == TGV_F32 && c.compute == TGV_F32 &&
          c.accumulate == TGV_F32))
      return TGV_ERR_UNSUPPORTED;
    if (c.split_form != TGV_SPLIT_BLAISDELL && c.split_form != TGV_SPLIT_DIVERGENCE)
      return TGV_ERR_UNSUPPORTED;
    if (!q_a[i] || !q_b[i] || !qt[i] || q_a[i] == q_b[i]) return TGV_ERR_ARG;
    if (!std::isfinite(dts[i]) || !(dts[i] > 0.0)) return TGV_ERR_ARG;
    if (!(c.flags & TGV_FLAG_ALLOW_UNSTABLE_DT) && dts[i] > tgv_dt_max(&c)) return TGV_ERR_UNSTABLE_DT;
  }
  return TGV_OK;
}

// Time `reps` first-stage launches of a candidate (reads Q_a only).
static float ens_time(const EnsTable& T, int tile, int grid, int reps, cudaStream_t st,
                      cudaEvent_t e0, cudaEvent_t e1) {
  if (ENS_FN[tile](T, grid, RK_A[0], RK_B[0], 0, 1, 0, st) != cudaSuccess) return -1.f;
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps; ++r)
    if (ENS_FN[tile](T, grid, RK_A[0], RK_B[0], 0, 1, 0, st) != cudaSuccess) return -1.f;
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
    const int occ = ENS_OCC[t]();
    if (occ <= 0) continue;
    for (int zc : ZC_CANDIDATES) {
      if (pin_zc > 0 && zc != pin_zc) continue;
      EnsTable T;
      build_table(T, E->in, t, zc);
      const int grid = std::min(T.total_items, occ * sms);
      const float ms = ens_time(T, t, grid, 3, st, e0, e1);
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
      const float ms = ens_time(T, t, grid, 1, st, e0, e1);
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
      ok = ENS_FN[E->tile](E->table, E->grid, RK_A[i], RK_B[i], i != 0, i != 2, (3 * m + i) & 1,
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
