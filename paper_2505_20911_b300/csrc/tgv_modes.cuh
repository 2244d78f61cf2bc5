// tgv_modes.cuh - precision modes and the per-mode launcher table.
//
// Each built (q_storage, qt_storage, compute, accumulate) combination is one
// "mode".  Its kernels are instantiated in a translation unit of its own
// (tgv_mode_<m>.cu) so the modes compile in parallel; the C ABI dispatches
// through the table returned by mode_table().
#pragma once

#include "tgv_common.cuh"
#include "tgv_stage.cuh"
#include "tgv_init_diag.cuh"

namespace tgv {

struct ModeKey { int qs, qts, comp, acc; };

constexpr int NUM_MODES = 8;
constexpr ModeKey MODE_KEYS[NUM_MODES] = {
    {TGV_F64, TGV_F64, TGV_F64, TGV_F64},    // 0 double
    {TGV_F64, TGV_F64, TGV_F32, TGV_F64},    // 1 single-double (Q FP64, R FP32)
    {TGV_F32, TGV_F32, TGV_F64, TGV_F64},    // 2 FP32 storage / FP64 compute
    {TGV_F32, TGV_F32, TGV_F32, TGV_F32},    // 3 single
    {TGV_BF16, TGV_BF16, TGV_F32, TGV_F32},  // 4 bf16 storage / FP32 compute
    {TGV_F16, TGV_F16, TGV_F32, TGV_F32},    // 5 half-single
    {TGV_F16, TGV_F16, TGV_F16, TGV_F32},    // 6 pure half
    {TGV_F32, TGV_F16, TGV_F32, TGV_F32},    // 7 Q FP32, Qt FP16
};

// Tile shapes (TX, TY); tile id t is 1-based in the C ABI.
constexpr int NUM_TILES = 3;
constexpr int TILE_TX[NUM_TILES] = {32, 16, 16};
constexpr int TILE_TY[NUM_TILES] = {8, 16, 8};

using StageFn = cudaError_t (*)(const Problem&, const StageArgs&, int zchunk, cudaStream_t);
using SmemFn = size_t (*)();
using OccFn = int (*)();
using InitFn = cudaError_t (*)(const Problem&, void*, cudaStream_t);
using DiagFn = cudaError_t (*)(const Problem&, const void*, double*, int, cudaStream_t);

struct ModeLaunchers {
  StageFn stage[NUM_TILES];   // EPI_RK
  StageFn rhs[NUM_TILES];     // EPI_RHS
  SmemFn smem[NUM_TILES];
  OccFn occupancy[NUM_TILES]; // resident CTAs per SM of the EPI_RK kernel
  InitFn init;
  DiagFn diag_partial;
};

const ModeLaunchers& mode_launchers(int mode);

template <class TS, class TT, class TC, class TA, int TX, int TY, int EPI>
cudaError_t launch_stage(const Problem& P, const StageArgs& S, int zchunk, cudaStream_t st) {
  auto kern = stage_kernel<TS, TT, TC, TA, TX, TY, EPI>;
  const size_t smem = stage_smem_bytes<TC, TX, TY>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int n = P.n;
  dim3 grid((n + TX - 1) / TX, (n + TY - 1) / TY, (n + zchunk - 1) / zchunk);
  dim3 block(TX, TY);
  kern<<<grid, block, smem, st>>>(P, S);
  return cudaGetLastError();
}

template <class TS, class TT, class TC, class TA, int TX, int TY>
int stage_occupancy() {
  auto kern = stage_kernel<TS, TT, TC, TA, TX, TY, EPI_RK>;
  const size_t smem = stage_smem_bytes<TC, TX, TY>();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, TX * TY, smem) != cudaSuccess) return 0;
  return nb;
}

template <class TS>
cudaError_t launch_init(const Problem& P, void* q, cudaStream_t st) {
  const long long n3 = (long long)P.n * P.n * P.n;
  const int threads = 256;
  const long long blocks = (n3 + threads - 1) / threads;
  init_kernel<TS><<<(unsigned)(blocks < 148 * 64 ? blocks : 148 * 64), threads, 0, st>>>(
      P, static_cast<TS*>(q));
  return cudaGetLastError();
}

template <class TS>
cudaError_t launch_diag_partial(const Problem& P, const void* q, double* part, int nblocks,
                                cudaStream_t st) {
  diag_partial_kernel<TS><<<nblocks, DIAG_THREADS, 0, st>>>(P, static_cast<const TS*>(q), part);
  return cudaGetLastError();
}

template <class TS, class TT, class TC, class TA>
ModeLaunchers make_launchers() {
  ModeLaunchers L;
  L.stage[0] = launch_stage<TS, TT, TC, TA, 32, 8, EPI_RK>;
  L.stage[1] = launch_stage<TS, TT, TC, TA, 16, 16, EPI_RK>;
  L.stage[2] = launch_stage<TS, TT, TC, TA, 16, 8, EPI_RK>;
  L.rhs[0] = launch_stage<TS, TT, TC, TA, 32, 8, EPI_RHS>;
  L.rhs[1] = launch_stage<TS, TT, TC, TA, 16, 16, EPI_RHS>;
  L.rhs[2] = launch_stage<TS, TT, TC, TA, 16, 8, EPI_RHS>;
  L.smem[0] = stage_smem_bytes<TC, 32, 8>;
  L.smem[1] = stage_smem_bytes<TC, 16, 16>;
  L.smem[2] = stage_smem_bytes<TC, 16, 8>;
  L.occupancy[0] = stage_occupancy<TS, TT, TC, TA, 32, 8>;
  L.occupancy[1] = stage_occupancy<TS, TT, TC, TA, 16, 16>;
  L.occupancy[2] = stage_occupancy<TS, TT, TC, TA, 16, 8>;
  L.init = launch_init<TS>;
  L.diag_partial = launch_diag_partial<TS>;
  return L;
}

}  // namespace tgv
