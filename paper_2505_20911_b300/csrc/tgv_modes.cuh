// tgv_modes.cuh - precision modes and the per-mode launcher table.
//
// Each built (q_storage, qt_storage, compute, accumulate) combination is one
// "mode".  Its kernels are instantiated in a translation unit of its own
// (tgv_mode_<m>.cu) so the modes compile in parallel; the C ABI dispatches
// through the table returned by mode_launchers().
#pragma once

#include "tgv_common.cuh"
#include "tgv_stage.cuh"
#include "tgv_init_diag.cuh"
#include "tgv_ensemble.cuh"

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

// Tile shapes (TX, TY) and points per thread; tile id t is 1-based in the C
// ABI, in order of preference (larger tiles carry less halo).  FP32/FP16
// compute uses two x points per thread; FP64 compute one, on smaller tiles
// (an FP64 ring of a 32x16 tile would not fit shared memory).  A tile whose
// shared memory exceeds STAGE_SMEM_LIMIT for a mode's storage types is not
// used for that mode.
constexpr int NUM_TILES = 3;
constexpr int TILE_TX[NUM_TILES] = {32, 16, 16};
constexpr int TILE_TY[NUM_TILES] = {16, 16, 8};
constexpr int TILE_TX_F64[NUM_TILES] = {16, 16, 8};
constexpr int TILE_TY_F64[NUM_TILES] = {16, 8, 8};

inline int tile_tx(int comp, int t) { return comp == TGV_F64 ? TILE_TX_F64[t] : TILE_TX[t]; }
inline int tile_ty(int comp, int t) { return comp == TGV_F64 ? TILE_TY_F64[t] : TILE_TY[t]; }

using StageFn = cudaError_t (*)(const Problem&, const StageArgs&, int zchunk, cudaStream_t);
using OccFn = int (*)();
using InitFn = cudaError_t (*)(const Problem&, void*, const ZLayout&, cudaStream_t);
using DiagFn = cudaError_t (*)(const Problem&, const void*, double*, int, cudaStream_t);

// Kernel variants by convective split family (SPL_QUAD, SPL_KGP, SPL_KEEP,
// SPL_FEIER); only SPL_QUAD is built for every mode.
constexpr int NUM_SPL = 4;
struct ModeLaunchers {
  StageFn stage[NUM_SPL][NUM_TILES];      // EPI_RK (null where a mode does not build it)
  StageFn stage_rk[3][NUM_TILES];         // EPI_RK, quadratic split, flags RKF_STAGE(i)
  StageFn stage_diag[NUM_SPL][NUM_TILES]; // EPI_RK with the fused diagnostics of its input
  StageFn stage_rk_diag[NUM_TILES];       // rk_step's first stage with the fused diagnostics
  StageFn rhs[NUM_SPL][NUM_TILES];        // EPI_RHS
  OccFn occupancy[NUM_TILES];    // resident CTAs per SM of the EPI_RK kernel
  size_t smem[NUM_TILES];        // dynamic shared memory per CTA
  int first_tile = 0;            // tile tried before the table order
  EnsFn ens[NUM_TILES];          // batched-ensemble stage (quadratic splits)
  OccFn ens_occ[NUM_TILES];      // its resident CTAs per SM
  InitFn init;
  DiagFn diag_partial;
};

const ModeLaunchers& mode_launchers(int mode);
// Index into MODE_KEYS of a config's (q_storage, qt_storage, compute,
// accumulate), or -1 if that combination is not built.
int find_mode(const tgv_config& c);

template <class TS, class TT, class TC, class TA, int TX, int TY, int NP, int EPI, bool DIAG,
          int SPL = SPL_QUAD, int RKF = RKF_RUNTIME>
cudaError_t launch_stage(const Problem& P, const StageArgs& S, int zchunk, cudaStream_t st) {
  auto kern = stage_kernel<TS, TT, TC, TA, TX, TY, NP, EPI, DIAG, SPL, RKF>;
  const size_t smem = stage_smem_bytes<TS, TT, TC, TX, TY, NP>();
  if (smem > STAGE_SMEM_LIMIT) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int n = P.n;
  const int nzl = S.nzl > 0 ? S.nzl : n;
  dim3 grid((n + TX - 1) / TX, (n + TY - 1) / TY, (nzl + zchunk - 1) / zchunk);
  dim3 block(TX / NP, TY);
  kern<<<grid, block, smem, st>>>(P, S);
  return cudaGetLastError();
}

// Stage i of rk_step (quadratic split, no diagnostics): the kernel with the
// RK flags of that stage fixed at compile time.  Its plain-encoding flag
// matters only to FP32 storage with FP32 arithmetic; a config with another
// encoding there takes the runtime-flag kernel.
template <class TS, class TT, class TC, class TA, int TX, int TY, int NP, int I>
cudaError_t launch_stage_rk(const Problem& P, const StageArgs& S, int zchunk, cudaStream_t st) {
  constexpr bool QIN_FC = std::is_same<TS, float>::value && std::is_same<TC, float>::value;
  if (QIN_FC && P.encoding != TGV_ENC_PLAIN)
    return launch_stage<TS, TT, TC, TA, TX, TY, NP, EPI_RK, false, SPL_QUAD>(P, S, zchunk, st);
  return launch_stage<TS, TT, TC, TA, TX, TY, NP, EPI_RK, false, SPL_QUAD, RKF_STAGE(I)>(P, S, zchunk,
                                                                                       st);
}

// rk_step's first stage of a logged step: the fused-diagnostics kernel with the
// flags of stage 0 built in (as launch_stage_rk).
template <class TS, class TT, class TC, class TA, int TX, int TY, int NP>
cudaError_t launch_stage_rk_diag(const Problem& P, const StageArgs& S, int zchunk, cudaStream_t st) {
  constexpr bool QIN_FC = std::is_same<TS, float>::value && std::is_same<TC, float>::value;
  if (QIN_FC && P.encoding != TGV_ENC_PLAIN)
    return launch_stage<TS, TT, TC, TA, TX, TY, NP, EPI_RK, true, SPL_QUAD>(P, S, zchunk, st);
  return launch_stage<TS, TT, TC, TA, TX, TY, NP, EPI_RK, true, SPL_QUAD, RKF_STAGE(0)>(P, S, zchunk,
                                                                                      st);
}

template <class TS, class TT, class TC, class TA, int TX, int TY, int NP>
int stage_occupancy() {
  auto kern = stage_kernel<TS, TT, TC, TA, TX, TY, NP, EPI_RK, false>;
  const size_t smem = stage_smem_bytes<TS, TT, TC, TX, TY, NP>();
  if (smem > STAGE_SMEM_LIMIT) return 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, (TX / NP) * TY, smem) != cudaSuccess)
    return 0;
  return nb;
}

template <class TS>
cudaError_t launch_init(const Problem& P, void* q, const ZLayout& L, cudaStream_t st) {
  const long long cnt = (long long)P.n * P.n * L.nzl;
  const int threads = 256;
  const long long blocks = (cnt + threads - 1) / threads;
  init_kernel<TS><<<(unsigned)(blocks < 148 * 64 ? blocks : 148 * 64), threads, 0, st>>>(
      P, static_cast<TS*>(q), L);
  return cudaGetLastError();
}

template <class TS, class TC>
cudaError_t launch_diag_partial(const Problem& P, const void* q, double* part, int nblocks,
                                cudaStream_t st) {
  diag_partial_kernel<TS, TC><<<nblocks, dim3(DIAG_TX, DIAG_TY), 0, st>>>(
      P, static_cast<const TS*>(q), part);
  return cudaGetLastError();
}

template <class TS, class TT, class TC, class TA, int TX, int TY, int NP, int SPL>
void set_split(ModeLaunchers& L, int t) {
  L.stage[SPL][t] = launch_stage<TS, TT, TC, TA, TX, TY, NP, EPI_RK, false, SPL>;
  L.stage_diag[SPL][t] = launch_stage<TS, TT, TC, TA, TX, TY, NP, EPI_RK, true, SPL>;
  L.rhs[SPL][t] = launch_stage<TS, TT, TC, TA, TX, TY, NP, EPI_RHS, false, SPL>;
}

template <class TS, class TT, class TC, class TA, int TX, int TY, int NP, bool WITH_KGP>
void set_tile(ModeLaunchers& L, int t) {
  for (int v = 0; v < NUM_SPL; ++v) L.stage[v][t] = L.stage_diag[v][t] = L.rhs[v][t] = nullptr;
  set_split<TS, TT, TC, TA, TX, TY, NP, SPL_QUAD>(L, t);
  L.stage_rk[0][t] = launch_stage_rk<TS, TT, TC, TA, TX, TY, NP, 0>;
  L.stage_rk[1][t] = launch_stage_rk<TS, TT, TC, TA, TX, TY, NP, 1>;
  L.stage_rk[2][t] = launch_stage_rk<TS, TT, TC, TA, TX, TY, NP, 2>;
  L.stage_rk_diag[t] = launch_stage_rk_diag<TS, TT, TC, TA, TX, TY, NP>;
  if constexpr (WITH_KGP) {
    set_split<TS, TT, TC, TA, TX, TY, NP, SPL_KGP>(L, t);
    set_split<TS, TT, TC, TA, TX, TY, NP, SPL_KEEP>(L, t);
    set_split<TS, TT, TC, TA, TX, TY, NP, SPL_FEIER>(L, t);
  }
  L.occupancy[t] = stage_occupancy<TS, TT, TC, TA, TX, TY, NP>;
  L.smem[t] = stage_smem_bytes<TS, TT, TC, TX, TY, NP>();
  L.ens[t] = ens_launch<TS, TT, TC, TA, TX, TY, NP>;
  L.ens_occ[t] = ens_occupancy<TS, TT, TC, TA, TX, TY, NP>;
}

// WITH_KGP: also build the KGP, KEEP and Feiereisen splits (the FP64, FP32
// and Q FP32 / Qt FP16 modes: the precisions of the paper's split-form study).
template <class TS, class TT, class TC, class TA, bool WITH_KGP = false>
ModeLaunchers make_launchers() {
  ModeLaunchers L;
  if constexpr (std::is_same<TC, double>::value) {
    set_tile<TS, TT, TC, TA, TILE_TX_F64[0], TILE_TY_F64[0], 1, WITH_KGP>(L, 0);
    set_tile<TS, TT, TC, TA, TILE_TX_F64[1], TILE_TY_F64[1], 1, WITH_KGP>(L, 1);
    set_tile<TS, TT, TC, TA, TILE_TX_F64[2], TILE_TY_F64[2], 1, WITH_KGP>(L, 2);
  } else {
    set_tile<TS, TT, TC, TA, TILE_TX[0], TILE_TY[0], 2, WITH_KGP>(L, 0);
    set_tile<TS, TT, TC, TA, TILE_TX[1], TILE_TY[1], 2, WITH_KGP>(L, 1);
    set_tile<TS, TT, TC, TA, TILE_TX[2], TILE_TY[2], 2, WITH_KGP>(L, 2);
  }
  L.init = launch_init<TS>;
  L.diag_partial = launch_diag_partial<TS, TC>;
  return L;
}

}  // namespace tgv
