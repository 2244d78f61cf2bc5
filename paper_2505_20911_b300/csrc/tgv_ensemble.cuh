// tgv_ensemble.cuh - the batched-ensemble stage kernel: many TGV instances of
// uneven size, each with its own constants and buffers, advanced by one
// persistent launch per RK stage (see tgv_ensemble.cu for the driver).
#pragma once

#include "tgv_stage.cuh"

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

// The per-instance table travels in the launch's parameter block (no device
// allocation): 64 instances take about 11 KB.
struct EnsTable {
  int count;
  int total_items;
  EnsInstance inst[ENS_MAX];
};

// The grid-sized set of CTAs walks the flattened list of work items
// (instance, x tile, y tile, z chunk) in a fixed round-robin order and runs
// the single-instance stage body on each, with rk_step's epilogue (the
// increment kept divided by dt), so an instance matches a single-instance
// rk_step with the same tile and z chunk bit for bit.
template <class TS, class TT, class TC, class TA, int TX, int TY, int NP>
__global__ void __launch_bounds__(Geo<TX, TY, NP>::NT, stage_min_blocks<TC>())
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
    stage_tile<TS, TT, TC, TA, TX, TY, NP, EPI_RK, false>(I.P, S, bx * TX, by * TY,
                                                          bz * I.zchunk, 0);
    __syncthreads();  // the next item reuses the shared-memory ring
  }
}

using EnsFn = cudaError_t (*)(const EnsTable&, int grid, double a, double b, int read_qt,
                              int write_qt, int parity, cudaStream_t);

template <class TS, class TT, class TC, class TA, int TX, int TY, int NP>
cudaError_t ens_launch(const EnsTable& T, int grid, double a, double b, int read_qt,
                       int write_qt, int parity, cudaStream_t st) {
  auto kern = ensemble_stage_kernel<TS, TT, TC, TA, TX, TY, NP>;
  const size_t smem = stage_smem_bytes<TS, TT, TC, TX, TY, NP>();
  if (smem > STAGE_SMEM_LIMIT) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, dim3(TX / NP, TY), smem, st>>>(T, a, b, read_qt, write_qt, parity);
  return cudaGetLastError();
}

template <class TS, class TT, class TC, class TA, int TX, int TY, int NP>
int ens_occupancy() {
  auto kern = ensemble_stage_kernel<TS, TT, TC, TA, TX, TY, NP>;
  const size_t smem = stage_smem_bytes<TS, TT, TC, TX, TY, NP>();
  if (smem > STAGE_SMEM_LIMIT) return 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, (TX / NP) * TY, smem) != cudaSuccess)
    return 0;
  return nb;
}

}  // namespace tgv
