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
// increment kept divided by dt; stage i's flags RKF_STAGE_ENC_RT(i) built in,
// the encoding read per instance), so an instance matches a single-instance
// rk_step with the same tile and z chunk bit for bit.
template <class TS, class TT, class TC, class TA, int TX, int TY, int NP, int I>
__global__ void __launch_bounds__(Geo<TX, TY, NP>::NT, stage_min_blocks<TC, TX, TY, NP>())
ensemble_stage_kernel(const EnsTable T, const double a, const double b, const int parity) {
  for (int item = blockIdx.x; item < T.total_items; item += gridDim.x) {
    int ii = 0;
    while (ii + 1 < T.count && T.inst[ii + 1].item_off <= item) ++ii;
    const EnsInstance& In = T.inst[ii];
    const int local = item - In.item_off;
    const int bx = local % In.tiles_x;
    const int rest = local / In.tiles_x;
    const int by = rest % In.tiles_y;
    const int bz = rest / In.tiles_y;
    StageArgs S;
    S.q_in = parity ? In.q_b : In.q_a;
    S.q_out = parity ? In.q_a : In.q_b;
    S.qt = In.qt;
    S.r_out = nullptr;
    S.diag_part = nullptr;
    S.a = a;
    S.b = b;
    S.dt = In.dt;
    S.read_qt = I != 0;
    S.write_qt = I != 2;
    S.scaled_qt = 1;  // as rk_step: Qt is internal scratch kept divided by dt
    S.bdt = b * In.dt;
    S.zchunk = In.zchunk;
    S.zg = 0;  // the periodic box
    S.nzl = 0;
    S.fs_q = S.fs_t = 0;
    S.zoff = 0;
    stage_tile<TS, TT, TC, TA, TX, TY, NP, EPI_RK, false, SPL_QUAD, RKF_STAGE_ENC_RT(I)>(
        In.P, S, bx * TX, by * TY, bz * In.zchunk, 0);
    __syncthreads();  // the next item reuses the shared-memory ring
  }
}

using EnsFn = cudaError_t (*)(const EnsTable&, int grid, double a, double b, int read_qt,
                              int write_qt, int parity, cudaStream_t);

template <class TS, class TT, class TC, class TA, int TX, int TY, int NP, int I>
cudaError_t ens_launch_stage(const EnsTable& T, int grid, double a, double b, int parity,
                             cudaStream_t st) {
  auto kern = ensemble_stage_kernel<TS, TT, TC, TA, TX, TY, NP, I>;
  const size_t smem = stage_smem_bytes<TS, TT, TC, TX, TY, NP>();
  if (smem > STAGE_SMEM_LIMIT) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, dim3(TX / NP, TY), smem, st>>>(T, a, b, parity);
  return cudaGetLastError();
}

// Stage launch by rk_step's flags: (read, write) = (0, 1), (1, 1), (1, 0) are
// stages 0, 1, 2; (0, 0) does not occur in an RK3 step.
template <class TS, class TT, class TC, class TA, int TX, int TY, int NP>
cudaError_t ens_launch(const EnsTable& T, int grid, double a, double b, int read_qt,
                       int write_qt, int parity, cudaStream_t st) {
  if (!read_qt && !write_qt) return cudaErrorInvalidValue;
  if (!read_qt) return ens_launch_stage<TS, TT, TC, TA, TX, TY, NP, 0>(T, grid, a, b, parity, st);
  if (write_qt) return ens_launch_stage<TS, TT, TC, TA, TX, TY, NP, 1>(T, grid, a, b, parity, st);
  return ens_launch_stage<TS, TT, TC, TA, TX, TY, NP, 2>(T, grid, a, b, parity, st);
}

template <class TS, class TT, class TC, class TA, int TX, int TY, int NP>
int ens_occupancy() {
  auto kern = ensemble_stage_kernel<TS, TT, TC, TA, TX, TY, NP, 1>;
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
