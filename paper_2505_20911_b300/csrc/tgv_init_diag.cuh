// tgv_init_diag.cuh - Taylor-Green initial condition and FP64 diagnostics.
#pragma once

#include "tgv_common.cuh"

namespace tgv {

// Where a state's planes live: owned planes are global z = z0 .. z0+nzl-1,
// stored after zg ghost planes, fields fs elements apart.  The periodic box is
// {0, N, 0, N^3}; a z-slab has zg = 2 and fs = (nzl + 4) N^2.
struct ZLayout {
  int z0, nzl, zg;
  long long fs;
};

// Taylor-Green initial field (Sec. 4.1, Eqs. 6-10), evaluated in FP64 and
// rounded once to the storage type (offset-encoded if requested), on the
// owned planes of layout L (ghost planes are not written).
template <class TS>
__global__ void init_kernel(const Problem P, TS* __restrict__ q, const ZLayout L) {
  const long long n = P.n, nn = n * n, cnt = nn * L.nzl, fs = L.fs;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < cnt;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % n), j = (int)((o / n) % n), kl = (int)(o / nn);
    const int k = L.z0 + kl;
    const long long d = o + (long long)L.zg * nn;
    const double x = (i + P.offset) * P.h, y = (j + P.offset) * P.h, z = (k + P.offset) * P.h;
    double sx, cx, sy, cy, sz, cz;
    sincos(x, &sx, &cx);
    sincos(y, &sy, &cy);
    sincos(z, &sz, &cz);
    const double u = sx * cy * cz, v = -cx * sy * cz;
    const double c2x = cx * cx - sx * sx, c2y = cy * cy - sy * sy, c2z = cz * cz - sz * sz;
    const double p = 1.0 / P.gM2 + (c2x + c2y) * (2.0 + c2z) / 16.0;
    const double rho = P.gM2 * p;
    const double rhoE = p / P.gm1 + 0.5 * rho * (u * u + v * v);
    q[d] = Num<TS>::from_f64(rho - P.rho0);
    q[d + fs] = Num<TS>::from_f64(rho * u);
    q[d + 2 * fs] = Num<TS>::from_f64(rho * v);
    q[d + 3 * fs] = Num<TS>::from_f64(0.0);
    q[d + 4 * fs] = Num<TS>::from_f64(rhoE - P.rhoE0);
  }
}

constexpr int DIAG_TX = 32, DIAG_TY = 8, DIAG_THREADS = DIAG_TX * DIAG_TY;
constexpr int DIAG_MAX_BLOCKS = 148 * 8;

// Per-point arithmetic type of the standalone diagnostics: FP64 for FP64
// compute, FP32 otherwise (the sums are FP64 in every mode).
template <class TC> struct DiagT { using T = float; };
template <> struct DiagT<double> { using T = double; };

template <class TS, class DT>
__device__ __forceinline__ void load_vel(const TS* __restrict__ q, long long o, long long n3,
                                         DT rho0, DT* u) {
  const DT rho = (DT)Num<TS>::to_f64(q[o]) + rho0;
  const DT ri = DT(1) / rho;
  u[0] = (DT)Num<TS>::to_f64(q[o + n3]) * ri;
  u[1] = (DT)Num<TS>::to_f64(q[o + 2 * n3]) * ri;
  u[2] = (DT)Num<TS>::to_f64(q[o + 3 * n3]) * ri;
}

// Per-block FP64 partial sums of the TGV_DIAG_COUNT diagnostics (sums, not
// means).  Work items are (32 x 8 tile, z plane) pairs, assigned to blocks in
// a fixed grid-stride order, so the result is deterministic.
template <class TS, class TC>
__global__ void __launch_bounds__(DIAG_THREADS)
diag_partial_kernel(const Problem P, const TS* __restrict__ q, double* __restrict__ part) {
  using DT = typename DiagT<TC>::T;
  const int n = P.n;
  const long long nn = (long long)n * n, n3 = nn * n;
  const int tilesx = (n + DIAG_TX - 1) / DIAG_TX, tilesy = (n + DIAG_TY - 1) / DIAG_TY;
  const long long items = (long long)tilesx * tilesy * n;
  const DT s = (DT)P.inv12h, rho0 = (DT)P.rho0, rhoE0 = (DT)P.rhoE0;
  double acc[TGV_DIAG_COUNT];
#pragma unroll
  for (int m = 0; m < TGV_DIAG_COUNT; ++m) acc[m] = 0.0;
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const int k = (int)(item / (tilesx * tilesy));
    const int t = (int)(item - (long long)k * tilesx * tilesy);
    const int i = (t % tilesx) * DIAG_TX + threadIdx.x;
    const int j = (t / tilesx) * DIAG_TY + threadIdx.y;
    if (i >= n || j >= n) continue;
    const long long o = (long long)k * nn + (long long)j * n + i;
    DT qc[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) qc[c] = (DT)Num<TS>::to_f64(q[o + c * n3]);
    qc[0] += rho0;
    qc[4] += rhoE0;
    bool bad = false;
#pragma unroll
    for (int c = 0; c < 5; ++c) bad |= !isfinite((double)qc[c]);
    const DT ri = DT(1) / qc[0];
    const DT u = qc[1] * ri, v = qc[2] * ri, w = qc[3] * ri;
    const DT u2 = u * u + v * v + w * w;
    DT g[3][3];  // g[a][b] = D_b u_a
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      DT um2[3], um1[3], up1[3], up2[3];
      DT* dst[4] = {um2, um1, up1, up2};
      const int off[4] = {-2, -1, 1, 2};
#pragma unroll
      for (int tt = 0; tt < 4; ++tt) {
        int xi = i, yj = j, zk = k;
        int* c = (b == 0) ? &xi : (b == 1) ? &yj : &zk;
        bool flipped;
        *c = wrap_index(*c + off[tt], n, P.symmetric != 0, &flipped);
        load_vel<TS, DT>(q, (long long)zk * nn + (long long)yj * n + xi, n3, rho0, dst[tt]);
        if (flipped) dst[tt][b] = -dst[tt][b];  // mirror ghost: normal velocity odd
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) g[a][b] = s * (DT(8) * (up1[a] - um1[a]) - (up2[a] - um2[a]));
    }
    const DT wx = g[2][1] - g[1][2], wy = g[0][2] - g[2][0], wz = g[1][0] - g[0][1];
    acc[0] += (double)(DT(0.5) * u2);
    acc[1] += (double)(DT(0.5) * qc[0] * u2);
    acc[2] += (double)(wx * wx + wy * wy + wz * wz);
    acc[4] += (double)qc[0];
    acc[5] += (double)qc[1];
    acc[6] += (double)qc[2];
    acc[7] += (double)qc[3];
    acc[8] += (double)qc[4];
    acc[9] += bad ? 1.0 : 0.0;
  }
  // block reduction: warp shuffles, then a fixed-order pass over warps
  __shared__ double red[DIAG_THREADS / 32][TGV_DIAG_COUNT];
  const int tid = threadIdx.y * DIAG_TX + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int m = 0; m < TGV_DIAG_COUNT; ++m) {
    double v = acc[m];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][m] = v;
  }
  __syncthreads();
  if (tid < TGV_DIAG_COUNT) {
    double v = 0.0;
    for (int w = 0; w < DIAG_THREADS / 32; ++w) v += red[w][tid];
    part[blockIdx.x * TGV_DIAG_COUNT + tid] = v;
  }
}

// Second pass: fixed-order sum of the block partials, then means.
__global__ void diag_final_kernel(const Problem P, const double* __restrict__ part, int nblocks,
                                  double* __restrict__ out);

}  // namespace tgv
