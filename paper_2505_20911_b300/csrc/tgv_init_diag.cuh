// tgv_init_diag.cuh - Taylor-Green initial condition and FP64 diagnostics.
#pragma once

#include "tgv_common.cuh"

namespace tgv {

// Taylor-Green initial field (Sec. 4.1, Eqs. 6-10), evaluated in FP64 and
// rounded once to the storage type (offset-encoded if requested).
template <class TS>
__global__ void init_kernel(const Problem P, TS* __restrict__ q) {
  const long long n = P.n, nn = n * n, n3 = nn * n;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n3;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % n), j = (int)((o / n) % n), k = (int)(o / nn);
    const double x = i * P.h, y = j * P.h, z = k * P.h;
    double sx, cx, sy, cy, sz, cz;
    sincos(x, &sx, &cx);
    sincos(y, &sy, &cy);
    sincos(z, &sz, &cz);
    const double u = sx * cy * cz, v = -cx * sy * cz;
    const double c2x = cx * cx - sx * sx, c2y = cy * cy - sy * sy, c2z = cz * cz - sz * sz;
    const double p = 1.0 / P.gM2 + (c2x + c2y) * (2.0 + c2z) / 16.0;
    const double rho = P.gM2 * p;
    const double rhoE = p / P.gm1 + 0.5 * rho * (u * u + v * v);
    q[o] = Num<TS>::from_f64(rho - P.rho0);
    q[o + n3] = Num<TS>::from_f64(rho * u);
    q[o + 2 * n3] = Num<TS>::from_f64(rho * v);
    q[o + 3 * n3] = Num<TS>::from_f64(0.0);
    q[o + 4 * n3] = Num<TS>::from_f64(rhoE - P.rhoE0);
  }
}

constexpr int DIAG_THREADS = 256;
constexpr int DIAG_MAX_BLOCKS = 148 * 8;

template <class TS>
__device__ __forceinline__ void load_vel(const TS* __restrict__ q, long long o, long long n3,
                                         double rho0, double* u) {
  const double rho = Num<TS>::to_f64(q[o]) + rho0;
  u[0] = Num<TS>::to_f64(q[o + n3]) / rho;
  u[1] = Num<TS>::to_f64(q[o + 2 * n3]) / rho;
  u[2] = Num<TS>::to_f64(q[o + 3 * n3]) / rho;
}

// Per-block FP64 partial sums of the TGV_DIAG_COUNT diagnostics (sums, not
// means); a fixed grid-stride assignment keeps the result deterministic.
template <class TS>
__global__ void __launch_bounds__(DIAG_THREADS)
diag_partial_kernel(const Problem P, const TS* __restrict__ q, double* __restrict__ part) {
  const int n = P.n;
  const long long nn = (long long)n * n, n3 = nn * n;
  double acc[TGV_DIAG_COUNT];
#pragma unroll
  for (int m = 0; m < TGV_DIAG_COUNT; ++m) acc[m] = 0.0;
  const double s = P.inv12h;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n3;
       o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % n), j = (int)((o / n) % n), k = (int)(o / nn);
    double qc[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) qc[c] = Num<TS>::to_f64(q[o + c * n3]);
    qc[0] += P.rho0;
    qc[4] += P.rhoE0;
    bool bad = false;
#pragma unroll
    for (int c = 0; c < 5; ++c) bad |= !isfinite(qc[c]);
    const double u = qc[1] / qc[0], v = qc[2] / qc[0], w = qc[3] / qc[0];
    const double u2 = u * u + v * v + w * w;
    // velocity derivatives du_a/dx_b (4th-order central, periodic)
    double g[3][3];  // g[a][b] = D_b u_a
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double um2[3], um1[3], up1[3], up2[3];
      const int ii[4] = {-2, -1, 1, 2};
      double* dst[4] = {um2, um1, up1, up2};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        int xi = i, yj = j, zk = k;
        if (b == 0) xi = (i + ii[t] + n) % n;
        if (b == 1) yj = (j + ii[t] + n) % n;
        if (b == 2) zk = (k + ii[t] + n) % n;
        load_vel(q, (long long)zk * nn + (long long)yj * n + xi, n3, P.rho0, dst[t]);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a)
        g[a][b] = s * (8.0 * (up1[a] - um1[a]) - (up2[a] - um2[a]));
    }
    const double wx = g[2][1] - g[1][2], wy = g[0][2] - g[2][0], wz = g[1][0] - g[0][1];
    const double ens = wx * wx + wy * wy + wz * wz;
    acc[0] += 0.5 * u2;
    acc[1] += 0.5 * qc[0] * u2;
    acc[2] += ens;
    acc[4] += qc[0];
    acc[5] += qc[1];
    acc[6] += qc[2];
    acc[7] += qc[3];
    acc[8] += qc[4];
    acc[9] += bad ? 1.0 : 0.0;
  }
  // block reduction: warp shuffles, then a fixed-order pass over warps
  __shared__ double red[DIAG_THREADS / 32][TGV_DIAG_COUNT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < TGV_DIAG_COUNT; ++m) {
    double v = acc[m];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][m] = v;
  }
  __syncthreads();
  if (threadIdx.x < TGV_DIAG_COUNT) {
    double v = 0.0;
    for (int w = 0; w < DIAG_THREADS / 32; ++w) v += red[w][threadIdx.x];
    part[blockIdx.x * TGV_DIAG_COUNT + threadIdx.x] = v;
  }
}

// Second pass: fixed-order sum of the block partials, then means.
__global__ void diag_final_kernel(const Problem P, const double* __restrict__ part, int nblocks,
                                  double* __restrict__ out);

}  // namespace tgv
