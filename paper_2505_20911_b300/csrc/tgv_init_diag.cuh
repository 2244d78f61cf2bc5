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
constexpr int DIAG_ZC = 16;  // z planes per work item
constexpr int DIAG_MAX_BLOCKS = 148 * 8;
constexpr int DIAG_RX = DIAG_TX + 4, DIAG_RY = DIAG_TY + 4, DIAG_PL = DIAG_RX * DIAG_RY;

// Work items of the standalone diagnostics: (32 x 8 column tile, chunk of
// DIAG_ZC planes) pairs.
inline long long diag_items(int n) {
  return (long long)((n + DIAG_TX - 1) / DIAG_TX) * ((n + DIAG_TY - 1) / DIAG_TY) *
         ((n + DIAG_ZC - 1) / DIAG_ZC);
}

// Per-point arithmetic type of the standalone diagnostics: FP64 for FP64
// compute, FP32 otherwise (the sums are FP64 in every mode).
template <class TC> struct DiagT { using T = float; };
template <> struct DiagT<double> { using T = double; };

// Per-block FP64 partial sums of the TGV_DIAG_COUNT diagnostics (sums, not
// means).  A block takes work items (32 x 8 column tile, chunk of DIAG_ZC
// planes) in a fixed grid-stride order, so the result is deterministic, and
// marches up the chunk: each plane's velocities on the tile and a 2-point
// halo (one division per point) go to shared memory for the x and y
// derivatives, and each thread keeps its column's u and v of the last five
// planes in registers for the z derivatives of the vorticity.  In the
// symmetric box the halo points are mirror images with the normal velocity
// component negated (the vorticity uses only derivatives of the tangential
// components across a face, which are even).
template <class TS, class TC>
__global__ void __launch_bounds__(DIAG_THREADS)
diag_partial_kernel(const Problem P, const TS* __restrict__ q, double* __restrict__ part) {
  using DT = typename DiagT<TC>::T;
  __shared__ DT su[DIAG_PL], sv[DIAG_PL], sw[DIAG_PL];
  const int n = P.n;
  const long long nn = (long long)n * n, n3 = nn * n;
  const int tilesx = (n + DIAG_TX - 1) / DIAG_TX, tilesy = (n + DIAG_TY - 1) / DIAG_TY;
  const int chunks = (n + DIAG_ZC - 1) / DIAG_ZC;
  const long long items = (long long)tilesx * tilesy * chunks;
  const DT s = (DT)P.inv12h, rho0 = (DT)P.rho0, rhoE0 = (DT)P.rhoE0;
  const bool sym = P.symmetric != 0;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * DIAG_TX + tx;
  typename DiagAcc<DT>::A acc[TGV_DIAG_COUNT];
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const int ck = (int)(item / ((long long)tilesx * tilesy));
    const int t = (int)(item - (long long)ck * tilesx * tilesy);
    const int x0 = (t % tilesx) * DIAG_TX, y0 = (t / tilesx) * DIAG_TY;
    const int z0 = ck * DIAG_ZC, z1 = min(z0 + DIAG_ZC, n);
    const bool active = (x0 + tx < n) && (y0 + ty < n);
    // region units of this thread: unit q < 256 is its own tile point,
    // units 256..431 the halo (rows 0-1, the side columns, rows TY+2..TY+3)
    int goff[2], eoff[2], flip[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int qq = tid + r * DIAG_THREADS;
      goff[r] = -1;
      eoff[r] = 0;
      flip[r] = 0;
      if (qq < DIAG_PL) {
        int rx, ry;
        if (qq < DIAG_THREADS) { rx = 2 + qq % DIAG_TX; ry = 2 + qq / DIAG_TX; }
        else {
          int h = qq - DIAG_THREADS;
          if (h < 2 * DIAG_RX) { ry = h / DIAG_RX; rx = h % DIAG_RX; }
          else if ((h -= 2 * DIAG_RX) < DIAG_TY * 4) { ry = 2 + h / 4; rx = (h % 4) < 2 ? h % 4 : DIAG_TX + (h % 4); }
          else { h -= DIAG_TY * 4; ry = DIAG_TY + 2 + h / DIAG_RX; rx = h % DIAG_RX; }
        }
        bool fx, fy;
        const int gx = wrap_index(x0 - 2 + rx, n, sym, &fx), gy = wrap_index(y0 - 2 + ry, n, sym, &fy);
        goff[r] = gy * n + gx;
        eoff[r] = ry * DIAG_RX + rx;
        flip[r] = (fx ? 1 : 0) | (fy ? 2 : 0);
      }
    }
    const int ec = (2 + ty) * DIAG_RX + 2 + tx;
    DT uq[5], vq[5], pdw[3], pxw[3], pxv[3], pdu[3];  // z queues (planes zl-4..zl / zl-2..zl)
#pragma unroll
    for (int d = 0; d < 5; ++d) uq[d] = vq[d] = DT(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) pdw[d] = pxw[d] = pxv[d] = pdu[d] = DT(0);
    for (int zl = z0 - 2; zl < z1 + 2; ++zl) {
      bool fz;
      const int zw = wrap_near(zl, n, sym, &fz);
      const long long zoff = (long long)zw * nn;
      __syncthreads();  // the previous plane's shared values have been read
      DT own_u = 0, own_v = 0;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (goff[r] < 0) continue;
        const long long o = zoff + goff[r];
        DT qc[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) qc[c] = cvt<DT>(q[o + c * n3]);
        qc[0] += rho0;
        qc[4] += rhoE0;
        const DT ri = DT(1) / qc[0];
        DT u = qc[1] * ri, v = qc[2] * ri, w = qc[3] * ri;
        if (flip[r] & 1) u = -u;
        if (flip[r] & 2) v = -v;
        if (fz) w = -w;
        su[eoff[r]] = u;
        sv[eoff[r]] = v;
        sw[eoff[r]] = w;
        if (r == 0) {
          own_u = u;
          own_v = v;
          if (active && zl >= z0 && zl < z1) {  // point-local sums of this plane
            const DT u2 = u * u + v * v + w * w;
            bool bad = false;
#pragma unroll
            for (int c = 0; c < 5; ++c) bad |= !isfinite(qc[c]);
            acc[0].add(DT(0.5) * u2);
            acc[1].add(DT(0.5) * qc[0] * u2);
            acc[4].add(qc[0]);
            acc[5].add(qc[1]);
            acc[6].add(qc[2]);
            acc[7].add(qc[3]);
            acc[8].add(qc[4]);
            acc[9].add(bad ? DT(1) : DT(0));
          }
        }
      }
      __syncthreads();
      // in-plane derivatives of this plane at the own point, and the z queues
      auto dx = [&](const DT* f) {
        return s * (DT(8) * (f[ec + 1] - f[ec - 1]) - (f[ec + 2] - f[ec - 2]));
      };
      auto dy = [&](const DT* f) {
        return s * (DT(8) * (f[ec + DIAG_RX] - f[ec - DIAG_RX]) -
                    (f[ec + 2 * DIAG_RX] - f[ec - 2 * DIAG_RX]));
      };
#pragma unroll
      for (int d = 0; d < 4; ++d) { uq[d] = uq[d + 1]; vq[d] = vq[d + 1]; }
      uq[4] = own_u;
      vq[4] = own_v;
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        pdw[d] = pdw[d + 1]; pxw[d] = pxw[d + 1]; pxv[d] = pxv[d + 1]; pdu[d] = pdu[d + 1];
      }
      pdw[2] = dy(sw);
      pxw[2] = dx(sw);
      pxv[2] = dx(sv);
      pdu[2] = dy(su);
      const int k = zl - 2;  // the plane whose z window is now complete
      if (active && k >= z0 && k < z1) {
        const DT dzu = s * (DT(8) * (uq[3] - uq[1]) - (uq[4] - uq[0]));
        const DT dzv = s * (DT(8) * (vq[3] - vq[1]) - (vq[4] - vq[0]));
        const DT wx = pdw[0] - dzv, wy = dzu - pxw[0], wz = pxv[0] - pdu[0];
        acc[2].add(wx * wx + wy * wy + wz * wz);
      }
    }
  }
  // block reduction: warp shuffles, then a fixed-order pass over warps
  __shared__ double red[DIAG_THREADS / 32][TGV_DIAG_COUNT];
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int m = 0; m < TGV_DIAG_COUNT; ++m) {
    double v = acc[m].value();
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
