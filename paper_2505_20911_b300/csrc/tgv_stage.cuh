// tgv_stage.cuh - the fused RHS + low-storage-RK stage kernel.
//
// One launch evaluates the residual R(Q) of the compressible Navier-Stokes
// equations (4th-order central differences, Blaisdell split convective terms,
// Sec. 2.3.1) at every grid point and folds the RK update of Sec. 3.1,
// Eqs. 3-4, into its epilogue:  Qt <- A Qt + dt R,  Q_out <- Q_in + B Qt.
// With EPI_RHS it writes R instead.
//
// Discretisation (the same discrete operator the FP64 oracle defines):
//   D f   = (-f[+2] + 8 f[+1] - 8 f[-1] + f[-2]) / 12h
//   D2 f  = (-f[+2] + 16 f[+1] - 30 f[0] + 16 f[-1] - f[-2]) / 12h^2
//   C_phi = 1/2 sum_j [D_j(u_j f) + u_j D_j f + f D_j u_j]      (Blaisdell; f = rho phi)
//   momentum i viscous = nu [sum_j D2_j u_i + 1/3 D2_i u_i + 1/3 D_i s_i],
//                        s_i = sum_{k != i} D_k u_k
//   energy   = -C_E - sum_j D_j(p u_j) + sum_j D2_j H_j
//              + nu [2 sum_{i<j} D_i D_j(u_i u_j) - 5/3 sum_j D_j(u_j s_j)],
//              H_j = kappa T + nu (|u|^2/2 + u_j^2/6)
//   (the viscous work d(u_i tau_ij)/dx_j and the heat flux rewritten exactly
//   in telescoping form, so mass, momentum and total energy are conserved to
//   round-off).
//
// Work decomposition (B300): a CTA owns a TX x TY column tile and marches in z
// over `zchunk` planes.  Each z plane of the tile plus a 2-point halo is read
// once from HBM (periodic wrap), converted to the compute type, and turned into
// primitives in a 5-plane shared-memory ring; every stencil tap afterwards is
// a shared-memory read.  Per plane:
//   load   : plane z+2 -> ring (conserved, u, v, w, p, T); sync
//   grads  : D_x u, D_y v of plane z+2 on the halo strips that need them;
//            centre plane z: D_z w, D_y(uv), D_z(uw), D_z(vw) on strips; sync
//   output : all terms at plane z for the TX x TY points, RK epilogue; sync
#pragma once

#include "tgv_common.cuh"

namespace tgv {

enum { EPI_RK = 0, EPI_RHS = 1 };

struct StageArgs {
  const void* q_in;   // Q layout, storage type TS
  void* q_out;        // Q layout, TS (EPI_RK)
  void* qt;           // Q layout, TT (EPI_RK)
  void* r_out;        // Q layout, TC (EPI_RHS)
  double a, b, dt;    // A_i, B_i, dt
  int read_qt;        // 0 when A_i == 0
  int write_qt;       // 0 on the last substep
  int zchunk;         // z planes per CTA
};

// Shared-memory fields of a ring plane.
enum { F_RHO = 0, F_RU, F_RV, F_RW, F_RE, F_U, F_V, F_W, F_P, F_T, F_DXU, F_DYV, NF };
// Per-centre-plane strip fields.
enum { S_DZW = 0, S_EYUV, S_EZUW, S_EZVW, NS };

template <int TX, int TY>
struct Tile {
  static constexpr int RX = TX + 4, RY = TY + 4, PL = RX * RY, NT = TX * TY;
  static constexpr int PER = (PL + NT - 1) / NT;
};

template <class TC, int TX, int TY>
constexpr size_t stage_smem_bytes() {
  return (size_t)(5 * NF + NS) * Tile<TX, TY>::PL * sizeof(TC);
}

template <class TS, class TT, class TC, class TA, int TX, int TY, int EPI>
__global__ void __launch_bounds__(TX * TY)
stage_kernel(const Problem P, const StageArgs S) {
  using TL = Tile<TX, TY>;
  constexpr int RX = TL::RX, PL = TL::PL, NT = TL::NT, PER = TL::PER;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* ring = reinterpret_cast<TC*>(smem_raw);  // [5][NF][PL]
  TC* scr = ring + 5 * NF * PL;                // [NS][PL]

  const int n = P.n;
  const long long nn = (long long)n * n, n3 = nn * n;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * S.zchunk;
  const int z1 = min(z0 + S.zchunk, n);
  const TS* __restrict__ q_in = static_cast<const TS*>(S.q_in);

  const TC c_inv12h = cvt<TC>(P.inv12h), c_inv12h2 = cvt<TC>(P.inv12h2);
  const TC c_gm1 = cvt<TC>(P.gm1), c_gM2 = cvt<TC>(P.gM2);
  const TC c_nu = cvt<TC>(P.nu), c_kappa = cvt<TC>(P.kappa);
  const TC c_rho0 = cvt<TC>(P.rho0), c_rhoE0 = cvt<TC>(P.rhoE0);
  const TC c_half = cvt<TC>(0.5), c_sixth = cvt<TC>(1.0 / 6.0), c_third = cvt<TC>(1.0 / 3.0);
  const TC c_8 = cvt<TC>(8.0), c_16 = cvt<TC>(16.0), c_30 = cvt<TC>(30.0);
  const TC c_2 = cvt<TC>(2.0), c_53 = cvt<TC>(5.0 / 3.0), c_zero = cvt<TC>(0.0);
  const bool blaisdell = (P.split == TGV_SPLIT_BLAISDELL);

  // In-plane global offsets of the halo-region points this thread loads.
  int roff[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int idx = tid + r * NT;
    roff[r] = -1;
    if (idx < PL) {
      int gx = (x0 - 2 + idx % RX) % n;
      if (gx < 0) gx += n;
      int gy = (y0 - 2 + idx / RX) % n;
      if (gy < 0) gy += n;
      roff[r] = gy * n + gx;
    }
  }

  auto D = [&](TC fm2, TC fm1, TC fp1, TC fp2) -> TC {  // raw first-derivative sum
    return c_8 * (fp1 - fm1) - (fp2 - fm2);
  };

  const int zbase = z0 - 2;
  for (int zl = z0 - 2; zl < z1 + 2; ++zl) {
    // ---------------------------------------------------------- load plane zl
    const int slot = (zl - zbase) % 5;
    {
      int zw = zl % n;
      if (zw < 0) zw += n;
      const long long zoff = (long long)zw * nn;
      TC* base = ring + slot * NF * PL;
#pragma unroll
      for (int r = 0; r < PER; ++r) {
        const int idx = tid + r * NT;
        if (idx < PL) {
          const long long o = zoff + roff[r];
          const TC rho = cvt<TC>(q_in[o]) + c_rho0;
          const TC ru = cvt<TC>(q_in[o + n3]);
          const TC rv = cvt<TC>(q_in[o + 2 * n3]);
          const TC rw = cvt<TC>(q_in[o + 3 * n3]);
          const TC rE = cvt<TC>(q_in[o + 4 * n3]) + c_rhoE0;
          const TC ri = recip(rho);
          const TC u = ru * ri, v = rv * ri, w = rw * ri;
          const TC ke = c_half * (ru * u + rv * v + rw * w);
          const TC p = c_gm1 * (rE - ke);
          base[F_RHO * PL + idx] = rho;
          base[F_RU * PL + idx] = ru;
          base[F_RV * PL + idx] = rv;
          base[F_RW * PL + idx] = rw;
          base[F_RE * PL + idx] = rE;
          base[F_U * PL + idx] = u;
          base[F_V * PL + idx] = v;
          base[F_W * PL + idx] = w;
          base[F_P * PL + idx] = p;
          base[F_T * PL + idx] = c_gM2 * p * ri;
        }
      }
    }
    __syncthreads();

    const int k = zl - 2;  // centre plane
    int sl[5];             // ring slots of planes k-2 .. k+2
#pragma unroll
    for (int d = 0; d < 5; ++d) sl[d] = (zl - 4 + d - zbase + 5) % 5;

    // --------------------------------- in-plane gradients of plane zl; strips
    {
      TC* base = ring + slot * NF * PL;
      const TC* U = base + F_U * PL;
      const TC* V = base + F_V * PL;
      for (int idx = tid; idx < PL; idx += NT) {
        const int rx = idx % RX, ry = idx / RX;
        if (rx >= 2 && rx < TX + 2)
          base[F_DXU * PL + idx] = c_inv12h * D(U[idx - 2], U[idx - 1], U[idx + 1], U[idx + 2]);
        if (ry >= 2 && ry < TY + 2)
          base[F_DYV * PL + idx] =
              c_inv12h * D(V[idx - 2 * RX], V[idx - RX], V[idx + RX], V[idx + 2 * RX]);
      }
      if (k >= z0) {
        const TC* P0 = ring + sl[2] * NF * PL;
        const TC* Pm2 = ring + sl[0] * NF * PL;
        const TC* Pm1 = ring + sl[1] * NF * PL;
        const TC* Pp1 = ring + sl[3] * NF * PL;
        const TC* Pp2 = ring + sl[4] * NF * PL;
        for (int idx = tid; idx < PL; idx += NT) {
          const int rx = idx % RX, ry = idx / RX;
          const bool xrow = (ry >= 2 && ry < TY + 2);  // x-strip (incl. tile)
          const bool ycol = (rx >= 2 && rx < TX + 2);  // y-strip (incl. tile)
          if (!(xrow || ycol)) continue;
          const TC wm2 = Pm2[F_W * PL + idx], wm1 = Pm1[F_W * PL + idx];
          const TC wp1 = Pp1[F_W * PL + idx], wp2 = Pp2[F_W * PL + idx];
          scr[S_DZW * PL + idx] = c_inv12h * D(wm2, wm1, wp1, wp2);
          if (xrow) {
            const TC* U0 = P0 + F_U * PL;
            const TC* V0 = P0 + F_V * PL;
            scr[S_EYUV * PL + idx] = c_inv12h * D(U0[idx - 2 * RX] * V0[idx - 2 * RX],
                                                  U0[idx - RX] * V0[idx - RX],
                                                  U0[idx + RX] * V0[idx + RX],
                                                  U0[idx + 2 * RX] * V0[idx + 2 * RX]);
            scr[S_EZUW * PL + idx] =
                c_inv12h * D(Pm2[F_U * PL + idx] * wm2, Pm1[F_U * PL + idx] * wm1,
                             Pp1[F_U * PL + idx] * wp1, Pp2[F_U * PL + idx] * wp2);
          }
          if (ycol) {
            scr[S_EZVW * PL + idx] =
                c_inv12h * D(Pm2[F_V * PL + idx] * wm2, Pm1[F_V * PL + idx] * wm1,
                             Pp1[F_V * PL + idx] * wp1, Pp2[F_V * PL + idx] * wp2);
          }
        }
      }
    }
    __syncthreads();

    // ------------------------------------------------------ output at plane k
    if (k >= z0 && x0 + tx < n && y0 + ty < n) {
      const int c = (ty + 2) * RX + (tx + 2);
      const TC* P0 = ring + sl[2] * NF * PL;
      TC fc[5];
#pragma unroll
      for (int f = 0; f < 5; ++f) fc[f] = P0[f * PL + c];
      const TC uc[3] = {P0[F_U * PL + c], P0[F_V * PL + c], P0[F_W * PL + c]};
      const TC Tc = P0[F_T * PL + c];
      const TC ke2c = c_half * (uc[0] * uc[0] + uc[1] * uc[1] + uc[2] * uc[2]);

      TC suf[5], udf[5];
#pragma unroll
      for (int f = 0; f < 5; ++f) { suf[f] = c_zero; udf[f] = c_zero; }
      TC div_raw = c_zero, dpu = c_zero, d2h = c_zero, dus = c_zero;
      TC dp[3], ds[3], d2u[3], d2own[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) { d2u[i] = c_zero; }

#pragma unroll
      for (int j = 0; j < 3; ++j) {
        TC dF[5];
#pragma unroll
        for (int f = 0; f < 5; ++f) dF[f] = c_zero;
        TC duj = c_zero, dpj = c_zero, dsj = c_zero, d2own_j = c_zero;
        TC d2uj[3] = {c_zero, c_zero, c_zero};
        TC d2hj = c_zero;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int s = (t < 2) ? (t - 2) : (t - 1);       // -2, -1, +1, +2
          const TC cs = (s == -2) ? cvt<TC>(1.0) : (s == -1) ? -c_8 : (s == 1) ? c_8 : cvt<TC>(-1.0);
          const TC ds2 = (s == -2 || s == 2) ? cvt<TC>(-1.0) : c_16;
          const TC* Pl;
          int e;
          if (j == 2) { Pl = ring + sl[2 + s] * NF * PL; e = c; }
          else { Pl = P0; e = c + (j == 0 ? s : s * RX); }
          TC f[5];
#pragma unroll
          for (int q = 0; q < 5; ++q) f[q] = Pl[q * PL + e];
          const TC uu = Pl[F_U * PL + e], vv = Pl[F_V * PL + e], ww = Pl[F_W * PL + e];
          const TC uj = (j == 0) ? uu : (j == 1) ? vv : ww;
          const TC pp = Pl[F_P * PL + e], TT = Pl[F_T * PL + e];
          TC sj;
          if (j == 0) sj = P0[F_DYV * PL + e] + scr[S_DZW * PL + e];
          else if (j == 1) sj = P0[F_DXU * PL + e] + scr[S_DZW * PL + e];
          else sj = Pl[F_DXU * PL + e] + Pl[F_DYV * PL + e];
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            dF[q] = dF[q] + cs * f[q];
            suf[q] = suf[q] + cs * (uj * f[q]);
          }
          duj = duj + cs * uj;
          dpj = dpj + cs * pp;
          dpu = dpu + cs * (pp * uj);
          d2uj[0] = d2uj[0] + ds2 * uu;
          d2uj[1] = d2uj[1] + ds2 * vv;
          d2uj[2] = d2uj[2] + ds2 * ww;
          const TC H = c_kappa * TT + c_nu * (c_half * (uu * uu + vv * vv + ww * ww) + c_sixth * (uj * uj));
          d2hj = d2hj + ds2 * H;
          dsj = dsj + cs * sj;
          dus = dus + cs * (uj * sj);
        }
        // centre tap of the second derivatives
        const TC Hc = c_kappa * Tc + c_nu * (ke2c + c_sixth * (uc[j] * uc[j]));
        d2hj = d2hj - c_30 * Hc;
#pragma unroll
        for (int i = 0; i < 3; ++i) d2u[i] = d2u[i] + (d2uj[i] - c_30 * uc[i]);
        d2own_j = d2uj[j] - c_30 * uc[j];
        d2own[j] = d2own_j;
        d2h = d2h + d2hj;
        div_raw = div_raw + duj;
        dp[j] = dpj;
        ds[j] = dsj;
#pragma unroll
        for (int q = 0; q < 5; ++q) udf[q] = udf[q] + uc[j] * dF[q];
      }

      // mixed second derivatives of u_i u_j (outer D over the strip fields)
      const TC mix =
          D(scr[S_EYUV * PL + c - 2], scr[S_EYUV * PL + c - 1], scr[S_EYUV * PL + c + 1],
            scr[S_EYUV * PL + c + 2]) +
          D(scr[S_EZUW * PL + c - 2], scr[S_EZUW * PL + c - 1], scr[S_EZUW * PL + c + 1],
            scr[S_EZUW * PL + c + 2]) +
          D(scr[S_EZVW * PL + c - 2 * RX], scr[S_EZVW * PL + c - RX], scr[S_EZVW * PL + c + RX],
            scr[S_EZVW * PL + c + 2 * RX]);

      const TC div = c_inv12h * div_raw;
      TC R[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        TC conv;
        if (blaisdell) conv = c_half * (c_inv12h * (suf[q] + udf[q]) + fc[q] * div);
        else conv = c_inv12h * suf[q];
        R[q] = -conv;
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const TC visc = c_nu * (c_inv12h2 * (d2u[i] + c_third * d2own[i]) + c_third * c_inv12h * ds[i]);
        R[1 + i] = R[1 + i] - c_inv12h * dp[i] + visc;
      }
      R[4] = R[4] - c_inv12h * dpu + c_inv12h2 * d2h + c_nu * c_inv12h * (c_2 * mix - c_53 * dus);

      const long long o = (long long)k * nn + (long long)(y0 + ty) * n + (x0 + tx);
      if constexpr (EPI == EPI_RHS) {
        TC* r_out = static_cast<TC*>(S.r_out);
#pragma unroll
        for (int q = 0; q < 5; ++q) r_out[o + q * n3] = R[q];
      } else {
        TS* q_out = static_cast<TS*>(S.q_out);
        TT* qt = static_cast<TT*>(S.qt);
        const TA a = cvt<TA>(S.a), b = cvt<TA>(S.b), dt = cvt<TA>(S.dt);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          TA qtn = dt * cvt<TA>(R[q]);
          if (S.read_qt) qtn = a * cvt<TA>(qt[o + q * n3]) + qtn;
          const TA qo = cvt<TA>(q_in[o + q * n3]) + b * qtn;
          q_out[o + q * n3] = cvt<TS>(qo);
          if (S.write_qt) qt[o + q * n3] = cvt<TT>(qtn);
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace tgv
