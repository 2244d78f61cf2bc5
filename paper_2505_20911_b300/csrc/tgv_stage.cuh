// tgv_stage.cuh - the fused RHS + low-storage-RK stage kernel.
//
// One launch evaluates the residual R(Q) of the compressible Navier-Stokes
// equations (4th-order central differences, split convective terms,
// Sec. 2.3.1) at every grid point and folds the RK update of Sec. 3.1,
// Eqs. 3-4, into its epilogue:  Qt <- A Qt + dt R,  Q_out <- Q_in + B Qt
// (rk_step keeps W = Qt/dt instead: W <- A W + R, Q_out <- Q_in + (B dt) W).
// With EPI_RHS it writes R instead.  With DIAG it also reduces the
// diagnostics of Sec. 4.1, Eqs. 11-12 of its input state.
//
// Discrete operator (identical to the FP64 oracle's, up to rounding order):
//   D f  = (-f[+2] + 8 f[+1] - 8 f[-1] + f[-2]) / 12h
//   D2 f = (-f[+2] + 16 f[+1] - 30 f[0] + 16 f[-1] - f[-2]) / 12h^2
//   C_c  = a sum_j D_j(u_j f_c) + b [sum_j u_j D_j f_c + f_c div u] (+ g kx_c)
//          (Blaisdell: a = b = 1/2;  divergence form: a = 1, b = 0; the
//          KGP, KEEP and Feiereisen variants add the terms kx of kgp_extra
//          and keep_extra)
//   R_rho   = -C_rho
//   R_m(i)  = -C_m(i) - D_i p + nu [sum_j (1 + delta_ij/3) D2_j u_i + 1/3 D_i s_i]
//   R_E     = -C_E - sum_j D_j(p u_j) + sum_j D2_j H_j
//             + nu [2 sum_{i<j} D_i D_j(u_i u_j) - 5/3 sum_j D_j(u_j s_j)]
//   s_i = sum_{k != i} D_k u_k,  H_j = kappa T + nu (|u|^2/2 + u_j^2/6).
// The pressure terms are merged with the convective fluxes of the same
// direction: a D_j(u_j rho u_j) + D_j p = D_j(a u_j rho u_j + p) and
// a D_j(u_j rho E) + D_j(p u_j) = D_j(u_j (a rho E + p)) (linearity of D).
//
// B300 work decomposition.  A CTA owns a TX x TY column tile and marches in z
// over `zchunk` planes; each thread owns NP consecutive x points (a "unit";
// NP = 2 pairs the FP32 arithmetic into f32x2 instructions and the shared
// loads into 64-bit accesses).  Each z plane of the tile plus a 2-point halo
// is read once from HBM (periodic wrap, or mirror images in the symmetric
// box; the next plane is staged into shared memory by cp.async while the
// current one is computed), converted to the compute type, and turned into
// primitives in a 5-plane shared-memory ring.  Per plane, with two CTA
// barriers:
//   1. primitives of the prefetched plane zl -> ring slot            | barrier
//   2. prefetch plane zl+1 (and the next centre plane's Qt); D_x u + D_y v
//      of plane zl (z-taps of s_z); centre plane k = zl-2: s_x, s_y and the
//      mixed-derivative fields on the tile and its x/y halo strips (and,
//      when the z taps come from the ring, every z-direction term of the
//      thread's unit)                                                | barrier
//   3. (the z-direction terms, when the thread's z taps come from its
//      register queue,) the x- and y-direction terms at plane k (centre
//      plane and strips only), assembly of R, RK epilogue.
#pragma once

#include "tgv_common.cuh"
#include "tgv_vec.cuh"

namespace tgv {

enum { EPI_RK = 0, EPI_RHS = 1 };
// Convective split families built as kernel variants: the quadratic forms
// (Blaisdell, divergence: runtime coefficients), the cubic KGP split, and KEEP
// (KGP for mass and momentum, the kinetic-energy and entropy preserving
// energy split of the two-point fluxes rho_bar u_bar e_bar
// + rho_bar u_bar (u_i u_i)~/2 + (p u)~).
// The Feiereisen quadratic split (printed in Sec. 2.3.1) is the fourth:
// 1/2 D_j(rho u_j phi) + 1/2 (phi D_j(rho u_j) + rho u_j D_j phi).
enum { SPL_QUAD = 0, SPL_KGP = 1, SPL_KEEP = 2, SPL_FEIER = 3 };
// RK epilogue flags fixed at compile time (kernel template argument RKF):
// read the increment, write it, keep it divided by dt, and (FP32 storage and
// arithmetic) plain encoding.  RKF_RUNTIME takes them from StageArgs/Problem.
// rk_step's three stages are the combinations RKF_STAGE(i).
// RKF_ENC_RT keeps only the encoding a run-time choice (the ensemble, whose
// instances may differ in it).
enum { RKF_RUNTIME = -1, RKF_READ = 1, RKF_WRITE = 2, RKF_SCALED = 4, RKF_PLAIN = 8, RKF_ENC_RT = 16 };
__host__ __device__ constexpr int RKF_STAGE(int i) {
  return (i != 0 ? RKF_READ : 0) | (i != 2 ? RKF_WRITE : 0) | RKF_SCALED | RKF_PLAIN;
}
__host__ __device__ constexpr int RKF_STAGE_ENC_RT(int i) {
  return (i != 0 ? RKF_READ : 0) | (i != 2 ? RKF_WRITE : 0) | RKF_SCALED | RKF_ENC_RT;
}

struct StageArgs {
  const void* q_in;   // Q layout, storage type TS
  void* q_out;        // Q layout, TS (EPI_RK)
  void* qt;           // Q layout, TT (EPI_RK)
  void* r_out;        // Q layout, TC (EPI_RHS)
  double* diag_part;  // [gridDim.x*gridDim.y*gridDim.z][TGV_DIAG_COUNT] (DIAG)
  double a, b, dt;    // A_i, B_i, dt
  int read_qt;        // 0 when A_i == 0
  int write_qt;       // 0 on the last substep
  int scaled_qt;      // 1: the increment is kept divided by dt (W = Qt/dt:
                      //    W <- A W + R, Q <- Q + (B dt) W), saving the dt
                      //    multiply; rk_step's Qt is internal scratch
  double bdt;         // B_i * dt (scaled_qt)
  int zchunk;         // z planes per CTA
  // z extent (0 = the periodic box: N planes, z wraps, field stride N^3).
  // A z-slab: nzl owned planes, stored after zg ghost planes and followed by
  // zg more in q_in / q_out (no wrap in z), field stride fs_q there; Qt and
  // r_out hold the owned planes only, field stride fs_t.
  int zg;
  int nzl;
  long long fs_q, fs_t;
  // A slab's global z of its first owned plane: in the symmetric box the
  // slab's ghost planes beyond a mirror face hold the raw values of the
  // mirrored planes, and the kernel recognises them by their global index.
  int zoff;
};

// Ring-plane fields (compute type).  The momenta are not kept: the taps of
// rho u, rho v and rho w are formed as rho * u, rho * v and rho * w (one
// multiply per tap instead of one shared-memory load; the stage is bound by
// shared-memory bandwidth, not by FP32 issue).
enum { F_RHO = 0, F_RE, F_U, F_V, F_W, F_P, F_H0, NFLD };
// Ring field of conserved component c (the momenta: none).
__host__ __device__ constexpr int cons_field(int c) { return c == 0 ? F_RHO : (c == 4 ? F_RE : -1); }
// Strip fields of the centre plane.
enum { S_SX = 0, S_SY, S_GX, S_GY, NSTRIP };
// Ring depth: phase A of centre plane k reads planes k-2..k+2; phase B reads
// only plane k and the strips, so the commit of plane k+3 (which follows the
// phase-B of plane k-1 and precedes the first barrier) may overwrite plane
// k-3's slot: 5 slots.
constexpr int NSLOT = 5;

template <int TX, int TY, int NP>
struct Geo {
  static_assert(TX % NP == 0, "tile width must be a multiple of the unit");
  static constexpr int TXU = TX / NP;       // threads per tile row
  static constexpr int NT = TXU * TY;       // threads per CTA
  static constexpr int RX = TX + 4, RY = TY + 4, PL = RX * RY;
  static constexpr int RXU = RX / NP;       // units per halo-region row
  static constexpr int PLU = RXU * RY;      // units in the halo region
  static constexpr int PERU = (PLU + NT - 1) / NT;  // region units per thread
  static constexpr int HALO_UNITS = PLU - NT;        // region units outside the tile
  static constexpr int HXU = 2 * (2 / NP) * TY;  // x-halo strip units (both sides)
  static constexpr int HYU = 4 * TXU;            // y-halo strip units (both sides)
  static constexpr int HU = HXU + HYU;
  static constexpr int PERH = (HU + NT - 1) / NT;
};

// Shared memory: ring, strips (compute type), then the cp.async staging of
// the raw planes (storage type) and one raw Qt plane of the tile.
template <class TS, class TT, class TC, int TX, int TY, int NP>
constexpr size_t stage_smem_bytes() {
  using G = Geo<TX, TY, NP>;
  return sizeof(TC) * ((size_t)NSLOT * NFLD * G::PL + (size_t)NSTRIP * G::PL) +
         sizeof(TS) * NP * 5 * (size_t)G::PLU +
         sizeof(TT) * NP * 5 * (size_t)G::NT;
}
// Largest dynamic shared memory a stage CTA may request (B300: 227 KB per CTA,
// less the static reduction buffer of the fused-diagnostics variant).
constexpr size_t STAGE_SMEM_LIMIT = 232448 - 2048;

// Asynchronous global -> shared copies of 4 or 8 bytes (one unit).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gmem_src), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <class V> struct Taps { V m2, m1, p1, p2; };

template <class V> __device__ __forceinline__ V dsum(const Taps<V>& t, V c8) {
  return fma(c8, t.p1 - t.m1, t.m2 - t.p2);  // 8(f+1 - f-1) - (f+2 - f-2)
}
template <class V> __device__ __forceinline__ V d2sum(const Taps<V>& t, V c, V c16, V cm30) {
  return fma(c16, t.p1 + t.m1, fma(cm30, c, -(t.p2 + t.m2)));
}
template <class V> __device__ __forceinline__ Taps<V> tmul(const Taps<V>& a, const Taps<V>& b) {
  return {a.m2 * b.m2, a.m1 * b.m1, a.p1 * b.p1, a.p2 * b.p2};
}
template <class V> __device__ __forceinline__ Taps<V> tfma(const Taps<V>& a, const Taps<V>& b,
                                                           const Taps<V>& c) {
  return {fma(a.m2, b.m2, c.m2), fma(a.m1, b.m1, c.m1), fma(a.p1, b.p1, c.p1), fma(a.p2, b.p2, c.p2)};
}
template <class V> __device__ __forceinline__ Taps<V> tscale(V s, const Taps<V>& a) {
  return {s * a.m2, s * a.m1, s * a.p1, s * a.p2};
}
template <class V> __device__ __forceinline__ Taps<V> taxpy(V s, const Taps<V>& a, const Taps<V>& c) {
  return {fma(s, a.m2, c.m2), fma(s, a.m1, c.m1), fma(s, a.p1, c.p1), fma(s, a.p2, c.p2)};
}

template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// The work of one CTA: the TX x TY column tile at (x0, y0), planes z0 to
// min(z0 + S.zchunk, n); `cta` indexes its diagnostics partials.
// Extra terms of the cubic KGP split for one direction j (the quarter weights
// of u_j D f_c and f_c D u_j are shared with the quadratic forms):
//   kx_c += rho D(u_j phi_c) + phi_c D(rho u_j) + (rho u_j) D phi_c + u_j phi_c D rho
// with phi = (1, u, v, w, E), E = rho E / rho; raw sums, scaled by 1/12h later.
// FULL = false keeps only phi D_j(rho u_j) + rho u_j D_j phi (the Feiereisen
// split's second part).
template <bool FULL = true, class V>
__device__ __forceinline__ void kgp_extra(const int j, const Taps<V>& U, const Taps<V>* Ui,
                                          const Taps<V>& F0, const Taps<V>& F4, const V* dF,
                                          const V* fc, const V* uc, const V& c8, V* kx) {
  const Taps<V> Et = tmul(F4, {rcp(F0.m2), rcp(F0.m1), rcp(F0.p1), rcp(F0.p2)});
  const V Ec = fc[4] * rcp(fc[0]);
  const V mj = fc[1 + j];
  // c = 0 (phi = 1): rho D u_j + D(rho u_j) + u_j D rho
  if constexpr (FULL) kx[0] = kx[0] + fma(fc[0], dsum(U, c8), fma(uc[j], dF[0], dF[1 + j]));
  else kx[0] = kx[0] + dF[1 + j];
#pragma unroll
  for (int c = 1; c < 5; ++c) {
    const Taps<V>& Ph = (c == 4) ? Et : Ui[c - 1];
    const V phc = (c == 4) ? Ec : uc[c - 1];
    const V dphi = dsum(Ph, c8);
    if constexpr (FULL) {
      const V duphi = dsum(tmul(U, Ph), c8);
      kx[c] = kx[c] + fma(fc[0], duphi, fma(phc, dF[1 + j], fma(mj, dphi, uc[j] * phc * dF[0])));
    } else {
      kx[c] = kx[c] + fma(phc, dF[1 + j], mj * dphi);
    }
  }
}

// KEEP energy terms of direction j beyond the KGP split of the internal
// energy, as raw sums added to kx[4] (which the assembly scales by 1/4 and
// 1/12h): the kinetic-energy split
//   sum_c [ m_j v_c D v_c + v_c D(u_j rho v_c) + rho v_c D(u_j v_c) + u_j v_c D(rho v_c) ]
// and four times the pressure work u_j D p + p D u_j.  Fm: taps of rho v_c.
template <class V>
__device__ __forceinline__ void keep_extra(const int j, const Taps<V>& U, const Taps<V>* Ui,
                                           const Taps<V>* Fm, const Taps<V>& Pt, const V* dF,
                                           const V* fc, const V* uc, const V& pc, const V& c8,
                                           const V& c4, V* kx) {
  const V mj = fc[1 + j];
  V acc = c4 * fma(uc[j], dsum(Pt, c8), pc * dsum(U, c8));
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const V vc = uc[c];
    acc = fma(mj * vc, dsum(Ui[c], c8), acc);
    acc = fma(vc, dsum(tmul(U, Fm[c]), c8), acc);
    acc = fma(fc[1 + c], dsum(tmul(U, Ui[c]), c8), acc);
    acc = fma(uc[j] * vc, dF[1 + c], acc);
  }
  kx[4] = kx[4] + acc;
}

template <class TS, class TT, class TC, class TA, int TX, int TY, int NP, int EPI, bool DIAG,
          int SPL = SPL_QUAD, int RKF = RKF_RUNTIME>
__device__ __forceinline__ void stage_tile(const Problem& P, const StageArgs& S, const int x0,
                                           const int y0, const int z0, const long long cta) {
  using G = Geo<TX, TY, NP>;
  using V = Vec<TC, NP>;
  using IO = UnitIO<TC, NP, TS>;
  constexpr int RX = G::RX, PL = G::PL, NT = G::NT, RXU = G::RXU, PLU = G::PLU;
  constexpr int PERU = G::PERU, TXU = G::TXU;
  constexpr int NF = NFLD;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* ring = reinterpret_cast<TC*>(smem_raw);         // [NSLOT][NF][PL]
  TC* strips = ring + NSLOT * NF * PL;                 // [NSTRIP][PL]

  const int n = P.n;
  const long long nn = (long long)n * n, n3 = nn * n;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TXU + tx;
  __builtin_assume(tx < TXU && ty < TY);  // the launch's block shape
  const int zg = S.zg, nzl = S.nzl > 0 ? S.nzl : n;
  const long long fsq = S.fs_q > 0 ? S.fs_q : n3, fst = S.fs_t > 0 ? S.fs_t : n3;
  const int z1 = min(z0 + S.zchunk, nzl);
  const TS* __restrict__ q_in = static_cast<const TS*>(S.q_in);

  const V c_inv12h = V::splat(cvt<TC>(P.inv12h)), c_inv12h2 = V::splat(cvt<TC>(P.inv12h2));
  const V c_gm1 = V::splat(cvt<TC>(P.gm1)), c_gM2 = V::splat(cvt<TC>(P.gM2));
  const V c_nu = V::splat(cvt<TC>(P.nu)), c_kappa = V::splat(cvt<TC>(P.kappa));
  const V c_rho0 = V::splat(cvt<TC>(P.rho0)), c_rhoE0 = V::splat(cvt<TC>(P.rhoE0));
  const V c_half = V::splat(cvt<TC>(0.5)), c_nu6 = V::splat(cvt<TC>(P.nu / 6.0));
  const V c_nuh = V::splat(cvt<TC>(0.5 * P.nu));
  const V c_8 = V::splat(cvt<TC>(8.0)), c_16 = V::splat(cvt<TC>(16.0));
  const V c_m30 = V::splat(cvt<TC>(-30.0)), c_2 = V::splat(cvt<TC>(2.0));
  const V c_43 = V::splat(cvt<TC>(4.0 / 3.0)), c_13 = V::splat(cvt<TC>(1.0 / 3.0));
  const V c_m53 = V::splat(cvt<TC>(-5.0 / 3.0)), c_one = V::splat(cvt<TC>(1.0));
  // convective split: a sum_j D_j(u_j f) + b (sum_j u_j D_j f + f div u) [+ b kx]
  const bool blaisdell = (P.split == TGV_SPLIT_BLAISDELL);
  constexpr bool CUBIC = SPL == SPL_KGP || SPL == SPL_KEEP, KEEP = SPL == SPL_KEEP;
  constexpr bool FEIER = SPL == SPL_FEIER, XTRA = SPL != SPL_QUAD;  // XTRA: kgp_extra terms
  // C = alpha sum_j D_j(u_j f) + beta (sum_j u_j D_j f + f div u) + gamma kx
  const V c_alpha = V::splat(cvt<TC>(CUBIC ? 0.25 : (FEIER || blaisdell ? 0.5 : 1.0)));
  const V c_beta = V::splat(cvt<TC>(CUBIC ? 0.25 : (!FEIER && blaisdell ? 0.5 : 0.0)));
  const V c_gam = V::splat(cvt<TC>(CUBIC ? 0.25 : (FEIER ? 0.5 : 0.0)));
  const V c_ig1 = V::splat(cvt<TC>(1.0 / P.gm1)), c_4 = V::splat(cvt<TC>(4.0));

  // ---- region units this thread loads and converts each plane.  Unit q < NT
  // is thread q's own tile unit; units q >= NT are the halo (rows 0-1, the
  // left/right columns of rows 2..TY+1, rows TY+2..TY+3).
  using RawS = typename UnitIO<TC, NP, TS>::Raw;
  using RawT = typename UnitIO<TA, NP, TT>::Raw;
  RawS* stage_q = reinterpret_cast<RawS*>(strips + NSTRIP * PL);       // [5][PLU]
  RawT* stage_t = reinterpret_cast<RawT*>(stage_q + 5 * PLU);         // [5][NT]
  const int zbase = z0 - 2;
  // one staging plane: the next raw plane is copied into it after every thread
  // has converted the current one (the commit precedes the CTA barrier)
  auto raw_plane = [&](int) -> RawS* { return stage_q; };
  // Global addresses are formed as a CTA-uniform 64-bit base (plane,
  // component) plus a 32-bit per-thread offset within the plane (n <= 1024).
  unsigned goff[PERU];
  int eoff[PERU], tform[PERU];  // tform: 1 swap lanes, 2 -rho u, 4 -rho v
  const bool sym = P.symmetric != 0;
#pragma unroll
  for (int r = 0; r < PERU; ++r) {
    const int q = tid + r * NT;
    goff[r] = 0;
    eoff[r] = 0;
    tform[r] = 0;
    if (q < PLU) {
      int rx, ry;
      if (q < NT) {
        rx = 2 + NP * (q % TXU);
        ry = 2 + q / TXU;
      } else {
        int h = q - NT;
        constexpr int side = 2 / NP;  // units per row on each side
        if (h < 2 * RXU) { ry = h / RXU; rx = (h % RXU) * NP; }
        else if ((h -= 2 * RXU) < TY * 2 * side) {
          ry = 2 + h / (2 * side);
          const int qq = h % (2 * side);
          rx = qq < side ? qq * NP : TX + 2 + (qq - side) * NP;
        } else {
          h -= TY * 2 * side;
          ry = TY + 2 + h / RXU;
          rx = (h % RXU) * NP;
        }
      }
      int gx = x0 - 2 + rx, gy = y0 - 2 + ry;
      bool fx = false, fy = false;
      // a unit starts at an even x and n is even, so it never straddles a face;
      // mirrored, its last point lands first: load from the mirror of that one
      gx = wrap_index(gx + (sym ? NP - 1 : 0), n, sym, &fx);
      if (!fx && sym) gx -= NP - 1;
      gy = wrap_index(gy, n, sym, &fy);
      goff[r] = (unsigned)(gy * n + gx);
      eoff[r] = ry * RX + rx;
      tform[r] = (fx && NP == 2 ? 1 : 0) | (fx ? 2 : 0) | (fy ? 4 : 0);
    }
  }
  const unsigned tile_off = (unsigned)((y0 + ty) * n + (x0 + NP * tx));
  const bool active_xy = (x0 + NP * tx < n) && (y0 + ty < n);
  auto prefetch = [&](int zl) {  // cp.async of raw plane zl into its staging slot
    bool fz;
    const int zw = zg ? zl + zg : wrap_near(zl, n, sym, &fz);
    const TS* plane = q_in + (long long)zw * nn;
    RawS* dst = raw_plane(zl);
#pragma unroll
    for (int r = 0; r < PERU; ++r) {
      const int q = tid + r * NT;
      if (q < PLU) {
#pragma unroll
        for (int c = 0; c < 5; ++c)
          cp_async<sizeof(RawS)>(dst + c * PLU + q, plane + c * fsq + goff[r]);
      }
    }
  };
  auto prefetch_qt = [&](int kq) {  // cp.async of this unit's Qt at plane kq
    if (!active_xy) return;
    const TT* qt = static_cast<const TT*>(S.qt);
    RawT* dst = stage_t;
#pragma unroll
    for (int c = 0; c < 5; ++c)
      cp_async<sizeof(RawT)>(dst + c * NT + tid, qt + (long long)kq * nn + c * fst + tile_off);
  };
  // The epilogue's Q_in of the own unit, in storage precision:
  //  - FP32 storage and arithmetic, plain encoding: rho and rho E of the
  //    centre plane are already in registers as exact copies of the stored
  //    values (fc below); the momenta, which the ring does not hold, come from
  //    global memory in the register-queue kernels (QM_GLOBAL) and otherwise
  //    from a three-plane register queue of the raw values carried from the
  //    plane loader (planes zl, zl-1, zl-2; zeroed first, so no entry is read
  //    before it is written);
  //  - otherwise: re-read from global memory at the start of phase B (a cache
  //    hit: the loader read it two planes earlier).
  constexpr bool QIN_FC = std::is_same<TS, float>::value && std::is_same<TC, float>::value;
  // Own-unit z taps from registers (FP32 or FP16 arithmetic, quadratic splits): the
  // loader keeps the primitives of its own unit for the last five planes
  // (zq[s][field] holds the plane committed to ring slot s), so the
  // z-direction terms read no shared memory; the ring still serves the x and
  // y taps and the z taps of the halo strips.  The z march is unrolled by the
  // ring depth, so every slot index is a compile-time constant and the
  // register queues are never shifted.  Only the 32x16 tile: the smaller
  // tiles hold two region units per thread and would spill (their FP32
  // kernel serves the FP64-state mode, two CTAs per SM).  Not in the
  // fused-diagnostics stage with run-time RK flags and the ensemble's
  // persistent kernel, whose extra live values would then spill.  Either
  // path computes the same values.
  constexpr bool ZQ = (std::is_same<TC, float>::value || std::is_same<TC, __half>::value) &&
                      NP == 2 && NT >= 256 && SPL == SPL_QUAD &&
                      !(DIAG && RKF == RKF_RUNTIME) && !(RKF != RKF_RUNTIME && (RKF & RKF_ENC_RT));
  V zq[ZQ ? NSLOT : 1][NF];
#pragma unroll
  for (int d = 0; d < (ZQ ? 5 : 1); ++d)
#pragma unroll
    for (int f = 0; f < NF; ++f) zq[d][f] = V::splat(cvt<TC>(0.0));
  constexpr bool RK_CT = RKF != RKF_RUNTIME;
  const bool read_qt = RK_CT ? (RKF & RKF_READ) != 0 : S.read_qt != 0;
  const bool write_qt = RK_CT ? (RKF & RKF_WRITE) != 0 : S.write_qt != 0;
  const bool scaled_qt = RK_CT ? (RKF & RKF_SCALED) != 0 : S.scaled_qt != 0;
  const bool qin_fc = QIN_FC && (RK_CT && !(RKF & RKF_ENC_RT) ? (RKF & RKF_PLAIN) != 0
                                                              : P.encoding == TGV_ENC_PLAIN);
  RawS qin_raw[5];
  // raw rho u, rho v, rho w of planes zl, zl-1, zl-2 (ring-path kernels; the
  // register-queue kernels re-read the momenta from global memory)
  constexpr bool QM_GLOBAL = ZQ;  // momenta re-read from global memory
  constexpr int NQM = QIN_FC && !QM_GLOBAL ? 3 : 1;
  RawS qm_q[NQM][3];
#pragma unroll
  for (int d = 0; d < NQM; ++d)
#pragma unroll
    for (int m = 0; m < 3; ++m) qm_q[d][m] = RawS{};
  auto commit = [&](int slot, int zl) {  // staged raw plane -> primitives in the ring
    TC* base = ring + slot * NF * PL;
    bool fz;  // a mirror image (symmetric box): beyond a face in global z
    wrap_near(zl + S.zoff, n, sym, &fz);
    const RawS* src = raw_plane(zl);
    // every unit's staged values are read before the first ring store (a
    // store may alias the staging for the compiler and hold later loads back)
    RawS raws[PERU][5];
#pragma unroll
    for (int r = 0; r < PERU; ++r) {
      const int q = tid + r * NT;
      if (q < PLU) {
#pragma unroll
        for (int c = 0; c < 5; ++c) raws[r][c] = src[c * PLU + q];
      }
    }
#pragma unroll
    for (int r = 0; r < PERU; ++r) {
      const int q = tid + r * NT;
      if (q < PLU) {
        const RawS* raw = raws[r];
        if constexpr (QIN_FC) {
          if (r == 0) {
#pragma unroll
            for (int m = 0; m < 3; ++m) {
              if constexpr (!QM_GLOBAL) {
                qm_q[2][m] = qm_q[1][m];
                qm_q[1][m] = qm_q[0][m];
                qm_q[0][m] = raw[1 + m];
              }
            }
          }
        }
        const int e = eoff[r];
        V rho = IO::conv(raw[0]) + c_rho0;
        V ru = IO::conv(raw[1]), rv = IO::conv(raw[2]), rw = IO::conv(raw[3]);
        V rE = IO::conv(raw[4]) + c_rhoE0;
        if (sym) {  // ghost of the symmetric box: mirror image, normal momentum odd
          const int tf = tform[r];
          if (tf & 1) {
            rho = rho.swapped(); ru = ru.swapped(); rv = rv.swapped();
            rw = rw.swapped(); rE = rE.swapped();
          }
          if (tf & 2) ru = -ru;
          if (tf & 4) rv = -rv;
          if (fz) rw = -rw;
        }
        const V ri = rcp(rho);
        const V uu = ru * ri, vv = rv * ri, ww = rw * ri;
        const V ke = c_half * fma(ru, uu, fma(rv, vv, rw * ww));
        const V p = c_gm1 * (rE - ke);
        const V T = c_gM2 * p * ri;
        const V h0 = fma(c_kappa, T, c_nuh * fma(uu, uu, fma(vv, vv, ww * ww)));
        if constexpr (ZQ) {
          if (r == 0) {  // the own unit
            zq[slot][F_RHO] = rho;
            zq[slot][F_RE] = rE;
            zq[slot][F_U] = uu;
            zq[slot][F_V] = vv;
            zq[slot][F_W] = ww;
            zq[slot][F_P] = p;
            zq[slot][F_H0] = h0;
          }
        }
        rho.store(base + F_RHO * PL + e);
        rE.store(base + F_RE * PL + e);
        uu.store(base + F_U * PL + e);
        vv.store(base + F_V * PL + e);
        ww.store(base + F_W * PL + e);
        p.store(base + F_P * PL + e);
        h0.store(base + F_H0 * PL + e);
      }
    }
  };

  // tap loaders on a plane-layout array f (offsets of the unit at e)
  auto xt = [&](const TC* f, int e, V& ctr) -> Taps<V> {
    if constexpr (NP == 1) {
      ctr = V::load(f + e);
      return {V::load(f + e - 2), V::load(f + e - 1), V::load(f + e + 1), V::load(f + e + 2)};
    } else {
      const V A = V::load(f + e - 2), B = V::load(f + e), C = V::load(f + e + 2);
      ctr = B;
      return {A, V::mix(A, B), V::mix(B, C), C};
    }
  };
  auto yt = [&](const TC* f, int e) -> Taps<V> {
    return {V::load(f + e - 2 * RX), V::load(f + e - RX), V::load(f + e + RX), V::load(f + e + 2 * RX)};
  };

  // diagnostics accumulators (per thread; per-point values are formed in the
  // compute type and the NP lanes of a unit summed, then accumulated by
  // DiagAcc: compensated FP32 sums in the FP32/FP16 kernels, FP64 in the FP64
  // ones; every thread's sum is added in FP64)
  using DA = DiagAcc<TC>;
  typename DA::A dacc[TGV_DIAG_COUNT];

  const int rxc = 2 + NP * tx, ryc = 2 + ty;
  const int ec = ryc * RX + rxc;        // unit centre in plane layout
  const V zero = V::splat(cvt<TC>(0.0));
  V szq[5];  // s_z = D_x u + D_y v of the own unit: of ring slot s (ZQ), else of planes zl-4 .. zl
#pragma unroll
  for (int d = 0; d < 5; ++d) szq[d] = zero;

  // halo-strip unit of this thread (fixed for the whole z march): its offset
  // in the plane layout and kind (1: x-halo unit, s_x and G_x; 2: y-halo
  // unit, s_y and G_y; 0: none)
  int strip_e[G::PERH], strip_kind[G::PERH];
#pragma unroll
  for (int r = 0; r < G::PERH; ++r) {
    const int h = tid + r * NT;
    strip_e[r] = 0;
    strip_kind[r] = 0;
    if (h < G::HXU) {
      constexpr int per_side = 2 / NP;
      const int row = h / (2 * per_side), q = h % (2 * per_side);
      const int rx = q < per_side ? q * NP : TX + 2 + (q - per_side) * NP;
      strip_e[r] = (2 + row) * RX + rx;
      strip_kind[r] = 1;
    } else if (h < G::HU) {
      const int hy = h - G::HXU;
      const int rowsel = hy / TXU, col = hy % TXU;
      const int ry = rowsel < 2 ? rowsel : TY + rowsel;  // 0,1,TY+2,TY+3
      strip_e[r] = ry * RX + 2 + col * NP;
      strip_kind[r] = 2;
    }
  }

  // s_z = D_x u + D_y v of the own unit at plane pl, pushed onto its queue
  auto push_sz = [&](const TC* pl, int slot) {
    V cdummy;
    const V dxu = dsum(xt(pl + F_U * PL, ec, cdummy), c_8);
    const V dyv = dsum(yt(pl + F_V * PL, ec), c_8);
    if constexpr (ZQ) {
      szq[slot] = c_inv12h * (dxu + dyv);
    } else {
#pragma unroll
      for (int d = 0; d < 4; ++d) szq[d] = szq[d + 1];
      szq[4] = c_inv12h * (dxu + dyv);
    }
  };

  prefetch(zbase);
  cp_async_commit();
  // Prologue: planes z0-2 .. z0+1 are no centre plane yet; they only fill the
  // ring and the s_z queue.  Each goes to a fresh ring slot and every thread
  // reads back only the staging units it copied itself, so one barrier per
  // plane suffices.
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int zl = zbase + i;  // ring slot i
    cp_async_wait<0>();
    commit(i, zl);
    __syncthreads();
    prefetch(zl + 1);  // z0 + 2 < z1 + 2: the main loop below consumes it
    cp_async_commit();
    push_sz(ring + i * NF * PL, i);
  }
  // ring slot of plane zl: (zl - zbase) mod NSLOT; the first centre plane's
  // iteration commits to slot 4
  constexpr int UNR = ZQ ? NSLOT : 1;
  for (int zl0 = z0 + 2; zl0 < z1 + 2; zl0 += NSLOT) {
#pragma unroll UNR
   for (int u = 0; u < NSLOT; ++u) {
    const int zl = zl0 + u;
    if (zl >= z1 + 2) break;
    const int slot = (4 + u) % NSLOT;
    // slots of planes k-2, k-1, k, k+1 of the centre plane k = zl - 2 (k+2: slot)
    const int sm2 = (slot + 1) % NSLOT, sm1 = (slot + 2) % NSLOT, sc0 = (slot + 3) % NSLOT,
              sp1 = (slot + 4) % NSLOT;
    cp_async_wait<0>();
    commit(slot, zl);
    __syncthreads();
    // this centre plane's Qt (its own group, which the epilogue waits for),
    // then the next raw plane (a second group, waited for by the next
    // iteration); one Qt staging plane suffices because every thread reads
    // only the unit it copied, in the epilogue of this same iteration
    if (EPI == EPI_RK && read_qt) {
      prefetch_qt(zl - 2);
      cp_async_commit();
    }
    if (zl + 1 < z1 + 2) prefetch(zl + 1);
    cp_async_commit();

    const int k = zl - 2;  // centre plane, z0 <= k < z1
    const TC* pk[5];  // ring planes k-2 .. k+2 = zl-4 .. zl: slots slot+1 .. slot+5 (mod NSLOT)
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      const int sd = slot + 1 + d;
      pk[d] = ring + (sd >= NSLOT ? sd - NSLOT : sd) * NF * PL;
    }
    TC* st = strips;

    // ---- phase A: s_z of plane zl (own unit, kept in registers) ...
    push_sz(ring + slot * NF * PL, slot);
    // ... then, for centre plane k: the strip fields of the tile and its halo,
    // and every z-direction term of the own unit (its z taps of u, v, w are
    // shared with the strips).  The partial sums stay in registers across the
    // barrier and phase B adds the x and y directions.
    // Per-unit values of the centre plane.  Phase A assigns each of them (the
    // z-direction terms are the first contribution to every sum, so no sum
    // starts from a zero fill).
    V fc[5], uc[3], h0c, div;
    V fcc[5];  // rho phi of the convective split (KEEP: rho e in place of rho E)
    V pc;      // centre pressure (KEEP)
    V suf[5], udf[5], d2u[3], ds[3], kx[5];
    V d2h, dus;
    V grad[3][3];  // grad[i][j] = raw D_j u_i (diagnostics)
    Taps<V> ux_c, uy_c, vy_c;  // x taps of u, y taps of u and v: phase A loads them, phase B reuses
    if constexpr (XTRA) {
#pragma unroll
      for (int c = 0; c < 5; ++c) kx[c] = zero;
    }
    const TC* P0 = pk[2];
    auto ztw = [&](int fld, int e) -> Taps<V> {
      return {V::load(pk[0] + fld * PL + e), V::load(pk[1] + fld * PL + e),
              V::load(pk[3] + fld * PL + e), V::load(pk[4] + fld * PL + e)};
    };
    // the own unit's z taps and centre values: the register queue (ZQ) or the ring
    auto zt = [&](int fld) -> Taps<V> {
      if constexpr (ZQ) {
        Taps<V> t{zq[sm2][fld], zq[sm1][fld], zq[sp1][fld], zq[slot][fld]};
        pin(t.m2);
        pin(t.m1);
        pin(t.p1);
        pin(t.p2);
        return t;
      } else {
        return ztw(fld, ec);
      }
    };
    auto zc = [&](int fld) -> V {
      if constexpr (ZQ) {
        V c = zq[sc0][fld];
        pin(c);
        return c;
      } else {
        return V::load(P0 + fld * PL + ec);
      }
    };
    // centre-plane values of the own unit (ucx: u, when the ring serves it)
    auto centre_values = [&](const V& ucx) {
      h0c = zc(F_H0);
      uc[0] = ZQ ? zc(F_U) : ucx;
      uc[1] = zc(F_V);
      uc[2] = zc(F_W);
      fc[0] = zc(F_RHO);
      fc[4] = zc(F_RE);
#pragma unroll
      for (int i = 0; i < 3; ++i) fc[1 + i] = fc[0] * uc[i];
#pragma unroll
      for (int c = 0; c < 5; ++c) fcc[c] = fc[c];
      if constexpr (KEEP) {
        pc = zc(F_P);
        fcc[4] = c_ig1 * pc;
      }
    };
    // z-direction terms (j = 2), the first contribution to every sum: in
    // phase A when the z taps come from the ring (they fill the warps that
    // have no halo strip), in phase B from the register queue (fewer values
    // live across the barrier)
    auto z_terms = [&]() {
      const Taps<V> uz = zt(F_U), vz = zt(F_V), wz = zt(F_W);
      const Taps<V>& U = wz;
      const Taps<V> aU = tscale(c_alpha, U);
      const Taps<V> Pt = zt(F_P);
      V dFz[5];
      Taps<V> F0z, F4z, Fmz[3];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const Taps<V> F = c == 3 ? tmul(F0z, U)
                          : c == 1 ? tmul(F0z, uz)
                          : c == 2 ? tmul(F0z, vz)
                          : ((KEEP && c == 4) ? tscale(c_ig1, Pt) : zt(cons_field(c)));
        const V dF = dsum(F, c_8);
        dFz[c] = dF;
        if (c == 0) F0z = F;
        if constexpr (XTRA) {
          if (c == 4) F4z = F;
        }
        if constexpr (KEEP) {
          if (c >= 1 && c <= 3) Fmz[c - 1] = F;
        }
        udf[c] = uc[2] * dF;
        if (c == 0) continue;
        Taps<V> g;
        if (c == 3) g = tfma(aU, F, Pt);                      // a w rho w + p
        else if (c == 4 && !KEEP) g = tmul(U, taxpy(c_alpha, F, Pt));  // w (a rho E + p)
        else g = tmul(aU, F);
        suf[c] = dsum(g, c_8);
        if (c == 3) suf[0] = c_alpha * dF;  // D_z(rho w)
      }
      if constexpr (XTRA) {
        const Taps<V> UZall[3] = {uz, vz, wz};
        kgp_extra<!FEIER>(2, U, UZall, F0z, F4z, dFz, fcc, uc, c_8, kx);
        if constexpr (KEEP) keep_extra(2, U, UZall, Fmz, Pt, dFz, fc, uc, pc, c_8, c_4, kx);
      }
      const Taps<V>* UZ[3] = {&uz, &vz, &wz};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const V d2 = d2sum(*UZ[i], uc[i], c_16, c_m30);
        d2u[i] = i == 2 ? c_43 * d2 : d2;
        if constexpr (DIAG) grad[i][2] = dsum(*UZ[i], c_8);
      }
      {
        const Taps<V> H = tfma(tscale(c_nu6, U), U, zt(F_H0));
        const V Hc = fma(c_nu6 * uc[2], uc[2], h0c);
        d2h = d2sum(H, Hc, c_16, c_m30);
      }
      {
        const Taps<V> Sj = ZQ ? Taps<V>{szq[sm2], szq[sm1], szq[sp1], szq[slot]}
                              : Taps<V>{szq[0], szq[1], szq[3], szq[4]};
        ds[2] = dsum(Sj, c_8);
        dus = dsum(tmul(U, Sj), c_8);
      }
    };
    {
      // own unit (tile point); its strip values are stored at the end of the
      // phase, after every ring load of the phase (a shared store may alias
      // the ring for the compiler, which then keeps later loads behind it)
      V own_sx, own_sy, own_gx, own_gy;
      {
        V ucx;
        const Taps<V> ux = xt(P0 + F_U * PL, ec, ucx);
        const Taps<V> uy = yt(P0 + F_U * PL, ec), vy = yt(P0 + F_V * PL, ec);
        ux_c = ux;
        uy_c = uy;
        vy_c = vy;
        const Taps<V> uz = zt(F_U), vz = zt(F_V), wz = zt(F_W);
        const V dxu = c_inv12h * dsum(ux, c_8);
        const V dyv = c_inv12h * dsum(vy, c_8);
        const V dzw = c_inv12h * dsum(wz, c_8);
        div = dxu + dyv + dzw;
        own_sx = dyv + dzw;
        own_sy = dxu + dzw;
        const V eyuv = dsum(tmul(uy, vy), c_8);
        const V ezuw = dsum(tmul(uz, wz), c_8);
        const V ezvw = dsum(tmul(vz, wz), c_8);
        own_gx = c_2 * c_inv12h * (eyuv + ezuw);
        own_gy = c_2 * c_inv12h * ezvw;
        if constexpr (!ZQ) {
          centre_values(ucx);
          z_terms();
        }
      }
      // halo strips: x-halo units need s_x and G_x, y-halo units s_y and G_y
#pragma unroll
      for (int r = 0; r < G::PERH; ++r) {
        const int e = strip_e[r];
        if (strip_kind[r] == 1) {
          const Taps<V> vy = yt(P0 + F_V * PL, e), wz = ztw(F_W, e);
          const V dyv = c_inv12h * dsum(vy, c_8);
          const V dzw = c_inv12h * dsum(wz, c_8);
          const V eyuv = dsum(tmul(yt(P0 + F_U * PL, e), vy), c_8);
          const V ezuw = dsum(tmul(ztw(F_U, e), wz), c_8);
          (dyv + dzw).store(st + S_SX * PL + e);
          (c_2 * c_inv12h * (eyuv + ezuw)).store(st + S_GX * PL + e);
        } else if (strip_kind[r] == 2) {
          V cd;
          const V dxu = c_inv12h * dsum(xt(P0 + F_U * PL, e, cd), c_8);
          const Taps<V> wz = ztw(F_W, e);
          const V dzw = c_inv12h * dsum(wz, c_8);
          const V ezvw = dsum(tmul(ztw(F_V, e), wz), c_8);
          (dxu + dzw).store(st + S_SY * PL + e);
          (c_2 * c_inv12h * ezvw).store(st + S_GY * PL + e);
        }
      }
      own_sx.store(st + S_SX * PL + ec);
      own_sy.store(st + S_SY * PL + ec);
      own_gx.store(st + S_GX * PL + ec);
      own_gy.store(st + S_GY * PL + ec);
    }
    __syncthreads();

    // ---- phase B: (z-direction terms from the register queue,) x- and
    // y-direction terms of the own unit, assembly, epilogue
    if (active_xy) {
      if constexpr (ZQ) {
        centre_values(zc(F_U));
        z_terms();
      }
      // the epilogue's Q_in of the own unit at plane k (see qin_raw), issued
      // here so that its latency hides behind the x/y terms
      if constexpr (EPI == EPI_RK) {
        {
          if (!qin_fc) {
#pragma unroll
            for (int c = 0; c < 5; ++c)
              qin_raw[c] = IO::load(q_in + (long long)(k + zg) * nn + c * fsq + tile_off);
          } else if constexpr (QM_GLOBAL) {
#pragma unroll
            for (int c = 1; c < 4; ++c)
              qin_raw[c] = IO::load(q_in + (long long)(k + zg) * nn + c * fsq + tile_off);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        auto tap = [&](int fld) -> Taps<V> {
          if (j == 0) { V cd; return xt(P0 + fld * PL, ec, cd); }
          return yt(P0 + fld * PL, ec);
        };
        const Taps<V> U = j == 0 ? ux_c : vy_c;
        const Taps<V> aU = tscale(c_alpha, U);
        const Taps<V> Pt = tap(F_P);
        const Taps<V> Wt = tap(F_W);
        Taps<V> Uall[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          Uall[i] = (i == j) ? U : (i == 2 ? Wt : ((j == 1 && i == 0) ? uy_c : tap(F_U + i)));
        V dFj[5];
        Taps<V> F0j, F4j, Fmj[3];
        // conserved components: D_j f_c, a D_j(u_j f_c) with merged pressure
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const Taps<V> F = c == 3 ? tmul(F0j, Wt)
                            : (c == 1 || c == 2) ? tmul(F0j, Uall[c - 1])
                            : ((KEEP && c == 4) ? tscale(c_ig1, Pt) : tap(cons_field(c)));
          const V dF = dsum(F, c_8);
          dFj[c] = dF;
          if (c == 0) F0j = F;
          if constexpr (XTRA) {
            if (c == 4) F4j = F;
          }
          if constexpr (KEEP) {
            if (c >= 1 && c <= 3) Fmj[c - 1] = F;
          }
          udf[c] = fma(uc[j], dF, udf[c]);
          if (c == 0) continue;
          Taps<V> g;
          if (c == 1 + j) g = tfma(aU, F, Pt);                 // a u_j rho u_j + p
          else if (c == 4 && !KEEP) g = tmul(U, taxpy(c_alpha, F, Pt));  // u_j (a rho E + p)
          else g = tmul(aU, F);
          suf[c] = suf[c] + dsum(g, c_8);
          if (c == 1 + j) suf[0] = fma(c_alpha, dF, suf[0]);  // D_j(rho u_j)
        }
        if constexpr (XTRA) kgp_extra<!FEIER>(j, U, Uall, F0j, F4j, dFj, fcc, uc, c_8, kx);
        if constexpr (KEEP) keep_extra(j, U, Uall, Fmj, Pt, dFj, fc, uc, pc, c_8, c_4, kx);
        // velocity second derivatives (and first derivatives for diagnostics)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const Taps<V>& Ui = Uall[i];
          const V w8 = (i == j) ? c_43 : c_one;
          d2u[i] = fma(w8, d2sum(Ui, uc[i], c_16, c_m30), d2u[i]);
          if constexpr (DIAG) grad[i][j] = dsum(Ui, c_8);
        }
        // heat flux + viscous kinetic-energy flux: D2_j H_j
        {
          const Taps<V> H = tfma(tscale(c_nu6, U), U, tap(F_H0));
          const V Hc = fma(c_nu6 * uc[j], uc[j], h0c);
          d2h = d2h + d2sum(H, Hc, c_16, c_m30);
        }
        // dilatation cross terms: D_j s_j and D_j(u_j s_j)
        {
          Taps<V> Sj;
          if (j == 0) { V cd; Sj = xt(st + S_SX * PL, ec, cd); }
          else Sj = yt(st + S_SY * PL, ec);
          ds[j] = dsum(Sj, c_8);
          dus = dus + dsum(tmul(U, Sj), c_8);
        }
      }
      // mixed second derivatives: outer D_x of G_x, outer D_y of G_y
      V gmix;
      {
        V cd;
        gmix = dsum(xt(st + S_GX * PL, ec, cd), c_8) + dsum(yt(st + S_GY * PL, ec), c_8);
      }

      V R[5];
#pragma unroll
      for (int c = 0; c < 5; ++c)
        R[c] = -(fma(c_inv12h, fma(c_beta, udf[c], XTRA ? fma(c_gam, kx[c], suf[c]) : suf[c]),
                     c_beta * fcc[c] * div));
#pragma unroll
      for (int i = 0; i < 3; ++i)
        R[1 + i] = fma(c_nu, fma(c_inv12h2, d2u[i], c_13 * c_inv12h * ds[i]), R[1 + i]);
      R[4] = fma(c_inv12h2, d2h, fma(c_nu * c_inv12h, fma(c_m53, dus, gmix), R[4]));

      if constexpr (DIAG) {
        // per-point diagnostics of the input state, in the compute type
        const V wx = c_inv12h * (grad[2][1] - grad[1][2]);
        const V wy = c_inv12h * (grad[0][2] - grad[2][0]);
        const V wz = c_inv12h * (grad[1][0] - grad[0][1]);
        const V ens = fma(wx, wx, fma(wy, wy, wz * wz));
        const V u2h = c_half * fma(uc[0], uc[0], fma(uc[1], uc[1], uc[2] * uc[2]));
        const V vals[8] = {u2h, fc[0] * u2h, ens, fc[0], fc[1], fc[2], fc[3], fc[4]};
        const int slot_of[8] = {0, 1, 2, 4, 5, 6, 7, 8};
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          TC t = vals[m].get(0);
#pragma unroll
          for (int e = 1; e < NP; ++e) t = t + vals[m].get(e);
          dacc[slot_of[m]].add(cvt<typename DA::In>(t));
        }
        int bad = 0;
#pragma unroll
        for (int e = 0; e < NP; ++e) {
          bool ok = true;
#pragma unroll
          for (int c = 0; c < 5; ++c) ok = ok && finite_val(fc[c].get(e));
          bad += ok ? 0 : 1;
        }
        dacc[9].add((typename DA::In)bad);
      }

      const long long ko = (long long)k * nn;  // centre plane (plus tile_off per thread)
      if constexpr (EPI == EPI_RHS) {
        TC* r_out = static_cast<TC*>(S.r_out);
#pragma unroll
        for (int c = 0; c < 5; ++c) R[c].store(r_out + ko + c * fst + tile_off);
      } else {
        TS* q_out = static_cast<TS*>(S.q_out);
        TT* qt = static_cast<TT*>(S.qt);
        const TA a = cvt<TA>(S.a), b = cvt<TA>(S.b), dt = cvt<TA>(S.dt);
        const TA bdt = cvt<TA>(S.bdt);
        if (read_qt) cp_async_wait<1>();  // all but the newest group (the next raw plane)
        const RawT* qts = stage_t;
        // With FP32 accumulation on two lanes the update runs as paired
        // instructions (f32x2): per lane the same fused multiply-adds, with the
        // same rounding, as the scalar form, which every other kernel that
        // inlines this epilogue (the ensemble's) shares.
        constexpr bool PAIRED = std::is_same<TA, float>::value && NP == 2;
        using VA = Vec<TA, NP>;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          TA qtn[NP], qo[NP], qin[NP], qold[NP], rc[NP];
          if constexpr (QIN_FC) {
            if (qin_fc) {
              if (c >= 1 && c <= 3) raw_elems<TA, NP>(QM_GLOBAL ? qin_raw[c] : qm_q[2][c - 1], qin);
              else {
#pragma unroll
                for (int e = 0; e < NP; ++e) qin[e] = cvt<TA>(fc[c].get(e));
              }
            } else {
              raw_elems<TA, NP>(qin_raw[c], qin);
            }
          } else {
            raw_elems<TA, NP>(qin_raw[c], qin);
          }
          if (read_qt) raw_elems<TA, NP>(qts[c * NT + tid], qold);
#pragma unroll
          for (int e = 0; e < NP; ++e) rc[e] = cvt<TA>(R[c].get(e));
          if constexpr (PAIRED) {
            VA v = scaled_qt ? VA(rc[0], rc[1]) : VA::splat(dt) * VA(rc[0], rc[1]);
            if (read_qt) v = fma(VA::splat(a), VA(qold[0], qold[1]), v);
            const VA w = fma(VA::splat(scaled_qt ? bdt : b), v, VA(qin[0], qin[1]));
            qtn[0] = v.get(0);
            qtn[1] = v.get(1);
            qo[0] = w.get(0);
            qo[1] = w.get(1);
          } else {
#pragma unroll
            for (int e = 0; e < NP; ++e) {
              // explicit fused multiply-adds (the rounding of the paired form)
              TA v = scaled_qt ? rc[e] : dt * rc[e];
              if (read_qt) v = fma_rn(a, qold[e], v);
              qtn[e] = v;
              qo[e] = fma_rn(scaled_qt ? bdt : b, v, qin[e]);
            }
          }
          UnitStore<TS, NP>::put(q_out + ko + zg * nn + c * fsq + tile_off, qo);
          if (write_qt) UnitStore<TT, NP>::put(qt + ko + c * fst + tile_off, qtn);
        }
      }
    }
   }
  }

  if constexpr (DIAG) {
    // CTA reduction: warp sums, then a fixed-order pass over warps
    __shared__ double red[NT / 32 + 1][TGV_DIAG_COUNT];
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int m = 0; m < TGV_DIAG_COUNT; ++m) {
      const double v = warp_sum(dacc[m].value());
      if (lane == 0) red[warp][m] = v;
    }
    __syncthreads();
    if (tid < TGV_DIAG_COUNT) {
      double v = 0.0;
      for (int w = 0; w < NT / 32; ++w) v += red[w][tid];
      S.diag_part[(size_t)cta * TGV_DIAG_COUNT + tid] = v;
    }
  }
}

// Resident CTAs per SM the register allocation targets: two for FP16
// arithmetic (128 registers per thread; its shared memory allows two CTAs,
// and 16 warps per SM run the pure-half stage about 20% faster than 8),
// otherwise one (the FP32/FP64 ring allows one CTA per SM).
template <class TC, int TX, int TY, int NP> constexpr int stage_min_blocks() {
  return std::is_same<TC, __half>::value ? 2 : 1;
}

template <class TS, class TT, class TC, class TA, int TX, int TY, int NP, int EPI, bool DIAG,
          int SPL = SPL_QUAD, int RKF = RKF_RUNTIME>
__global__ void __launch_bounds__(Geo<TX, TY, NP>::NT, stage_min_blocks<TC, TX, TY, NP>())
stage_kernel(const Problem P, const StageArgs S) {
  const long long cta = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  stage_tile<TS, TT, TC, TA, TX, TY, NP, EPI, DIAG, SPL, RKF>(
      P, S, blockIdx.x * TX, blockIdx.y * TY, blockIdx.z * S.zchunk, cta);
}

}  // namespace tgv
