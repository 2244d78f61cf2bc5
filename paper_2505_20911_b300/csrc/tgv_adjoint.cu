// tgv_adjoint.cu - hand-written discrete adjoint of the residual and of the
// low-storage RK3 step, and the gradient of the final kinetic energy.
//
// The paper has no adjoint; this differentiates the discrete scheme the
// forward kernels implement (4th-order central differences, Sec. 2.3.1; the
// RK update of Sec. 3.1, Eqs. 3-5), exactly (up to rounding), in FP64.
//
// Residual (the forward stage kernel's operator), D first / D2 second
// derivative, f_c = Q_c, u = m / rho, p, T, s_i = sum_{k!=i} D_k u_k:
//   R_c    = -a sum_j D_j(u_j f_c) - b sum_j u_j D_j f_c - b f_c div u
//   R_m(i) += -D_i p + nu [sum_j w_ij D2_j u_i + 1/3 D_i s_i],  w_ij = 1 + d_ij/3
//   R_E    += -sum_j D_j(p u_j) + sum_j D2_j H_j
//             + nu [2 sum_{i<j} D_i D_j(u_i u_j) - 5/3 sum_j D_j(u_j s_j)],
//   H_j = kappa T + nu (|u|^2/2 + u_j^2/6).
// On the periodic grid D^T = -D, D2^T = D2, (D_i D_j)^T = D_j D_i, so for a
// cotangent lam of R the cotangents of the pointwise quantities are
//   u_j : sum_c a (D_j lam_c) f_c - b sum_c lam_c D_j f_c + b D_j(sum_c lam_c f_c)
//         + p D_j lam_E + nu sum_j' w_jj' D2_j' lam_m(j)
//         + nu u_j sum_j' D2_j' lam_E + nu/3 u_j D2_j lam_E
//         + sum_{i!=j} 2 nu (D_i D_j lam_E) u_i + 5/3 nu (D_j lam_E) s_j
//         - sum_{i!=j} D_j sbar_i,
//   sbar_i = -nu/3 D_i lam_m(i) + 5/3 nu u_i D_i lam_E,
//   f_c : a sum_j u_j D_j lam_c + b sum_j D_j(lam_c u_j) - b lam_c div u,
//   p   : sum_i D_i lam_m(i) + sum_j u_j D_j lam_E,      T : kappa sum_j D2_j lam_E,
// and the pointwise chain rule through u = m/rho, p = (g-1)(E - |m|^2/(2 rho)),
// T = g M^2 p / rho gives the cotangent of Q.
//
// Kernels (one thread per grid point, FP64, periodic wrap by index):
//   adj_prim : W = (u, v, w, p, T) from Q
//   adj_s    : S = (s_x, s_y, s_z, sbar_x, sbar_y, sbar_z)
//   adj_main : everything else, qbar_out = qbar_in + scale * (dR/dQ)^T lam
//   adj_axpy : lam = a lam + b qbar (the Qt cotangent recursion)
#include <cmath>
#include <cstring>

#include "tgv_modes.cuh"

namespace tgv {

constexpr int ADJ_BX = 32, ADJ_BY = 8;

struct AdjGrid {
  int n;
  long long nn, n3;
  __device__ __forceinline__ long long at(int i, int j, int k) const {
    i = i < 0 ? i + n : (i >= n ? i - n : i);
    j = j < 0 ? j + n : (j >= n ? j - n : j);
    k = k < 0 ? k + n : (k >= n ? k - n : k);
    return (long long)k * nn + (long long)j * n + i;
  }
};

__device__ __forceinline__ void shift3(int d, int s, int& di, int& dj, int& dk) {
  di = (d == 0) ? s : 0;
  dj = (d == 1) ? s : 0;
  dk = (d == 2) ? s : 0;
}

// raw first/second-derivative sums of a field accessor g(i, j, k) in direction d
template <class F>
__device__ __forceinline__ double dsum(F g, int i, int j, int k, int d) {
  int a, b, c;
  shift3(d, 1, a, b, c);
  const double p1 = g(i + a, j + b, k + c), m1 = g(i - a, j - b, k - c);
  const double p2 = g(i + 2 * a, j + 2 * b, k + 2 * c), m2 = g(i - 2 * a, j - 2 * b, k - 2 * c);
  return 8.0 * (p1 - m1) - (p2 - m2);
}
template <class F>
__device__ __forceinline__ double d2sum(F g, int i, int j, int k, int d) {
  int a, b, c;
  shift3(d, 1, a, b, c);
  const double p1 = g(i + a, j + b, k + c), m1 = g(i - a, j - b, k - c);
  const double p2 = g(i + 2 * a, j + 2 * b, k + 2 * c), m2 = g(i - 2 * a, j - 2 * b, k - 2 * c);
  return 16.0 * (p1 + m1) - (p2 + m2) - 30.0 * g(i, j, k);
}

#define ADJ_INDEX                                                  \
  const int i = blockIdx.x * ADJ_BX + threadIdx.x;                 \
  const int j = blockIdx.y * ADJ_BY + threadIdx.y;                 \
  const int k = blockIdx.z;                                        \
  if (i >= P.n || j >= P.n) return;                                \
  const AdjGrid G{P.n, (long long)P.n * P.n, (long long)P.n * P.n * P.n}; \
  const long long o = G.at(i, j, k);

template <class TS>
__device__ __forceinline__ double qval(const TS* q, const Problem& P, long long o, long long n3, int c) {
  double v = Num<TS>::to_f64(q[o + c * n3]);
  if (c == 0) v += P.rho0;
  if (c == 4) v += P.rhoE0;
  return v;
}

// W = (u, v, w, p, T)
template <class TS>
__global__ void adj_prim_kernel(const Problem P, const TS* __restrict__ q, double* __restrict__ W) {
  ADJ_INDEX
  const long long n3 = G.n3;
  const double rho = qval(q, P, o, n3, 0);
  const double u = qval(q, P, o, n3, 1) / rho, v = qval(q, P, o, n3, 2) / rho,
               w = qval(q, P, o, n3, 3) / rho;
  const double p = P.gm1 * (qval(q, P, o, n3, 4) - 0.5 * rho * (u * u + v * v + w * w));
  W[o] = u;
  W[o + n3] = v;
  W[o + 2 * n3] = w;
  W[o + 3 * n3] = p;
  W[o + 4 * n3] = P.gM2 * p / rho;
}

// S = (s_i, sbar_i), i = x, y, z
__global__ void adj_s_kernel(const Problem P, const double* __restrict__ W,
                             const double* __restrict__ lam, double* __restrict__ S) {
  ADJ_INDEX
  const long long n3 = G.n3;
  const double s = P.inv12h;
  double dd[3];  // D_k u_k
  for (int d = 0; d < 3; ++d)
    dd[d] = s * dsum([&](int a, int b, int c) { return W[G.at(a, b, c) + d * n3]; }, i, j, k, d);
  for (int d = 0; d < 3; ++d) {
    S[o + d * n3] = dd[0] + dd[1] + dd[2] - dd[d];
    const double dlm = s * dsum([&](int a, int b, int c) { return lam[G.at(a, b, c) + (1 + d) * n3]; }, i, j, k, d);
    const double dle = s * dsum([&](int a, int b, int c) { return lam[G.at(a, b, c) + 4 * n3]; }, i, j, k, d);
    S[o + (3 + d) * n3] = -P.nu / 3.0 * dlm + 5.0 / 3.0 * P.nu * W[o + d * n3] * dle;
  }
}

// qbar_out = qbar_in + scale * (dR/dQ)^T lam   (qbar_in may be null: zero)
template <class TS>
__global__ void adj_main_kernel(const Problem P, const TS* __restrict__ q, const double* __restrict__ W,
                                const double* __restrict__ S, const double* __restrict__ lam,
                                const double* __restrict__ qbar_in, double* __restrict__ qbar_out,
                                double scale) {
  ADJ_INDEX
  const long long n3 = G.n3;
  const double s = P.inv12h, s2 = P.inv12h2, nu = P.nu;
  const bool blaisdell = (P.split == TGV_SPLIT_BLAISDELL);
  const double al = blaisdell ? 0.5 : 1.0, be = blaisdell ? 0.5 : 0.0;

  double f[5], lm[5];
  for (int c = 0; c < 5; ++c) {
    f[c] = qval(q, P, o, n3, c);
    lm[c] = lam[o + c * n3];
  }
  const double rho = f[0];
  const double u[3] = {W[o], W[o + n3], W[o + 2 * n3]};
  const double p = W[o + 3 * n3], T = W[o + 4 * n3];
  const double sv[3] = {S[o], S[o + n3], S[o + 2 * n3]};

  auto LAM = [&](int c) { return [&, c](int a, int b, int cc) { return lam[G.at(a, b, cc) + c * n3]; }; };
  auto QF = [&](int c) { return [&, c](int a, int b, int cc) { return qval(q, P, G.at(a, b, cc), n3, c); }; };

  double Dl[3][5];  // D_j lam_c
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 5; ++c) Dl[d][c] = s * dsum(LAM(c), i, j, k, d);
  double D2lE[3], D2lm[3][3];  // D2_j lam_E ; D2_j lam_m(i) as [i][j]
  for (int d = 0; d < 3; ++d) {
    D2lE[d] = s2 * d2sum(LAM(4), i, j, k, d);
    for (int c = 0; c < 3; ++c) D2lm[c][d] = s2 * d2sum(LAM(1 + c), i, j, k, d);
  }
  double div = 0.0;
  for (int d = 0; d < 3; ++d)
    div += s * dsum([&](int a, int b, int cc) { return W[G.at(a, b, cc) + d * n3]; }, i, j, k, d);

  double ub[3] = {0.0, 0.0, 0.0}, fb[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  double pb = 0.0, Tb = 0.0;
  // [A] -a D_j(u_j f_c)   [B] -b u_j D_j f_c   [C] -b f_c div
  for (int d = 0; d < 3; ++d) {
    for (int c = 0; c < 5; ++c) {
      ub[d] += al * Dl[d][c] * f[c];
      fb[c] += al * u[d] * Dl[d][c];
      const double dfc = s * dsum(QF(c), i, j, k, d);
      ub[d] -= be * lm[c] * dfc;
      fb[c] += be * s * dsum([&](int a, int b, int cc) {
        const long long y = G.at(a, b, cc);
        return lam[y + c * n3] * W[y + d * n3];
      }, i, j, k, d);
    }
    ub[d] += be * s * dsum([&](int a, int b, int cc) {
      const long long y = G.at(a, b, cc);
      double acc = 0.0;
      for (int c = 0; c < 5; ++c) acc += lam[y + c * n3] * qval(q, P, y, n3, c);
      return acc;
    }, i, j, k, d);
  }
  for (int c = 0; c < 5; ++c) fb[c] -= be * lm[c] * div;
  // [D] -D_i p  [E] -D_j(p u_j)
  for (int d = 0; d < 3; ++d) {
    pb += Dl[d][1 + d] + u[d] * Dl[d][4];
    ub[d] += p * Dl[d][4];
  }
  // [F] viscous momentum  [H] heat + viscous kinetic-energy flux
  double sumH = D2lE[0] + D2lE[1] + D2lE[2];
  Tb += P.kappa * sumH;
  for (int c = 0; c < 3; ++c) {
    for (int d = 0; d < 3; ++d) ub[c] += nu * (d == c ? 4.0 / 3.0 : 1.0) * D2lm[c][d];
    ub[c] += nu * u[c] * sumH + nu / 3.0 * u[c] * D2lE[c];
  }
  // [I] 2 nu D_i D_j (u_i u_j), i < j: cotangent 2 nu D_j D_i lam_E
  for (int a = 0; a < 3; ++a)
    for (int b2 = a + 1; b2 < 3; ++b2) {
      const double Mab = 2.0 * nu * s * s * dsum([&](int x, int y, int z) {
        return dsum(LAM(4), x, y, z, a);
      }, i, j, k, b2);
      ub[a] += Mab * u[b2];
      ub[b2] += Mab * u[a];
    }
  // [J] -5/3 nu D_j(u_j s_j)
  for (int d = 0; d < 3; ++d) ub[d] += 5.0 / 3.0 * nu * Dl[d][4] * sv[d];
  // [S] s_i = sum_{k != i} D_k u_k  ->  u_k : -sum_{i != k} D_k sbar_i
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 3; ++c) {
      if (c == d) continue;
      ub[d] -= s * dsum([&](int a, int b, int cc) { return S[G.at(a, b, cc) + (3 + c) * n3]; }, i, j, k, d);
    }
  // chain rule to Q
  const double pbt = pb + Tb * P.gM2 / rho;
  const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double qb[5];
  qb[0] = fb[0] - (ub[0] * u[0] + ub[1] * u[1] + ub[2] * u[2]) / rho + pbt * P.gm1 * 0.5 * u2 -
          Tb * T / rho;
  for (int c = 0; c < 3; ++c) qb[1 + c] = fb[1 + c] + ub[c] / rho - pbt * P.gm1 * u[c];
  qb[4] = fb[4] + pbt * P.gm1;
  for (int c = 0; c < 5; ++c) {
    const double base = qbar_in ? qbar_in[o + c * n3] : 0.0;
    qbar_out[o + c * n3] = base + scale * qb[c];
  }
}

// lam = a * lam + b * qbar (5 fields)
__global__ void adj_axpy_kernel(long long total, double a, double b, double* __restrict__ lam,
                                const double* __restrict__ qbar) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    lam[t] = (a == 0.0 ? 0.0 : a * lam[t]) + b * qbar[t];  // a = 0: lam is not read
}

// Cotangent of J = <|u|^2 / 2> = <|m|^2 / (2 rho^2)> (mean over points) at Q:
// dJ/drho = -|u|^2 / (rho N^3), dJ/dm_i = u_i / (rho N^3), dJ/dE = 0.
template <class TS>
__global__ void ke_grad_kernel(const Problem P, const TS* __restrict__ q, double* __restrict__ qbar) {
  ADJ_INDEX
  const long long n3 = G.n3;
  const double inv = 1.0 / (double)n3;
  const double rho = qval(q, P, o, n3, 0);
  double u2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double uc = qval(q, P, o, n3, 1 + c) / rho;
    u2 += uc * uc;
    qbar[o + (1 + c) * n3] = uc / rho * inv;
  }
  qbar[o] = -u2 / rho * inv;
  qbar[o + 4 * n3] = 0.0;
}

// ------------------------------------------------------------- host drivers
static dim3 adj_grid(int n) { return dim3((n + ADJ_BX - 1) / ADJ_BX, (n + ADJ_BY - 1) / ADJ_BY, n); }

// (dR/dQ)^T lam at state q into qbar_out (+ qbar_in, scaled); ws: 11 fields.
template <class TS>
static cudaError_t vjp_launch(const Problem& P, const void* q, const double* lam,
                              const double* qbar_in, double* qbar_out, double scale, double* ws,
                              cudaStream_t st) {
  const long long n3 = (long long)P.n * P.n * P.n;
  double* W = ws;
  double* S = ws + 5 * n3;
  const dim3 g = adj_grid(P.n), b(ADJ_BX, ADJ_BY);
  adj_prim_kernel<TS><<<g, b, 0, st>>>(P, static_cast<const TS*>(q), W);
  adj_s_kernel<<<g, b, 0, st>>>(P, W, lam, S);
  adj_main_kernel<TS><<<g, b, 0, st>>>(P, static_cast<const TS*>(q), W, S, lam, qbar_in, qbar_out,
                                       scale);
  return cudaGetLastError();
}

static cudaError_t vjp_dispatch(const tgv_config& c, const Problem& P, const void* q,
                                const double* lam, const double* qbar_in, double* qbar_out,
                                double scale, double* ws, cudaStream_t st) {
  if (c.q_storage == TGV_F64) return vjp_launch<double>(P, q, lam, qbar_in, qbar_out, scale, ws, st);
  return vjp_launch<float>(P, q, lam, qbar_in, qbar_out, scale, ws, st);
}

static cudaError_t axpy_launch(long long total, double a, double b, double* lam, const double* qbar,
                               cudaStream_t st) {
  const long long blocks = (total + 255) / 256;
  adj_axpy_kernel<<<(unsigned)(blocks < 148 * 32 ? blocks : 148 * 32), 256, 0, st>>>(total, a, b,
                                                                                     lam, qbar);
  return cudaGetLastError();
}

// Adjoint modes: FP64 forward/adjoint, or the FP32 forward with an FP64 adjoint.
static bool adjoint_mode_ok(const tgv_config& c) {
  const bool f64 = c.q_storage == TGV_F64 && c.qt_storage == TGV_F64 && c.compute == TGV_F64 &&
                   c.accumulate == TGV_F64;
  const bool f32 = c.q_storage == TGV_F32 && c.qt_storage == TGV_F32 && c.compute == TGV_F32 &&
                   c.accumulate == TGV_F32;
  return (f64 || f32) && c.encoding == TGV_ENC_PLAIN &&
         (c.split_form == TGV_SPLIT_BLAISDELL || c.split_form == TGV_SPLIT_DIVERGENCE) &&
         !(c.flags & TGV_FLAG_SYMMETRIC);
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace tgv

using namespace tgv;

extern "C" {

size_t tgv_adjoint_workspace_bytes(const tgv_config* cfg) {
  if (tgv_check_config(cfg) != TGV_OK || !adjoint_mode_ok(*cfg)) return 0;
  const size_t n3 = (size_t)cfg->n * cfg->n * cfg->n;
  return al256(16 * n3 * sizeof(double));
}

int32_t rhs_vjp(const tgv_config* cfg, const void* q, const double* lam, double* q_bar,
                void* workspace, size_t ws_bytes, void* stream) {
  int32_t s = tgv_check_config(cfg);
  if (s != TGV_OK) return s;
  if (!adjoint_mode_ok(*cfg)) return TGV_ERR_UNSUPPORTED;
  if (!q || !lam || !q_bar) return TGV_ERR_ARG;
  if (!workspace || ws_bytes < tgv_adjoint_workspace_bytes(cfg)) return TGV_ERR_WORKSPACE;
  const Problem P = make_problem(*cfg);
  cudaError_t e = vjp_dispatch(*cfg, P, q, lam, nullptr, q_bar, 1.0, static_cast<double*>(workspace),
                               static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? TGV_OK : TGV_ERR_CUDA;
}

// One reverse RK3 step: q_bar (in: cotangent of Q^{n+1}, out: of Q^n).
static int32_t step_adjoint_impl(const tgv_config& c, const Problem& P, const void* const st_in[3],
                                 double* q_bar, double dt, double* lam, double* ws,
                                 cudaStream_t st) {
  const long long total = 5LL * c.n * c.n * c.n;
  for (int i = 2; i >= 0; --i) {
    const double a_next = (i == 2) ? 0.0 : RK_A[i + 1];
    cudaError_t e = axpy_launch(total, a_next, RK_B[i], lam, q_bar, st);
    if (e != cudaSuccess) return TGV_ERR_CUDA;
    e = vjp_dispatch(c, P, st_in[i], lam, q_bar, q_bar, dt, ws, st);
    if (e != cudaSuccess) return TGV_ERR_CUDA;
  }
  return TGV_OK;
}

int32_t rk_step_adjoint(const tgv_config* cfg, const void* stage_inputs, double* q_bar, double dt,
                        void* workspace, size_t ws_bytes, void* stream) {
  int32_t s = tgv_check_config(cfg);
  if (s != TGV_OK) return s;
  if (!adjoint_mode_ok(*cfg)) return TGV_ERR_UNSUPPORTED;
  if (!stage_inputs || !q_bar || !std::isfinite(dt)) return TGV_ERR_ARG;
  const size_t need = tgv_adjoint_workspace_bytes(cfg);
  if (!workspace || ws_bytes < need) return TGV_ERR_WORKSPACE;
  const Problem P = make_problem(*cfg);
  const size_t qb = tgv_state_bytes(cfg);
  const char* base = static_cast<const char*>(stage_inputs);
  const void* st_in[3] = {base, base + qb, base + 2 * qb};
  const long long n3 = (long long)cfg->n * cfg->n * cfg->n;
  double* ws = static_cast<double*>(workspace);
  return step_adjoint_impl(*cfg, P, st_in, q_bar, dt, ws + 11 * n3, ws,
                           static_cast<cudaStream_t>(stream));
}

size_t tgv_grad_workspace_bytes(const tgv_config* cfg, int32_t nsteps, int32_t ckpt_every) {
  if (tgv_check_config(cfg) != TGV_OK || !adjoint_mode_ok(*cfg) || nsteps < 1 || ckpt_every < 1)
    return 0;
  const size_t n3 = (size_t)cfg->n * cfg->n * cfg->n;
  const size_t qb = al256(tgv_state_bytes(cfg)), qtb = al256(tgv_qt_bytes(cfg));
  const size_t nck = (size_t)(nsteps + ckpt_every - 1) / ckpt_every;
  const size_t seg = 3 * (size_t)ckpt_every + 1;
  return nck * qb + seg * qb + qtb + al256(5 * n3 * sizeof(double)) +
         tgv_adjoint_workspace_bytes(cfg) + al256(tgv_workspace_bytes(cfg)) + 256;
}

int32_t tgv_grad_final_ke(const tgv_config* cfg, const void* q0, double dt, int32_t nsteps,
                          int32_t ckpt_every, double* grad_mom, double* j_out, void* workspace,
                          size_t ws_bytes, void* stream) {
  int32_t s = tgv_check_config(cfg);
  if (s != TGV_OK) return s;
  if (!adjoint_mode_ok(*cfg)) return TGV_ERR_UNSUPPORTED;
  if (!q0 || !grad_mom || !j_out || nsteps < 1 || ckpt_every < 1 || !std::isfinite(dt) || !(dt > 0))
    return TGV_ERR_ARG;
  if (!(cfg->flags & TGV_FLAG_ALLOW_UNSTABLE_DT) && dt > tgv_dt_max(cfg)) return TGV_ERR_UNSTABLE_DT;
  if (!workspace || ws_bytes < tgv_grad_workspace_bytes(cfg, nsteps, ckpt_every))
    return TGV_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Problem P = make_problem(*cfg);
  const long long n3 = (long long)cfg->n * cfg->n * cfg->n;
  const size_t qb = al256(tgv_state_bytes(cfg)), qraw = tgv_state_bytes(cfg);
  const size_t qtb = al256(tgv_qt_bytes(cfg));
  const int nck = (nsteps + ckpt_every - 1) / ckpt_every;
  const int segn = 3 * ckpt_every + 1;
  char* w = static_cast<char*>(workspace);
  char* ckpt = w;
  char* seg = ckpt + (size_t)nck * qb;
  void* qt = seg + (size_t)segn * qb;
  double* qbar = reinterpret_cast<double*>(static_cast<char*>(qt) + qtb);
  double* adjws = reinterpret_cast<double*>(reinterpret_cast<char*>(qbar) + al256(5 * n3 * 8));
  double* lam = adjws + 11 * n3;
  char* diagws = reinterpret_cast<char*>(adjws) + tgv_adjoint_workspace_bytes(cfg);
  double* diag_out = reinterpret_cast<double*>(diagws + al256(tgv_workspace_bytes(cfg)));
  auto slot = [&](int m) -> void* { return seg + (size_t)m * qb; };

  // forward with checkpoints Q_0, Q_c, Q_2c, ... (seg slots 0/1 as ping-pong)
  NvtxRange fwd_range("tgv adjoint: forward with checkpoints");
  TGV_CUDA_TRY(cudaMemcpyAsync(slot(0), q0, qraw, cudaMemcpyDeviceToDevice, st));
  int cur = 0;
  for (int m = 0; m < nsteps; ++m) {
    if (m % ckpt_every == 0)
      TGV_CUDA_TRY(cudaMemcpyAsync(ckpt + (size_t)(m / ckpt_every) * qb, slot(cur), qraw,
                                   cudaMemcpyDeviceToDevice, st));
    for (int i = 0; i < 3; ++i) {
      s = rk_substep(cfg, slot(cur), slot(cur ^ 1), qt, i, dt, stream);
      if (s != TGV_OK) return s;
      cur ^= 1;
    }
  }
  // J = K(Q_N) and its cotangent
  s = diagnostics_reduce(cfg, slot(cur), diag_out, diagws, tgv_workspace_bytes(cfg), stream);
  if (s != TGV_OK) return s;
  TGV_CUDA_TRY(cudaMemcpyAsync(j_out, diag_out, sizeof(double), cudaMemcpyDeviceToDevice, st));
  const dim3 g = adj_grid(cfg->n), b(ADJ_BX, ADJ_BY);
  if (cfg->q_storage == TGV_F64)
    ke_grad_kernel<double><<<g, b, 0, st>>>(P, static_cast<const double*>(slot(cur)), qbar);
  else
    ke_grad_kernel<float><<<g, b, 0, st>>>(P, static_cast<const float*>(slot(cur)), qbar);
  TGV_CUDA_TRY(cudaGetLastError());

  // reverse sweep, one checkpoint segment at a time: recompute the segment
  // keeping every stage input, then run the step adjoints backwards
  for (int sgi = nck - 1; sgi >= 0; --sgi) {
    NvtxRange seg_range("tgv adjoint: segment recompute + reverse");
    const int m0 = sgi * ckpt_every;
    const int m1 = (m0 + ckpt_every < nsteps) ? m0 + ckpt_every : nsteps;
    TGV_CUDA_TRY(cudaMemcpyAsync(slot(0), ckpt + (size_t)sgi * qb, qraw, cudaMemcpyDeviceToDevice, st));
    for (int m = m0; m < m1; ++m) {
      const int b0 = 3 * (m - m0);
      for (int i = 0; i < 3; ++i) {
        s = rk_substep(cfg, slot(b0 + i), slot(b0 + i + 1), qt, i, dt, stream);
        if (s != TGV_OK) return s;
      }
    }
    for (int m = m1 - 1; m >= m0; --m) {
      const int b0 = 3 * (m - m0);
      const void* st_in[3] = {slot(b0), slot(b0 + 1), slot(b0 + 2)};
      s = step_adjoint_impl(*cfg, P, st_in, qbar, dt, lam, adjws, st);
      if (s != TGV_OK) return s;
    }
  }
  // dJ/d(rho u_0, rho v_0, rho w_0)
  TGV_CUDA_TRY(cudaMemcpyAsync(grad_mom, qbar + n3, 3 * n3 * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
  return TGV_OK;
}

}  // extern "C"
