/*
 * tgv.h - C ABI of the B300 (sm_103a) Taylor-Green-vortex hot path.
 *
 * The library advances the compressible Navier-Stokes equations on a periodic
 * N^3 grid (or the mirror-symmetric box of the paper's TGSym runs, see
 * TGV_FLAG_SYMMETRIC) with explicit 4th-order central differences
 * (arXiv 2505.20911, Sec. 2.3.1) and the low-storage 3-stage Runge-Kutta
 * scheme of Sec. 3.1, Eqs. 3-5, starting from the Taylor-Green field of
 * Sec. 4.1, Eqs. 6-10.
 *
 * Conventions shared by every entry point
 *  - Layout: a state Q is 5 planar fields (rho, rho*u, rho*v, rho*w, rho*E),
 *    each N^3 contiguous elements, x fastest: element (c, k, j, i) lives at
 *    offset (c*N + k)*N*N + j*N + i  (c field, k = z, j = y, i = x index),
 *    grid point x_i = i*L/N.  Qt (the Runge-Kutta increment) has the same
 *    layout.  Element types are given by the config (tgv_dtype).
 *  - Ownership: the caller allocates every buffer (device memory unless the
 *    name says host) and keeps ownership.  Apart from the ensemble handle
 *    (tgv_ensemble_create / tgv_ensemble_destroy), the library allocates no
 *    memory; scratch space is a caller-provided device workspace whose size a
 *    *_workspace_bytes query returns.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *    Work is enqueued on it; functions return without synchronising unless
 *    stated.  Buffers must not be touched by other streams meanwhile.
 *  - Errors: every function returns a tgv_status.  Arguments are validated on
 *    the host before any CUDA call; a failing CUDA call maps to TGV_ERR_CUDA.
 *    Nothing aborts, traps on the device, or prints.
 *  - Encoding (reading of Sec. 4.2's failure of pure FP16 storage): with
 *    TGV_ENC_OFFSET, stored rho and rho*E are the deviations from the uniform
 *    base state rho0 = 1 and (rho E)0 = 1/(gamma (gamma-1) M^2); kernels add the
 *    offsets back in the compute type.  TGV_ENC_PLAIN stores the plain values.
 */
#ifndef TGV_H_
#define TGV_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TGV_ABI_VERSION 1
#define TGV_DIAG_COUNT 10

typedef enum { TGV_F64 = 0, TGV_F32 = 1, TGV_BF16 = 2, TGV_F16 = 3 } tgv_dtype;

typedef enum {
  TGV_OK = 0,
  TGV_ERR_ARG = -1,          /* invalid argument (null pointer, bad size)      */
  TGV_ERR_UNSUPPORTED = -2,  /* valid but not built (precision combination)    */
  TGV_ERR_CUDA = -3,         /* a CUDA runtime call failed                     */
  TGV_ERR_NONFINITE = -4,    /* a diagnostic found NaN/Inf in the state        */
  TGV_ERR_UNSTABLE_DT = -5,  /* dt above the acoustic stability limit          */
  TGV_ERR_TIMEOUT = -6,      /* a bounded device wait ran out                  */
  TGV_ERR_WORKSPACE = -7     /* workspace null or smaller than required        */
} tgv_status;

/* Convective split forms (Sec. 2.3.1, Eq. 1; the study of Sec. 4.2):
 * Blaisdell quadratic (default), plain divergence form, the Feiereisen
 * quadratic form printed in Sec. 2.3.1 (1/2 D_j(rho u_j phi)
 * + 1/2 (phi D_j(rho u_j) + rho u_j D_j phi)), KGP cubic, and KEEP
 * (kinetic energy and entropy preserving: KGP for mass and momentum; for the
 * energy, KGP of the internal energy, the kinetic-energy split of the
 * two-point flux rho_bar u_bar (u_i u_i)~/2 and the pressure work
 * u_j D_j p + p D_j u_j; the paper cites it without printing it).
 * Every split is built for every precision mode of rk_step, rk_substep,
 * rhs_eval and the slab stage; Feiereisen, KGP and KEEP return
 * TGV_ERR_UNSUPPORTED in the adjoint and in the ensemble. */
typedef enum {
  TGV_SPLIT_BLAISDELL = 0,
  TGV_SPLIT_DIVERGENCE = 1,
  TGV_SPLIT_KGP = 2,
  TGV_SPLIT_KEEP = 3,
  TGV_SPLIT_FEIEREISEN = 4
} tgv_split;
typedef enum { TGV_ENC_PLAIN = 0, TGV_ENC_OFFSET = 1 } tgv_encoding;

/* Flags of tgv_config.flags */
#define TGV_FLAG_ALLOW_UNSTABLE_DT 1  /* skip the dt stability check            */
#define TGV_FLAG_CHECK_FINITE 2       /* rk_step: after each diagnostics record,
                                         synchronise the stream and stop with
                                         TGV_ERR_NONFINITE if the state holds a
                                         NaN or Inf (costs one sync per record) */
#define TGV_FLAG_CELL_CENTERED 4      /* grid points at (i + 1/2) L/N            */
#define TGV_FLAG_SYMMETRIC 8          /* the symmetric box of Sec. 4.1 (TGSym):
                                         [0, L]^3, cell-centred, every face a
                                         mirror plane (ghost i -> -1-i and
                                         2N-1-i, the momentum component normal
                                         to the face odd, the rest even).  With
                                         L = pi it holds one octant of the
                                         periodic 2pi problem with 2N points.
                                         Not supported by the adjoint. */

/*
 * One TGV problem.  Physics follows Sec. 3.1 / Sec. 4.1 (nondimensional):
 * p = (gamma-1)(rho E - rho|u|^2/2), T = gamma M^2 p / rho,
 * tau_ij = (mu/Re)(du_i/dx_j + du_j/dx_i - 2/3 delta_ij div u),
 * q_j = -mu/((gamma-1) M^2 Pr Re) dT/dx_j.  mu = 0 gives the inviscid limit.
 *
 * Precision (Sec. 3.1 storage of Q / Qt and the precision of R and W): Q is
 * stored as q_storage, Qt as qt_storage, the residual is computed in
 * `compute`, the RK axpy of Eqs. 3-4 in `accumulate`.  Built combinations
 * (q_storage, qt_storage, compute, accumulate):
 *   F64 F64 F64 F64  double                 F64 F64 F32 F64  single-double (Q FP64)
 *   F32 F32 F64 F64  FP32 storage/FP64 comp F32 F32 F32 F32  single
 *   BF16 BF16 F32 F32 bf16-single           F16 F16 F32 F32  half-single
 *   F16 F16 F16 F32  pure half              F32 F16 F32 F32  Q FP32 / Qt FP16
 * Anything else returns TGV_ERR_UNSUPPORTED.
 */
typedef struct tgv_config {
  int32_t n;          /* N: grid points per direction, even, 8..1024          */
  int32_t split_form; /* tgv_split                                            */
  int32_t q_storage;  /* tgv_dtype of Q                                       */
  int32_t qt_storage; /* tgv_dtype of Qt                                      */
  int32_t compute;    /* tgv_dtype of the residual arithmetic (F64/F32/F16)   */
  int32_t accumulate; /* tgv_dtype of the RK update arithmetic (F64/F32)      */
  int32_t encoding;   /* tgv_encoding                                         */
  int32_t tile;       /* stencil tile id, 0 = default (see tgv_tile_count)    */
  int32_t zchunk;     /* z planes per thread block, 0 = chosen by the library */
  int32_t flags;      /* TGV_FLAG_*                                           */
  double length;      /* periodic box edge L (2*pi for the TGV)               */
  double gamma;       /* ratio of specific heats (1.4)                        */
  double mach;        /* reference Mach number M                              */
  double re;          /* Reynolds number                                      */
  double pr;          /* Prandtl number (0.71)                                */
  double mu;          /* constant nondimensional viscosity (1, or 0: inviscid) */
} tgv_config;

/* ABI version (TGV_ABI_VERSION) and a static message for a status code. */
int32_t tgv_abi_version(void);
const char* tgv_strerror(int32_t status);

/* Host-only validation of a config: TGV_OK, TGV_ERR_ARG or TGV_ERR_UNSUPPORTED. */
int32_t tgv_check_config(const tgv_config* cfg);

/* Bytes of one Q (5*N^3*sizeof(q_storage)) and one Qt; 0 if cfg is invalid. */
size_t tgv_state_bytes(const tgv_config* cfg);
size_t tgv_qt_bytes(const tgv_config* cfg);

/* Number of stencil tile shapes built, and the shape of tile id t (1-based). */
int32_t tgv_tile_count(void);
int32_t tgv_tile_shape(int32_t t, int32_t* tx, int32_t* ty);

/*
 * Largest stable time step (host only).  Reading of the paper's time-step
 * choice (Sec. 4.2, heat-map study): the RK3 stability boundary on the
 * imaginary axis, sqrt(3), divided by the largest modified acoustic wave
 * speed of the 4th-order central difference, 1.3722/h * (sqrt(3)/M + |u|max),
 * with |u|max = 1 for the TGV.  Returns 0 for an invalid config.
 */
double tgv_dt_max(const tgv_config* cfg);

/*
 * Taylor-Green initial condition (Sec. 4.1, Eqs. 6-10) into q (device, Q
 * layout, q_storage, encoded), at the grid points i*h, or (i + 1/2)*h with
 * TGV_FLAG_CELL_CENTERED or TGV_FLAG_SYMMETRIC.  Evaluated in FP64 on the
 * device, then rounded.
 */
int32_t tgv_init(const tgv_config* cfg, void* q, void* stream);

/*
 * Residual R(Q) = dQ/dt of Sec. 3.1 (the "remaining terms" of the governing
 * equations): Blaisdell-split convective terms (Sec. 2.3.1), pressure terms,
 * viscous stress and heat flux, all 4th-order central.
 * q: device, Q layout, q_storage.  r: device, Q layout, 5 fields of the
 * compute type (not encoded).  Same stencil kernel as rk_step, with the
 * residual written out instead of the RK update.
 */
int32_t rhs_eval(const tgv_config* cfg, const void* q, void* r, void* stream);

/*
 * Advance nsteps full RK3 steps (3 fused stage kernels each, Sec. 3.1,
 * Eqs. 3-5; Williamson's 2N coefficients A = (0, -5/9, -153/128),
 * B = (1/3, 15/16, 8/15)).
 * q_a: device, holds Q^n on entry.  q_b: device, same size, scratch.  Stages
 *   ping-pong between the two buffers (Q is never updated in place because
 *   neighbouring blocks still read its halo); *parity_out (nullable) is set to
 *   the buffer holding Q^(n+nsteps): 0 = q_a, 1 = q_b (that is, nsteps % 2).
 * qt: device, Qt layout, qt_storage; its contents on entry are ignored
 *   (A_1 = 0) and are garbage on return.
 * diag_every > 0: diagnostics (as diagnostics_reduce) of Q^(n+m) for every m
 *   in [0, nsteps] with m % diag_every == 0 are written to diag_dev
 *   (device, double[(nsteps/diag_every + 1) * TGV_DIAG_COUNT]) in order.
 *   diag_every = 0: diag_dev is not touched (may be NULL).
 * workspace: device scratch of tgv_workspace_bytes(cfg) bytes (nullable
 *   when diag_every = 0).
 * Returns TGV_ERR_UNSTABLE_DT if dt > tgv_dt_max(cfg) and the flag
 * TGV_FLAG_ALLOW_UNSTABLE_DT is not set.  With TGV_FLAG_CHECK_FINITE (and
 * diag_every > 0) it stops at the first record whose non-finite count is not
 * zero and returns TGV_ERR_NONFINITE; *parity_out then names the buffer
 * holding that recorded state, and the records up to it are valid.
 */
int32_t rk_step(const tgv_config* cfg, void* q_a, void* q_b, void* qt, double dt,
                int32_t nsteps, int32_t diag_every, double* diag_dev,
                void* workspace, size_t ws_bytes, int32_t* parity_out, void* stream);

/*
 * One RK substep i in {0,1,2} (Sec. 3.1, Eqs. 3-4) from q_in to q_out:
 * Qt <- A_i Qt + dt R(q_in); q_out <- q_in + B_i Qt.  q_in and q_out must
 * differ.  For i = 0 the incoming Qt is ignored.
 */
int32_t rk_substep(const tgv_config* cfg, const void* q_in, void* q_out, void* qt,
                   int32_t i, double dt, void* stream);

/* Device scratch needed by rk_step (with diagnostics) and diagnostics_reduce. */
size_t tgv_workspace_bytes(const tgv_config* cfg);

/*
 * Diagnostics of Sec. 4.1, Eqs. 11-12, reduced in FP64 (reading: eps^S as a
 * volume average, like K).  out_dev (device, double[TGV_DIAG_COUNT]):
 *   [0] K = <|u|^2/2>        [1] <rho |u|^2/2>      [2] <omega.omega>
 *   [3] eps^S = <omega.omega>/Re                     [4] <rho>
 *   [5] <rho u>  [6] <rho v>  [7] <rho w>  [8] <rho E>
 *   [9] number of grid points where any component of Q is NaN or Inf.
 * <.> is the mean over the N^3 grid points; omega uses the 4th-order D.
 * Deterministic: per-block FP64 partials, then a fixed-order second pass.
 */
int32_t diagnostics_reduce(const tgv_config* cfg, const void* q, double* out_dev,
                           void* workspace, size_t ws_bytes, void* stream);

/*
 * Discrete adjoint (the paper has none; this is the exact transpose of the
 * discrete forward operator of rhs_eval / rk_step, evaluated in FP64).
 * Supported configs: the FP64 mode, and the FP32 mode (FP32 forward states,
 * FP64 adjoint arithmetic), both with TGV_ENC_PLAIN; others return
 * TGV_ERR_UNSUPPORTED.  Cotangents (lam, q_bar, grad_mom) are FP64 device
 * arrays in the Q layout (grad_mom: the 3 momentum fields only).
 *
 * tgv_adjoint_workspace_bytes: device scratch for rhs_vjp / rk_step_adjoint.
 * rhs_vjp: q_bar = (dR/dQ)^T lam at state q (q: device, Q layout, q_storage).
 * rk_step_adjoint: one RK3 step backwards.  stage_inputs: device, the three
 *   stage input states Q^n, Q^(n,1), Q^(n,2) of the forward step, stored
 *   back to back (tgv_state_bytes apart).  q_bar: in, the cotangent of
 *   Q^(n+1); out, the cotangent of Q^n.  Reverse of Eqs. 3-4 (Sec. 3.1),
 *   for i = 3, 2, 1:  lam <- A_(i+1) lam + B_i q_bar (A_4 = 0);
 *   q_bar <- q_bar + dt (dR/dQ(Q^(n,i-1)))^T lam.
 * tgv_grad_final_ke: J = K(Q_nsteps) (Sec. 4.1, Eq. 11, the grid mean of
 *   |u|^2/2) and dJ/d(rho u, rho v, rho w) at Q_0 with rho and rho E held
 *   fixed, by the forward run with a checkpoint every ckpt_every steps, then
 *   a reverse sweep that recomputes each segment keeping its stage inputs.
 *   q0: device, Q layout; grad_mom: device double[3 N^3]; j_out: device
 *   double[1]; workspace: tgv_grad_workspace_bytes(cfg, nsteps, ckpt_every).
 */
size_t tgv_adjoint_workspace_bytes(const tgv_config* cfg);
int32_t rhs_vjp(const tgv_config* cfg, const void* q, const double* lam, double* q_bar,
                void* workspace, size_t ws_bytes, void* stream);
int32_t rk_step_adjoint(const tgv_config* cfg, const void* stage_inputs, double* q_bar, double dt,
                        void* workspace, size_t ws_bytes, void* stream);
size_t tgv_grad_workspace_bytes(const tgv_config* cfg, int32_t nsteps, int32_t ckpt_every);
int32_t tgv_grad_final_ke(const tgv_config* cfg, const void* q0, double dt, int32_t nsteps,
                          int32_t ckpt_every, double* grad_mom, double* j_out, void* workspace,
                          size_t ws_bytes, void* stream);

/*
 * Batched ensemble (a library feature; the paper runs one problem at a
 * time): `count` independent TGV problems, each with its own N, Re, M and
 * dt, advanced together by one persistent launch per RK stage over a
 * flattened list of (instance, tile, z chunk) work items, the launches of
 * steps_per_graph steps captured in a CUDA graph that tgv_ensemble_run
 * replays.  Built for every precision mode; all instances of one ensemble
 * share the mode (TGV_ERR_ARG otherwise) and use a quadratic split form
 * (Blaisdell or divergence; TGV_ERR_UNSUPPORTED otherwise).
 * cfgs[i], q_a[i], q_b[i], qt[i], dts[i]: instance i (device buffers of that
 *   instance's size; q_a holds Q on entry and again after every replay,
 *   q_b and qt are scratch).  count: 1..64.  steps_per_graph: even, >= 2.
 * Tile shape and z-chunk length are autotuned at creation by timing
 *   first-stage launches, which read q_a and write only q_b and qt; if
 *   cfgs[0].tile / cfgs[0].zchunk are non-zero they are used instead.
 *   Instance i then matches a single-instance rk_step with tile = the chosen
 *   tile and zchunk = min(N_i, chosen z-chunk) bit for bit.
 * The handle (host memory, the graph and its executable) is owned by the
 * library and released by tgv_ensemble_destroy; no device memory is
 * allocated.  create synchronises `stream` once.
 */
typedef struct tgv_ensemble tgv_ensemble;
int32_t tgv_ensemble_create(const tgv_config* cfgs, int32_t count, void* const* q_a,
                            void* const* q_b, void* const* qt, const double* dts,
                            int32_t steps_per_graph, void* stream, tgv_ensemble** out);
int32_t tgv_ensemble_run(tgv_ensemble* ens, int32_t replays, void* stream);
int32_t tgv_ensemble_info(const tgv_ensemble* ens, int32_t* tile, int32_t* zchunk_target,
                          int32_t* grid, int32_t* items, int32_t* steps_per_graph);
int32_t tgv_ensemble_destroy(tgv_ensemble* ens);

/*
 * diagnostics_reduce without a workspace argument: the same diagnostics
 * (same kernels, same result) with the per-block partials kept in a fixed
 * array inside the library's device memory (1184 * TGV_DIAG_COUNT doubles,
 * about 95 KB, held on every device that loads the library until the process
 * exits).  For callers that cannot allocate device memory where they need
 * the diagnostics (a framework that owns all device allocations, a loop that
 * must not take cudaMalloc's implicit synchronisation, a plug-in given only
 * the state).  The paper has no counterpart; this is a library convenience.
 * q: device, Q layout; out_dev: device, double[TGV_DIAG_COUNT].
 * The first call on a device looks up the array's address (cudaGetSymbolAddress)
 * with that device current and caches it with the device's CUDA context; make
 * that first call before any stream capture.  A call in another context (after
 * a device reset, which recreates the context) looks the address up again.
 * All calls share the array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Allocates nothing; returns TGV_ERR_ARG if a problem needed more partials
 * than the array holds (no valid N does).
 */
int32_t diagnostics_reduce_noalloc(const tgv_config* cfg, const void* q, double* out_dev,
                                   void* stream);

/*
 * End-to-end call with HOST buffers: copies q_host_in (Q layout, q_storage,
 * encoded) to the device, advances nsteps RK3 steps with diagnostics every
 * diag_every steps, copies Q^(n+nsteps) to q_host_out and the diagnostics
 * ((nsteps/diag_every + 1) * TGV_DIAG_COUNT doubles) to diag_host (nullable),
 * and synchronises the stream.  Device memory (two Q buffers, Qt, the
 * diagnostics scratch and records) comes from dev_workspace, of at least
 * tgv_run_host_workspace_bytes(cfg, nsteps, diag_every) bytes (0 = invalid).
 * Pinned host memory is fastest.
 */
size_t tgv_run_host_workspace_bytes(const tgv_config* cfg, int32_t nsteps, int32_t diag_every);
int32_t tgv_run_host(const tgv_config* cfg, const void* q_host_in, void* q_host_out,
                     double dt, int32_t nsteps, int32_t diag_every, double* diag_host,
                     void* dev_workspace, size_t ws_bytes, void* stream);

/*
 * `count` independent states from host memory, each advanced exactly as by
 * tgv_run_host (H2D of Q, nsteps RK3 steps with diagnostics every diag_every,
 * D2H of Q and of its records), with the copies overlapped with computation:
 * state i is copied in and state i-1 out on copy_stream while the steps run on
 * compute_stream, through two device buffer sets used in turn.  No paper
 * counterpart (a pipeline for many runs, e.g. an ensemble of initial fields
 * held on the host).
 * q_host_in[i], q_host_out[i]: host, Q layout, q_storage (pinned for the
 *   copies to overlap); in and out may be the same buffer.
 * diag_host: nullable; count consecutive blocks of
 *   (nsteps/diag_every + 1) * TGV_DIAG_COUNT doubles.
 * dev_workspace: tgv_run_host_stream_workspace_bytes(cfg, nsteps, diag_every)
 *   bytes (two tgv_run_host workspaces).
 * compute_stream, copy_stream: may be equal (then nothing overlaps).  Four
 *   CUDA events are created and destroyed inside the call.  Returns after both
 *   streams are synchronised; on an error the results of later states are
 *   not written.
 */
size_t tgv_run_host_stream_workspace_bytes(const tgv_config* cfg, int32_t nsteps,
                                           int32_t diag_every);
int32_t tgv_run_host_stream(const tgv_config* cfg, int32_t count, const void* const* q_host_in,
                            void* const* q_host_out, double dt, int32_t nsteps,
                            int32_t diag_every, double* diag_host, void* dev_workspace,
                            size_t ws_bytes, void* compute_stream, void* copy_stream);

/*
 * Z-slab domain decomposition (the parallel strategy of Sec. 4.3: every
 * process owns a block of the grid and exchanges halo points with its
 * neighbours before each residual evaluation; here a block is a slab of
 * whole z planes of the periodic box, one per GPU, and the halos are
 * exchanged in the storage type of Q).
 *
 * tgv_slab: owned planes z0 .. z0+nz-1 of the N^3 box (nz >= 2).
 * Slab state layout: 5 fields, each (nz + 4) planes of N x N points, x
 * fastest: planes 0-1 are ghosts (copies of global planes z0-2, z0-1, wrapped),
 * planes 2 .. nz+1 the owned planes, planes nz+2, nz+3 ghosts (global z0+nz,
 * z0+nz+1, wrapped): element (c, k, j, i) at ((c*(nz+4) + k)*N + j)*N + i.
 * In the symmetric box (TGV_FLAG_SYMMETRIC) the ghosts beyond a mirror face
 * hold the raw values of the mirrored owned planes (global plane -1 <- 0,
 * -2 <- 1, N <- N-1, N+1 <- N-2); the stage kernel applies the sign change of
 * the normal momentum.
 * Two ghost planes match the z reach of every term of the residual.
 * A slab's Qt holds only the owned planes: ((c*nz + k)*N + j)*N + i.
 */
typedef struct tgv_slab {
  int32_t z0; /* first owned global plane */
  int32_t nz; /* owned planes, >= 2      */
} tgv_slab;

/* Bytes of a slab state (5 (nz+4) N^2 elements of q_storage) and of its Qt
 * (5 nz N^2 of qt_storage); 0 if cfg or slab is invalid. */
size_t tgv_slab_state_bytes(const tgv_config* cfg, const tgv_slab* slab);
size_t tgv_slab_qt_bytes(const tgv_config* cfg, const tgv_slab* slab);

/* Taylor-Green initial condition (Sec. 4.1, Eqs. 6-10) on the owned planes
 * of a slab state q (device); the ghost planes are not written. */
int32_t tgv_slab_init(const tgv_config* cfg, const tgv_slab* slab, void* q, void* stream);

/*
 * One RK substep i in {0,1,2} (Sec. 3.1, Eqs. 3-4) of a slab: the fused stage
 * kernel of rk_step on the owned planes of q_in (device, slab layout; its
 * ghost planes must hold the neighbours' current planes), written to the
 * owned planes of q_out (device, slab layout, != q_in; ghosts untouched).
 * qt (device, slab Qt layout) is internal scratch as in rk_step (the
 * increment kept divided by dt; ignored on entry for i = 0, not written for
 * i = 2), so three substeps with an exchange before each equal one rk_step
 * step of the whole box, bit for bit, on every owned plane.
 * diag_dev (nullable; device double[TGV_DIAG_COUNT]): the diagnostics of
 * q_in's owned planes as contributions to the whole box's means (sums over
 * the slab divided by N^3; eps^S by N^3 Re): summed over all slabs they are
 * diagnostics_reduce of the box.  workspace: tgv_workspace_bytes(cfg) bytes
 * when diag_dev is given.  Returns TGV_ERR_UNSTABLE_DT like rk_step.
 */
int32_t tgv_slab_substep(const tgv_config* cfg, const tgv_slab* slab, const void* q_in,
                         void* q_out, void* qt, int32_t i, double dt, double* diag_dev,
                         void* workspace, size_t ws_bytes, void* stream);

/*
 * Ghost exchange among `count` slabs of one box that all live on the current
 * device: slabs[r] must tile [0, N) in order (slabs[0].z0 = 0, each slab
 * starting where the previous ends); q[r] is slab r's state (device, slab
 * layout).  Fills every slab's four ghost planes from its periodic
 * neighbours in one kernel launch (per field, the two top owned planes of the
 * slab below and the two bottom owned planes of the slab above); one slab
 * (count = 1) wraps onto itself; in the symmetric box the first slab's lower
 * and the last slab's upper ghosts are filled as mirror images instead (see
 * tgv_slab).  1 <= count <= 512, else TGV_ERR_ARG.
 * Between processes on different GPUs the same planes are exchanged with
 * point-to-point messages instead (the Python binding, over NCCL).
 */
int32_t tgv_slab_exchange_local(const tgv_config* cfg, int32_t count, const tgv_slab* slabs,
                                void* const* q, void* stream);

/*
 * Measurement support (no paper counterpart): throughput probe of the FMA
 * pipe in the three arithmetic forms the stage kernels use, for the ALU
 * roofline and the choice between FP32 pairs and packed FP16.  Launches
 * `blocks` blocks of 256 threads on `stream`; every thread runs 8
 * independent chains of x <- x*a + b for `iters` iterations and writes one
 * float to sink (device, at least blocks*256 floats).  *flops (host) receives
 * the floating-point operations the launch performs (2 per lane per FMA); the
 * caller times the launch.  TGV_ERR_ARG on a bad argument.
 */
#define TGV_PROBE_FFMA 0   /* scalar FP32 fused multiply-add            */
#define TGV_PROBE_FFMA2 1  /* paired FP32 (two lanes per instruction)   */
#define TGV_PROBE_HFMA2 2  /* packed FP16 (half2, two lanes)            */
int32_t tgv_probe_fma(int32_t kind, int32_t iters, int32_t blocks, float* sink,
                      size_t sink_floats, double* flops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TGV_H_ */
