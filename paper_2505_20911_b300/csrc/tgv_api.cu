// tgv_api.cu - the C ABI declared in include/tgv.h.
//
// Host-side validation, mode dispatch, z-chunk selection and the RK3 driver
// loop (three fused stage launches per step, buffers ping-ponged).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <vector>

#include "tgv_modes.cuh"

namespace tgv {

static const char* const STAGE_NAMES[3] = {"tgv stage 1", "tgv stage 2", "tgv stage 3"};

const ModeLaunchers& mode_launchers_0();
const ModeLaunchers& mode_launchers_1();
const ModeLaunchers& mode_launchers_2();
const ModeLaunchers& mode_launchers_3();
const ModeLaunchers& mode_launchers_4();
const ModeLaunchers& mode_launchers_5();
const ModeLaunchers& mode_launchers_6();
const ModeLaunchers& mode_launchers_7();

const ModeLaunchers& mode_launchers(int m) {
  switch (m) {
    case 0: return mode_launchers_0();
    case 1: return mode_launchers_1();
    case 2: return mode_launchers_2();
    case 3: return mode_launchers_3();
    case 4: return mode_launchers_4();
    case 5: return mode_launchers_5();
    case 6: return mode_launchers_6();
    default: return mode_launchers_7();
  }
}

Problem make_problem(const tgv_config& c) {
  Problem P;
  P.n = c.n;
  P.split = c.split_form;
  P.encoding = c.encoding;
  P.h = c.length / c.n;
  P.inv12h = 1.0 / (12.0 * P.h);
  P.inv12h2 = 1.0 / (12.0 * P.h * P.h);
  P.gamma = c.gamma;
  P.gm1 = c.gamma - 1.0;
  P.gM2 = c.gamma * c.mach * c.mach;
  P.nu = c.mu / c.re;
  P.kappa = c.mu / ((c.gamma - 1.0) * c.mach * c.mach * c.pr * c.re);
  if (c.encoding == TGV_ENC_OFFSET) {
    P.rho0 = 1.0;
    P.rhoE0 = 1.0 / (c.gamma * (c.gamma - 1.0) * c.mach * c.mach);
  } else {
    P.rho0 = 0.0;
    P.rhoE0 = 0.0;
  }
  P.mach = c.mach;
  P.re = c.re;
  P.symmetric = (c.flags & TGV_FLAG_SYMMETRIC) ? 1 : 0;
  P.offset = (c.flags & (TGV_FLAG_SYMMETRIC | TGV_FLAG_CELL_CENTERED)) ? 0.5 : 0.0;
  return P;
}

int find_mode(const tgv_config& c) {
  for (int m = 0; m < NUM_MODES; ++m) {
    const ModeKey& k = MODE_KEYS[m];
    if (k.qs == c.q_storage && k.qts == c.qt_storage && k.comp == c.compute && k.acc == c.accumulate)
      return m;
  }
  return -1;
}

static bool valid_dtype(int d) { return d >= TGV_F64 && d <= TGV_F16; }

static int32_t check(const tgv_config* c) {
  if (!c) return TGV_ERR_ARG;
  if (c->n < 8 || c->n > 1024 || (c->n & 1)) return TGV_ERR_ARG;
  if (c->split_form != TGV_SPLIT_BLAISDELL && c->split_form != TGV_SPLIT_DIVERGENCE &&
      c->split_form != TGV_SPLIT_KGP && c->split_form != TGV_SPLIT_KEEP &&
      c->split_form != TGV_SPLIT_FEIEREISEN)
    return TGV_ERR_ARG;
  if (!valid_dtype(c->q_storage) || !valid_dtype(c->qt_storage) || !valid_dtype(c->compute) ||
      !valid_dtype(c->accumulate))
    return TGV_ERR_ARG;
  if (c->encoding != TGV_ENC_PLAIN && c->encoding != TGV_ENC_OFFSET) return TGV_ERR_ARG;
  if (c->tile < 0 || c->tile > NUM_TILES) return TGV_ERR_ARG;
  if (c->zchunk < 0 || c->zchunk > c->n) return TGV_ERR_ARG;
  if (!(c->length > 0.0) || !(c->gamma > 1.0) || !(c->mach > 0.0) || !(c->re > 0.0) ||
      !(c->pr > 0.0) || !(c->mu >= 0.0) || !std::isfinite(c->length) || !std::isfinite(c->re) ||
      !std::isfinite(c->mu))
    return TGV_ERR_ARG;
  if (find_mode(*c) < 0) return TGV_ERR_UNSUPPORTED;
  return TGV_OK;
}

// Default tile: among the tiles whose shared memory fits, the one that pads
// N x N least (ties go to the larger tile).  -1 if none fits.
static int pick_tile(const tgv_config& c) {
  const ModeLaunchers& L = mode_launchers(find_mode(c));
  if (c.tile > 0) return L.smem[c.tile - 1] <= STAGE_SMEM_LIMIT ? c.tile - 1 : -1;
  // the first tile (the mode's own first choice, then the table order) whose
  // padded plane is within 4% of the smallest padded plane of the tiles that fit
  long long area[NUM_TILES], min_area = -1;
  for (int t = 0; t < NUM_TILES; ++t) {
    const int tx = tile_tx(c.compute, t), ty = tile_ty(c.compute, t);
    area[t] = L.smem[t] > STAGE_SMEM_LIMIT
                  ? -1
                  : (long long)((c.n + tx - 1) / tx) * tx * ((c.n + ty - 1) / ty) * ty;
    if (area[t] > 0 && (min_area < 0 || area[t] < min_area)) min_area = area[t];
  }
  for (int i = -1; i < NUM_TILES; ++i) {
    const int t = i < 0 ? L.first_tile : i;
    if (area[t] > 0 && area[t] * 25 <= min_area * 26) return t;
  }
  return -1;
}

// Upper bound on the z chunks of one stage launch (bounds the CTA count, and
// with it the diagnostics partials of a fused launch).
constexpr int MAX_ZCHUNKS = 16;

// CTAs of one stage launch over nzl planes (N for the periodic box).
static long long stage_ctas(const tgv_config& c, int tile, int zc, int nzl) {
  const int tx = tile_tx(c.compute, tile), ty = tile_ty(c.compute, tile);
  return (long long)((c.n + tx - 1) / tx) * ((c.n + ty - 1) / ty) * ((nzl + zc - 1) / zc);
}

// Per-device caches (SM count; resident CTAs per SM of each stage kernel).
constexpr int MAX_DEVICES = 64;
static std::atomic<int> g_sms[MAX_DEVICES];
static std::atomic<int> g_occ[MAX_DEVICES][NUM_MODES][NUM_TILES];

static int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return -1;
  return dev;
}

static int device_sms(int dev) {
  int v = g_sms[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  g_sms[dev].store(v, std::memory_order_relaxed);
  return v;
}

static int stage_occ(int dev, int mode, int tile) {
  int v = g_occ[dev][mode][tile].load(std::memory_order_relaxed);
  if (v > 0) return v;
  v = mode_launchers(mode).occupancy[tile]();
  if (v > 0) g_occ[dev][mode][tile].store(v, std::memory_order_relaxed);
  return v;
}

// z planes per CTA: balance whole waves of resident CTAs against the 4 extra
// halo planes each chunk reads; nzl planes are advanced (N for the periodic
// box, the owned planes of a slab).
static int pick_zchunk(const tgv_config& c, int tile, int occupancy, int sms, int nzl) {
  if (c.zchunk > 0) return c.zchunk < nzl ? c.zchunk : nzl;
  const int n = c.n;
  const int tx = tile_tx(c.compute, tile), ty = tile_ty(c.compute, tile);
  const long long tiles = (long long)((n + tx - 1) / tx) * ((n + ty - 1) / ty);
  const long long conc = (long long)(occupancy > 0 ? occupancy : 1) * (sms > 0 ? sms : 148);
  double best = -1.0;
  int best_zc = nzl;
  for (int chunks = 1; chunks <= nzl / 8 && chunks <= MAX_ZCHUNKS; ++chunks) {
    const int zc = (nzl + chunks - 1) / chunks;
    const long long ctas = tiles * ((nzl + zc - 1) / zc);
    const long long waves = (ctas + conc - 1) / conc;
    const double fill = (double)ctas / (double)(waves * conc);
    const double eff = fill * (double)zc / (double)(zc + 4);
    if (eff > best + 1e-9) { best = eff; best_zc = zc; }
  }
  return best_zc;
}

// Ghost exchange among slabs on one device, one launch: block (x, 2c + side, r)
// copies, for field c of slab r, either its two lower ghost planes from the two
// top owned planes of the slab below (side 0) or its two upper ghost planes
// from the two bottom owned planes of the slab above (side 1).  In the
// symmetric box the first slab's lower and the last slab's upper ghosts lie
// beyond a mirror face instead: they take the slab's own two outermost owned
// planes in reverse order (plane -1 <- 0, -2 <- 1; N <- N-1, N+1 <- N-2), as
// raw values (the stage kernel applies the mirror's sign change).  Ghost
// planes are written and owned planes read, so no copy overlaps another.  A
// two-plane block is 2 N^2 elements of 2, 4 or 8 bytes with N even: a whole
// number of 32-bit words, at offsets that are multiples of 4 bytes.
constexpr int SLAB_XCH_MAX = 512;
struct SlabXchTable {
  const void* q[SLAB_XCH_MAX];
  int nz[SLAB_XCH_MAX];
};

__global__ void slab_exchange_kernel(const SlabXchTable T, int count, long long nn, int es,
                                     int symmetric) {
  const int r = blockIdx.z, c = blockIdx.y >> 1, side = blockIdx.y & 1;
  const bool mirror = symmetric && (side ? r == count - 1 : r == 0);
  const int src_r = mirror ? r : (side ? (r + 1) % count : (r + count - 1) % count);
  const long long fs_dst = (T.nz[r] + 4) * nn, fs_src = (T.nz[src_r] + 4) * nn;
  const long long dst_el = c * fs_dst + (side ? (long long)(T.nz[r] + 2) * nn : 0);
  // the source block: the neighbour's outermost owned planes facing this
  // slab, or (mirror) this slab's own outermost owned planes at the face
  const long long src_el =
      c * fs_src + ((side != 0) != mirror ? 2 * nn : (long long)T.nz[src_r] * nn);
  unsigned* dst = reinterpret_cast<unsigned*>(const_cast<char*>(static_cast<const char*>(T.q[r])) +
                                              dst_el * es);
  const unsigned* src =
      reinterpret_cast<const unsigned*>(static_cast<const char*>(T.q[src_r]) + src_el * es);
  const long long wpp = nn * es / 4, words = 2 * wpp;  // 32-bit words per plane, per block
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < words;
       i += (long long)gridDim.x * blockDim.x) {
    const long long j = mirror ? (i < wpp ? i + wpp : i - wpp) : i;  // planes swapped
    dst[i] = src[j];
  }
}

}  // namespace tgv

using namespace tgv;

extern "C" {

int32_t tgv_abi_version(void) { return TGV_ABI_VERSION; }

const char* tgv_strerror(int32_t s) {
  switch (s) {
    case TGV_OK: return "ok";
    case TGV_ERR_ARG: return "invalid argument";
    case TGV_ERR_UNSUPPORTED: return "unsupported precision combination";
    case TGV_ERR_CUDA: return "CUDA runtime error";
    case TGV_ERR_NONFINITE: return "non-finite value in the state";
    case TGV_ERR_UNSTABLE_DT: return "dt above the stability limit";
    case TGV_ERR_TIMEOUT: return "bounded device wait timed out";
    case TGV_ERR_WORKSPACE: return "workspace missing or too small";
  }
  return "unknown status";
}

int32_t tgv_check_config(const tgv_config* cfg) { return check(cfg); }

size_t tgv_state_bytes(const tgv_config* cfg) {
  if (check(cfg) != TGV_OK) return 0;
  const size_t n = (size_t)cfg->n;
  return 5 * n * n * n * dtype_size(cfg->q_storage);
}

size_t tgv_qt_bytes(const tgv_config* cfg) {
  if (check(cfg) != TGV_OK) return 0;
  const size_t n = (size_t)cfg->n;
  return 5 * n * n * n * dtype_size(cfg->qt_storage);
}

int32_t tgv_tile_count(void) { return NUM_TILES; }

int32_t tgv_tile_shape(int32_t t, int32_t* tx, int32_t* ty) {
  if (t < 1 || t > NUM_TILES || !tx || !ty) return TGV_ERR_ARG;
  *tx = TILE_TX[t - 1];  // FP32/FP16 compute; FP64 compute uses TILE_TX_F64
  *ty = TILE_TY[t - 1];
  return TGV_OK;
}

double tgv_dt_max(const tgv_config* cfg) {
  if (check(cfg) != TGV_OK) return 0.0;
  const double h = cfg->length / cfg->n;
  const double kmax = 1.3722 / h;  // max of (8 sin t - sin 2t)/(6h)
  const double lam = kmax * (std::sqrt(3.0) / cfg->mach + 1.0);
  return std::sqrt(3.0) / lam;
}

size_t tgv_workspace_bytes(const tgv_config* cfg) {
  if (check(cfg) != TGV_OK) return 0;
  long long blocks = DIAG_MAX_BLOCKS;
  for (int t = 0; t < NUM_TILES; ++t) {
    const int zc = cfg->zchunk > 0 ? cfg->zchunk : (cfg->n + MAX_ZCHUNKS - 1) / MAX_ZCHUNKS;
    const long long b = stage_ctas(*cfg, t, zc, cfg->n);
    if (b > blocks) blocks = b;
  }
  return (size_t)blocks * TGV_DIAG_COUNT * sizeof(double);
}

int32_t tgv_init(const tgv_config* cfg, void* q, void* stream) {
  int32_t s = check(cfg);
  if (s != TGV_OK) return s;
  if (!q) return TGV_ERR_ARG;
  const Problem P = make_problem(*cfg);
  const long long n3 = (long long)cfg->n * cfg->n * cfg->n;
  const ZLayout L{0, cfg->n, 0, n3};
  TGV_CUDA_TRY(mode_launchers(find_mode(*cfg)).init(P, q, L, (cudaStream_t)stream));
  return TGV_OK;
}

// Launch one stage kernel (rhs: residual epilogue; S.diag_part != nullptr:
// the fused-diagnostics variant, whose CTA count is returned in *ctas).
static int32_t launch_stage_common(const tgv_config* cfg, const StageArgs& S, bool rhs,
                                   cudaStream_t st, long long* ctas = nullptr) {
  const int m = find_mode(*cfg);
  const ModeLaunchers& L = mode_launchers(m);
  const int tile = pick_tile(*cfg);
  if (tile < 0) return TGV_ERR_UNSUPPORTED;
  const int dev = current_device();
  if (dev < 0) return TGV_ERR_CUDA;
  const int occ = stage_occ(dev, m, tile);
  if (occ <= 0) return TGV_ERR_CUDA;
  const int nzl = S.nzl > 0 ? S.nzl : cfg->n;
  const int zc = pick_zchunk(*cfg, tile, occ, device_sms(dev), nzl);
  StageArgs A = S;
  A.zchunk = zc;
  const Problem P = make_problem(*cfg);
  if (ctas) *ctas = stage_ctas(*cfg, tile, zc, nzl);
  const int v = cfg->split_form == TGV_SPLIT_KGP      ? SPL_KGP
                : cfg->split_form == TGV_SPLIT_KEEP     ? SPL_KEEP
                : cfg->split_form == TGV_SPLIT_FEIEREISEN ? SPL_FEIER
                                                         : SPL_QUAD;
  StageFn fn = rhs ? L.rhs[v][tile] : (S.diag_part ? L.stage_diag[v][tile] : L.stage[v][tile]);
  // rk_step's stages (increment kept divided by dt, written by all but the
  // last, read by all but the first) have kernels with those flags built in
  if (!rhs && !S.diag_part && v == SPL_QUAD && S.scaled_qt && (S.read_qt || S.write_qt)) {
    const int i = !S.read_qt ? 0 : (S.write_qt ? 1 : 2);
    fn = L.stage_rk[i][tile];
  }
  if (!rhs && S.diag_part && v == SPL_QUAD && S.scaled_qt && !S.read_qt && S.write_qt)
    fn = L.stage_rk_diag[tile];
  if (!fn) return TGV_ERR_UNSUPPORTED;
  cudaError_t e = fn(P, A, zc, st);
  return e == cudaSuccess ? TGV_OK : TGV_ERR_CUDA;
}

int32_t rhs_eval(const tgv_config* cfg, const void* q, void* r, void* stream) {
  int32_t s = check(cfg);
  if (s != TGV_OK) return s;
  if (!q || !r || q == r) return TGV_ERR_ARG;
  StageArgs S;
  std::memset(&S, 0, sizeof(S));
  S.q_in = q;
  S.r_out = r;
  return launch_stage_common(cfg, S, true, (cudaStream_t)stream);
}

static int32_t substep_impl(const tgv_config* cfg, const void* q_in, void* q_out, void* qt,
                            int32_t i, double dt, double* diag_part, long long* ctas,
                            void* stream, bool write_qt = true, bool scaled_qt = false) {
  StageArgs S;
  std::memset(&S, 0, sizeof(S));
  S.q_in = q_in;
  S.q_out = q_out;
  S.qt = qt;
  S.diag_part = diag_part;
  S.a = RK_A[i];
  S.b = RK_B[i];
  S.dt = dt;
  S.read_qt = (i != 0);
  S.write_qt = write_qt ? 1 : 0;
  S.scaled_qt = scaled_qt ? 1 : 0;
  S.bdt = RK_B[i] * dt;
  return launch_stage_common(cfg, S, false, (cudaStream_t)stream, ctas);
}

int32_t rk_substep(const tgv_config* cfg, const void* q_in, void* q_out, void* qt, int32_t i,
                   double dt, void* stream) {
  int32_t s = check(cfg);
  if (s != TGV_OK) return s;
  if (!q_in || !q_out || !qt || q_in == q_out || i < 0 || i > 2 || !std::isfinite(dt))
    return TGV_ERR_ARG;
  return substep_impl(cfg, q_in, q_out, qt, i, dt, nullptr, nullptr, stream);
}

int32_t diagnostics_reduce(const tgv_config* cfg, const void* q, double* out_dev, void* workspace,
                           size_t ws_bytes, void* stream) {
  int32_t s = check(cfg);
  if (s != TGV_OK) return s;
  if (!q || !out_dev) return TGV_ERR_ARG;
  if (!workspace || ws_bytes < tgv_workspace_bytes(cfg)) return TGV_ERR_WORKSPACE;
  const Problem P = make_problem(*cfg);
  const long long items = diag_items(cfg->n);
  const long long nb = items < DIAG_MAX_BLOCKS ? items : DIAG_MAX_BLOCKS;
  cudaStream_t st = (cudaStream_t)stream;
  double* part = static_cast<double*>(workspace);
  TGV_CUDA_TRY(mode_launchers(find_mode(*cfg)).diag_partial(P, q, part, (int)nb, st));
  diag_final_kernel<<<1, 32 * TGV_DIAG_COUNT, 0, st>>>(P, part, (int)nb, out_dev);
  TGV_CUDA_TRY(cudaGetLastError());
  return TGV_OK;
}

int32_t rk_step(const tgv_config* cfg, void* q_a, void* q_b, void* qt, double dt, int32_t nsteps,
                int32_t diag_every, double* diag_dev, void* workspace, size_t ws_bytes,
                int32_t* parity_out, void* stream) {
  int32_t s = check(cfg);
  if (s != TGV_OK) return s;
  if (!q_a || !q_b || !qt || q_a == q_b || nsteps < 0 || diag_every < 0 || !std::isfinite(dt) ||
      !(dt > 0.0))
    return TGV_ERR_ARG;
  if (diag_every > 0) {
    if (!diag_dev) return TGV_ERR_ARG;
    if (!workspace || ws_bytes < tgv_workspace_bytes(cfg)) return TGV_ERR_WORKSPACE;
  }
  if (!(cfg->flags & TGV_FLAG_ALLOW_UNSTABLE_DT) && dt > tgv_dt_max(cfg)) return TGV_ERR_UNSTABLE_DT;
  void* buf[2] = {q_a, q_b};
  int cur = 0;
  int rec = 0;
  const Problem P = make_problem(*cfg);
  for (int32_t m = 0; m < nsteps; ++m) {
    const bool log = diag_every > 0 && m % diag_every == 0;
    NvtxRange step_range("tgv rk_step");
    for (int i = 0; i < 3; ++i) {
      NvtxRange stage_range(STAGE_NAMES[i]);
      // the first substep of a logged step also reduces the diagnostics of Q^m
      long long ctas = 0;
      double* part = (log && i == 0) ? static_cast<double*>(workspace) : nullptr;
      // the last substep's Qt is never read (A_1 = 0 restarts it): not stored
      s = substep_impl(cfg, buf[cur], buf[cur ^ 1], qt, i, dt, part, &ctas, stream, i != 2, true);
      if (s != TGV_OK) return s;
      if (part) {
        double* record = diag_dev + (size_t)rec * TGV_DIAG_COUNT;
        diag_final_kernel<<<1, 32 * TGV_DIAG_COUNT, 0, (cudaStream_t)stream>>>(P, part, (int)ctas,
                                                                              record);
        TGV_CUDA_TRY(cudaGetLastError());
        ++rec;
        if (cfg->flags & TGV_FLAG_CHECK_FINITE) {
          double bad = 0.0;
          TGV_CUDA_TRY(cudaMemcpyAsync(&bad, record + 9, sizeof(double), cudaMemcpyDeviceToHost,
                                       (cudaStream_t)stream));
          TGV_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
          if (bad != 0.0) {  // the recorded state is the stage-1 input, buf[cur]
            if (parity_out) *parity_out = cur;
            return TGV_ERR_NONFINITE;
          }
        }
      }
      cur ^= 1;
    }
  }
  if (diag_every > 0 && nsteps % diag_every == 0) {
    double* record = diag_dev + (size_t)rec * TGV_DIAG_COUNT;
    s = diagnostics_reduce(cfg, buf[cur], record, workspace, ws_bytes, stream);
    if (s != TGV_OK) return s;
    if (cfg->flags & TGV_FLAG_CHECK_FINITE) {
      double bad = 0.0;
      TGV_CUDA_TRY(cudaMemcpyAsync(&bad, record + 9, sizeof(double), cudaMemcpyDeviceToHost,
                                   (cudaStream_t)stream));
      TGV_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
      if (bad != 0.0) {
        if (parity_out) *parity_out = cur;
        return TGV_ERR_NONFINITE;
      }
    }
  }
  if (parity_out) *parity_out = cur;
  return TGV_OK;
}

static size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t tgv_run_host_workspace_bytes(const tgv_config* cfg, int32_t nsteps, int32_t diag_every) {
  if (check(cfg) != TGV_OK || nsteps < 0 || diag_every < 0) return 0;
  const size_t nrec = diag_every > 0 ? (size_t)(nsteps / diag_every + 1) : 0;
  return 2 * up256(tgv_state_bytes(cfg)) + up256(tgv_qt_bytes(cfg)) +
         up256(tgv_workspace_bytes(cfg)) + up256(nrec * TGV_DIAG_COUNT * sizeof(double));
}

int32_t tgv_run_host(const tgv_config* cfg, const void* q_host_in, void* q_host_out, double dt,
                     int32_t nsteps, int32_t diag_every, double* diag_host, void* dev_workspace,
                     size_t ws_bytes, void* stream) {
  int32_t s = check(cfg);
  if (s != TGV_OK) return s;
  if (!q_host_in || !q_host_out || nsteps < 0 || diag_every < 0) return TGV_ERR_ARG;
  if (!dev_workspace || ws_bytes < tgv_run_host_workspace_bytes(cfg, nsteps, diag_every))
    return TGV_ERR_WORKSPACE;
  const size_t qb = tgv_state_bytes(cfg), qtb = tgv_qt_bytes(cfg);
  const size_t wsb = tgv_workspace_bytes(cfg);
  char* w = static_cast<char*>(dev_workspace);
  void* qa = w;
  void* qbuf = w + up256(qb);
  void* qt = w + 2 * up256(qb);
  void* diag_ws = w + 2 * up256(qb) + up256(qtb);
  double* diag_dev = reinterpret_cast<double*>(w + 2 * up256(qb) + up256(qtb) + up256(wsb));
  const int nrec = diag_every > 0 ? nsteps / diag_every + 1 : 0;
  cudaStream_t st = (cudaStream_t)stream;
  TGV_CUDA_TRY(cudaMemcpyAsync(qa, q_host_in, qb, cudaMemcpyHostToDevice, st));
  int32_t parity = 0;
  s = rk_step(cfg, qa, qbuf, qt, dt, nsteps, diag_every, nrec > 0 ? diag_dev : nullptr, diag_ws,
              wsb, &parity, stream);
  if (s != TGV_OK) return s;
  TGV_CUDA_TRY(cudaMemcpyAsync(q_host_out, parity ? qbuf : qa, qb, cudaMemcpyDeviceToHost, st));
  if (nrec > 0 && diag_host)
    TGV_CUDA_TRY(cudaMemcpyAsync(diag_host, diag_dev, (size_t)nrec * TGV_DIAG_COUNT * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
  TGV_CUDA_TRY(cudaStreamSynchronize(st));
  return TGV_OK;
}

size_t tgv_run_host_stream_workspace_bytes(const tgv_config* cfg, int32_t nsteps,
                                           int32_t diag_every) {
  const size_t one = tgv_run_host_workspace_bytes(cfg, nsteps, diag_every);
  return one ? 2 * up256(one) : 0;
}

int32_t tgv_run_host_stream(const tgv_config* cfg, int32_t count, const void* const* q_host_in,
                            void* const* q_host_out, double dt, int32_t nsteps,
                            int32_t diag_every, double* diag_host, void* dev_workspace,
                            size_t ws_bytes, void* compute_stream, void* copy_stream) {
  int32_t s = check(cfg);
  if (s != TGV_OK) return s;
  if (count < 0 || (count > 0 && (!q_host_in || !q_host_out)) || nsteps < 0 || diag_every < 0)
    return TGV_ERR_ARG;
  for (int32_t i = 0; i < count; ++i)
    if (!q_host_in[i] || !q_host_out[i]) return TGV_ERR_ARG;
  if (!dev_workspace || ws_bytes < tgv_run_host_stream_workspace_bytes(cfg, nsteps, diag_every))
    return TGV_ERR_WORKSPACE;
  if (count == 0) return TGV_OK;
  const size_t qb = tgv_state_bytes(cfg), qtb = tgv_qt_bytes(cfg), wsb = tgv_workspace_bytes(cfg);
  const size_t one = up256(tgv_run_host_workspace_bytes(cfg, nsteps, diag_every));
  const int nrec = diag_every > 0 ? nsteps / diag_every + 1 : 0;
  const size_t rec_bytes = (size_t)nrec * TGV_DIAG_COUNT * sizeof(double);
  struct Set { void *qa, *qb, *qt, *dws; double* diag; } set[2];
  for (int b = 0; b < 2; ++b) {
    char* w = static_cast<char*>(dev_workspace) + b * one;
    set[b] = {w, w + up256(qb), w + 2 * up256(qb), w + 2 * up256(qb) + up256(qtb),
              reinterpret_cast<double*>(w + 2 * up256(qb) + up256(qtb) + up256(wsb))};
  }
  cudaStream_t cs = (cudaStream_t)compute_stream, xs = (cudaStream_t)copy_stream;
  cudaEvent_t in_done[2] = {nullptr, nullptr}, out_ready[2] = {nullptr, nullptr};
  std::vector<int32_t> parity((size_t)count, 0);
  auto cleanup = [&](int32_t status) {
    cudaStreamSynchronize(cs);
    cudaStreamSynchronize(xs);
    for (int b = 0; b < 2; ++b) {
      if (in_done[b]) cudaEventDestroy(in_done[b]);
      if (out_ready[b]) cudaEventDestroy(out_ready[b]);
    }
    return status;
  };
  for (int b = 0; b < 2; ++b)
    if (cudaEventCreateWithFlags(&in_done[b], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&out_ready[b], cudaEventDisableTiming) != cudaSuccess)
      return cleanup(TGV_ERR_CUDA);
  // copy-out of state j (issued after the copy-in of state j + 1, so that a
  // copy-in never waits behind a copy-out that waits for the computation)
  auto copy_out = [&](int32_t j) -> int32_t {
    const Set& S = set[j & 1];
    if (cudaStreamWaitEvent(xs, out_ready[j & 1], 0) != cudaSuccess) return TGV_ERR_CUDA;
    if (cudaMemcpyAsync(q_host_out[j], parity[j] ? S.qb : S.qa, qb, cudaMemcpyDeviceToHost,
                        xs) != cudaSuccess)
      return TGV_ERR_CUDA;
    if (nrec > 0 && diag_host &&
        cudaMemcpyAsync(diag_host + (size_t)j * nrec * TGV_DIAG_COUNT, S.diag, rec_bytes,
                        cudaMemcpyDeviceToHost, xs) != cudaSuccess)
      return TGV_ERR_CUDA;
    return TGV_OK;
  };
  for (int32_t i = 0; i < count; ++i) {
    const Set& S = set[i & 1];
    // set i&1 is free: the copy-out of state i-2 precedes this copy-in on xs
    if (cudaMemcpyAsync(S.qa, q_host_in[i], qb, cudaMemcpyHostToDevice, xs) != cudaSuccess ||
        cudaEventRecord(in_done[i & 1], xs) != cudaSuccess ||
        cudaStreamWaitEvent(cs, in_done[i & 1], 0) != cudaSuccess)
      return cleanup(TGV_ERR_CUDA);
    s = rk_step(cfg, S.qa, S.qb, S.qt, dt, nsteps, diag_every, nrec > 0 ? S.diag : nullptr, S.dws,
                wsb, &parity[i], cs);
    if (s != TGV_OK) return cleanup(s);
    if (cudaEventRecord(out_ready[i & 1], cs) != cudaSuccess) return cleanup(TGV_ERR_CUDA);
    if (i > 0 && (s = copy_out(i - 1)) != TGV_OK) return cleanup(s);
  }
  if ((s = copy_out(count - 1)) != TGV_OK) return cleanup(s);
  return cleanup(TGV_OK);
}

// ------------------------------------------------------------ z-slabs
static int32_t check_slab(const tgv_config* cfg, const tgv_slab* sl) {
  int32_t s = check(cfg);
  if (s != TGV_OK) return s;
  if (!sl || sl->nz < 2 || sl->z0 < 0 || sl->z0 + sl->nz > cfg->n) return TGV_ERR_ARG;
  return TGV_OK;
}

static long long slab_fs(const tgv_config* cfg, const tgv_slab* sl) {
  return (long long)(sl->nz + 4) * cfg->n * cfg->n;
}

size_t tgv_slab_state_bytes(const tgv_config* cfg, const tgv_slab* slab) {
  if (check_slab(cfg, slab) != TGV_OK) return 0;
  return 5 * (size_t)slab_fs(cfg, slab) * dtype_size(cfg->q_storage);
}

size_t tgv_slab_qt_bytes(const tgv_config* cfg, const tgv_slab* slab) {
  if (check_slab(cfg, slab) != TGV_OK) return 0;
  return 5 * (size_t)slab->nz * cfg->n * cfg->n * dtype_size(cfg->qt_storage);
}

int32_t tgv_slab_init(const tgv_config* cfg, const tgv_slab* slab, void* q, void* stream) {
  int32_t s = check_slab(cfg, slab);
  if (s != TGV_OK) return s;
  if (!q) return TGV_ERR_ARG;
  const Problem P = make_problem(*cfg);
  const ZLayout L{slab->z0, slab->nz, 2, slab_fs(cfg, slab)};
  TGV_CUDA_TRY(mode_launchers(find_mode(*cfg)).init(P, q, L, (cudaStream_t)stream));
  return TGV_OK;
}

int32_t tgv_slab_substep(const tgv_config* cfg, const tgv_slab* slab, const void* q_in,
                         void* q_out, void* qt, int32_t i, double dt, double* diag_dev,
                         void* workspace, size_t ws_bytes, void* stream) {
  int32_t s = check_slab(cfg, slab);
  if (s != TGV_OK) return s;
  if (!q_in || !q_out || !qt || q_in == q_out || i < 0 || i > 2 || !std::isfinite(dt) ||
      !(dt > 0.0))
    return TGV_ERR_ARG;
  if (diag_dev && (!workspace || ws_bytes < tgv_workspace_bytes(cfg))) return TGV_ERR_WORKSPACE;
  if (!(cfg->flags & TGV_FLAG_ALLOW_UNSTABLE_DT) && dt > tgv_dt_max(cfg)) return TGV_ERR_UNSTABLE_DT;
  StageArgs S;
  std::memset(&S, 0, sizeof(S));
  S.q_in = q_in;
  S.q_out = q_out;
  S.qt = qt;
  S.diag_part = diag_dev ? static_cast<double*>(workspace) : nullptr;
  S.a = RK_A[i];
  S.b = RK_B[i];
  S.dt = dt;
  S.read_qt = (i != 0);
  S.write_qt = (i != 2);   // as rk_step: the last substep's increment is never read
  S.scaled_qt = 1;         // as rk_step: the increment is kept divided by dt
  S.bdt = RK_B[i] * dt;
  S.zg = 2;
  S.nzl = slab->nz;
  S.zoff = slab->z0;
  S.fs_q = slab_fs(cfg, slab);
  S.fs_t = (long long)slab->nz * cfg->n * cfg->n;
  long long ctas = 0;
  NvtxRange stage_range(STAGE_NAMES[i]);
  s = launch_stage_common(cfg, S, false, (cudaStream_t)stream, &ctas);
  if (s != TGV_OK) return s;
  if (diag_dev) {
    const Problem P = make_problem(*cfg);
    diag_final_kernel<<<1, 32 * TGV_DIAG_COUNT, 0, (cudaStream_t)stream>>>(P, S.diag_part,
                                                                         (int)ctas, diag_dev);
    TGV_CUDA_TRY(cudaGetLastError());
  }
  return TGV_OK;
}

int32_t tgv_slab_exchange_local(const tgv_config* cfg, int32_t count, const tgv_slab* slabs,
                                void* const* q, void* stream) {
  int32_t s = check(cfg);
  if (s != TGV_OK) return s;
  if (count < 1 || count > SLAB_XCH_MAX || !slabs || !q) return TGV_ERR_ARG;
  int32_t z = 0;
  SlabXchTable T;
  for (int32_t r = 0; r < count; ++r) {  // the slabs tile [0, N) in order
    if ((s = check_slab(cfg, &slabs[r])) != TGV_OK) return s;
    if (slabs[r].z0 != z || !q[r]) return TGV_ERR_ARG;
    z += slabs[r].nz;
    T.q[r] = q[r];
    T.nz[r] = slabs[r].nz;
  }
  if (z != cfg->n) return TGV_ERR_ARG;
  const int es = (int)dtype_size(cfg->q_storage);
  const long long nn = (long long)cfg->n * cfg->n;
  const long long words = 2 * nn * es / 4;  // one two-plane block in 32-bit words
  const int bx = (int)std::min<long long>((words + 255) / 256, 64);
  NvtxRange range("tgv slab ghost exchange");
  const int sym = (cfg->flags & TGV_FLAG_SYMMETRIC) ? 1 : 0;
  slab_exchange_kernel<<<dim3(bx, 10, count), 256, 0, (cudaStream_t)stream>>>(T, count, nn, es,
                                                                               sym);
  TGV_CUDA_TRY(cudaGetLastError());
  return TGV_OK;
}

}  // extern "C"

namespace tgv {
__global__ void diag_final_kernel(const Problem P, const double* __restrict__ part, int nblocks,
                                  double* __restrict__ out) {
  // 32 lanes per diagnostic: each lane sums a fixed strided subset in order,
  // then a fixed shuffle tree combines the lanes.
  const int m = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (m >= TGV_DIAG_COUNT) return;
  double v = 0.0;
  const int src = (m == 3) ? 2 : m;  // eps^S = <omega.omega> / Re
  for (int b = lane; b < nblocks; b += 32) v += part[b * TGV_DIAG_COUNT + src];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if (lane == 0) {
    const double n3 = (double)P.n * P.n * P.n;
    if (m == 9) out[9] = v;
    else if (m == 3) out[3] = v / n3 / P.re;
    else out[m] = v / n3;
  }
}
}  // namespace tgv
