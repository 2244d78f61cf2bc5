// tgv_noalloc.cu - diagnostics_reduce without a caller-provided workspace.
//
// diagnostics_reduce needs a device scratch buffer for its per-block FP64
// partial sums, which the caller normally allocates (tgv_workspace_bytes).
// Some callers cannot allocate device memory at the point where they want the
// diagnostics: code that runs inside a framework that owns every device
// allocation, real-time loops where the implicit synchronisation of
// cudaMalloc is unacceptable, or plug-ins handed only the state pointer.  For
// them, diagnostics_reduce_noalloc keeps the partials in a fixed array in the
// library's own device memory instead.
//
// The array lives for the lifetime of the process on every device that loads
// the library (NOALLOC_PARTIALS doubles, about 95 KB).  Host code cannot use
// its name as a device address, so the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and caches
// it; that first call should therefore come before any stream capture.
#include <atomic>

#include "tgv_modes.cuh"

namespace tgv {

// Capacity: one FP64 partial per diagnostic per block of the standalone
// diagnostics kernel, which never launches more than DIAG_MAX_BLOCKS blocks.
constexpr int NOALLOC_BLOCKS = DIAG_MAX_BLOCKS;
constexpr size_t NOALLOC_PARTIALS = (size_t)NOALLOC_BLOCKS * TGV_DIAG_COUNT;

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_PARTIALS];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::atomic<double*> g_noalloc_ptr[NOALLOC_MAX_DEVICES];

// Device address of the partials array on the current device (looked up once).
static double* noalloc_scratch(int dev) {
  double* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (p) return p;
  void* addr = nullptr;
  if (cudaGetSymbolAddress(&addr, g_noalloc_partials) != cudaSuccess || !addr) return nullptr;
  p = static_cast<double*>(addr);
  g_noalloc_ptr[dev].store(p, std::memory_order_release);
  return p;
}

static int noalloc_mode(const tgv_config& c) {
  for (int m = 0; m < NUM_MODES; ++m) {
    const ModeKey& k = MODE_KEYS[m];
    if (k.qs == c.q_storage && k.qts == c.qt_storage && k.comp == c.compute && k.acc == c.accumulate)
      return m;
  }
  return -1;
}

}  // namespace tgv

using namespace tgv;

extern "C" int32_t diagnostics_reduce_noalloc(const tgv_config* cfg, const void* q,
                                              double* out_dev, void* stream) {
  const int32_t s = tgv_check_config(cfg);
  if (s != TGV_OK) return s;
  if (!q || !out_dev) return TGV_ERR_ARG;
  const long long items = (long long)((cfg->n + DIAG_TX - 1) / DIAG_TX) *
                          ((cfg->n + DIAG_TY - 1) / DIAG_TY) * cfg->n;
  const long long nb = items < DIAG_MAX_BLOCKS ? items : DIAG_MAX_BLOCKS;
  if (nb > NOALLOC_BLOCKS) return TGV_ERR_ARG;  // more partials than the fixed array holds
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return TGV_ERR_CUDA;
  double* part = noalloc_scratch(dev);
  if (!part) return TGV_ERR_CUDA;
  // Every partial the final pass reads is written by this call's first pass,
  // so nothing in the array has to be cleared beforehand.
  const Problem P = make_problem(*cfg);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (mode_launchers(noalloc_mode(*cfg)).diag_partial(P, q, part, (int)nb, st) != cudaSuccess)
    return TGV_ERR_CUDA;
  diag_final_kernel<<<1, 32 * TGV_DIAG_COUNT, 0, st>>>(P, part, (int)nb, out_dev);
  if (cudaGetLastError() != cudaSuccess) return TGV_ERR_CUDA;
  return TGV_OK;
}
