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
// its name as a device address, so a call looks the address up with
// cudaGetSymbolAddress (with the device current) and caches it per device
// together with the CUDA context it belongs to; a call in another context (a
// device reset recreates the primary context and reloads the module) looks it
// up again.  The first call on a device, which does the lookup, should come
// before any stream capture.
#include <cuda.h>  // the CUcontext type only; the driver function is obtained at run time

#include <mutex>

#include "tgv_modes.cuh"

namespace tgv {

// Capacity: one FP64 partial per diagnostic per block of the standalone
// diagnostics kernel, which never launches more than DIAG_MAX_BLOCKS blocks.
constexpr int NOALLOC_BLOCKS = DIAG_MAX_BLOCKS;
constexpr size_t NOALLOC_PARTIALS = (size_t)NOALLOC_BLOCKS * TGV_DIAG_COUNT;

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_PARTIALS];

constexpr int NOALLOC_MAX_DEVICES = 64;
struct NoallocCache {
  CUcontext ctx;
  double* ptr;
};
static NoallocCache g_noalloc_cache[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

// cuCtxGetCurrent through the runtime's driver entry-point query (null if the
// driver does not provide it; the cache then keys on the device alone).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
static CtxGetCurrentFn ctx_get_current() {
  static const CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 2000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  return fn;
}

static CUcontext current_ctx() {
  CUcontext ctx = nullptr;
  const CtxGetCurrentFn fn = ctx_get_current();
  if (fn && fn(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  return ctx;
}

// Device address of the partials array on the current device and context.
static double* noalloc_scratch(int dev) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoallocCache& c = g_noalloc_cache[dev];
  if (c.ptr && c.ctx == current_ctx()) return c.ptr;
  void* addr = nullptr;
  if (cudaGetSymbolAddress(&addr, g_noalloc_partials) != cudaSuccess || !addr) return nullptr;
  c.ptr = static_cast<double*>(addr);
  c.ctx = current_ctx();  // the lookup has made the device's context current
  return c.ptr;
}

}  // namespace tgv

using namespace tgv;

extern "C" int32_t diagnostics_reduce_noalloc(const tgv_config* cfg, const void* q,
                                              double* out_dev, void* stream) {
  const int32_t s = tgv_check_config(cfg);
  if (s != TGV_OK) return s;
  if (!q || !out_dev) return TGV_ERR_ARG;
  const long long items = diag_items(cfg->n);
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
  if (mode_launchers(find_mode(*cfg)).diag_partial(P, q, part, (int)nb, st) != cudaSuccess)
    return TGV_ERR_CUDA;
  diag_final_kernel<<<1, 32 * TGV_DIAG_COUNT, 0, st>>>(P, part, (int)nb, out_dev);
  if (cudaGetLastError() != cudaSuccess) return TGV_ERR_CUDA;
  return TGV_OK;
}
