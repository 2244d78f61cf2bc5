// tgv_mode_7.cu - kernels of precision mode 7: Q float, Qt __half,
// compute float, accumulate float.
#include "tgv_modes.cuh"

namespace tgv {
const ModeLaunchers& mode_launchers_7() {
  static const ModeLaunchers L = make_launchers<float, __half, float, float, true>();
  return L;
}
}  // namespace tgv
