// tgv_mode_6.cu - kernels of precision mode 6: Q __half, Qt __half,
// compute __half, accumulate float.
#include "tgv_modes.cuh"

namespace tgv {
const ModeLaunchers& mode_launchers_6() {
  static const ModeLaunchers L = make_launchers<__half, __half, __half, float, true>();
  return L;
}
}  // namespace tgv
