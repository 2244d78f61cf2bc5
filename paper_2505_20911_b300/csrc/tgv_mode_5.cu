// tgv_mode_5.cu - kernels of precision mode 5: Q __half, Qt __half,
// compute float, accumulate float.
#include "tgv_modes.cuh"

namespace tgv {
const ModeLaunchers& mode_launchers_5() {
  static const ModeLaunchers L = make_launchers<__half, __half, float, float, true>();
  return L;
}
}  // namespace tgv
