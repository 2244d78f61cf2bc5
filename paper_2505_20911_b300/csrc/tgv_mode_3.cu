// tgv_mode_3.cu - kernels of precision mode 3: Q float, Qt float,
// compute float, accumulate float.
#include "tgv_modes.cuh"

namespace tgv {
const ModeLaunchers& mode_launchers_3() {
  static const ModeLaunchers L = make_launchers<float, float, float, float, true>();
  return L;
}
}  // namespace tgv
