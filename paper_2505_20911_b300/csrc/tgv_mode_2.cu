// tgv_mode_2.cu - kernels of precision mode 2: Q float, Qt float,
// compute double, accumulate double.
#include "tgv_modes.cuh"

namespace tgv {
const ModeLaunchers& mode_launchers_2() {
  static const ModeLaunchers L = make_launchers<float, float, double, double, true>();
  return L;
}
}  // namespace tgv
