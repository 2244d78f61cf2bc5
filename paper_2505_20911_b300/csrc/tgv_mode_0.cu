// tgv_mode_0.cu - kernels of precision mode 0: Q double, Qt double,
// compute double, accumulate double.
#include "tgv_modes.cuh"

namespace tgv {
const ModeLaunchers& mode_launchers_0() {
  static const ModeLaunchers L = make_launchers<double, double, double, double, true>();
  return L;
}
}  // namespace tgv
