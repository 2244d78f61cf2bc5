// tgv_mode_1.cu - kernels of precision mode 1: Q double, Qt double,
// compute float, accumulate double.
#include "tgv_modes.cuh"

namespace tgv {
const ModeLaunchers& mode_launchers_1() {
  static const ModeLaunchers L = make_launchers<double, double, float, double>();
  return L;
}
}  // namespace tgv
