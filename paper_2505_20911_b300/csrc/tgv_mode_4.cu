// tgv_mode_4.cu - kernels of precision mode 4: Q __nv_bfloat16, Qt __nv_bfloat16,
// compute float, accumulate float.
#include "tgv_modes.cuh"

namespace tgv {
const ModeLaunchers& mode_launchers_4() {
  static const ModeLaunchers L = make_launchers<__nv_bfloat16, __nv_bfloat16, float, float, true>();
  return L;
}
}  // namespace tgv
