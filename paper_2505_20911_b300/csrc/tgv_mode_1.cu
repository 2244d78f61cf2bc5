// tgv_mode_1.cu - kernels of precision mode 1: Q double, Qt double,
// compute float, accumulate double.
#include "tgv_modes.cuh"

namespace tgv {
const ModeLaunchers& mode_launchers_1() {
  // The FP64 state makes the 32x16 tile's shared memory (211 KB) allow one
  // CTA per SM; two 16x16 CTAs per SM overlap one CTA's FP64 epilogue with
  // the other's FP32 stencil work and measured about 10% faster at 256^3.
  static const ModeLaunchers L = [] {
    ModeLaunchers m = make_launchers<double, double, float, double, true>();
    m.first_tile = 1;
    return m;
  }();
  return L;
}
}  // namespace tgv
