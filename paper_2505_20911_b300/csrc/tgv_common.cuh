// tgv_common.cuh - shared device/host definitions of the TGV kernels.
//
// Number types: storage types (double, float, __nv_bfloat16, __half) convert
// to and from the compute/accumulate types through the helpers below; all
// arithmetic of a kernel runs in one compute type TC.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "tgv.h"

namespace tgv {

// NVTX range for profilers (a no-op unless a tool is attached): the RK steps,
// stages, adjoint sweeps and ensemble replays the library enqueues are named
// in a timeline.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- conversions
template <class T> struct Num;
template <> struct Num<double> {
  static __host__ __device__ __forceinline__ double to_f64(double v) { return v; }
  static __host__ __device__ __forceinline__ double from_f64(double v) { return v; }
};
template <> struct Num<float> {
  static __host__ __device__ __forceinline__ double to_f64(float v) { return (double)v; }
  static __host__ __device__ __forceinline__ float from_f64(double v) { return (float)v; }
};
template <> struct Num<__half> {
  static __device__ __forceinline__ double to_f64(__half v) { return (double)__half2float(v); }
  static __device__ __forceinline__ __half from_f64(double v) { return __double2half(v); }
};
template <> struct Num<__nv_bfloat16> {
  static __device__ __forceinline__ double to_f64(__nv_bfloat16 v) {
    return (double)__bfloat162float(v);
  }
  static __device__ __forceinline__ __nv_bfloat16 from_f64(double v) {
    return __double2bfloat16(v);
  }
};

// cvt<To>(from): one rounding, from any supported type to any other.
template <class To, class From> struct Cvt {
  static __device__ __forceinline__ To go(From v) { return Num<To>::from_f64(Num<From>::to_f64(v)); }
};
template <class T> struct Cvt<T, T> {
  static __device__ __forceinline__ T go(T v) { return v; }
};
template <> struct Cvt<float, __half> {
  static __device__ __forceinline__ float go(__half v) { return __half2float(v); }
};
template <> struct Cvt<__half, float> {
  static __device__ __forceinline__ __half go(float v) { return __float2half_rn(v); }
};
template <> struct Cvt<float, __nv_bfloat16> {
  static __device__ __forceinline__ float go(__nv_bfloat16 v) { return __bfloat162float(v); }
};
template <> struct Cvt<__nv_bfloat16, float> {
  static __device__ __forceinline__ __nv_bfloat16 go(float v) { return __float2bfloat16_rn(v); }
};
// FP64 <-> FP32 conversions in integer arithmetic (IEEE 754 binary64 and
// binary32 bit layouts; round to nearest, ties to even).  On B300 the
// hardware conversions share the FP64 pipe, which runs at 1/64 of the FP32
// rate; these run on the integer pipes.  Values below the FP32 normal range
// (|x| < 2^-126) become signed zeros.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned s = hi & 0x80000000u;
  const unsigned e = (hi >> 20) & 0x7FFu;               // biased binary64 exponent
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // top 23 fraction bits
  const unsigned rem = lo & 0x1FFFFFFFu;                // the 29 dropped bits
  unsigned f = s | ((e - 896u) << 23) | m;               // rebias 1023 -> 127
  f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
  if (e <= 896u) f = s;                                   // below the normal range
  if (e >= 1151u) f = s | 0x7F800000u | (e == 2047u && (m | rem) ? 0x400000u : 0u);
  return __uint_as_float(f);
}
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned f = __float_as_uint(x);
  const unsigned s = f & 0x80000000u, e = (f >> 23) & 0xFFu, m = f & 0x7FFFFFu;
  unsigned hi = s | ((e + 896u) << 20) | (m >> 3);
  if (e == 0u) hi = s;                                    // zero (subnormals flushed)
  if (e == 255u) hi = s | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u);
  const unsigned lo = (e == 0u) ? 0u : (m << 29);
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}
template <> struct Cvt<float, double> {
  static __device__ __forceinline__ float go(double v) { return f64_to_f32(v); }
};
template <> struct Cvt<double, float> {
  static __device__ __forceinline__ double go(float v) { return f32_to_f64(v); }
};
template <class To, class From>
__device__ __forceinline__ To cvt(From v) { return Cvt<To, From>::go(v); }

// Reciprocal in the compute type (IEEE-rounded division for float/double).
__device__ __forceinline__ double recip(double v) { return 1.0 / v; }
__device__ __forceinline__ float recip(float v) { return 1.0f / v; }
__device__ __forceinline__ __half recip(__half v) { return hrcp(v); }

// Fused multiply-add a*b + c with one rounding, in the accumulate type.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Per-thread accumulators of the diagnostics.  FP64 arithmetic runs at about
// 1/64 of the FP32 rate on B300, so in the FP32-arithmetic kernels each
// thread sums its per-point values with compensated (Kahan) FP32 summation,
// whose result is within about one FP32 rounding of the exact sum of its
// terms, and converts once to FP64, where the partials of all threads are
// added; FP64-arithmetic kernels add in FP64 directly.
struct KahanF {
  float s = 0.f, c = 0.f;  // running sum and its negated rounding error
  __device__ __forceinline__ void add(float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
struct PlainD {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <class T> struct DiagAcc { using A = KahanF; using In = float; };
template <> struct DiagAcc<double> { using A = PlainD; using In = double; };

// Finite (neither NaN nor +-Inf): the exponent field is not all ones.
__device__ __forceinline__ bool finite_val(float v) {
  return (__float_as_uint(v) & 0x7F800000u) != 0x7F800000u;
}
__device__ __forceinline__ bool finite_val(__half v) {
  return (__half_as_ushort(v) & 0x7C00u) != 0x7C00u;
}
__device__ __forceinline__ bool finite_val(double v) { return isfinite(v); }

// ------------------------------------------------------------ problem params
// Per-problem constants, precomputed on the host in FP64.
struct Problem {
  int n;            // grid points per direction
  int split;        // tgv_split
  int encoding;     // tgv_encoding
  double h;         // grid spacing L/N
  double inv12h;    // 1/(12 h): first-derivative stencil scale
  double inv12h2;   // 1/(12 h^2): second-derivative stencil scale
  double gamma, gm1, gM2;  // gamma, gamma-1, gamma*M^2
  double nu;        // mu/Re
  double kappa;     // mu/((gamma-1) M^2 Pr Re)
  double rho0, rhoE0;      // encoding offsets (0 for TGV_ENC_PLAIN)
  double mach, re;
  double offset;    // grid points at (i + offset) h: 0, or 0.5 (cell-centred)
  int symmetric;    // 1: mirror planes on every face (TGV_FLAG_SYMMETRIC)
};

// Grid index of a neighbour at i (possibly outside [0, n)) and whether the
// mirror flipped it: periodic wrap, or reflection about the faces of the
// cell-centred symmetric box (i -> -1-i, i -> 2n-1-i).  Indices more than one
// box length outside are clamped (they only feed points outside the grid).
__host__ __device__ __forceinline__ int wrap_index(int i, int n, bool symmetric, bool* flipped) {
  *flipped = false;
  if (!symmetric) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  if (i < 0) { i = -1 - i; *flipped = true; }
  else if (i >= n) { i = 2 * n - 1 - i; *flipped = true; }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// wrap_index for an index within one box length of the grid (i in [-n, 2n)),
// without a division: the z planes a stage kernel visits (z0 - 2 .. z1 + 1).
__host__ __device__ __forceinline__ int wrap_near(int i, int n, bool symmetric, bool* flipped) {
  *flipped = false;
  if (i < 0) {
    if (symmetric) { *flipped = true; return -1 - i; }
    return i + n;
  }
  if (i >= n) {
    if (symmetric) { *flipped = true; return 2 * n - 1 - i; }
    return i - n;
  }
  return i;
}

Problem make_problem(const tgv_config& c);

// Storage-type tag -> C++ type.
template <int D> struct DType;
template <> struct DType<TGV_F64> { using T = double; };
template <> struct DType<TGV_F32> { using T = float; };
template <> struct DType<TGV_BF16> { using T = __nv_bfloat16; };
template <> struct DType<TGV_F16> { using T = __half; };

inline size_t dtype_size(int d) {
  switch (d) {
    case TGV_F64: return 8;
    case TGV_F32: return 4;
    case TGV_BF16: return 2;
    case TGV_F16: return 2;
  }
  return 0;
}

// Williamson 2N coefficients (reading of Sec. 3.1, Eqs. 3-4).
constexpr double RK_A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
constexpr double RK_B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

#define TGV_CUDA_TRY(expr)                                    \
  do {                                                        \
    cudaError_t e__ = (expr);                                 \
    if (e__ != cudaSuccess) { return TGV_ERR_CUDA; }          \
  } while (0)

}  // namespace tgv
