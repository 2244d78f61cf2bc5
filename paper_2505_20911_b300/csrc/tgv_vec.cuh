// tgv_vec.cuh - a "unit" of NP consecutive x points handled by one thread.
//
// Vec<T, 1> is a scalar; Vec<float, 2> packs two FP32 lanes and uses the
// sm_100+ paired FP32 operations (PTX add/sub/mul/fma .rn .f32x2), which
// issue once for both lanes; Vec<__half, 2> is __half2.  All stencil arithmetic of the
// stage kernel is written once against this interface.
#pragma once

#include "tgv_common.cuh"

namespace tgv {

template <class T, int NP> struct Vec;

// ------------------------------------------------------------------ scalars
template <class T> struct Vec<T, 1> {
  T v;
  __device__ __forceinline__ Vec() {}
  __device__ __forceinline__ explicit Vec(T a) : v(a) {}
  static __device__ __forceinline__ Vec splat(T a) { return Vec(a); }
  static __device__ __forceinline__ Vec load(const T* p) { return Vec(p[0]); }
  __device__ __forceinline__ void store(T* p) const { p[0] = v; }
  __device__ __forceinline__ T get(int) const { return v; }
  // (a.hi, b.lo) of two consecutive units; for one-point units it is b
  static __device__ __forceinline__ Vec mix(const Vec&, const Vec& b) { return b; }
  __device__ __forceinline__ Vec swapped() const { return *this; }
};
template <class T> __device__ __forceinline__ Vec<T, 1> operator+(Vec<T, 1> a, Vec<T, 1> b) { return Vec<T, 1>(a.v + b.v); }
template <class T> __device__ __forceinline__ Vec<T, 1> operator-(Vec<T, 1> a, Vec<T, 1> b) { return Vec<T, 1>(a.v - b.v); }
template <class T> __device__ __forceinline__ Vec<T, 1> operator*(Vec<T, 1> a, Vec<T, 1> b) { return Vec<T, 1>(a.v * b.v); }
template <class T> __device__ __forceinline__ Vec<T, 1> operator-(Vec<T, 1> a) { return Vec<T, 1>(-a.v); }
__device__ __forceinline__ Vec<double, 1> fma(Vec<double, 1> a, Vec<double, 1> b, Vec<double, 1> c) {
  return Vec<double, 1>(__fma_rn(a.v, b.v, c.v));
}
__device__ __forceinline__ Vec<float, 1> fma(Vec<float, 1> a, Vec<float, 1> b, Vec<float, 1> c) {
  return Vec<float, 1>(__fmaf_rn(a.v, b.v, c.v));
}
__device__ __forceinline__ Vec<double, 1> rcp(Vec<double, 1> a) { return Vec<double, 1>(1.0 / a.v); }
__device__ __forceinline__ Vec<float, 1> rcp(Vec<float, 1> a) { return Vec<float, 1>(__frcp_rn(a.v)); }

// ------------------------------------------------------ two FP32 lanes (f32x2)
template <> struct Vec<float, 2> {
  float2 v;
  __device__ __forceinline__ Vec() {}
  __device__ __forceinline__ explicit Vec(float2 a) : v(a) {}
  __device__ __forceinline__ Vec(float a, float b) : v(make_float2(a, b)) {}
  static __device__ __forceinline__ Vec splat(float a) { return Vec(a, a); }
  static __device__ __forceinline__ Vec load(const float* p) {
    return Vec(*reinterpret_cast<const float2*>(p));
  }
  __device__ __forceinline__ void store(float* p) const { *reinterpret_cast<float2*>(p) = v; }
  __device__ __forceinline__ float get(int e) const { return e ? v.y : v.x; }
  static __device__ __forceinline__ Vec mix(const Vec& a, const Vec& b) { return Vec(a.v.y, b.v.x); }
  __device__ __forceinline__ Vec swapped() const { return Vec(v.y, v.x); }
};
// The paired operations are written as PTX with an explicit rounding mode
// (add/sub/mul/fma .rn .f32x2): an explicit rounding mode forbids the code
// generator to fuse a multiply into a following add, so every kernel that
// evaluates the same expression rounds it the same way, whatever the
// surrounding code (the CUDA paired intrinsics were fused in some code shapes
// and not in others, and results then differed in the last bit between
// kernels that compute the same grid point).
#define TGV_F32X2_OP2(NAME, OP)                                                         \
  __device__ __forceinline__ float2 NAME(float2 a, float2 b) {                           \
    float2 d;                                                                            \
    asm("{ .reg .b64 ra, rb, rd; mov.b64 ra, {%2, %3}; mov.b64 rb, {%4, %5}; " OP        \
        " rd, ra, rb; mov.b64 {%0, %1}, rd; }"                                           \
        : "=f"(d.x), "=f"(d.y)                                                           \
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                       \
    return d;                                                                            \
  }
TGV_F32X2_OP2(f32x2_add, "add.rn.f32x2")
TGV_F32X2_OP2(f32x2_sub, "sub.rn.f32x2")
TGV_F32X2_OP2(f32x2_mul, "mul.rn.f32x2")
#undef TGV_F32X2_OP2
__device__ __forceinline__ float2 f32x2_fma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{ .reg .b64 ra, rb, rc, rd; mov.b64 ra, {%2, %3}; mov.b64 rb, {%4, %5}; "
      "mov.b64 rc, {%6, %7}; fma.rn.f32x2 rd, ra, rb, rc; mov.b64 {%0, %1}, rd; }"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ Vec<float, 2> operator+(Vec<float, 2> a, Vec<float, 2> b) {
  return Vec<float, 2>(f32x2_add(a.v, b.v));
}
__device__ __forceinline__ Vec<float, 2> operator-(Vec<float, 2> a) { return Vec<float, 2>(-a.v.x, -a.v.y); }
__device__ __forceinline__ Vec<float, 2> operator-(Vec<float, 2> a, Vec<float, 2> b) {
  return Vec<float, 2>(f32x2_sub(a.v, b.v));
}
__device__ __forceinline__ Vec<float, 2> operator*(Vec<float, 2> a, Vec<float, 2> b) {
  return Vec<float, 2>(f32x2_mul(a.v, b.v));
}
__device__ __forceinline__ Vec<float, 2> fma(Vec<float, 2> a, Vec<float, 2> b, Vec<float, 2> c) {
  return Vec<float, 2>(f32x2_fma(a.v, b.v, c.v));
}
__device__ __forceinline__ Vec<float, 2> rcp(Vec<float, 2> a) {
  return Vec<float, 2>(__frcp_rn(a.v.x), __frcp_rn(a.v.y));
}

// ------------------------------------------------------------ two FP16 lanes
template <> struct Vec<__half, 2> {
  __half2 v;
  __device__ __forceinline__ Vec() {}
  __device__ __forceinline__ explicit Vec(__half2 a) : v(a) {}
  __device__ __forceinline__ Vec(__half a, __half b) : v(__halves2half2(a, b)) {}
  static __device__ __forceinline__ Vec splat(__half a) { return Vec(__half2half2(a)); }
  static __device__ __forceinline__ Vec load(const __half* p) {
    return Vec(*reinterpret_cast<const __half2*>(p));
  }
  __device__ __forceinline__ void store(__half* p) const { *reinterpret_cast<__half2*>(p) = v; }
  __device__ __forceinline__ __half get(int e) const { return e ? __high2half(v) : __low2half(v); }
  static __device__ __forceinline__ Vec mix(const Vec& a, const Vec& b) {
    return Vec(__halves2half2(__high2half(a.v), __low2half(b.v)));
  }
  __device__ __forceinline__ Vec swapped() const { return Vec(__lowhigh2highlow(v)); }
};
__device__ __forceinline__ Vec<__half, 2> operator+(Vec<__half, 2> a, Vec<__half, 2> b) { return Vec<__half, 2>(__hadd2(a.v, b.v)); }
__device__ __forceinline__ Vec<__half, 2> operator-(Vec<__half, 2> a, Vec<__half, 2> b) { return Vec<__half, 2>(__hsub2(a.v, b.v)); }
__device__ __forceinline__ Vec<__half, 2> operator*(Vec<__half, 2> a, Vec<__half, 2> b) { return Vec<__half, 2>(__hmul2(a.v, b.v)); }
__device__ __forceinline__ Vec<__half, 2> operator-(Vec<__half, 2> a) { return Vec<__half, 2>(__hneg2(a.v)); }
__device__ __forceinline__ Vec<__half, 2> fma(Vec<__half, 2> a, Vec<__half, 2> b, Vec<__half, 2> c) {
  return Vec<__half, 2>(__hfma2(a.v, b.v, c.v));
}
__device__ __forceinline__ Vec<__half, 2> rcp(Vec<__half, 2> a) { return Vec<__half, 2>(h2rcp(a.v)); }

// pin(v): an empty assembly statement that makes the value opaque to the
// compiler.  The stage kernel passes its register-queue taps through it.
// Without it the register-queue kernel and the shared-memory-ring kernel,
// which apply the same operations to the same values, differed in the last
// bit at rare grid points (measured: first after 320 steps of a 32^3 run);
// with it they agree bit for bit (the ensemble and slab tests compare them).
template <class T, int NP> __device__ __forceinline__ void pin(Vec<T, NP>&) {}
__device__ __forceinline__ void pin(Vec<float, 2>& a) {
  asm volatile("" : "+f"(a.v.x), "+f"(a.v.y));
}
__device__ __forceinline__ void pin(Vec<__half, 2>& a) {
  unsigned r = *reinterpret_cast<unsigned*>(&a.v);
  asm volatile("" : "+r"(r));
  a.v = *reinterpret_cast<__half2*>(&r);
}

// ---------------------------------------------------- storage <-> compute units
// Load NP consecutive storage elements and convert to the compute type.
template <class TC, int NP, class TS> struct UnitIO;

template <class TC, class TS> struct UnitIO<TC, 1, TS> {
  using Raw = TS;
  static __device__ __forceinline__ Raw load(const TS* p) { return p[0]; }
  static __device__ __forceinline__ Vec<TC, 1> conv(Raw r) { return Vec<TC, 1>(cvt<TC>(r)); }
};

template <class TC, class TS> struct UnitIO<TC, 2, TS> {
  struct alignas(2 * sizeof(TS)) Raw { TS a, b; };
  static __device__ __forceinline__ Raw load(const TS* p) { return *reinterpret_cast<const Raw*>(p); }
  static __device__ __forceinline__ Vec<TC, 2> conv(Raw r) { return Vec<TC, 2>(cvt<TC>(r.a), cvt<TC>(r.b)); }
};

// Load NP consecutive storage elements as NP values of type TA.
template <class TA, int NP, class TS>
__device__ __forceinline__ void load_elems(const TS* p, TA* out) {
  if constexpr (NP == 1) {
    out[0] = cvt<TA>(p[0]);
  } else {
    struct alignas(2 * sizeof(TS)) Raw { TS a, b; };
    const Raw r = *reinterpret_cast<const Raw*>(p);
    out[0] = cvt<TA>(r.a);
    out[1] = cvt<TA>(r.b);
  }
}

// The NP values of a raw unit (UnitIO<...>::Raw) as type TA.
template <class TA, int NP, class Raw>
__device__ __forceinline__ void raw_elems(const Raw& r, TA* out) {
  if constexpr (NP == 1) {
    out[0] = cvt<TA>(r);
  } else {
    out[0] = cvt<TA>(r.a);
    out[1] = cvt<TA>(r.b);
  }
}

// Store NP accumulate-type values as NP consecutive storage elements.
template <class TS, int NP> struct UnitStore;
template <class TS> struct UnitStore<TS, 1> {
  template <class TA> static __device__ __forceinline__ void put(TS* p, const TA* v) { p[0] = cvt<TS>(v[0]); }
};
template <class TS> struct UnitStore<TS, 2> {
  struct alignas(2 * sizeof(TS)) Raw { TS a, b; };
  template <class TA> static __device__ __forceinline__ void put(TS* p, const TA* v) {
    Raw r;
    r.a = cvt<TS>(v[0]);
    r.b = cvt<TS>(v[1]);
    *reinterpret_cast<Raw*>(p) = r;
  }
};

}  // namespace tgv
