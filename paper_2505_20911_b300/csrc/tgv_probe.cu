// tgv_probe.cu - arithmetic-pipe throughput probe (measurement support for
// the benchmark's ALU roofline; no paper counterpart).
//
// Every thread runs CHAINS independent chains of fused multiply-adds
// x <- x * a + b for `iters` iterations in one of three forms: scalar FP32,
// paired FP32 (f32x2, two lanes per instruction) or packed FP16 (half2), and
// writes the sum of its chains to `sink` so that nothing is dead code.  With
// enough resident warps the chains keep the FMA pipe busy, so flops / time is
// the pipe's throughput for that form.
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "tgv.h"

namespace {

constexpr int CHAINS = 8;
constexpr int PROBE_THREADS = 256;

template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS)
fma_probe_kernel(float* __restrict__ sink, int iters, float a, float b) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (KIND == TGV_PROBE_FFMA) {
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = 1e-3f * (float)(t & 255) + (float)c;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) x[c] = __fmaf_rn(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    sink[t] = s;
  } else if constexpr (KIND == TGV_PROBE_FFMA2) {
    float2 x[CHAINS];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = make_float2(1e-3f * (float)(t & 255) + (float)c, (float)c);
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c].x + x[c].y;
    sink[t] = s;
  } else {
    __half2 x[CHAINS];
    const __half2 a2 = __float2half2_rn(a), b2 = __float2half2_rn(b);
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = __floats2half2_rn(1e-3f * (float)(t & 255), (float)c);
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) x[c] = __hfma2(x[c], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += __low2float(x[c]) + __high2float(x[c]);
    sink[t] = s;
  }
}

}  // namespace

extern "C" int32_t tgv_probe_fma(int32_t kind, int32_t iters, int32_t blocks, float* sink,
                                 size_t sink_floats, double* flops, void* stream) {
  if (kind < TGV_PROBE_FFMA || kind > TGV_PROBE_HFMA2 || iters < 1 || blocks < 1 || !sink ||
      sink_floats < (size_t)blocks * PROBE_THREADS || !flops)
    return TGV_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const float a = 0.9999f, b = 1e-4f;
  if (kind == TGV_PROBE_FFMA)
    fma_probe_kernel<TGV_PROBE_FFMA><<<blocks, PROBE_THREADS, 0, st>>>(sink, iters, a, b);
  else if (kind == TGV_PROBE_FFMA2)
    fma_probe_kernel<TGV_PROBE_FFMA2><<<blocks, PROBE_THREADS, 0, st>>>(sink, iters, a, b);
  else
    fma_probe_kernel<TGV_PROBE_HFMA2><<<blocks, PROBE_THREADS, 0, st>>>(sink, iters, a, b);
  if (cudaGetLastError() != cudaSuccess) return TGV_ERR_CUDA;
  const double lanes = kind == TGV_PROBE_FFMA ? 1.0 : 2.0;
  *flops = 2.0 * lanes * CHAINS * (double)iters * (double)blocks * PROBE_THREADS;
  return TGV_OK;
}
