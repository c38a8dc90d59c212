// Split-FP32 ("double-float") arithmetic on the FP32 pipe.
//
// GB300 executes FP64 FMAs at 2 lanes per clock per SM, 1/63 of its FP32
// rate, so even streaming FP64 vector work (dot products, axpy) is bound by
// the FP64 pipe rather than by HBM. A value is kept here as an unevaluated
// sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2 (48 significant
// bits, 8 bytes, the same storage as an FP64 number) and operated on with
// error-free transformations: Knuth's two-sum, Dekker's product through a
// fused multiply-add. Reference: T. J. Dekker, "A floating-point technique
// for extending the available precision", Numer. Math. 18 (1971); D. E.
// Knuth, TAOCP vol. 2, 4.2.2.
#pragma once
#include <cuda_runtime.h>

namespace mehdg {

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// renormalise (h, l) so that |l| <= ulp(h) / 2
__device__ __forceinline__ float2 df_norm(float h, float l) {
  const float s = h + l;
  return make_float2(s, l - (s - h));
}

// FP64 -> (hi, lo)
__device__ __forceinline__ float2 df_from(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

__device__ __forceinline__ double df_to(float2 a) { return (double)a.x + (double)a.y; }

// (ah, al) += a * b, products and sum of the high words error-free; the low
// words collect the rounding terms (a.lo * b.lo, below 2^-48 relative, is dropped)
__device__ __forceinline__ void df_fma(float& ah, float& al, float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  float s, t;
  two_sum(ah, p, s, t);
  ah = s;
  al += t + e;
}

// (ah, al) += (bh, bl)
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  float s, t;
  two_sum(ah, bh, s, t);
  ah = s;
  al += t + bl;
}

// warp-wide sum of (h, l) pairs (all lanes receive the result)
__device__ __forceinline__ void df_warp_sum(float& h, float& l) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, off);
    const float ol = __shfl_xor_sync(0xffffffffu, l, off);
    df_add(h, l, oh, ol);
  }
}

}  // namespace mehdg
