// Float-float arithmetic shared by the float-float Cholesky updates of the
// log-det and the float-float products of the gradient.
#pragma once

#include <cuda_runtime.h>

namespace rpa {

// ---------------------------------------------------------------- float-float arithmetic
// A value is the unevaluated sum hi + lo of two FP32 numbers; products use
// Dekker's exact product via FMA, sums Knuth's two-sum (about 44 significant
// bits after a panel of multiply-adds).  A complex value is a float4
// (re hi, re lo, im hi, im lo).  The _rn intrinsics keep the compiler from
// contracting the steps into FMAs, which would break the exact error terms.
__device__ __forceinline__ float4 ff_split(double2 x) {
  const float rh = __double2float_rn(x.x), ih = __double2float_rn(x.y);
  return make_float4(rh, __double2float_rn(x.x - (double)rh), ih, __double2float_rn(x.y - (double)ih));
}

// (sh, sl) += (xh, xl) * (yh, yl)
__device__ __forceinline__ void ff_mac(float& sh, float& sl, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  float e = __fmaf_rn(xh, yh, -p);  // p + e == xh * yh exactly
  e = __fmaf_rn(xh, yl, e);
  e = __fmaf_rn(xl, yh, e);
  const float t = __fadd_rn(sh, p);  // t + d == sh + p exactly
  const float z = __fsub_rn(t, sh);
  const float d = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(d, e));
}

// (h, l) <- h + l with |l| <= ulp(h) / 2 (fast two-sum; |h| >= |l| holds)
__device__ __forceinline__ void ff_norm(float& h, float& l) {
  const float s = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(s, h));
  h = s;
}

// (ah, al) - (bh, bl), normalised
__device__ __forceinline__ void ff_sub(float& ah, float& al, float bh, float bl) {
  const float t = __fsub_rn(ah, bh);
  const float z = __fsub_rn(t, ah);
  float d = __fadd_rn(__fsub_rn(ah, __fsub_rn(t, z)), __fsub_rn(-bh, z));  // t + d == ah - bh exactly
  d = __fadd_rn(d, __fsub_rn(al, bl));
  ah = t;
  al = d;
  ff_norm(ah, al);
}

__device__ __forceinline__ double2 ff_to_double(float4 v) {
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

}  // namespace rpa
