// fr_df.cuh -- double-float arithmetic: a value carried as an unevaluated sum hi + lo of
// two FP32 numbers (|lo| <= ulp(hi) / 2 after normalisation, about 48 significant bits),
// built from error-free transformations (Knuth's two-sum, the exact FMA residual of a
// product).  Every rounding step uses the __f*_rn intrinsics, which the compiler never
// contracts into a fused multiply-add: contraction would break the transformations.
#pragma once
#include <cuda_runtime.h>

namespace fr {

// hi + lo = v to about 2^-48 |v|.
__device__ __forceinline__ float2 df_split(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(__dsub_rn(v, (double)h)));
}

__device__ __forceinline__ double df_value(float h, float l) { return __dadd_rn((double)h, (double)l); }

// (sh, sl) += (bh, bl) (two-sum of the high parts; the low parts are added).
__device__ __forceinline__ void df_merge(float& sh, float& sl, float bh, float bl) {
  const float sn = __fadd_rn(sh, bh);
  const float bv = __fsub_rn(sn, sh);
  const float er = __fadd_rn(__fsub_rn(sh, __fsub_rn(sn, bv)), __fsub_rn(bh, bv));
  sh = sn;
  sl = __fadd_rn(sl, __fadd_rn(bl, er));
}

// (sh, sl) += a (xh + xl), a a plain FP32 number.
__device__ __forceinline__ void df_add(float& sh, float& sl, float a, float2 xv) {
  const float ph = __fmul_rn(a, xv.x);
  float pl = fmaf(a, xv.x, -ph);   // exact low part of a x_hi
  pl = fmaf(a, xv.y, pl);           // + a x_lo
  df_merge(sh, sl, ph, pl);
}

// (sh, sl) += (ah + al)(bh + bl); the al bl term (below 2^-48 of the product) is dropped.
__device__ __forceinline__ void df_fma(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float ph = __fmul_rn(ah, bh);
  float pl = fmaf(ah, bh, -ph);
  pl = fmaf(ah, bl, pl);
  pl = fmaf(al, bh, pl);
  df_merge(sh, sl, ph, pl);
}

// (xh, xl) -= (ah + al)(bh + bl), then renormalised so that the pair keeps its ~48 bits
// over long update chains.
__device__ __forceinline__ void df_fms(float& xh, float& xl, float ah, float al, float bh, float bl) {
  const float ph = __fmul_rn(ah, bh);
  float pl = fmaf(ah, bh, -ph);
  pl = fmaf(ah, bl, pl);
  pl = fmaf(al, bh, pl);
  df_merge(xh, xl, -ph, -pl);
  const float s = __fadd_rn(xh, xl);
  xl = __fsub_rn(xl, __fsub_rn(s, xh));
  xh = s;
}

// Sum of a double-float over the 32 lanes of a warp (every lane gets it).
__device__ __forceinline__ void df_warp_sum(float& h, float& l) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, off);
    const float ol = __shfl_xor_sync(0xffffffffu, l, off);
    df_merge(h, l, oh, ol);
  }
}

}  // namespace fr
