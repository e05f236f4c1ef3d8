// Double-float ("df32") arithmetic: a value is an unevaluated sum hi + lo of
// two float32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.
// Error-free transformations (Dekker, "A floating-point technique for
// extending the available precision", 1971; Knuth TAOCP Vol. 2, two-sum):
//   two_sum(a, b) = (s, e) with s = fl(a + b), a + b = s + e exactly;
//   a*b = p + e exactly with p = fl(a*b), e = fma(a, b, -p).
// GB300 runs float32 at 70x its float64 rate, so the memory-bound solve
// kernels use df32 (float32 FMA pipe) instead of float64 FMAs.  Operands are
// stored pre-split (8 bytes per element, as float64 would be).
// Every operation uses the _rn intrinsics so that the compiler cannot fuse
// or reassociate the error-free sequences.
#pragma once
#include <cuda_runtime.h>

__device__ __forceinline__ float2 df_split(double a) {
  const float h = __double2float_rn(a);
  return make_float2(h, __double2float_rn(a - (double)h));
}

__device__ __forceinline__ double df_to_double(float h, float l) { return (double)h + (double)l; }

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// (sh, sl) += a * x, a and x double-floats; sl collects all low-order terms.
__device__ __forceinline__ void df_mac(float& sh, float& sl, float2 a, float2 x) {
  const float p = __fmul_rn(a.x, x.x);
  const float e = __fmaf_rn(a.x, x.x, -p);
  float t, e2;
  df_two_sum(sh, p, t, e2);
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(e, e2), __fmaf_rn(a.x, x.y, __fmul_rn(a.y, x.x))));
}

// (sh, sl) += a * x with the low-order terms added by FMAs straight into sl:
// the same terms as df_mac (exact product error, exact two-sum error, the two
// cross products), 12 float32 instructions instead of 13.
__device__ __forceinline__ void df_mac_f(float& sh, float& sl, float2 a, float2 x) {
  const float p = __fmul_rn(a.x, x.x);
  const float e = __fmaf_rn(a.x, x.x, -p);
  float t, e2;
  df_two_sum(sh, p, t, e2);
  sh = t;
  sl = __fmaf_rn(a.x, x.y, __fmaf_rn(a.y, x.x, __fadd_rn(sl, __fadd_rn(e, e2))));
}

// df_mac_f for two independent accumulators at once, lanes .x and .y of each
// float2 (sh, sl: the accumulators' high and low parts; ah, al and xh, xl:
// the two products' operands), with the packed float32x2 operations of
// sm_100 and later (__fmul2_rn, __ffma2_rn, __fadd2_rn: one issue slot per
// pair of float32 operations).  Every lane takes the same IEEE
// round-to-nearest steps in the same order as df_mac_f, so the results are
// bit for bit those of two df_mac_f calls; a - b is formed as fma(b, -1, a)
// (one rounding of the exact a - b, the packed add having no negated
// operand) and -p as p * -1 (exact).
__device__ __forceinline__ void df_mac_f_x2(float2& sh, float2& sl, float2 ah, float2 al, float2 xh, float2 xl) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 p = __fmul2_rn(ah, xh);
  const float2 e = __ffma2_rn(ah, xh, __fmul2_rn(p, m1));                  // ah xh - p, exact
  const float2 t = __fadd2_rn(sh, p);                                      // two-sum of sh and p
  const float2 bp = __ffma2_rn(sh, m1, t);                                 // t - sh
  const float2 e2 = __fadd2_rn(__ffma2_rn(__ffma2_rn(bp, m1, t), m1, sh),  // (sh - (t - bp))
                               __ffma2_rn(bp, m1, p));                     //   + (p - bp)
  sh = t;
  sl = __ffma2_rn(ah, xl, __ffma2_rn(al, xh, __fadd2_rn(sl, __fadd2_rn(e, e2))));
}

// df_mac_f_x2 with the negated high part nxh = -xh also at hand (an operand
// shared by many products): q = ah nxh is -p exactly, so the product error
// fma(ah, xh, q), the sum sh - q and p - bp = -(q + bp) need no separate
// negation; every step rounds the same exact value as in df_mac_f_x2, so the
// results are the same bits, in 12 packed instructions instead of 13.
__device__ __forceinline__ void df_mac_f_x2n(float2& sh, float2& sl, float2 ah, float2 al, float2 xh, float2 xl,
                                             float2 nxh) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 q = __fmul2_rn(ah, nxh);                                    // -p
  const float2 e = __ffma2_rn(ah, xh, q);                                  // ah xh - p, exact
  const float2 t = __ffma2_rn(q, m1, sh);                                  // sh + p
  const float2 bp = __ffma2_rn(sh, m1, t);                                 // t - sh
  const float2 e2 = __ffma2_rn(__fadd2_rn(q, bp), m1,                      // (sh - (t - bp))
                               __ffma2_rn(__ffma2_rn(bp, m1, t), m1, sh)); //   + (p - bp)
  sh = t;
  sl = __ffma2_rn(ah, xl, __ffma2_rn(al, xh, __fadd2_rn(sl, __fadd2_rn(e, e2))));
}

// (h0, l0) += a0 x0 and (h1, l1) += a1 x1: df_mac_f_x2 on two scalar accumulators.
__device__ __forceinline__ void df_mac_2(float& h0, float& l0, float& h1, float& l1, float2 a0, float2 x0, float2 a1,
                                         float2 x1) {
  float2 H = make_float2(h0, h1), L = make_float2(l0, l1);
  df_mac_f_x2(H, L, make_float2(a0.x, a1.x), make_float2(a0.y, a1.y), make_float2(x0.x, x1.x), make_float2(x0.y, x1.y));
  h0 = H.x;
  h1 = H.y;
  l0 = L.x;
  l1 = L.y;
}

// The two double-float entries of a float4 (h0, l0, h1, l1) times those of
// x, accumulated into (h0, l0) and (h1, l1): df_mac_f_x2 on the pair.
__device__ __forceinline__ void df_mac_pair(float& h0, float& l0, float& h1, float& l1, float4 a, float4 x) {
  float2 H = make_float2(h0, h1), L = make_float2(l0, l1);
  df_mac_f_x2(H, L, make_float2(a.x, a.z), make_float2(a.y, a.w), make_float2(x.x, x.z), make_float2(x.y, x.w));
  h0 = H.x;
  h1 = H.y;
  l0 = L.x;
  l1 = L.y;
}

// Fold the low part into the high part (fast two-sum, |sh| >= |sl| not required
// for the exactness of the sum, only for normalisation).
__device__ __forceinline__ void df_renorm(float& sh, float& sl) {
  float s, e;
  df_two_sum(sh, sl, s, e);
  sh = s;
  sl = e;
}

// (ah, al) += (bh, bl)
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  float s, e;
  df_two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  df_two_sum(s, e, ah, al);
}

// Warp-wide double-float sum (result valid in every lane).
__device__ __forceinline__ void df_warp_sum(float& h, float& l) {
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_add(h, l, oh, ol);
  }
}

// (h, l) += (bh, bl) inside a reduction: the high parts by an error-free
// two-sum whose error joins the low part, the low parts added plainly, and
// no renormalisation until the reduction is done (df_renorm).  The only
// roundings are those of the low-part additions, relative to the low parts
// (about 2^-24 of 2^-24 of the terms), as in df_add.
__device__ __forceinline__ void df_reduce_add(float& h, float& l, float bh, float bl) {
  float s, e;
  df_two_sum(h, bh, s, e);
  h = s;
  l = __fadd_rn(l, __fadd_rn(bl, e));
}
// df_reduce_add on two independent pairs at once (lanes .x and .y).
__device__ __forceinline__ void df_reduce_add_x2(float2& h, float2& l, float2 bh, float2 bl) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 s = __fadd2_rn(h, bh);
  const float2 bp = __ffma2_rn(h, m1, s);                                  // s - h
  const float2 e = __fadd2_rn(__ffma2_rn(__ffma2_rn(bp, m1, s), m1, h),    // (h - (s - bp))
                              __ffma2_rn(bp, m1, bh));                     //   + (bh - bp)
  h = s;
  l = __fadd2_rn(l, __fadd2_rn(bl, e));
}
// Warp-wide double-float sum by df_reduce_add, renormalised at the end
// (result valid in every lane).
__device__ __forceinline__ void df_warp_sum_lazy(float& h, float& l) {
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_reduce_add(h, l, oh, ol);
  }
  df_renorm(h, l);
}

// fast two-sum (|a| >= |b| or a == 0): s + e = a + b exactly
__device__ __forceinline__ float2 df_fast(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// a * b in double-float (Dekker 1971): exact product of the high parts, the
// cross terms added to its error, one fast renormalisation.
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = __fmaf_rn(a.x, b.x, -p);
  const float t = __fadd_rn(e, __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
  return df_fast(p, t);
}

// a / b in double-float (Dekker 1971): q1 = a_h / b_h, r = a - q1 b formed with
// an exact product, q2 = r_h / b_h; about 2^-46 relative.
__device__ __forceinline__ float2 df_div(float2 a, float2 b) {
  const float q1 = __fdiv_rn(a.x, b.x);
  const float p = __fmul_rn(q1, b.x);
  const float pe = __fmaf_rn(q1, b.x, -p);             // q1 b_h = p + pe exactly
  float rh, re;
  df_two_sum(a.x, -p, rh, re);
  const float r = __fadd_rn(rh, __fsub_rn(__fadd_rn(re, a.y), __fmaf_rn(q1, b.y, pe)));
  return df_fast(q1, __fdiv_rn(r, b.x));
}

// sqrt(a) in double-float, a >= 0: y = sqrt(a_h) (float32), then one Heron step
// y + (a - y^2) / (2 y) with the residual formed exactly (Karp & Markstein,
// "High-precision division and square root", ACM TOMS 23, 1997).
__device__ __forceinline__ float2 df_sqrt(float2 a) {
  if (!(a.x > 0.f)) return make_float2(0.f, 0.f);
  const float y = __fsqrt_rn(a.x);
  const float p = __fmul_rn(y, y);
  const float pe = __fmaf_rn(y, y, -p);                // y^2 = p + pe exactly
  const float e = __fadd_rn(__fsub_rn(__fsub_rn(a.x, p), pe), a.y);
  return df_fast(y, __fdiv_rn(e, __fmul_rn(2.f, y)));
}
