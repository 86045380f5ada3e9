// Double-word ("float-float") arithmetic for the extended-precision branch of
// the preprocess. A value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi) / 2, about 48 significant bits. GB300 runs FP32
// arithmetic at 64x its FP64 rate, so a double-word operation (2 to 20 FP32
// operations) is several times cheaper than the FP64 one it replaces, and the
// 48 bits are far more than the cancellations of the thin-Gaussian geometry
// consume.
//
// The building blocks are the error-free transformations 2Sum (Knuth),
// Fast2Sum (Dekker) and 2Prod (with FMA), and the double-word algorithms of
// Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic" (ACM TOMS 44(2), 2017):
// AccurateDWPlusDW (relative error <= 3u^2 + 13u^3), DWTimesDW3 (<= 4u^2) and
// DWTimesFP3 (<= 2u^2), u = 2^-24. Every FP32 operation is an explicit
// round-to-nearest intrinsic, so the compiler can neither contract nor
// reorder them: each kernel that evaluates the same expression gets the same
// bits.
#pragma once

#include <cuda_runtime.h>

namespace ug {

struct dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dd(float x) : hi(x), lo(0.f) {}
  __host__ __device__ constexpr dd(int x) : hi((float)x), lo(0.f) {}  // exact for |x| < 2^24
  // constants only: the split is evaluated by the compiler
  __host__ __device__ constexpr dd(double x)
      : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __device__ __forceinline__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float ap = __fsub_rn(s, b);
  const float bp = __fsub_rn(s, ap);
  const float da = __fsub_rn(a, ap);
  const float db = __fsub_rn(b, bp);
  return dd(s, __fadd_rn(da, db));
}

// requires |a| >= |b| (or a = 0)
__device__ __forceinline__ dd fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return dd(s, __fsub_rn(b, z));
}

__device__ __forceinline__ dd two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return dd(p, __fmaf_rn(a, b, -p));
}

// AccurateDWPlusDW
__device__ __forceinline__ dd dd_add(dd x, dd y) {
  const dd s = two_sum(x.hi, y.hi);
  const dd t = two_sum(x.lo, y.lo);
  const float c = __fadd_rn(s.lo, t.hi);
  const dd v = fast_two_sum(s.hi, c);
  const float w = __fadd_rn(t.lo, v.lo);
  return fast_two_sum(v.hi, w);
}

// SloppyDWPlusDW (Joldes, Muller and Popescu): 11 operations instead of 20.
// Its error is bounded relative to the operands, |err| <= 2u^2 (|x| + |y|)
// roughly, not to the result; that is all the geometry's sums need (their
// operands already carry errors of that size), and it is the bound of the
// accurate form's dot products as well.
__device__ __forceinline__ dd dd_add_sloppy(dd x, dd y) {
  const dd s = two_sum(x.hi, y.hi);
  const float v = __fadd_rn(x.lo, y.lo);
  const float w = __fadd_rn(s.lo, v);
  return fast_two_sum(s.hi, w);
}

// DWTimesDW3
__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  const dd c = two_prod(x.hi, y.hi);
  const float tl0 = __fmul_rn(x.lo, y.lo);
  const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  const float cl3 = __fadd_rn(c.lo, cl2);
  return fast_two_sum(c.hi, cl3);
}

// DWTimesFP3
__device__ __forceinline__ dd dd_mul(dd x, float y) {
  const dd c = two_prod(x.hi, y);
  const float cl3 = __fmaf_rn(x.lo, y, c.lo);
  return fast_two_sum(c.hi, cl3);
}

__device__ __forceinline__ dd operator-(dd x) { return dd(-x.hi, -x.lo); }
__device__ __forceinline__ dd operator+(dd x, dd y) { return dd_add(x, y); }
__device__ __forceinline__ dd operator-(dd x, dd y) { return dd_add(x, -y); }
__device__ __forceinline__ dd operator*(dd x, dd y) { return dd_mul(x, y); }

__device__ __forceinline__ bool operator<(dd a, dd b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool operator>(dd a, dd b) { return b < a; }
__device__ __forceinline__ bool operator<=(dd a, dd b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo);
}
__device__ __forceinline__ bool operator>=(dd a, dd b) { return b <= a; }

// Compensated three-term dot products (the scheme of Ogita, Rump and Oishi's
// Dot2, kept as a double word): the high parts' products by 2Prod and summed
// by 2Sum, every error term and every low-part product summed in FP32, one
// Fast2Sum at the end. |err| <= about 6u^2 sum |a_k b_k|, as for the chain of
// double-word FMAs it replaces, at a third of the operations.
__device__ __forceinline__ dd dd_dot3(const dd a[3], const float b[3]) {
  const dd p0 = two_prod(a[0].hi, b[0]), p1 = two_prod(a[1].hi, b[1]),
           p2 = two_prod(a[2].hi, b[2]);
  float e = __fmaf_rn(a[0].lo, b[0], p0.lo);
  e = __fmaf_rn(a[1].lo, b[1], __fadd_rn(e, p1.lo));
  e = __fmaf_rn(a[2].lo, b[2], __fadd_rn(e, p2.lo));
  const dd s = two_sum(p0.hi, p1.hi);
  const dd t = two_sum(s.hi, p2.hi);
  e = __fadd_rn(e, __fadd_rn(s.lo, t.lo));
  return fast_two_sum(t.hi, e);
}
__device__ __forceinline__ dd dd_dot3(const dd a[3], const dd b[3]) {
  const dd p0 = two_prod(a[0].hi, b[0].hi), p1 = two_prod(a[1].hi, b[1].hi),
           p2 = two_prod(a[2].hi, b[2].hi);
  float e = __fmaf_rn(a[0].hi, b[0].lo, __fmaf_rn(a[0].lo, b[0].hi, p0.lo));
  e = __fadd_rn(e, __fmaf_rn(a[1].hi, b[1].lo, __fmaf_rn(a[1].lo, b[1].hi, p1.lo)));
  e = __fadd_rn(e, __fmaf_rn(a[2].hi, b[2].lo, __fmaf_rn(a[2].lo, b[2].hi, p2.lo)));
  const dd s = two_sum(p0.hi, p1.hi);
  const dd t = two_sum(s.hi, p2.hi);
  e = __fadd_rn(e, __fadd_rn(s.lo, t.lo));
  return fast_two_sum(t.hi, e);
}

// The geometry's exact-rounding vocabulary for double words (sums by the
// sloppy addition; a double word times an FP32 number by DWTimesFP3).
__device__ __forceinline__ dd r_add(dd a, dd b) { return dd_add_sloppy(a, b); }
__device__ __forceinline__ dd r_sub(dd a, dd b) { return dd_add_sloppy(a, -b); }
__device__ __forceinline__ dd r_mul(dd a, dd b) { return dd_mul(a, b); }
__device__ __forceinline__ dd r_mul(dd a, float b) { return dd_mul(a, b); }
__device__ __forceinline__ dd r_fma(dd a, dd b, dd c) { return dd_add_sloppy(dd_mul(a, b), c); }
__device__ __forceinline__ dd r_fma(dd a, float b, dd c) { return dd_add_sloppy(dd_mul(a, b), c); }

// Division and square root of values that are already accurate run in FP32
// (see the FP32 and FP64 overloads beside the geometry).
__device__ __forceinline__ dd m_div(dd a, dd b) { return dd(__fdiv_rn((float)a, (float)b)); }
__device__ __forceinline__ dd m_sqrt(dd a) { return dd(__fsqrt_rn((float)a)); }

// 1/x and 1/sqrt(x) to double-word accuracy: an FP32 estimate r and one
// Newton step (the error of the estimate squares). The residual e, about
// 2^-23 in size, is formed from exact steps and needs only FP32 accuracy
// (its error is then about 2^-47), so r + r e comes out as a Fast2Sum.
//  1/x: 1 - x.hi r is exact in one FMA when r is the correctly rounded
//  reciprocal of x.hi (Markstein), then e = (1 - x.hi r) - x.lo r.
__device__ __forceinline__ dd dd_rcp(dd x) {
  const float r = __frcp_rn(x.hi);
  const float e = __fmaf_rn(-x.lo, r, __fmaf_rn(-x.hi, r, 1.f));
  return fast_two_sum(r, __fmul_rn(r, e));
}
//  1/sqrt(x): x r^2 = x.hi (t + t') + x.lo t with t + t' = r^2 exactly (2Prod)
//  and x.hi t = p + p' exactly; 1 - p is exact (Sterbenz: p is within a few
//  ulps of 1), so e = ((1 - p) - p') - (x.hi t' + x.lo t) and the result is
//  r + r e / 2.
__device__ __forceinline__ dd dd_rsqrt(dd x) {
  const float r = rsqrtf(x.hi);
  const dd t = two_prod(r, r);
  const dd p = two_prod(x.hi, t.hi);
  const float small = __fmaf_rn(x.hi, t.lo, __fmul_rn(x.lo, t.hi));
  const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.f, p.hi), p.lo), small);
  return fast_two_sum(r, __fmul_rn(__fmul_rn(0.5f, r), e));
}

__device__ __forceinline__ dd ceil(dd x) {
  const float c = ceilf(x.hi);
  return dd(c == x.hi && x.lo > 0.f ? __fadd_rn(c, 1.f) : c);
}
__device__ __forceinline__ dd floor(dd x) {
  const float f = floorf(x.hi);
  return dd(f == x.hi && x.lo < 0.f ? __fsub_rn(f, 1.f) : f);
}
__device__ __forceinline__ int dd_to_int(dd x) { return (int)x.hi; }  // integral values

}  // namespace ug
