// Per-Gaussian and per-(plane, Gaussian) geometry of the plane rasterizer.
//
// Everything that decides which pairs exist (the covariance factor, the
// extended-precision switch, the phase-1 test and the pixel box) is written
// with explicit round-to-nearest intrinsics, so the compiler cannot contract
// or reorder it: the counting pass and the emitting pass, compiled into
// different kernels, take bit-identical decisions.
#pragma once

#include "ug_dd.cuh"
#include "ug_internal.cuh"

namespace ug {

// ------------------------------------------------------------ exact-rounding ops
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float r_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float r_sqrt(float a) { return __fsqrt_rn(a); }

// Division and square root of values that are already accurate run in FP32
// in both branches (relative error 2^-24, far below the decision margins).
__device__ __forceinline__ float m_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float m_sqrt(float a) { return __fsqrt_rn(a); }

// Extended-precision reciprocal and reciprocal square root, by type.
__device__ __forceinline__ dd ext_rcp(dd x) { return dd_rcp(x); }
__device__ __forceinline__ dd ext_rsqrt(dd x) { return dd_rsqrt(x); }
__device__ __forceinline__ float ext_rcp(float x) { return r_div(1.f, x); }
__device__ __forceinline__ float ext_rsqrt(float x) { return r_div(1.f, r_sqrt(x)); }

__device__ __forceinline__ int to_int(float x) { return (int)x; }
__device__ __forceinline__ int to_int(dd x) { return dd_to_int(x); }

// Whether T is the extended-precision type of the thin-Gaussian branch.
template <typename T>
struct is_ext {
  static constexpr bool value = true;
};
template <>
struct is_ext<float> {
  static constexpr bool value = false;
};

template <typename T>
__device__ __forceinline__ T r_dot3(const T a[3], const T b[3]) {
  return r_fma(a[2], b[2], r_fma(a[1], b[1], r_mul(a[0], b[0])));
}
// double words: the compensated dot products (ug_dd.cuh)
__device__ __forceinline__ dd r_dot3(const dd a[3], const dd b[3]) { return dd_dot3(a, b); }
__device__ __forceinline__ dd r_dot3(const dd a[3], const float b[3]) { return dd_dot3(a, b); }
__device__ __forceinline__ dd r_dot3(const float b[3], const dd a[3]) { return dd_dot3(a, b); }

// Parameters of one Gaussian as loaded from the structure-of-arrays rows.
struct GaussParams {
  float mu[3];
  float cp[7];  // tri[6] or log_scale[3] + quat[4]
  float logit, c;
};

__device__ __forceinline__ void load_params(const ug_gaussians& g, int64_t n, int64_t i, int cov,
                                            GaussParams& p) {
#pragma unroll
  for (int k = 0; k < 3; ++k) p.mu[k] = __ldg(g.mean + k * n + i);
  if (cov == UG_COV_TRI) {
#pragma unroll
    for (int k = 0; k < 6; ++k) p.cp[k] = __ldg(g.tri + k * n + i);
    p.cp[6] = 0.f;
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) p.cp[k] = __ldg(g.log_scale + k * n + i);
#pragma unroll
    for (int k = 0; k < 4; ++k) p.cp[3 + k] = __ldg(g.quat + k * n + i);
  }
  p.logit = __ldg(g.opacity_logit + i);
  p.c = __ldg(g.intensity + i);
}

// Covariance factor of one Gaussian: Sigma^-1 = F F^T, Fi = F^-1.
// Triangular (Sec. 4.2, Eq. tri-param): F = L lower triangular with diagonal
// l_kk^2 + beta; Fi by forward substitution. Scale/rotation: F = R diag(1/s),
// Fi = diag(s) R^T with R from the normalised quaternion.
template <typename T>
struct Factor {
  T mu[3];
  T F[3][3];
  T Fi[3][3];
  T s[3];      // scales (scale/rotation only)
  T qn[4];     // normalised quaternion (scale/rotation only)
  T qnorm;
};

template <typename T, int COV>
__device__ __forceinline__ void make_factor(const GaussParams& p, float beta, Factor<T>& f) {
#pragma unroll
  for (int k = 0; k < 3; ++k) f.mu[k] = (T)p.mu[k];
  if (COV == UG_COV_TRI) {
    const T b = (T)beta;
    const T t0 = (T)p.cp[0], t1 = (T)p.cp[1], t2 = (T)p.cp[2];
    const T t3 = (T)p.cp[3], t4 = (T)p.cp[4], t5 = (T)p.cp[5];
    f.F[0][0] = r_fma(t0, t0, b);
    f.F[0][1] = (T)0;
    f.F[0][2] = (T)0;
    f.F[1][0] = t1;
    f.F[1][1] = r_fma(t3, t3, b);
    f.F[1][2] = (T)0;
    f.F[2][0] = t2;
    f.F[2][1] = t4;
    f.F[2][2] = r_fma(t5, t5, b);
    T i00, i11, i22;
    if constexpr (is_ext<T>::value) {
      i00 = ext_rcp(f.F[0][0]);
      i11 = ext_rcp(f.F[1][1]);
      i22 = ext_rcp(f.F[2][2]);
    } else {
      i00 = r_div((T)1, f.F[0][0]);
      i11 = r_div((T)1, f.F[1][1]);
      i22 = r_div((T)1, f.F[2][2]);
    }
    // L Fi = I column by column (forward substitution)
    const T i10 = -r_mul(r_mul(f.F[1][0], i00), i11);
    const T i21 = -r_mul(r_mul(f.F[2][1], i11), i22);
    const T i20 = -r_mul(r_fma(f.F[2][1], i10, r_mul(f.F[2][0], i00)), i22);
    f.Fi[0][0] = i00;
    f.Fi[0][1] = (T)0;
    f.Fi[0][2] = (T)0;
    f.Fi[1][0] = i10;
    f.Fi[1][1] = i11;
    f.Fi[1][2] = (T)0;
    f.Fi[2][0] = i20;
    f.Fi[2][1] = i21;
    f.Fi[2][2] = i22;
    f.s[0] = f.s[1] = f.s[2] = (T)0;
    f.qn[0] = f.qn[1] = f.qn[2] = f.qn[3] = (T)0;
    f.qnorm = (T)1;
  } else {
    const T q0 = (T)p.cp[3], q1 = (T)p.cp[4], q2 = (T)p.cp[5], q3 = (T)p.cp[6];
    const T nq2 = r_fma(q3, q3, r_fma(q2, q2, r_fma(q1, q1, r_mul(q0, q0))));
    T nq, w, x, y, z;
    if constexpr (is_ext<T>::value) {
      const T rq = ext_rsqrt(nq2);
      nq = nq2 * rq;
      w = q0 * rq;
      x = q1 * rq;
      y = q2 * rq;
      z = q3 * rq;
    } else {
      nq = r_sqrt(nq2);
      w = r_div(q0, nq);
      x = r_div(q1, nq);
      y = r_div(q2, nq);
      z = r_div(q3, nq);
    }
    f.qn[0] = w;
    f.qn[1] = x;
    f.qn[2] = y;
    f.qn[3] = z;
    f.qnorm = nq;
    T R[3][3];
    R[0][0] = (T)1 - (T)2 * r_fma(y, y, r_mul(z, z));
    R[0][1] = (T)2 * r_fma(x, y, -r_mul(w, z));
    R[0][2] = (T)2 * r_fma(x, z, r_mul(w, y));
    R[1][0] = (T)2 * r_fma(x, y, r_mul(w, z));
    R[1][1] = (T)1 - (T)2 * r_fma(x, x, r_mul(z, z));
    R[1][2] = (T)2 * r_fma(y, z, -r_mul(w, x));
    R[2][0] = (T)2 * r_fma(x, z, -r_mul(w, y));
    R[2][1] = (T)2 * r_fma(y, z, r_mul(w, x));
    R[2][2] = (T)1 - (T)2 * r_fma(x, x, r_mul(y, y));
    // the scales only rescale the rows of R (no cancellation follows), so FP32
    // exp and reciprocal are accurate enough for both branches
    T sinv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      f.s[a] = (T)expf(p.cp[a]);
      sinv[a] = (T)expf(-p.cp[a]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        f.F[k][a] = r_mul(R[k][a], sinv[a]);
        f.Fi[a][k] = r_mul(f.s[a], R[k][a]);
      }
  }
}

// Axis-ratio proxy: ||L||_F ||L^-1||_F (between the axis ratio and 3x it) for
// the triangular factor, max(s)/min(s) for scale/rotation.
template <int COV>
__device__ __forceinline__ float axis_ratio_proxy(const Factor<float>& f) {
  if (COV == UG_COV_TRI) {
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        a = r_fma(f.F[i][j], f.F[i][j], a);
        b = r_fma(f.Fi[i][j], f.Fi[i][j], b);
      }
    return r_sqrt(r_mul(a, b));
  } else {
    const float smax = fmaxf(f.s[0], fmaxf(f.s[1], f.s[2]));
    const float smin = fminf(f.s[0], fminf(f.s[1], f.s[2]));
    return r_div(smax, smin);
  }
}

// z = Fi r (Sigma3D_jk = z_j . z_k).
template <typename T, int COV, typename R>
__device__ __forceinline__ void apply_fi(const Factor<T>& f, const R r[3], T z[3]) {
  if (COV == UG_COV_TRI) {
    z[0] = r_mul(f.Fi[0][0], r[0]);
    z[1] = r_fma(f.Fi[1][1], r[1], r_mul(f.Fi[1][0], r[0]));
    z[2] = r_fma(f.Fi[2][2], r[2], r_fma(f.Fi[2][1], r[1], r_mul(f.Fi[2][0], r[0])));
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      z[a] = r_fma(f.Fi[a][2], r[2], r_fma(f.Fi[a][1], r[1], r_mul(f.Fi[a][0], r[0])));
  }
}

// b = F^T r (probe-frame precision P3D_jk = b_j . b_k).
template <typename T, int COV, typename R>
__device__ __forceinline__ void apply_ft(const Factor<T>& f, const R r[3], T b[3]) {
  if (COV == UG_COV_TRI) {
    b[0] = r_fma(f.F[2][0], r[2], r_fma(f.F[1][0], r[1], r_mul(f.F[0][0], r[0])));
    b[1] = r_fma(f.F[2][1], r[2], r_mul(f.F[1][1], r[1]));
    b[2] = r_mul(f.F[2][2], r[2]);
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      b[a] = r_fma(f.F[2][a], r[2], r_fma(f.F[1][a], r[1], r_mul(f.F[0][a], r[0])));
  }
}

// Plane axes: FP32 numbers as given (products with double words then take
// the cheaper double word x FP32 form).
struct Frame {
  float o[3], r[3][3];  // rows u, v, n
};

__device__ __forceinline__ void load_frame(const PlaneDev& pl, Frame& fr) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    fr.o[k] = pl.o[k];
    fr.r[0][k] = pl.u[k];
    fr.r[1][k] = pl.v[k];
    fr.r[2][k] = pl.n[k];
  }
}

// mu - o: exact as a double word (2Sum), rounded once in FP32.
__device__ __forceinline__ void mean_offset(const float mu[3], const float o[3], dd d[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = two_sum(mu[k], -o[k]);
}
__device__ __forceinline__ void mean_offset(const float mu[3], const float o[3], float d[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = __fsub_rn(mu[k], o[k]);
}

// Phase 1 and the pixel box of one (plane, Gaussian) pair.
struct PairBox {
  bool visible;
  int j0, j1, i0, i1;
};

template <typename T>
struct PairGeo {
  T d[3];     // mu - o (world)
  T m[3];     // probe-frame mean
  T z[3][3];  // Fi u, Fi v, Fi n
  T S11, S22, S33;
};

// Pixel range [ceil(lo), floor(hi)] of the closed interval in pixel units,
// clipped to [0, size - 1]; lo > hi or non-finite gives an empty range.
template <typename T>
__device__ __forceinline__ void pixel_range(T c, T h, T inv_pitch, T shift, int size, int& a,
                                            int& b) {
  const T lo = r_fma(r_sub(c, h), inv_pitch, shift);
  const T hi = r_fma(r_add(c, h), inv_pitch, shift);
  if (!(lo <= hi) || !(hi >= (T)0) || !(lo <= (T)(size - 1))) {
    a = 1;
    b = 0;
    return;
  }
  const T lo_c = lo < (T)0 ? (T)0 : lo;
  const T hi_c = hi > (T)(size - 1) ? (T)(size - 1) : hi;
  a = to_int(ceil(lo_c));
  b = to_int(floor(hi_c));
}

// Sec. 4.3-4.4: h_k = sqrt(chi2 Sigma3D_kk); reject unless m3 - h3 <= 0 <=
// m3 + h3; pixel j is inside iff m1 - h1 <= (j + 1/2 - W/2) pitch_u <= m1 + h1.
template <typename T, int COV>
__device__ __forceinline__ PairBox pair_box(const Factor<T>& f, const PlaneDev& pl, float chi2,
                                            PairGeo<T>& g) {
  PairBox pb;
  pb.visible = false;
  pb.j0 = 1;
  pb.j1 = 0;
  pb.i0 = 1;
  pb.i1 = 0;
  Frame fr;
  load_frame(pl, fr);
  T* d = g.d;
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = r_sub(f.mu[k], (T)fr.o[k]);
  g.m[2] = r_dot3(fr.r[2], d);
  apply_fi<T, COV>(f, fr.r[2], g.z[2]);
  g.S33 = r_dot3(g.z[2], g.z[2]);
  const T c2 = (T)chi2;
  const T h3 = m_sqrt(r_mul(c2, g.S33));
  if (!(r_sub(g.m[2], h3) <= (T)0 && r_add(g.m[2], h3) >= (T)0)) return pb;
  g.m[0] = r_dot3(fr.r[0], d);
  g.m[1] = r_dot3(fr.r[1], d);
  apply_fi<T, COV>(f, fr.r[0], g.z[0]);
  apply_fi<T, COV>(f, fr.r[1], g.z[1]);
  g.S11 = r_dot3(g.z[0], g.z[0]);
  g.S22 = r_dot3(g.z[1], g.z[1]);
  const T h1 = m_sqrt(r_mul(c2, g.S11));
  const T h2 = m_sqrt(r_mul(c2, g.S22));
  pixel_range<T>(g.m[0], h1, (T)pl.inv_pu, (T)pl.jshift, pl.w, pb.j0, pb.j1);
  pixel_range<T>(g.m[1], h2, (T)pl.inv_pv, (T)pl.ishift, pl.h, pb.i0, pb.i1);
  pb.visible = (pb.j0 <= pb.j1) && (pb.i0 <= pb.i1);
  return pb;
}

// The phase-1 test and pixel box of a pair in FP32 from any factor: the mean
// and the inverse factor rounded to FP32 (for a double-word factor, its
// inverse computed in double words, then rounded once). The decisions only
// need absolute accuracy (the oracle's ambiguity margins): the rounding of
// Fi r is a few ulps of |Fi| |r| whatever Fi's condition, and that of
// mu - o a few ulps of the scene's coordinates.
template <typename T, int COV>
__device__ __forceinline__ PairBox pair_box_f32(const Factor<T>& f, const PlaneDev& pl,
                                                float chi2) {
  if constexpr (!is_ext<T>::value) {
    PairGeo<float> g;
    return pair_box<float, COV>(f, pl, chi2, g);
  } else {
    Factor<float> ff;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ff.mu[k] = (float)f.mu[k];
#pragma unroll
      for (int j = 0; j < 3; ++j) ff.Fi[k][j] = (float)f.Fi[k][j];
    }
    PairGeo<float> g;
    return pair_box<float, COV>(ff, pl, chi2, g);
  }
}

// Render-side geometry of a visible pair in the plane's own coordinates. With
// X_w = o + x1 u + x2 v a point of the plane (x1, x2 in world units), the
// quadratic form of Eq. mahalanobis-3d is q = |F^T (X_w - mu)|^2 = |B x - c|^2,
// B = [F^T u, F^T v] (3 x 2), c = F^T (mu - o): a linear least-squares
// residual in x = (x1, x2). Gram-Schmidt B = [q1 q2] R (R upper triangular)
// gives
//   x* = R^-1 (q1.c, q2.c),  q = q0 + |R (x - x*)|^2,  q0 = (nh.c)^2,
// nh = q1 x q2. Unlike the conditional-Gaussian form through the probe frame,
// this uses u and v as given (the plane's FP32 axes are orthonormal only to
// about 1e-8, which thin Gaussians amplify beyond the output tolerance), so x*
// and q0 match the definition for any input pose.
template <typename T>
struct PairLsq {
  T X, Y;          // x* in pixel units (pixel (i, j) centred at (j + 1/2, i + 1/2))
  T kappa;         // r12 / r11 of the pixel-unit factor
  float r11, r22;  // pixel-unit factor of (log2 e / 2) D A D (see ug_internal.cuh)
  float rho3;      // nh.c: q0 = rho3^2
  float q1[3], q2[3], nh[3];  // orthonormal frame of the residual (backward chain)
  float ew[3];     // X_w(x*) - mu in world units (backward chain)
};

template <typename T>
__device__ __forceinline__ float to_f(T x) {
  return (float)x;
}

// x u + y v - d rounded to FP32. In double words the terms cancel to about
// the Gaussian's extent: the high parts' products by 2Prod and their sums by
// 2Sum, every error term and low part summed in FP32, one final rounding.
__device__ __forceinline__ float lin2_minus(float x, float y, float u, float v, float d) {
  return r_fma(x, u, r_fma(y, v, -d));
}
__device__ __forceinline__ float lin2_minus(dd x, dd y, float u, float v, dd d) {
  const dd p = two_prod(x.hi, u), q = two_prod(y.hi, v);
  const dd s = two_sum(p.hi, q.hi);
  const dd t = two_sum(s.hi, -d.hi);
  float e = __fmaf_rn(x.lo, u, p.lo);
  e = __fmaf_rn(y.lo, v, __fadd_rn(e, q.lo));
  e = __fadd_rn(e, __fsub_rn(__fadd_rn(s.lo, t.lo), d.lo));
  return __fadd_rn(t.hi, e);
}

template <typename T, int COV>
__device__ __forceinline__ void pair_lsq(const Factor<T>& f, const PlaneDev& pl,
                                         const PairGeo<T>& g, PairLsq<T>& o) {
  Frame fr;
  load_frame(pl, fr);
  T b1[3], b2[3], c[3];
  apply_ft<T, COV>(f, fr.r[0], b1);
  apply_ft<T, COV>(f, fr.r[1], b2);
  apply_ft<T, COV>(f, g.d, c);
  const T A11 = r_dot3(b1, b1);
  const T ir11 = ext_rsqrt(A11);
  const T r11 = r_mul(A11, ir11);
  T q1[3], q2[3], b2p[3], nh[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) q1[a] = r_mul(b1[a], ir11);
  const T r12 = r_dot3(q1, b2);
#pragma unroll
  for (int a = 0; a < 3; ++a) b2p[a] = r_fma(-r12, q1[a], b2[a]);
  const T A22 = r_dot3(b2p, b2p);
  const T ir22 = ext_rsqrt(A22);
  const T r22 = r_mul(A22, ir22);
#pragma unroll
  for (int a = 0; a < 3; ++a) q2[a] = r_mul(b2p[a], ir22);
  const T y = r_mul(r_dot3(q2, c), ir22);               // x2*
  const T x = r_mul(r_fma(-r12, y, r_dot3(q1, c)), ir11);  // x1*
  nh[0] = r_fma(q1[1], q2[2], -r_mul(q1[2], q2[1]));
  nh[1] = r_fma(q1[2], q2[0], -r_mul(q1[0], q2[2]));
  nh[2] = r_fma(q1[0], q2[1], -r_mul(q1[1], q2[0]));
  const T rho3 = r_dot3(nh, c);
  const T ipu = ext_rcp((T)pl.pu), ipv = ext_rcp((T)pl.pv);
  o.X = r_fma(x, ipu, (T)pl.half_w);
  o.Y = r_fma(y, ipv, (T)pl.half_h);
  // kappa = (r12 pv) / (r11 pu)
  o.kappa = r_mul(r_mul(r_mul(r12, ir11), pl.pv), ipu);
  const float sc = 0.84932180028801904272f;  // sqrt(log2(e) / 2)
  o.r11 = __fmul_rn(__fmul_rn(sc, pl.pu), to_f(r11));
  o.r22 = __fmul_rn(__fmul_rn(sc, pl.pv), to_f(r22));
  o.rho3 = to_f(rho3);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    o.q1[a] = to_f(q1[a]);
    o.q2[a] = to_f(q2[a]);
    o.nh[a] = to_f(nh[a]);
    // X_w(x*) - mu = x1* u + x2* v - (mu - o): the terms cancel to about the
    // Gaussian's extent, so this stays in T
    o.ew[a] = lin2_minus(x, y, fr.r[0][a], fr.r[1][a], g.d[a]);
  }
}

constexpr float kHalfLog2e = 0.72134752044448170368f;  // log2(e) / 2
constexpr float kLn2 = 0.69314718055994530942f;
constexpr float kLog2e = 1.44269504088896340736f;

// log2(sigmoid(x)) = -log2(1 + e^-x), computed without overflow.
__device__ __forceinline__ float log2_sigmoid(float x) {
  return x >= 0.f ? -log1pf(expf(-x)) * kLog2e : (x - log1pf(expf(x))) * kLog2e;
}

__device__ __forceinline__ float sigmoidf(float x) {
  return x >= 0.f ? 1.f / (1.f + expf(-x)) : expf(x) / (1.f + expf(x));
}

}  // namespace ug
