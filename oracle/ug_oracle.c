/*
 * FP64 CPU oracle of the UltraGauss ultrasound plane rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY: tests, the package's smoke check and the bench's
 * CPU-baseline leg may call this code; the product path never does.
 *
 * It is the plain definition, with no tiling and no sorting:
 *
 *   covariance   Sigma^-1 = L L^T, L lower triangular with diagonal
 *                l_kk^2 + beta (Sec. 4.2, Eq. tri-param), or
 *                Sigma = R diag(s^2) R^T from a normalised quaternion and
 *                s = exp(log_scale) (Sec. 4.2, the Kerbl et al. form);
 *   opacity      alpha_i = sigmoid(logit_i) (Sec. 4.5);
 *   probe frame  mu3D = W mu (rows u, v, n = u x v, origin o), Sigma3D =
 *                W Sigma W^T (Sec. 4.1, Eq. mahalanobis-3d and the line after);
 *   cut-off      half-extents of the p% ellipsoid (Sec. 4.3, Eq. ellipsoid
 *                and Eq. boundary): the box is the ellipsoid's axis-aligned
 *                bound in the probe frame, h_k = the largest probe coordinate
 *                r_k . (X - mu) over {(X - mu)^T Sigma^-1 (X - mu) <= chi2},
 *                i.e. h_k = sqrt(chi2 * r_k^T Sigma r_k) for the frame rows
 *                r_k = u, v, n. For an orthonormal frame this is the printed
 *                cofactor/determinant formula applied to the matrix of the
 *                quadratic form, P3D = (Sigma3D)^-1: sqrt(chi2 * cof_kk(P3D) /
 *                det(P3D)). The inputs' frames are FP32 (orthonormal to about
 *                1e-7), and the cofactor form of W Sigma^-1 W^T then differs
 *                from the ellipsoid's bound by up to (s_max / s_min)^2 * 1e-7
 *                (per cent at axis ratios of 1e4), so the oracle evaluates the
 *                bound itself: r_k^T Sigma r_k = |L^-1 r_k|^2 by forward
 *                substitution (triangular form) or sum_a s_a^2 (R_a . r_k)^2
 *                (scale and rotation), sums of squares without cancellation;
 *   phase 1      a Gaussian is rejected on a plane iff m3 - h3 > 0 or
 *                m3 + h3 < 0 (Sec. 4.4 load balancing, item 1);
 *   phase 2      pixel x is inside iff m1 - h1 <= x1 <= m1 + h1 and
 *                m2 - h2 <= x2 <= m2 + h2 (item 2); in the optional
 *                ellipsoid mode additionally q <= chi2;
 *   weight       w = alpha * exp(-q/2), q = (X - mu)^T Sigma^-1 (X - mu) with
 *                X = o + x1 u + x2 v the lifted pixel (Eq. mahalanobis-3d,
 *                evaluated in the world frame, which is the same number);
 *   image        C = (sum w c + a_bg c_bg) / (sum w + a_bg)
 *                (Eq. alpha-combine, Eq. colour-combine, Eq. us-render).
 *
 * Pixel (i, j) of a W x H plane has its centre at
 *   x1 = (j + 1/2 - W/2) * pitch_u,  x2 = (i + 1/2 - H/2) * pitch_v.
 *
 * The gradient is the analytic FP64 chain rule of the same formulas, with the
 * cut-off treated as a constant mask (as in all splatting rasterizers).
 *
 * Every inclusion decision whose margin is within amb * pitch + amb_abs
 * (in-plane), amb * h3 + amb_abs (plane test) or amb * chi2 (ellipsoid test)
 * is reported as ambiguous: an FP32 implementation may take either side of
 * it. amb_abs (world units) covers the FP32 rounding of the probe-frame mean
 * and half-extents, a few ulps of the scene's coordinates.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double chi2, beta, alpha_bg, c_bg, amb, amb_abs;
  int32_t cutoff;    /* 0: box (paper), 1: box and ellipsoid */
  int32_t cov_param; /* 0: triangular, 1: scale + quaternion */
} or_config;

/* Plane in FP64: origin, u, v, pitch_u, pitch_v (11 doubles); sizes are
 * width, height, pixel_offset (3 int64). */
typedef struct {
  double o[3], u[3], v[3], n[3], pu, pv;
  int64_t w, h, off;
} or_plane;

static void load_plane(const double* pl, const int64_t* sz, or_plane* p) {
  for (int k = 0; k < 3; ++k) {
    p->o[k] = pl[k];
    p->u[k] = pl[3 + k];
    p->v[k] = pl[6 + k];
  }
  p->n[0] = p->u[1] * p->v[2] - p->u[2] * p->v[1];
  p->n[1] = p->u[2] * p->v[0] - p->u[0] * p->v[2];
  p->n[2] = p->u[0] * p->v[1] - p->u[1] * p->v[0];
  p->pu = pl[9];
  p->pv = pl[10];
  p->w = sz[0];
  p->h = sz[1];
  p->off = sz[2];
}

/* Rotation matrix of the normalised quaternion (w, x, y, z). */
static void quat_rotation(const double* q4, double R[3][3], double* qn_out, double* norm_out) {
  double nrm = sqrt(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
  double w = q4[0] / nrm, x = q4[1] / nrm, y = q4[2] / nrm, z = q4[3] / nrm;
  R[0][0] = 1 - 2 * (y * y + z * z);
  R[0][1] = 2 * (x * y - w * z);
  R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);
  R[1][1] = 1 - 2 * (x * x + z * z);
  R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);
  R[2][1] = 2 * (y * z + w * x);
  R[2][2] = 1 - 2 * (x * x + y * y);
  if (qn_out) {
    qn_out[0] = w;
    qn_out[1] = x;
    qn_out[2] = y;
    qn_out[3] = z;
  }
  if (norm_out) *norm_out = nrm;
}

/* Lower-triangular factor L of Eq. tri-param from its six parameters
 * (l11, l21, l31, l22, l32, l33); the third-row middle entry is an independent
 * parameter (the printed L_12 there is read as L_32). */
static void tri_factor(const double* t, double beta, double L[3][3]) {
  memset(L, 0, sizeof(double) * 9);
  L[0][0] = t[0] * t[0] + beta;
  L[1][0] = t[1];
  L[2][0] = t[2];
  L[1][1] = t[3] * t[3] + beta;
  L[2][1] = t[4];
  L[2][2] = t[5] * t[5] + beta;
}

/* World-frame precision Sigma^-1 of one Gaussian. covp holds 6 (triangular)
 * or 7 (log_scale[3], quat[4]) parameters. */
static void precision(const double* covp, int cov_param, double beta, double Pi[3][3]) {
  if (cov_param == 0) {
    double L[3][3];
    tri_factor(covp, beta, L);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += L[i][k] * L[j][k];
        Pi[i][j] = s;
      }
  } else {
    double R[3][3];
    quat_rotation(covp + 3, R, NULL, NULL);
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = exp(-2.0 * covp[a]);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0;
        for (int a = 0; a < 3; ++a) s += R[i][a] * d[a] * R[j][a];
        Pi[i][j] = s;
      }
  }
}

/* r^T Sigma r of one Gaussian (Sigma = (L L^T)^-1 or R diag(s^2) R^T) for a
 * direction r, as a sum of squares: |y|^2 with L y = r by forward
 * substitution, or sum_a s_a^2 (R_a . r)^2 with R_a the a-th principal axis. */
static double sigma_quad(const double* covp, int cov_param, double beta, const double r[3]) {
  if (cov_param == 0) {
    double L[3][3];
    tri_factor(covp, beta, L);
    const double y0 = r[0] / L[0][0];
    const double y1 = (r[1] - L[1][0] * y0) / L[1][1];
    const double y2 = (r[2] - L[2][0] * y0 - L[2][1] * y1) / L[2][2];
    return y0 * y0 + y1 * y1 + y2 * y2;
  }
  double R[3][3];
  quat_rotation(covp + 3, R, NULL, NULL);
  double s = 0;
  for (int a = 0; a < 3; ++a) {
    const double p = R[0][a] * r[0] + R[1][a] * r[1] + R[2][a] * r[2];
    s += exp(2.0 * covp[a]) * p * p;
  }
  return s;
}

/* Cofactor matrix and determinant of a 3x3 matrix. */
static double cofactors(const double A[3][3], double C[3][3]) {
  C[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  C[0][1] = -(A[1][0] * A[2][2] - A[1][2] * A[2][0]);
  C[0][2] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  C[1][0] = -(A[0][1] * A[2][2] - A[0][2] * A[2][1]);
  C[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
  C[1][2] = -(A[0][0] * A[2][1] - A[0][1] * A[2][0]);
  C[2][0] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
  C[2][1] = -(A[0][0] * A[1][2] - A[0][2] * A[1][0]);
  C[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
  return A[0][0] * C[0][0] + A[0][1] * C[0][1] + A[0][2] * C[0][2];
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* Per-(plane, Gaussian) quantities of the definition. */
typedef struct {
  double mu[3];   /* world mean */
  double Pi[3][3];/* world precision */
  double m[3];    /* probe-frame mean */
  double h[3];    /* half-extents of the axis-aligned box in the probe frame */
  double alpha, c;
  int visible;    /* phase-1 accepted */
  int amb_plane;  /* phase-1 decision within the ambiguity margin */
} or_pg;

static void pg_compute(const or_plane* pl, const double* mean, const double* covp,
                       double logit, double intensity, const or_config* cfg, or_pg* g) {
  for (int k = 0; k < 3; ++k) g->mu[k] = mean[k];
  precision(covp, cfg->cov_param, cfg->beta, g->Pi);
  g->alpha = sigmoid(logit);
  g->c = intensity;
  const double* rows[3] = {pl->u, pl->v, pl->n};
  double d[3] = {mean[0] - pl->o[0], mean[1] - pl->o[1], mean[2] - pl->o[2]};
  for (int j = 0; j < 3; ++j) g->m[j] = rows[j][0] * d[0] + rows[j][1] * d[1] + rows[j][2] * d[2];
  /* the ellipsoid's bound along each frame row: sqrt(chi2 r_k^T Sigma r_k) */
  for (int k = 0; k < 3; ++k) g->h[k] = sqrt(cfg->chi2 * sigma_quad(covp, cfg->cov_param, cfg->beta, rows[k]));
  /* phase 1: reject iff b3min > 0 or b3max < 0 */
  double bmin = g->m[2] - g->h[2], bmax = g->m[2] + g->h[2];
  g->visible = !(bmin > 0.0 || bmax < 0.0);
  double margin = g->h[2] - fabs(g->m[2]);
  g->amb_plane = fabs(margin) <= cfg->amb * g->h[2] + cfg->amb_abs;
}

static inline double px_x1(const or_plane* p, int64_t j) { return ((double)j + 0.5 - 0.5 * (double)p->w) * p->pu; }
static inline double px_x2(const or_plane* p, int64_t i) { return ((double)i + 0.5 - 0.5 * (double)p->h) * p->pv; }

/* q at pixel (x1, x2) in the world frame. */
static double pair_q(const or_plane* p, const or_pg* g, double x1, double x2, double dl[3]) {
  for (int k = 0; k < 3; ++k) dl[k] = p->o[k] + x1 * p->u[k] + x2 * p->v[k] - g->mu[k];
  double q = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) q += dl[a] * g->Pi[a][b] * dl[b];
  return q;
}

/* Inclusion test of one pair. Returns 1 if included; *amb set if any decision
 * was within the margin. */
static int pair_included(const or_plane* p, const or_pg* g, const or_config* cfg, double x1,
                         double x2, double q, int* amb) {
  *amb = 0;
  const double t1 = cfg->amb * p->pu + cfg->amb_abs, t2 = cfg->amb * p->pv + cfg->amb_abs;
  if (!g->visible) {
    *amb = g->amb_plane && (fabs(x1 - g->m[0]) <= g->h[0] * (1 + cfg->amb) + t1) &&
           (fabs(x2 - g->m[1]) <= g->h[1] * (1 + cfg->amb) + t2);
    return 0;
  }
  double e1 = g->h[0] - fabs(x1 - g->m[0]);
  double e2 = g->h[1] - fabs(x2 - g->m[1]);
  int in = (g->m[0] - g->h[0] <= x1) && (x1 <= g->m[0] + g->h[0]) && (g->m[1] - g->h[1] <= x2) &&
           (x2 <= g->m[1] + g->h[1]);
  int near1 = fabs(e1) <= t1, near2 = fabs(e2) <= t2;
  /* a decision can only flip if the other axis is inside or also near */
  if ((near1 && (e2 >= 0 || near2)) || (near2 && (e1 >= 0 || near1))) *amb = 1;
  if (in && g->amb_plane) *amb = 1;
  if (cfg->cutoff == 1) {
    if (in && fabs(q - cfg->chi2) <= cfg->amb * cfg->chi2) *amb = 1;
    in = in && (q <= cfg->chi2);
  }
  return in;
}

static const double* gauss_mean(const double* mean, int64_t i) { return mean + 3 * i; }
static int ncovp(int cov_param) { return cov_param == 0 ? 6 : 7; }

/* ------------------------------------------------------------------ render
 * mode 0: dense, every pixel tests every Gaussian.
 * mode 1: scatter, each Gaussian visits only its box (one pixel of slack on
 *         each side) with the same per-pixel test; the per-pixel sums are
 *         accumulated in the same Gaussian order, so both modes give the same
 *         bits.
 * Outputs per pixel (total_px): image C, alpha = sum w + a_bg, sa = sum w,
 * sc = sum w c, amb = sum of w over ambiguous pairs (included or not).
 * Returns the number of included pairs. */
int64_t or_render(int64_t n, const double* mean, const double* covp, const double* logit,
                  const double* intensity, int32_t P, const double* planes, const int64_t* sizes,
                  const or_config* cfg, int32_t mode, double* image, double* alpha, double* sa,
                  double* sc, double* amb, int32_t nthreads) {
  int64_t pairs = 0;
  const int nc = ncovp(cfg->cov_param);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  or_pg* gs = (or_pg*)malloc(sizeof(or_pg) * (size_t)(n > 0 ? n : 1));
  for (int32_t pi = 0; pi < P; ++pi) {
    or_plane pl;
    load_plane(planes + 11 * pi, sizes + 3 * pi, &pl);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g)
      pg_compute(&pl, gauss_mean(mean, g), covp + nc * g, logit[g], intensity[g], cfg, &gs[g]);
    const int64_t W = pl.w, H = pl.h;
    if (mode == 0) {
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : pairs)
      for (int64_t pix = 0; pix < W * H; ++pix) {
        int64_t i = pix / W, j = pix % W;
        double x1 = px_x1(&pl, j), x2 = px_x2(&pl, i);
        double s_a = 0, s_c = 0, s_amb = 0;
        for (int64_t g = 0; g < n; ++g) {
          double dl[3];
          double q = pair_q(&pl, &gs[g], x1, x2, dl);
          int am;
          int in = pair_included(&pl, &gs[g], cfg, x1, x2, q, &am);
          double w = gs[g].alpha * exp(-0.5 * q);
          if (in) {
            s_a += w;
            s_c += w * gs[g].c;
            pairs++;
          }
          if (am) s_amb += w;
        }
        int64_t o = pl.off + pix;
        sa[o] = s_a;
        sc[o] = s_c;
        amb[o] = s_amb;
        alpha[o] = s_a + cfg->alpha_bg;
        image[o] = (s_c + cfg->alpha_bg * cfg->c_bg) / alpha[o];
      }
    } else {
      const int64_t band = 4;
      const int64_t nb = (H + band - 1) / band;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : pairs)
      for (int64_t b = 0; b < nb; ++b) {
        int64_t r0 = b * band, r1 = r0 + band < H ? r0 + band : H;
        for (int64_t pix = r0 * W; pix < r1 * W; ++pix) {
          sa[pl.off + pix] = 0;
          sc[pl.off + pix] = 0;
          amb[pl.off + pix] = 0;
        }
        for (int64_t g = 0; g < n; ++g) {
          const or_pg* G = &gs[g];
          if (!G->visible && !G->amb_plane) continue;
          double hx = G->h[0] * (1 + 2 * cfg->amb) + 2 * cfg->amb_abs;
          double hy = G->h[1] * (1 + 2 * cfg->amb) + 2 * cfg->amb_abs;
          double jlo = (G->m[0] - hx) / pl.pu + 0.5 * W - 0.5;
          double jhi = (G->m[0] + hx) / pl.pu + 0.5 * W - 0.5;
          double ilo = (G->m[1] - hy) / pl.pv + 0.5 * H - 0.5;
          double ihi = (G->m[1] + hy) / pl.pv + 0.5 * H - 0.5;
          if (!(jhi >= -1.0) || !(jlo <= (double)W) || !(ihi >= -1.0) || !(ilo <= (double)H)) continue;
          int64_t j0 = (int64_t)floor(jlo) - 1, j1 = (int64_t)ceil(jhi) + 1;
          int64_t i0 = (int64_t)floor(ilo) - 1, i1 = (int64_t)ceil(ihi) + 1;
          if (j0 < 0) j0 = 0;
          if (j1 > W - 1) j1 = W - 1;
          if (i0 < r0) i0 = r0;
          if (i1 > r1 - 1) i1 = r1 - 1;
          for (int64_t i = i0; i <= i1; ++i) {
            double x2 = px_x2(&pl, i);
            for (int64_t j = j0; j <= j1; ++j) {
              double x1 = px_x1(&pl, j);
              double dl[3];
              double q = pair_q(&pl, G, x1, x2, dl);
              int am;
              int in = pair_included(&pl, G, cfg, x1, x2, q, &am);
              double w = G->alpha * exp(-0.5 * q);
              int64_t o = pl.off + i * W + j;
              if (in) {
                sa[o] += w;
                sc[o] += w * G->c;
                pairs++;
              }
              if (am) amb[o] += w;
            }
          }
        }
        for (int64_t pix = r0 * W; pix < r1 * W; ++pix) {
          int64_t o = pl.off + pix;
          alpha[o] = sa[o] + cfg->alpha_bg;
          image[o] = (sc[o] + cfg->alpha_bg * cfg->c_bg) / alpha[o];
        }
      }
    }
  }
  free(gs);
  return pairs;
}

/* ------------------------------------------------------------- geometry
 * Per (plane, Gaussian): visible flag, ambiguity flag, probe-frame mean m,
 * half-extents h, and the exact pixel box [j0, j1] x [i0, i1] (first and last
 * column/row whose centre passes the in-plane test, clipped to the image;
 * j0 > j1 when empty). Arrays are indexed [plane * n + g]. */
void or_geometry(int64_t n, const double* mean, const double* covp, const double* logit,
                 const double* intensity, int32_t P, const double* planes, const int64_t* sizes,
                 const or_config* cfg, int32_t* visible, int32_t* amb_plane, double* m, double* h,
                 int64_t* box) {
  const int nc = ncovp(cfg->cov_param);
  for (int32_t pi = 0; pi < P; ++pi) {
    or_plane pl;
    load_plane(planes + 11 * pi, sizes + 3 * pi, &pl);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g) {
      or_pg G;
      pg_compute(&pl, gauss_mean(mean, g), covp + nc * g, logit[g], intensity[g], cfg, &G);
      int64_t k = (int64_t)pi * n + g;
      visible[k] = G.visible;
      amb_plane[k] = G.amb_plane;
      for (int a = 0; a < 3; ++a) {
        m[3 * k + a] = G.m[a];
        h[3 * k + a] = G.h[a];
      }
      /* first/last pixel centre inside the closed interval */
      int64_t j0 = pl.w, j1 = -1, i0 = pl.h, i1 = -1;
      for (int64_t j = 0; j < pl.w; ++j) {
        double x1 = px_x1(&pl, j);
        if (G.m[0] - G.h[0] <= x1 && x1 <= G.m[0] + G.h[0]) {
          if (j < j0) j0 = j;
          j1 = j;
        }
      }
      for (int64_t i = 0; i < pl.h; ++i) {
        double x2 = px_x2(&pl, i);
        if (G.m[1] - G.h[1] <= x2 && x2 <= G.m[1] + G.h[1]) {
          if (i < i0) i0 = i;
          i1 = i;
        }
      }
      box[4 * k + 0] = j0;
      box[4 * k + 1] = j1;
      box[4 * k + 2] = i0;
      box[4 * k + 3] = i1;
    }
  }
}

/* ------------------------------------------------------------- gradient
 * Analytic FP64 gradient of a scalar loss L given dL/dC per pixel
 * (grad_image), the rendered image C and alpha = sum w + a_bg. For each
 * Gaussian in `subset` (or all Gaussians if subset is NULL) it writes
 * nparam = 3 + ncovp + 2 values: dL/dmean[3], dL/dcovp[6|7], dL/dlogit,
 * dL/dintensity, and in grad_abs the same chain applied to absolute values of
 * every per-pair term (a scale for the rounding error of a sum that cancels).
 */
static void chain_covp(const double* covp, const or_config* cfg, double gPi[3][3], double* out) {
  if (cfg->cov_param == 0) {
    double L[3][3];
    tri_factor(covp, cfg->beta, L);
    /* dL/dL = (G + G^T) L = 2 G L for symmetric G */
    double gL[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += (gPi[i][k] + gPi[k][i]) * L[k][j];
        gL[i][j] = s;
      }
    out[0] = gL[0][0] * 2 * covp[0];
    out[1] = gL[1][0];
    out[2] = gL[2][0];
    out[3] = gL[1][1] * 2 * covp[3];
    out[4] = gL[2][1];
    out[5] = gL[2][2] * 2 * covp[5];
  } else {
    double R[3][3], qn[4], qnorm;
    quat_rotation(covp + 3, R, qn, &qnorm);
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = exp(-2.0 * covp[a]);
    /* Pi = R diag(d) R^T */
    for (int a = 0; a < 3; ++a) {
      double s = 0;
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) s += R[i][a] * gPi[i][k] * R[k][a];
      out[a] = s * (-2.0 * d[a]);
    }
    double gR[3][3];
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += (gPi[i][k] + gPi[k][i]) * R[k][a];
        gR[i][a] = s * d[a];
      }
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    double gw = 2 * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] +
                     x * gR[2][1]);
    double gx = 2 * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2 * x * gR[1][1] - w * gR[1][2] +
                     z * gR[2][0] + w * gR[2][1] - 2 * x * gR[2][2]);
    double gy = 2 * (-2 * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] -
                     w * gR[2][0] + z * gR[2][1] - 2 * y * gR[2][2]);
    double gz = 2 * (-2 * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] -
                     2 * z * gR[1][1] + y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
    double gq[4] = {gw, gx, gy, gz};
    double dot = gq[0] * qn[0] + gq[1] * qn[1] + gq[2] * qn[2] + gq[3] * qn[3];
    for (int k = 0; k < 4; ++k) out[3 + k] = (gq[k] - qn[k] * dot) / qnorm;
  }
}

/* Same linear chain with every coefficient replaced by its absolute value. */
static void chain_covp_abs(const double* covp, const or_config* cfg, double aPi[3][3], double* out) {
  if (cfg->cov_param == 0) {
    double L[3][3];
    tri_factor(covp, cfg->beta, L);
    double gL[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += (aPi[i][k] + aPi[k][i]) * fabs(L[k][j]);
        gL[i][j] = s;
      }
    out[0] = gL[0][0] * 2 * fabs(covp[0]);
    out[1] = gL[1][0];
    out[2] = gL[2][0];
    out[3] = gL[1][1] * 2 * fabs(covp[3]);
    out[4] = gL[2][1];
    out[5] = gL[2][2] * 2 * fabs(covp[5]);
  } else {
    double R[3][3], qn[4], qnorm;
    quat_rotation(covp + 3, R, qn, &qnorm);
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = exp(-2.0 * covp[a]);
    for (int a = 0; a < 3; ++a) {
      double s = 0;
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) s += fabs(R[i][a]) * aPi[i][k] * fabs(R[k][a]);
      out[a] = s * 2.0 * d[a];
    }
    double gR[3][3];
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += (aPi[i][k] + aPi[k][i]) * fabs(R[k][a]);
        gR[i][a] = s * d[a];
      }
    double sum = 0;
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) sum += gR[i][a];
    /* every rotation entry has partials of magnitude <= 4 in each unit-quaternion component */
    for (int k = 0; k < 4; ++k) out[3 + k] = 8.0 * sum / qnorm;
  }
}

void or_render_grad(int64_t n, const double* mean, const double* covp, const double* logit,
                    const double* intensity, int32_t P, const double* planes, const int64_t* sizes,
                    const or_config* cfg, const double* image, const double* alpha,
                    const double* grad_image, const int64_t* subset, int64_t nsub, double* grads,
                    double* grads_abs, double* grads_abs_pre, int32_t* amb_gauss,
                    int32_t nthreads) {
  const int nc = ncovp(cfg->cov_param);
  const int np = 3 + nc + 2;
  const int64_t count = subset ? nsub : n;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t s = 0; s < count; ++s) {
    int64_t g = subset ? subset[s] : s;
    double gmu[3] = {0, 0, 0}, amu[3] = {0, 0, 0}, pmu[3] = {0, 0, 0};
    double gPi[3][3] = {{0}}, aPi[3][3] = {{0}}, pPi[3][3] = {{0}};
    double glogit = 0, alogit = 0, plogit = 0, gc = 0, ac = 0;
    int any_amb = 0;
    for (int32_t pi = 0; pi < P; ++pi) {
      or_plane pl;
      load_plane(planes + 11 * pi, sizes + 3 * pi, &pl);
      or_pg G;
      pg_compute(&pl, gauss_mean(mean, g), covp + nc * g, logit[g], intensity[g], cfg, &G);
      if (G.amb_plane) any_amb = 1;
      if (!G.visible) continue;
      const int64_t W = pl.w, H = pl.h;
      double hx = G.h[0] * (1 + 2 * cfg->amb) + 2 * cfg->amb_abs;
      double hy = G.h[1] * (1 + 2 * cfg->amb) + 2 * cfg->amb_abs;
      double jlo = (G.m[0] - hx) / pl.pu + 0.5 * W - 0.5;
      double jhi = (G.m[0] + hx) / pl.pu + 0.5 * W - 0.5;
      double ilo = (G.m[1] - hy) / pl.pv + 0.5 * H - 0.5;
      double ihi = (G.m[1] + hy) / pl.pv + 0.5 * H - 0.5;
      if (!(jhi >= -1.0) || !(jlo <= (double)W) || !(ihi >= -1.0) || !(ilo <= (double)H)) continue;
      int64_t j0 = (int64_t)floor(jlo) - 1, j1 = (int64_t)ceil(jhi) + 1;
      int64_t i0 = (int64_t)floor(ilo) - 1, i1 = (int64_t)ceil(ihi) + 1;
      if (j0 < 0) j0 = 0;
      if (j1 > W - 1) j1 = W - 1;
      if (i0 < 0) i0 = 0;
      if (i1 > H - 1) i1 = H - 1;
      for (int64_t i = i0; i <= i1; ++i) {
        double x2 = px_x2(&pl, i);
        for (int64_t j = j0; j <= j1; ++j) {
          double x1 = px_x1(&pl, j);
          double dl[3];
          double q = pair_q(&pl, &G, x1, x2, dl);
          int am;
          int inc = pair_included(&pl, &G, cfg, x1, x2, q, &am);
          if (am) any_amb = 1;
          if (!inc) continue;
          int64_t o = pl.off + i * W + j;
          double w = G.alpha * exp(-0.5 * q);
          double Gp = grad_image[o], A = alpha[o], C = image[o];
          double dLdw = Gp * (G.c - C) / A;
          /* |dL/dw| before the cancellation in c - C */
          double pdLdw = fabs(Gp / A) * (fabs(G.c) + fabs(C));
          gc += Gp * w / A;
          ac += fabs(Gp * w / A);
          double dLdq = -0.5 * w * dLdw, pdLdq = 0.5 * w * pdLdw;
          double Pd[3];
          for (int a = 0; a < 3; ++a) Pd[a] = G.Pi[a][0] * dl[0] + G.Pi[a][1] * dl[1] + G.Pi[a][2] * dl[2];
          for (int a = 0; a < 3; ++a) {
            gmu[a] += dLdq * (-2.0 * Pd[a]);
            amu[a] += fabs(dLdq * 2.0 * Pd[a]);
            pmu[a] += pdLdq * fabs(2.0 * Pd[a]);
            for (int b = 0; b < 3; ++b) {
              gPi[a][b] += dLdq * dl[a] * dl[b];
              aPi[a][b] += fabs(dLdq * dl[a] * dl[b]);
              pPi[a][b] += pdLdq * fabs(dl[a] * dl[b]);
            }
          }
          glogit += dLdw * w * (1.0 - G.alpha);
          alogit += fabs(dLdw * w * (1.0 - G.alpha));
          plogit += pdLdw * w * (1.0 - G.alpha);
        }
      }
    }
    double* out = grads + np * s;
    double* aout = grads_abs + np * s;
    for (int a = 0; a < 3; ++a) {
      out[a] = gmu[a];
      aout[a] = amu[a];
    }
    chain_covp(covp + nc * g, cfg, gPi, out + 3);
    chain_covp_abs(covp + nc * g, cfg, aPi, aout + 3);
    out[3 + nc] = glogit;
    aout[3 + nc] = alogit;
    out[4 + nc] = gc;
    aout[4 + nc] = ac;
    if (grads_abs_pre) {
      double* pout = grads_abs_pre + np * s;
      for (int a = 0; a < 3; ++a) pout[a] = pmu[a];
      chain_covp_abs(covp + nc * g, cfg, pPi, pout + 3);
      pout[3 + nc] = plogit;
      pout[4 + nc] = ac; /* dL/dc = sum G w / alpha has no c - C */
    }
    if (amb_gauss) amb_gauss[s] = any_amb;
  }
}

/* ------------------------------------------------------------- contributions
 * Included pairs of ONE Gaussian (its parameters passed directly) on all
 * planes: writes up to cap (pixel index, w) pairs and returns the count (which
 * may exceed cap; then call again with a larger buffer). Used for
 * finite differences: perturbing one Gaussian changes only these pixels. */
int64_t or_contrib(const double* mean3, const double* covp, double logit, double intensity,
                   int32_t P, const double* planes, const int64_t* sizes, const or_config* cfg,
                   int64_t* pix_out, double* w_out, int64_t cap) {
  int64_t cnt = 0;
  for (int32_t pi = 0; pi < P; ++pi) {
    or_plane pl;
    load_plane(planes + 11 * pi, sizes + 3 * pi, &pl);
    or_pg G;
    pg_compute(&pl, mean3, covp, logit, intensity, cfg, &G);
    if (!G.visible) continue;
    for (int64_t i = 0; i < pl.h; ++i) {
      double x2 = px_x2(&pl, i);
      if (!(G.m[1] - G.h[1] <= x2 && x2 <= G.m[1] + G.h[1])) continue;
      for (int64_t j = 0; j < pl.w; ++j) {
        double x1 = px_x1(&pl, j);
        double dl[3];
        double q = pair_q(&pl, &G, x1, x2, dl);
        int am;
        if (!pair_included(&pl, &G, cfg, x1, x2, q, &am)) continue;
        if (cnt < cap) {
          pix_out[cnt] = pl.off + i * pl.w + j;
          w_out[cnt] = G.alpha * exp(-0.5 * q);
        }
        cnt++;
      }
    }
  }
  return cnt;
}

/* World-frame precision and covariance (explicit cofactor inverse) of n
 * Gaussians, 9 doubles each. */
void or_covariance(int64_t n, const double* covp, const or_config* cfg, double* prec, double* cov) {
  const int nc = ncovp(cfg->cov_param);
  for (int64_t g = 0; g < n; ++g) {
    double Pi[3][3], C[3][3];
    precision(covp + nc * g, cfg->cov_param, cfg->beta, Pi);
    double det = cofactors(Pi, C);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        prec[9 * g + 3 * a + b] = Pi[a][b];
        cov[9 * g + 3 * a + b] = C[b][a] / det; /* inverse = adjugate / det */
      }
  }
}

int32_t or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
