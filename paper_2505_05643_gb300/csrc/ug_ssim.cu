// SSIM and PSNR of rendered slices against targets (the paper's evaluation
// metrics, Sec. 5), and the L1 + D-SSIM training loss with its gradient (the
// loss of Kerbl et al., which Sec. 4.5 takes over): 11 x 11 Gaussian window with sigma 1.5 normalised to sum
// 1, C1 = (0.01)^2, C2 = (0.03)^2 (data range 1), every position where the
// window lies inside the image, mean over those positions; PSNR = 10
// log10(1 / MSE) per image.
//
// Three passes over P images of W x H pixels stored one after the other:
//   1. horizontal 11-tap sums of x, y, x^2, y^2, x y (taken about 1/2, which
//      keeps the variances free of cancellation) at every row and valid column,
//      and the per-row sum of squared differences;
//   2. vertical 11-tap sums at every valid position, the SSIM there, and the sum
//      over each valid row (a fixed-order block reduction);
//   3. per image (one block each), the rows' sums in a fixed order: mean SSIM
//      and PSNR (deterministic).
#include <cmath>

#include "ug_internal.cuh"

namespace ug {

namespace {

constexpr int kWin = 11;
constexpr float kC1 = 1e-4f, kC2 = 9e-4f;

__constant__ float c_gauss[kWin];

struct GaussInit {
  float g[kWin];
};

GaussInit gauss_taps() {
  GaussInit t;
  double s = 0.0, w[kWin];
  for (int a = 0; a < kWin; ++a) {
    const double r = a - (kWin - 1) / 2.0;
    w[a] = std::exp(-(r * r) / (2.0 * 1.5 * 1.5));
    s += w[a];
  }
  for (int a = 0; a < kWin; ++a) t.g[a] = (float)(w[a] / s);
  return t;
}

// Fixed-order sum of one float per thread of a 256-thread block, returned to
// thread 0: a pairwise tree within each warp (shuffles), then the eight warp
// sums in order. FP64 arithmetic runs at 1/64 of the FP32 rate on GB300, so
// the per-row sums stay in FP32; their pairwise order keeps the error near
// log2(256) roundings.
__device__ __forceinline__ float block_sum256f(float v) {
  __shared__ float ws[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = 0.f;
  if (threadIdx.x == 0) {
    r = ((ws[0] + ws[1]) + (ws[2] + ws[3])) + ((ws[4] + ws[5]) + (ws[6] + ws[7]));
  }
  return r;
}

__global__ void k_ssim_rows(const float* __restrict__ x, const float* __restrict__ y, int W, int H,
                            float* __restrict__ maps, float* __restrict__ row_sse) {
  const int p = blockIdx.z, i = blockIdx.y;
  const int Wv = W - (kWin - 1);
  const int64_t img = (int64_t)p * W * H + (int64_t)i * W;
  const int64_t plane_maps = (int64_t)H * Wv;
  for (int jv = blockIdx.x * blockDim.x + threadIdx.x; jv < Wv; jv += gridDim.x * blockDim.x) {
    float sx = 0.f, sy = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;
#pragma unroll
    for (int a = 0; a < kWin; ++a) {
      const float xv = __ldg(x + img + jv + a) - 0.5f, yv = __ldg(y + img + jv + a) - 0.5f;
      const float g = c_gauss[a];
      sx = fmaf(g, xv, sx);
      sy = fmaf(g, yv, sy);
      sxx = fmaf(g, xv * xv, sxx);
      syy = fmaf(g, yv * yv, syy);
      sxy = fmaf(g, xv * yv, sxy);
    }
    float* m = maps + (int64_t)p * 5 * plane_maps + (int64_t)i * Wv + jv;
    m[0] = sx;
    m[plane_maps] = sy;
    m[2 * plane_maps] = sxx;
    m[3 * plane_maps] = syy;
    m[4 * plane_maps] = sxy;
  }
  // sum of squared differences of row i (one block per row does it)
  if (blockIdx.x == 0) {
    float s = 0.f;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
      const float d = __ldg(x + img + j) - __ldg(y + img + j);
      s = fmaf(d, d, s);
    }
    s = block_sum256f(s);
    if (threadIdx.x == 0) row_sse[(int64_t)p * H + i] = s;
  }
}

__global__ void k_ssim_cols(const float* __restrict__ maps, int W, int H,
                            float* __restrict__ row_ssim) {
  const int p = blockIdx.y, iv = blockIdx.x;
  const int Wv = W - (kWin - 1), Hv = H - (kWin - 1);
  const int64_t plane_maps = (int64_t)H * Wv;
  const float* m = maps + (int64_t)p * 5 * plane_maps;
  float s = 0.f;
  for (int jv = threadIdx.x; jv < Wv; jv += blockDim.x) {
    float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
    for (int a = 0; a < kWin; ++a) {
      const int64_t o = (int64_t)(iv + a) * Wv + jv;
      const float g = c_gauss[a];
      mx = fmaf(g, m[o], mx);
      my = fmaf(g, m[plane_maps + o], my);
      exx = fmaf(g, m[2 * plane_maps + o], exx);
      eyy = fmaf(g, m[3 * plane_maps + o], eyy);
      exy = fmaf(g, m[4 * plane_maps + o], exy);
    }
    const float vx = exx - mx * mx, vy = eyy - my * my, cxy = exy - mx * my;  // about 1/2
    const float ux = mx + 0.5f, uy = my + 0.5f;
    const float num = (2.f * ux * uy + kC1) * (2.f * cxy + kC2);
    const float den = (ux * ux + uy * uy + kC1) * (vx + vy + kC2);
    s += num / den;
  }
  s = block_sum256f(s);
  if (threadIdx.x == 0) row_ssim[(int64_t)p * Hv + iv] = s;
}

// Fixed-order block sum of one value per thread (256 threads).
__device__ __forceinline__ double block_sum256(double v) {
  __shared__ double red[256];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Per image (one block each): mean SSIM over the valid positions and PSNR,
// from the rows' sums in a fixed order.
__global__ void k_ssim_final(const float* __restrict__ row_ssim, const float* __restrict__ row_sse,
                             int P, int W, int H, float* __restrict__ ssim,
                             float* __restrict__ psnr) {
  const int p = blockIdx.x;
  const int Wv = W - (kWin - 1), Hv = H - (kWin - 1);
  double s = 0.0, e = 0.0;
  for (int i = threadIdx.x; i < Hv; i += blockDim.x) s += (double)row_ssim[(int64_t)p * Hv + i];
  for (int i = threadIdx.x; i < H; i += blockDim.x) e += (double)row_sse[(int64_t)p * H + i];
  s = block_sum256(s);
  e = block_sum256(e);
  if (threadIdx.x == 0) {
    if (ssim) ssim[p] = (float)(s / ((double)Hv * (double)Wv));
    if (psnr) psnr[p] = (float)(10.0 * log10((double)W * (double)H / e));
  }
}

// ---------------------------------------------------------------- L1 + D-SSIM loss
// Gradient of the mean SSIM (per plane, over its valid positions p): with the
// window sums about 1/2 (mx = mu_x - 1/2, ...), A1 = 2 ux uy + C1, A2 = 2 cxy +
// C2, B1 = ux^2 + uy^2 + C1, B2 = vx + vy + C2, S = A1 A2 / (B1 B2):
//   dS/dux = 2 A2 (uy B1 - A1 ux) / (B1^2 B2), dS/dvx = -S / B2, dS/dcxy = 2 A1 / (B1 B2),
//   dS(p)/dx_q = w(q - p) (a(p) + b(p) x'_q + c(p) y'_q),  x' = x - 1/2,
//   a = dS/dux - 2 mx dS/dvx - my dS/dcxy,  b = 2 dS/dvx,  c = dS/dcxy;
// the per-pixel sums over the positions whose window holds q are two
// transposed 11-tap passes (rows, then columns) of the maps a, b, c.

// Vertical window sums at the valid positions of row iv: S, and the maps a, b, c.
__global__ void k_dssim_cols(const float* __restrict__ maps, int W, int H,
                             float* __restrict__ abc, float* __restrict__ row_ssim) {
  const int p = blockIdx.y, iv = blockIdx.x;
  const int Wv = W - (kWin - 1), Hv = H - (kWin - 1);
  const int64_t plane_maps = (int64_t)H * Wv, plane_abc = (int64_t)Hv * Wv;
  const float* m = maps + (int64_t)p * 5 * plane_maps;
  float* o = abc + (int64_t)p * 3 * plane_abc + (int64_t)iv * Wv;
  float s = 0.f;
  for (int jv = threadIdx.x; jv < Wv; jv += blockDim.x) {
    float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
    for (int a = 0; a < kWin; ++a) {
      const int64_t q = (int64_t)(iv + a) * Wv + jv;
      const float g = c_gauss[a];
      mx = fmaf(g, m[q], mx);
      my = fmaf(g, m[plane_maps + q], my);
      exx = fmaf(g, m[2 * plane_maps + q], exx);
      eyy = fmaf(g, m[3 * plane_maps + q], eyy);
      exy = fmaf(g, m[4 * plane_maps + q], exy);
    }
    const float vx = exx - mx * mx, vy = eyy - my * my, cxy = exy - mx * my;
    const float ux = mx + 0.5f, uy = my + 0.5f;
    const float A1 = 2.f * ux * uy + kC1, A2 = 2.f * cxy + kC2;
    const float B1 = ux * ux + uy * uy + kC1, B2 = vx + vy + kC2;
    const float S = (A1 * A2) / (B1 * B2);
    const float d_ux = 2.f * A2 * (uy * B1 - A1 * ux) / (B1 * B1 * B2);
    const float d_vx = -S / B2;
    const float d_cxy = 2.f * A1 / (B1 * B2);
    o[jv] = d_ux - 2.f * mx * d_vx - my * d_cxy;
    o[plane_abc + jv] = 2.f * d_vx;
    o[2 * plane_abc + jv] = d_cxy;
    s += S;
  }
  s = block_sum256f(s);
  if (threadIdx.x == 0) row_ssim[(int64_t)p * Hv + iv] = s;
}

// Transposed horizontal pass: T_f(iv, j) = sum_a w_a f(iv, j - a) over the
// valid columns j - a, for the three maps, at every column j of the plane.
__global__ void k_dssim_trows(const float* __restrict__ abc, int W, int H, float* __restrict__ t) {
  const int p = blockIdx.z, iv = blockIdx.y;
  const int Wv = W - (kWin - 1), Hv = H - (kWin - 1);
  const int64_t plane_abc = (int64_t)Hv * Wv, plane_t = (int64_t)Hv * W;
  const float* f = abc + (int64_t)p * 3 * plane_abc + (int64_t)iv * Wv;
  float* o = t + (int64_t)p * 3 * plane_t + (int64_t)iv * W;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < W; j += gridDim.x * blockDim.x) {
    float sa = 0.f, sb = 0.f, sc = 0.f;
#pragma unroll
    for (int a = 0; a < kWin; ++a) {
      const int c = j - a;
      if (c >= 0 && c < Wv) {
        const float g = c_gauss[a];
        sa = fmaf(g, f[c], sa);
        sb = fmaf(g, f[plane_abc + c], sb);
        sc = fmaf(g, f[2 * plane_abc + c], sc);
      }
    }
    o[j] = sa;
    o[plane_t + j] = sb;
    o[2 * plane_t + j] = sc;
  }
}

// Transposed vertical pass at every pixel of row i, the gradient
//   dL/dx = (1 - lam) sign(x - y) / N - lam / P * (Ga + x' Gb + y' Gc) / (Hv Wv),
// and the row's sum of |x - y| (one block per row, fixed order).
__global__ void k_dssim_grad(const float* __restrict__ x, const float* __restrict__ y,
                             const float* __restrict__ t, int W, int H, float k1, float k2,
                             float* __restrict__ grad, float* __restrict__ row_l1) {
  const int p = blockIdx.y, i = blockIdx.x;
  const int Hv = H - (kWin - 1);
  const int64_t plane_t = (int64_t)Hv * W;
  const float* tp = t + (int64_t)p * 3 * plane_t;
  const int64_t row = (int64_t)p * W * H + (int64_t)i * W;
  float s = 0.f;
  for (int j = threadIdx.x; j < W; j += blockDim.x) {
    float ga = 0.f, gb = 0.f, gc = 0.f;
#pragma unroll
    for (int a = 0; a < kWin; ++a) {
      const int r = i - a;
      if (r >= 0 && r < Hv) {
        const float g = c_gauss[a];
        const int64_t q = (int64_t)r * W + j;
        ga = fmaf(g, tp[q], ga);
        gb = fmaf(g, tp[plane_t + q], gb);
        gc = fmaf(g, tp[2 * plane_t + q], gc);
      }
    }
    const float xv = __ldg(x + row + j), yv = __ldg(y + row + j);
    const float d = xv - yv;
    const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    const float gs = fmaf(yv - 0.5f, gc, fmaf(xv - 0.5f, gb, ga));
    grad[row + j] = fmaf(k1, sg, -k2 * gs);
    s += fabsf(d);
  }
  s = block_sum256f(s);
  if (threadIdx.x == 0) row_l1[(int64_t)p * H + i] = s;
}

// Per plane (one block each): its mean SSIM and its sum of |x - y|.
__global__ void k_dssim_plane(const float* __restrict__ row_ssim, const float* __restrict__ row_l1,
                              int W, int H, double* __restrict__ plane) {
  const int p = blockIdx.x;
  const int Wv = W - (kWin - 1), Hv = H - (kWin - 1);
  double s = 0.0, l = 0.0;
  for (int i = threadIdx.x; i < Hv; i += blockDim.x) s += (double)row_ssim[(int64_t)p * Hv + i];
  for (int i = threadIdx.x; i < H; i += blockDim.x) l += (double)row_l1[(int64_t)p * H + i];
  s = block_sum256(s);
  l = block_sum256(l);
  if (threadIdx.x == 0) {
    plane[2 * p] = s / ((double)Hv * (double)Wv);
    plane[2 * p + 1] = l;
  }
}

__global__ void k_dssim_final(const double* __restrict__ plane, int P, int W, int H, float lam,
                              float* __restrict__ loss) {
  double s = 0.0, l = 0.0;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    s += plane[2 * p];
    l += plane[2 * p + 1];
  }
  s = block_sum256(s);
  l = block_sum256(l);
  if (threadIdx.x == 0) {
    const double n = (double)P * (double)W * (double)H;
    loss[0] = (float)((1.0 - lam) * l / n + lam * (1.0 - s / (double)P));
  }
}

}  // namespace

size_t dssim_scratch_floats(int32_t P, int32_t W, int32_t H) {
  const size_t Wv = (size_t)(W - (kWin - 1)), Hv = (size_t)(H - (kWin - 1));
  // window maps, gradient maps, their transposed row pass, per-row sums, and
  // per-plane sums (two doubles each, 8-byte aligned)
  return (size_t)P * (5 * (size_t)H * Wv + 3 * Hv * Wv + 3 * Hv * (size_t)W + Hv + (size_t)H) + 4 * (size_t)P + 2;
}

cudaError_t launch_l1_dssim(const float* image, const float* target, int32_t P, int32_t W,
                            int32_t H, float lam, float* scratch, float* grad, float* loss,
                            cudaStream_t s) {
  static const GaussInit taps = gauss_taps();
  cudaError_t e = cudaMemcpyToSymbolAsync(c_gauss, taps.g, sizeof(taps.g), 0,
                                          cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int Wv = W - (kWin - 1), Hv = H - (kWin - 1);
  float* maps = scratch;
  float* abc = maps + 5 * (size_t)P * (size_t)H * (size_t)Wv;
  float* t = abc + 3 * (size_t)P * (size_t)Hv * (size_t)Wv;
  float* row_ssim = t + 3 * (size_t)P * (size_t)Hv * (size_t)W;
  float* row_l1 = row_ssim + (size_t)P * (size_t)Hv;
  float* row_sse = row_l1;  // the row pass's squared differences are not needed; overwritten
  k_ssim_rows<<<dim3((unsigned)((Wv + 255) / 256), (unsigned)H, (unsigned)P), 256, 0, s>>>(
      image, target, W, H, maps, row_sse);
  k_dssim_cols<<<dim3((unsigned)Hv, (unsigned)P), 256, 0, s>>>(maps, W, H, abc, row_ssim);
  k_dssim_trows<<<dim3((unsigned)((W + 255) / 256), (unsigned)Hv, (unsigned)P), 256, 0, s>>>(
      abc, W, H, t);
  // the gradient's two constant factors, formed once here in FP64
  const double npx = (double)P * (double)W * (double)H;
  const float k1 = (float)((1.0 - (double)lam) / npx);
  const float k2 = (float)((double)lam / ((double)P * (double)Hv * (double)Wv));
  k_dssim_grad<<<dim3((unsigned)H, (unsigned)P), 256, 0, s>>>(image, target, t, W, H, k1, k2, grad,
                                                              row_l1);
  double* plane = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(row_l1 + (size_t)P * (size_t)H) + 7) & ~uintptr_t(7));
  k_dssim_plane<<<(unsigned)P, 256, 0, s>>>(row_ssim, row_l1, W, H, plane);
  k_dssim_final<<<1, 256, 0, s>>>(plane, P, W, H, lam, loss);
  return cudaGetLastError();
}

size_t ssim_scratch_floats(int32_t P, int32_t W, int32_t H) {
  const size_t Wv = (size_t)(W - (kWin - 1)), Hv = (size_t)(H - (kWin - 1));
  return 5 * (size_t)P * (size_t)H * Wv + (size_t)P * Hv + (size_t)P * (size_t)H;
}

cudaError_t launch_ssim(const float* image, const float* target, int32_t P, int32_t W, int32_t H,
                        float* scratch, float* ssim, float* psnr, cudaStream_t s) {
  static const GaussInit taps = gauss_taps();
  cudaError_t e = cudaMemcpyToSymbolAsync(c_gauss, taps.g, sizeof(taps.g), 0,
                                          cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int Wv = W - (kWin - 1), Hv = H - (kWin - 1);
  float* maps = scratch;
  float* row_ssim = maps + 5 * (size_t)P * (size_t)H * (size_t)Wv;
  float* row_sse = row_ssim + (size_t)P * (size_t)Hv;
  k_ssim_rows<<<dim3((unsigned)((Wv + 255) / 256), (unsigned)H, (unsigned)P), 256, 0, s>>>(
      image, target, W, H, maps, row_sse);
  k_ssim_cols<<<dim3((unsigned)Hv, (unsigned)P), 256, 0, s>>>(maps, W, H, row_ssim);
  k_ssim_final<<<(unsigned)P, 256, 0, s>>>(row_ssim, row_sse, P, W, H, ssim, psnr);
  return cudaGetLastError();
}

}  // namespace ug
