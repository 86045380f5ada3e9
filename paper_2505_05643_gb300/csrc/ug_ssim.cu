// SSIM and PSNR of rendered slices against targets (the paper's evaluation
// metrics, Sec. 5): 11 x 11 Gaussian window with sigma 1.5 normalised to sum
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
//   3. per image, the rows' sums in order: mean SSIM and PSNR (deterministic).
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
    double s = 0.0;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
      const double d = (double)__ldg(x + img + j) - (double)__ldg(y + img + j);
      s += d * d;
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) row_sse[(int64_t)p * H + i] = (float)red[0];
  }
}

__global__ void k_ssim_cols(const float* __restrict__ maps, int W, int H,
                            float* __restrict__ row_ssim) {
  const int p = blockIdx.y, iv = blockIdx.x;
  const int Wv = W - (kWin - 1), Hv = H - (kWin - 1);
  const int64_t plane_maps = (int64_t)H * Wv;
  const float* m = maps + (int64_t)p * 5 * plane_maps;
  double s = 0.0;
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
    s += (double)(num / den);
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) row_ssim[(int64_t)p * Hv + iv] = (float)red[0];
}

__global__ void k_ssim_final(const float* __restrict__ row_ssim, const float* __restrict__ row_sse,
                             int P, int W, int H, float* __restrict__ ssim,
                             float* __restrict__ psnr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int Wv = W - (kWin - 1), Hv = H - (kWin - 1);
  double s = 0.0, e = 0.0;
  for (int i = 0; i < Hv; ++i) s += (double)row_ssim[(int64_t)p * Hv + i];
  for (int i = 0; i < H; ++i) e += (double)row_sse[(int64_t)p * H + i];
  if (ssim) ssim[p] = (float)(s / ((double)Hv * (double)Wv));
  if (psnr) psnr[p] = (float)(10.0 * log10((double)W * (double)H / e));
}

}  // namespace

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
  k_ssim_final<<<(unsigned)((P + 127) / 128), 128, 0, s>>>(row_ssim, row_sse, P, W, H, ssim, psnr);
  return cudaGetLastError();
}

}  // namespace ug
