// Rows a6 and a9: the MSE loss gradient and the fused Adam step. Both are
// streaming, HBM-bound kernels (float4 loads where the rows allow it).
#include "ug_internal.cuh"

namespace ug {

// ------------------------------------------------------------------ MSE
__global__ void __launch_bounds__(256)
    k_mse(const float* __restrict__ image, const float* __restrict__ target, int64_t n,
          int64_t denom, float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ double red[8];
  const float scale = 2.0f / (float)denom;
  // a thread's few squares are summed in FP32 (FP64 arithmetic runs at a small
  // fraction of the FP32 rate), the threads' sums in FP64
  float accf = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool vec = (n % 4 == 0) && ((uintptr_t)image % 16 == 0) && ((uintptr_t)target % 16 == 0) &&
                   ((uintptr_t)grad % 16 == 0);
  if (vec) {
    const float4* im4 = reinterpret_cast<const float4*>(image);
    const float4* tg4 = reinterpret_cast<const float4*>(target);
    float4* gr4 = reinterpret_cast<float4*>(grad);
    for (int64_t i = t0; i < n / 4; i += stride) {
      const float4 a = im4[i], b = tg4[i];
      const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
      if (grad) gr4[i] = make_float4(scale * d.x, scale * d.y, scale * d.z, scale * d.w);
      accf = fmaf(d.x, d.x, accf);
      accf = fmaf(d.y, d.y, accf);
      accf = fmaf(d.z, d.z, accf);
      accf = fmaf(d.w, d.w, accf);
    }
  } else {
    for (int64_t i = t0; i < n; i += stride) {
      const float d = image[i] - target[i];
      if (grad) grad[i] = scale * d;
      accf = fmaf(d, d, accf);
    }
  }
  double acc = warp_sum((double)accf);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    loss[1 + blockIdx.x] = (float)s;
  }
}

__global__ void k_mse_final(float* loss, int64_t denom) {
  __shared__ double red[kMseBlocks];
  for (int b = threadIdx.x; b < kMseBlocks; b += blockDim.x) red[b] = (double)loss[1 + b];
  __syncthreads();
  for (int w = kMseBlocks / 2; w > 0; w >>= 1) {
    for (int b = threadIdx.x; b < w; b += blockDim.x) red[b] += red[b + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = (float)(red[0] / (double)denom);
}

// Sum of squared differences over n pixels divided by denom (denom = n: the
// mean), and its gradient 2 (image - target) / denom.
cudaError_t launch_mse(const float* image, const float* target, int64_t n, int64_t denom,
                       float* grad, float* loss, cudaStream_t s) {
  k_mse<<<kMseBlocks, 256, 0, s>>>(image, target, n, denom, grad, loss);
  k_mse_final<<<1, 256, 0, s>>>(loss, denom);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Adam
struct AdamScalars {
  float lr_over_bc1, inv_sqrt_bc2;
};

__device__ __forceinline__ AdamScalars adam_scalars(const ug_adam_row& row, int t, float b1,
                                                    float b2) {
  // bias corrections in FP64 once per block (1 - b^t cancels in FP32)
  const double bc1 = 1.0 - pow((double)b1, (double)t);
  const double bc2 = 1.0 - pow((double)b2, (double)t);
  double lr = row.lr_init;
  if (row.decay_steps > 0 && row.lr_final != row.lr_init) {
    const double frac = fmin((double)t / (double)row.decay_steps, 1.0);
    lr = (double)row.lr_init * pow((double)row.lr_final / (double)row.lr_init, frac);
  }
  AdamScalars a;
  a.lr_over_bc1 = (float)(lr / bc1);
  a.inv_sqrt_bc2 = (float)(1.0 / sqrt(bc2));
  return a;
}

__device__ __forceinline__ void adam_one(float& p, float g, float& m, float& v, float b1, float b2,
                                         float eps, const AdamScalars& a) {
  m = fmaf(b1, m, (1.f - b1) * g);
  v = fmaf(b2, v, (1.f - b2) * g * g);
  const float denom = sqrtf(v) * a.inv_sqrt_bc2 + eps;
  p -= a.lr_over_bc1 * (m / denom);
}

template <bool VEC>
__global__ void __launch_bounds__(256)
    k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
           float* __restrict__ v, int64_t n, const ug_adam_row* __restrict__ rows,
           const int32_t* __restrict__ d_step, float b1, float b2, float eps) {
  __shared__ AdamScalars sc;
  const int row = blockIdx.y;
  if (threadIdx.x == 0) sc = adam_scalars(rows[row], *d_step + 1, b1, b2);
  __syncthreads();
  const AdamScalars a = sc;
  const int64_t off = (int64_t)row * n;
  if (VEC) {
    const int64_t n4 = n >> 2;
    float4* p4 = reinterpret_cast<float4*>(p + off);
    const float4* g4 = reinterpret_cast<const float4*>(g + off);
    float4* m4 = reinterpret_cast<float4*>(m + off);
    float4* v4 = reinterpret_cast<float4*>(v + off);
    // two elements of four per thread in flight per iteration
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + stride < n4; i += 2 * stride) {
      float4 pp = p4[i], gg = g4[i], mm = m4[i], vv = v4[i];
      float4 pq = p4[i + stride], gq = g4[i + stride], mq = m4[i + stride], vq = v4[i + stride];
      adam_one(pp.x, gg.x, mm.x, vv.x, b1, b2, eps, a);
      adam_one(pp.y, gg.y, mm.y, vv.y, b1, b2, eps, a);
      adam_one(pp.z, gg.z, mm.z, vv.z, b1, b2, eps, a);
      adam_one(pp.w, gg.w, mm.w, vv.w, b1, b2, eps, a);
      adam_one(pq.x, gq.x, mq.x, vq.x, b1, b2, eps, a);
      adam_one(pq.y, gq.y, mq.y, vq.y, b1, b2, eps, a);
      adam_one(pq.z, gq.z, mq.z, vq.z, b1, b2, eps, a);
      adam_one(pq.w, gq.w, mq.w, vq.w, b1, b2, eps, a);
      p4[i] = pp;
      m4[i] = mm;
      v4[i] = vv;
      p4[i + stride] = pq;
      m4[i + stride] = mq;
      v4[i + stride] = vq;
    }
    for (; i < n4; i += stride) {
      float4 pp = p4[i], gg = g4[i], mm = m4[i], vv = v4[i];
      adam_one(pp.x, gg.x, mm.x, vv.x, b1, b2, eps, a);
      adam_one(pp.y, gg.y, mm.y, vv.y, b1, b2, eps, a);
      adam_one(pp.z, gg.z, mm.z, vv.z, b1, b2, eps, a);
      adam_one(pp.w, gg.w, mm.w, vv.w, b1, b2, eps, a);
      p4[i] = pp;
      m4[i] = mm;
      v4[i] = vv;
    }
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
      float pp = p[off + i], mm = m[off + i], vv = v[off + i];
      adam_one(pp, g[off + i], mm, vv, b1, b2, eps, a);
      p[off + i] = pp;
      m[off + i] = mm;
      v[off + i] = vv;
    }
  }
}

__global__ void k_step_inc(int32_t* d_step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *d_step += 1;
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int32_t rows, int64_t n,
                        const ug_adam_row* d_rows, int32_t* d_step, float b1, float b2,
                        float eps, cudaStream_t s) {
  const bool vec = (n % 4 == 0) && ((uintptr_t)p % 16 == 0) && ((uintptr_t)g % 16 == 0) &&
                   ((uintptr_t)m % 16 == 0) && ((uintptr_t)v % 16 == 0);
  // one wave: the SMs' resident blocks shared evenly among the rows
  static int resident[2] = {0, 0};
  int& occ = resident[vec ? 1 : 0];
  if (occ == 0) {
    if (vec) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adam<true>, 256, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adam<false>, 256, 0);
    if (occ < 1) occ = 1;
  }
  const int64_t work = vec ? n / 4 : n;
  int64_t bx = (work + 255) / 256;
  const int64_t cap = (int64_t)device_sms() * occ / (rows > 0 ? rows : 1);
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  dim3 grid((unsigned)bx, (unsigned)rows);
  if (vec)
    k_adam<true><<<grid, 256, 0, s>>>(p, g, m, v, n, d_rows, d_step, b1, b2, eps);
  else
    k_adam<false><<<grid, 256, 0, s>>>(p, g, m, v, n, d_rows, d_step, b1, b2, eps);
  k_step_inc<<<1, 32, 0, s>>>(d_step);
  return cudaGetLastError();
}

}  // namespace ug
