// The per-pixel sums of a Gaussian-sharded render. Image formation (Sec. 4.1,
// Eq. alpha-combine and Eq. colour-combine) divides two sums over Gaussians,
//   S_a = sum_i w_i,  S_c = sum_i w_i c_i,
//   alpha = S_a + a_bg,  C = (S_c + a_bg c_bg) / alpha,
// and neither sum depends on the order of its terms. A rank that renders a
// shard of the Gaussians therefore holds partial sums that add up, over the
// shards, to the full ones: one all-reduce of two floats per pixel, then the
// division. These two streaming kernels convert a shard's ug_render output to
// its partial sums, and the reduced sums back to image and alpha.
#include "ug_internal.cuh"

namespace ug {

// sums[2 i] = alpha_i - a_bg = S_a, sums[2 i + 1] = C_i alpha_i - a_bg c_bg = S_c.
__global__ void __launch_bounds__(256)
    k_shard_sums(const float* __restrict__ image, const float* __restrict__ alpha, int64_t n,
                 float abg, float cbg, float2* __restrict__ sums) {
  const float bc = abg * cbg;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float a = alpha[i];
    sums[i] = make_float2(a - abg, fmaf(image[i], a, -bc));
  }
}

// alpha_i = S_a + a_bg, C_i = (S_c + a_bg c_bg) / alpha_i, as the forward
// rasterizer forms them.
__global__ void __launch_bounds__(256)
    k_composite(const float2* __restrict__ sums, int64_t n, float abg, float cbg,
                float* __restrict__ image, float* __restrict__ alpha) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 s = sums[i];
    const float al = s.x + abg;
    image[i] = (s.y + abg * cbg) / al;
    alpha[i] = al;
  }
}

static int stream_grid(int64_t n) {
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)device_sms() * 8;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace ug

extern "C" ug_status ug_shard_sums(const float* image, const float* alpha, int64_t n,
                                   float alpha_bg, float c_bg, float* sums, ug_stream stream) {
  if (!image || !alpha || !sums || n < 1 || (uintptr_t)sums % 8 != 0)
    return UG_ERR_INVALID_ARGUMENT;
  if (!(alpha_bg > 0.f)) return UG_ERR_INVALID_ARGUMENT;
  ug::k_shard_sums<<<ug::stream_grid(n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      image, alpha, n, alpha_bg, c_bg, reinterpret_cast<float2*>(sums));
  return cudaGetLastError() == cudaSuccess ? UG_OK : UG_ERR_CUDA;
}

extern "C" ug_status ug_composite(const float* sums, int64_t n, float alpha_bg, float c_bg,
                                  float* image, float* alpha, ug_stream stream) {
  if (!image || !alpha || !sums || n < 1 || (uintptr_t)sums % 8 != 0)
    return UG_ERR_INVALID_ARGUMENT;
  if (!(alpha_bg > 0.f)) return UG_ERR_INVALID_ARGUMENT;
  ug::k_composite<<<ug::stream_grid(n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const float2*>(sums), n, alpha_bg, c_bg, image, alpha);
  return cudaGetLastError() == cudaSuccess ? UG_OK : UG_ERR_CUDA;
}
