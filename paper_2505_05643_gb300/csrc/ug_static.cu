// ug_mse_loss_grad_static: the MSE loss and its gradient for callers that
// cannot allocate device memory.
//
// ug_mse_loss_grad needs UG_MSE_LOSS_FLOATS floats from the caller, most of
// them scratch for per-block partial sums. Code that runs where it may not
// call cudaMalloc (inside a stream capture, in a plugin handed only the
// tensors it works on, or under a fixed memory budget owned by someone else)
// can call this variant instead: its partial sums live in one file-scope
// device array of this library, so the caller passes only the inputs, the
// gradient output and a single float for the loss.
//
// The array holds kStaticMaxBlocks partial sums (64 KiB) and stays allocated
// on every GPU that loads the library until the process exits. Each block
// reduces kStaticChunk consecutive elements, so n may not exceed
// UG_MSE_STATIC_MAX_N = kStaticMaxBlocks * kStaticChunk. All calls share the
// array: every partial is written before it is read in the same call, so
// nothing has to be cleared, but two calls whose kernels overlap on the GPU
// (different streams, no ordering between them) race on it.
#include <mutex>

#include "ug_internal.cuh"

namespace ug {

constexpr int kStaticChunk = 1 << 16;      // elements reduced by one block
constexpr int kStaticMaxBlocks = 1 << 14;  // partial sums in the scratch array
static_assert((long long)kStaticChunk * kStaticMaxBlocks == UG_MSE_STATIC_MAX_N, "limit");

// The scratch. Host code must not pass this name to a kernel: on the host it
// is only a stand-in for the device symbol; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) float g_mse_partials[kStaticMaxBlocks];

constexpr int kMaxDevices = 64;
static float* s_partials[kMaxDevices];
static std::mutex s_mutex;

// Device address of the scratch for the current device, looked up once per
// device (with that device current) on the first call made on it.
static cudaError_t static_scratch(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(s_mutex);
  if (!s_partials[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mse_partials);
    if (e != cudaSuccess) return e;
    s_partials[dev] = static_cast<float*>(p);
  }
  *out = s_partials[dev];
  return cudaSuccess;
}

__global__ void __launch_bounds__(256)
    k_mse_static_partial(const float* __restrict__ image, const float* __restrict__ target,
                         int64_t n, float* __restrict__ grad, float* __restrict__ partials) {
  __shared__ double red[8];
  const float scale = 2.0f / (float)n;
  const int64_t begin = (int64_t)blockIdx.x * kStaticChunk;
  const int64_t end = min(begin + (int64_t)kStaticChunk, n);
  // a thread's few squares are summed in FP32 (FP64 arithmetic runs at a small
  // fraction of the FP32 rate), the threads' sums in FP64
  float accf = 0.f;
  for (int64_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
    const float d = image[i] - target[i];
    if (grad) grad[i] = scale * d;
    accf = fmaf(d, d, accf);
  }
  const double acc = warp_sum((double)accf);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    partials[blockIdx.x] = (float)s;
  }
}

__global__ void __launch_bounds__(1024)
    k_mse_static_final(const float* __restrict__ partials, int nblk, int64_t n, float* loss) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 1024) s += (double)partials[b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = (float)(red[0] / (double)n);
}

}  // namespace ug

extern "C" ug_status ug_mse_loss_grad_static(const float* image, const float* target, int64_t n,
                                             float* grad_image, float* loss, ug_stream stream) {
  if (!image || !target || !loss || n < 1) return UG_ERR_INVALID_ARGUMENT;
  if (n > UG_MSE_STATIC_MAX_N) return UG_ERR_INVALID_ARGUMENT;  // beyond the static scratch
  float* partials = nullptr;
  if (ug::static_scratch(&partials) != cudaSuccess) return UG_ERR_CUDA;
  const int nblk = (int)((n + ug::kStaticChunk - 1) / ug::kStaticChunk);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ug::k_mse_static_partial<<<nblk, 256, 0, s>>>(image, target, n, grad_image, partials);
  ug::k_mse_static_final<<<1, 1024, 0, s>>>(partials, nblk, n, loss);
  return cudaGetLastError() == cudaSuccess ? UG_OK : UG_ERR_CUDA;
}
