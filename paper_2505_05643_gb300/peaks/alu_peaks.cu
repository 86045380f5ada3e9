// Throughput of the instruction classes the rasterizers are built from, per SM
// per SM clock: scalar FP32 FMA, packed FP32x2 FMA (__ffma2_rn), MUFU ex2
// (ex2.approx.ftz.f32), and warp shuffles. These give the FP32-pipe roofline
// of the raster kernels (unit counts x clock), which no vendor table lists for
// this part.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o alu_peaks alu_peaks.cu && ./alu_peaks
//
// Every kernel runs 8 independent dependency chains per thread (enough to hide
// the pipe latency at 16 warps per SM scheduler), 8 blocks of 256 threads per
// SM. The SM clock during each kernel is measured from clock64() in block 0
// against the CUDA-event time, so the per-clock figures do not assume a clock.
#include <cstdio>
#include <cuda_runtime.h>

#define CHECK(x)                                                                 \
  do {                                                                           \
    cudaError_t e_ = (x);                                                        \
    if (e_ != cudaSuccess) {                                                     \
      std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));             \
      return 1;                                                                  \
    }                                                                            \
  } while (0)

// Block 0 records its SM clock counter and the global nanosecond timer at its
// start and end; their ratio is the SM clock while it ran.
__device__ __forceinline__ void mark(long long* clk, int which) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long ns;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
    clk[2 * which] = clock64();
    clk[2 * which + 1] = (long long)ns;
  }
}

__global__ void k_ffma(float* out, long long* clk, int iters, float a, float b) {
  mark(clk, 0);
  float x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = threadIdx.x * 1e-3f + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  mark(clk, 1);
}

__global__ void k_ffma2(float* out, long long* clk, int iters, float a, float b) {
  mark(clk, 0);
  float2 x[8];
  const float2 av = make_float2(a, a), bv = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = make_float2(threadIdx.x * 1e-3f + c, c - 0.5f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = __ffma2_rn(x[c], av, bv);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c].x + x[c].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  mark(clk, 1);
}

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void k_ex2(float* out, long long* clk, int iters) {
  mark(clk, 0);
  float x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = -(threadIdx.x * 1e-3f) - c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = -ex2(x[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  mark(clk, 1);
}

__global__ void k_shfl(float* out, long long* clk, int iters) {
  mark(clk, 0);
  float x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = __shfl_xor_sync(0xffffffffu, x[c], 1 << (c & 3));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  mark(clk, 1);
}

struct Result {
  double ms, mhz;
};

template <typename F>
static int timed(F launch, long long* d_clk, cudaEvent_t a, cudaEvent_t b, Result* r) {
  launch();  // warm-up
  CHECK(cudaGetLastError());
  CHECK(cudaDeviceSynchronize());
  CHECK(cudaEventRecord(a));
  launch();
  CHECK(cudaEventRecord(b));
  CHECK(cudaEventSynchronize(b));
  float ms = 0.f;
  CHECK(cudaEventElapsedTime(&ms, a, b));
  long long clk[4];
  CHECK(cudaMemcpy(clk, d_clk, sizeof(clk), cudaMemcpyDeviceToHost));
  r->ms = ms;
  r->mhz = clk[3] > clk[1] ? (double)(clk[2] - clk[0]) / (double)(clk[3] - clk[1]) * 1e3 : 0.0;
  return 0;
}

int main() {
  int dev = 0, sms = 0, clk_khz = 0;
  CHECK(cudaGetDevice(&dev));
  CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CHECK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev));
  const int blocks = sms * 8, threads = 256, iters = 2048;
  float* out = nullptr;
  long long* d_clk = nullptr;
  CHECK(cudaMalloc(&out, sizeof(float) * blocks * threads));
  CHECK(cudaMalloc(&d_clk, 4 * sizeof(long long)));
  cudaEvent_t a, b;
  CHECK(cudaEventCreate(&a));
  CHECK(cudaEventCreate(&b));
  const double thr = (double)blocks * threads;
  std::printf("SMs %d, max SM clock %d MHz, %d blocks x %d threads\n", sms, clk_khz / 1000, blocks,
              threads);
  std::printf("%-6s %10s %9s %14s %16s %16s\n", "kind", "time_ms", "sm_MHz", "Tlane-ops/s",
              "lane-ops/SM/clk", "warp-inst/SM/clk");
  Result r{0.0, 0.0};
  auto report = [&](const char* name, double lane_ops, double per_inst) {
    const double per_s = thr * lane_ops / (r.ms * 1e-3);
    const double mhz = r.mhz > 0.0 ? r.mhz : clk_khz * 1e-3;
    const double per_clk = per_s / sms / (mhz * 1e6);
    std::printf("%-6s %10.3f %9.0f %14.2f %16.1f %16.2f\n", name, r.ms, r.mhz, per_s / 1e12, per_clk,
                per_clk / 32.0 / per_inst);
  };
  if (timed([&] { k_ffma<<<blocks, threads>>>(out, d_clk, iters, 0.999f, 1e-3f); }, d_clk, a, b, &r))
    return 1;
  report("FFMA", (double)iters * 16 * 8, 1.0);
  if (timed([&] { k_ffma2<<<blocks, threads>>>(out, d_clk, iters, 0.999f, 1e-3f); }, d_clk, a, b, &r))
    return 1;
  report("FFMA2", (double)iters * 16 * 8 * 2, 2.0);
  if (timed([&] { k_ex2<<<blocks, threads>>>(out, d_clk, iters / 4); }, d_clk, a, b, &r)) return 1;
  report("EX2", (double)(iters / 4) * 16 * 8, 1.0);
  if (timed([&] { k_shfl<<<blocks, threads>>>(out, d_clk, iters / 4); }, d_clk, a, b, &r)) return 1;
  report("SHFL", (double)(iters / 4) * 16 * 8, 1.0);
  CHECK(cudaFree(out));
  CHECK(cudaFree(d_clk));
  return 0;
}
