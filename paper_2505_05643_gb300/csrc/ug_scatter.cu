// The paper's own forward, kept as an ablation of the tile gather: phase 2 of
// Sec. 4.4 loops over every visible (plane, Gaussian) record's pixel box and
// adds the record's weight and weighted intensity to each pixel with atomics;
// a last pass forms C = (S_c + a_bg c_bg) / (S_a + a_bg) (Eq. alpha-combine,
// Eq. colour-combine). Same records and same per-pixel weight formula as the
// tile rasterizer, so the two differ only in the order of the sums.
#include "ug_internal.cuh"

namespace ug {

// One warp per record slot (grid-stride); lanes take the box's rows in
// segments of up to 8 pixels (each segment one item of item_geo, anchored at
// its first pixel). Zero weights add nothing and issue no atomic.
__global__ void __launch_bounds__(256) k_scatter(WsView v, int cut, float* __restrict__ sa,
                                                 float* __restrict__ sc) {
  if (dev_failed(v.hdr)) return;
  const uint32_t slots = v.hdr->slots;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; slot < slots; slot += warps) {
    const uint2 bx = v.rec_box[slot];
    const int j0 = bx.x & 0xffff, j1 = bx.x >> 16, i0 = bx.y & 0xffff, i1 = bx.y >> 16;
    if (j0 > j1 || i0 > i1) continue;
    const float4 a = v.rec_a[slot], b = v.rec_b[slot], c = v.rec_c[slot];
    const PlaneDev& pl = v.planes[v.rec_plane[slot]];
    const uint32_t nsx = (uint32_t)(j1 - j0 + 8) / 8u, nseg = nsx * (uint32_t)(i1 - i0 + 1);
    for (uint32_t k = lane; k < nseg; k += 32u) {
      const uint32_t di = k / nsx, ds = k - di * nsx;
      const int i = i0 + (int)di, fj0 = j0 + 8 * (int)ds;
      const ItemGeo g = item_geo(a, b, c, bx, fj0, i);
      const float t2 = b.x * __fadd_rn(g.nyh, g.nyl);
      const int64_t row = pl.px_off + (int64_t)i * pl.w;
      for (int q = 0; q < 8 && fj0 + q <= j1; ++q) {
        const float t1 = __fmaf_rn(g.r11, __fadd_rn((float)q, g.ns0q), g.a0);
        const float e = __fsub_rn(__fmaf_rn(-t1, t1, b.y), __fmul_rn(t2, t2));
        const float qq = __fmaf_rn(t1, t1, __fmul_rn(t2, t2));
        const bool in = cut == 0 || qq <= b.w;
        const float w = in ? fast_exp2(e) : 0.f;
        if (w > 0.f) {
          atomicAdd(sa + row + fj0 + q, w);
          atomicAdd(sc + row + fj0 + q, w * b.z);
        }
      }
    }
  }
}

__global__ void k_scatter_finish(int64_t n, float abg, float cbg, float* __restrict__ image,
                                 float* __restrict__ alpha) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float al = alpha[p] + abg;
    image[p] = (image[p] + abg * cbg) / al;
    alpha[p] = al;
  }
}

cudaError_t launch_render_scatter(const ug_plan* plan, WsView v, float* image, float* alpha,
                                  cudaStream_t s) {
  const size_t bytes = sizeof(float) * (size_t)plan->total_pixels;
  cudaError_t e = cudaMemsetAsync(image, 0, bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(alpha, 0, bytes, s);
  // this forward leaves no footprint tests for the backward rasterizer
  if (e != cudaSuccess) return e;
  const int sms = device_sms();
  k_scatter<<<sms * 8, 256, 0, s>>>(v, plan->cfg.cutoff, alpha, image);
  k_scatter_finish<<<sms * 4, 256, 0, s>>>(plan->total_pixels, plan->cfg.alpha_bg, plan->cfg.c_bg,
                                           image, alpha);
  return cudaGetLastError();
}

}  // namespace ug
