// Rows a5 and a7: the forward tile rasterizer and its gradient.
//
// One CTA owns one TILE x TILE pixel tile at a time and takes tiles from a
// device work counter (persistent launch over all tiles of all planes, so
// planes of different sizes share one launch). Each warp owns a WW x WH
// sub-rectangle (footprint) of the tile, PPT vertically adjacent pixels per
// lane. The tile's records are staged in shared memory in batches of one
// record per thread; the staging thread decides, for every warp, whether the
// record can touch that warp's footprint:
//   - its pixel box must overlap the footprint (warp-level culling), and
//   - a lower bound on t1^2 + t2^2 over the overlap must leave the exponent
//     above -127: below that every weight in the overlap is exactly 0 in
//     FP32 (ex2 flushes results below 2^-126 to zero), so skipping the pair
//     changes no bit of the output or the gradient;
// and whether the box covers the whole footprint (then the per-pixel box
// tests are dropped). Each warp then walks its own compacted list.
//
// Per pixel and record:
//   dx = j + 1/2 - xs_j, dy = i + 1/2 - xs_i, t1 = r11 dx + r12 dy, t2 = r22 dy,
//   w = 2^(lw2 - t1^2 - t2^2)      (= alpha exp(-q/2), Eq. mahalanobis-3d)
// accumulated as S_a += w, S_c += w c in tile-list order (ascending Gaussian
// id), then C = (S_c + a_bg c_bg)/(S_a + a_bg) (Eq. alpha-combine,
// Eq. colour-combine). The forward pass has no atomics.
#include "ug_internal.cuh"

namespace ug {

__device__ __forceinline__ int find_plane(const int32_t* tile_off, int P, int t) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_off[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

struct TileCtx {
  int tile, tx, ty, w, h;
  int64_t px_off;
};

__device__ __forceinline__ bool next_tile(WsView& v, int which, int P, int total_tiles,
                                          TileCtx& tc, int* s_tile, int* s_plane) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const int t = (int)atomicAdd(&v.hdr->tile_counter[which], 1u);
    *s_tile = t;
    *s_plane = t < total_tiles ? find_plane(v.tile_off, P, t) : 0;
  }
  __syncthreads();
  const int t = *s_tile;
  if (t >= total_tiles) return false;
  const PlaneDev& pl = v.planes[*s_plane];
  const int local = t - pl.tile_off;
  tc.tx = local % pl.tiles_x;
  tc.ty = local / pl.tiles_x;
  tc.w = pl.w;
  tc.h = pl.h;
  tc.px_off = pl.px_off;
  tc.tile = t;
  return true;
}

template <int TILE, int WW, int PPT>
struct Layout {
  static constexpr int NT = TILE * TILE / PPT;
  static constexpr int NW = NT / 32;
  static constexpr int LH = 32 / WW;       // lane rows per warp
  static constexpr int WH = LH * PPT;      // warp footprint height
  static constexpr int WPR = TILE / WW;    // warps per tile row
  static_assert(NT % 32 == 0, "whole warps");
  static_assert(WPR * (TILE / WH) == NW, "warps tile the tile");
  static_assert(NW <= 16, "mask layout");
};

// Shared-memory staging of one batch of records and the per-warp lists.
template <int NT, int NW, bool BWD>
struct Stage {
  float4 a[NT];
  float4 b[NT];
  uint2 box[NT];
  uint32_t rid[BWD ? NT : 1];
  uint32_t mask[NT];          // bit w: live for warp w; bit 16 + w: box covers its footprint
  uint16_t list[NW][NT];      // record index | full << 15
  int tile, plane;
};

// Lower bound of t1^2 + t2^2 over the rectangle [dxlo, dxhi] x [dylo, dyhi],
// t1 = r11 dx + r12 dy (r11 >= 0), t2 = r22 dy (r22 >= 0): (min |t1|)^2 +
// (min |t2|)^2, each minimum taken at the rectangle's corners (t1 is linear).
__device__ __forceinline__ float min_q_lower_bound(float r11, float r12, float r22, float dxlo,
                                                   float dxhi, float dylo, float dyhi) {
  const float a1 = r12 * dylo, a2 = r12 * dyhi;
  const float t1min = fmaf(r11, dxlo, fminf(a1, a2));
  const float t1max = fmaf(r11, dxhi, fmaxf(a1, a2));
  const float m1 = t1min > 0.f ? t1min : (t1max < 0.f ? -t1max : 0.f);
  const float m2 = dylo > 0.f ? r22 * dylo : (dyhi < 0.f ? -r22 * dyhi : 0.f);
  return fmaf(m1, m1, m2 * m2);
}

// Stage one batch: thread t < cnt loads record vals[b + t] and classifies it
// for every warp footprint; then every warp compacts its own list.
template <int TILE, int WW, int PPT, int CUT, bool BWD>
__device__ __forceinline__ int stage_batch(
    Stage<Layout<TILE, WW, PPT>::NT, Layout<TILE, WW, PPT>::NW, BWD>& S, const WsView& v,
    const uint32_t* __restrict__ vals, uint32_t b, int cnt, int tx, int ty) {
  using Lay = Layout<TILE, WW, PPT>;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __syncthreads();  // the previous batch is consumed
  if (tid < cnt) {
    const uint32_t rid = __ldg(vals + b + tid);
    const float4 a = __ldg(v.rec_a + rid);
    const float4 c = __ldg(v.rec_b + rid);
    const uint2 bx = __ldg(v.rec_box + rid);
    S.a[tid] = a;
    S.b[tid] = c;
    S.box[tid] = bx;
    if (BWD) S.rid[tid] = rid;
    const int j0 = bx.x & 0xffff, j1 = bx.x >> 16, i0 = bx.y & 0xffff, i1 = bx.y >> 16;
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < Lay::NW; ++w) {
      const int fj0 = tx * TILE + (w % Lay::WPR) * WW, fi0 = ty * TILE + (w / Lay::WPR) * Lay::WH;
      const int fj1 = fj0 + WW - 1, fi1 = fi0 + Lay::WH - 1;
      const int xa = max(fj0, j0), xb = min(fj1, j1), ya = max(fi0, i0), yb = min(fi1, i1);
      if (xa > xb || ya > yb) continue;
      const float qmin = min_q_lower_bound(a.z, a.w, c.x, (float)xa + 0.5f - a.x,
                                           (float)xb + 0.5f - a.x, (float)ya + 0.5f - a.y,
                                           (float)yb + 0.5f - a.y);
      if (c.y - qmin < -127.f) continue;                   // every weight is an FP32 zero
      if (CUT && qmin > c.w * 1.0001f + 1e-6f) continue;  // outside the ellipsoid everywhere
      m |= 1u << w;
      if (j0 <= fj0 && j1 >= fj1 && i0 <= fi0 && i1 >= fi1) m |= 1u << (16 + w);
    }
    S.mask[tid] = m;
  }
  __syncthreads();
  int count = 0;
  for (int base = 0; base < cnt; base += 32) {
    const int r = base + lane;
    const uint32_t m = r < cnt ? S.mask[r] : 0u;
    const bool live = (m >> warp) & 1u;
    const uint32_t full = (m >> (16 + warp)) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, live);
    if (live) S.list[warp][count + __popc(bal & lanemask_lt())] = (uint16_t)(r | (full << 15));
    count += __popc(bal);
  }
  __syncwarp();
  return count;
}

template <int TILE, int WW, int PPT, int CUT>
__global__ void __launch_bounds__(Layout<TILE, WW, PPT>::NT)
    k_render_fwd(WsView v, const uint32_t* __restrict__ vals, int P, int total_tiles, float abg,
                 float cbg, float* __restrict__ image, float* __restrict__ alpha) {
  using Lay = Layout<TILE, WW, PPT>;
  constexpr int NT = Lay::NT;
  __shared__ Stage<NT, Lay::NW, false> S;
  if (dev_failed(v.hdr)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wx = warp % Lay::WPR, wy = warp / Lay::WPR;
  const int lx = lane % WW, ly = lane / WW;
  TileCtx tc;
  unsigned long long evaluated = 0;  // (record, footprint) evaluations of this warp
  while (next_tile(v, 0, P, total_tiles, tc, &S.tile, &S.plane)) {
    const int fj0 = tc.tx * TILE + wx * WW, fi0 = tc.ty * TILE + wy * Lay::WH;
    const int j = fj0 + lx;
    const int ib = fi0 + ly * PPT;
    const float pxj = (float)j + 0.5f, pyi = (float)ib + 0.5f;
    const uint2 rg = v.ranges[tc.tile];
    float sa[PPT], sc[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) sa[k] = sc[k] = 0.f;
    for (uint32_t b = rg.x; b < rg.y; b += NT) {
      const int cnt = (int)min((uint32_t)NT, rg.y - b);
      const int nl = stage_batch<TILE, WW, PPT, CUT, false>(S, v, vals, b, cnt, tc.tx, tc.ty);
      evaluated += (unsigned long long)nl;
      for (int e = 0; e < nl; ++e) {
        const uint32_t ent = S.list[warp][e];
        const int r = ent & 0x7fff;
        const float4 a = S.a[r];
        const float4 c = S.b[r];
        const float dx = pxj - a.x, dy = pyi - a.y;
        const float t1 = fmaf(a.z, dx, a.w * dy);
        const float t2 = c.x * dy;
        if (ent & 0x8000u) {  // the box covers the footprint: no per-pixel tests
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            const float t1k = k ? fmaf((float)k, a.w, t1) : t1;
            const float t2k = k ? fmaf((float)k, c.x, t2) : t2;
            float w;
            if (CUT) {
              const float qq = fmaf(t1k, t1k, t2k * t2k);
              w = qq <= c.w ? fast_exp2(c.y - qq) : 0.f;
            } else {
              w = fast_exp2(fmaf(-t1k, t1k, fmaf(-t2k, t2k, c.y)));
            }
            sa[k] += w;
            sc[k] = fmaf(w, c.z, sc[k]);
          }
        } else {
          const uint2 bx = S.box[r];
          const int j0 = bx.x & 0xffff, j1 = bx.x >> 16, i0 = bx.y & 0xffff, i1 = bx.y >> 16;
          const bool jin = (unsigned)(j - j0) <= (unsigned)(j1 - j0);
          const float lw = jin ? c.y : -INFINITY;
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            const float t1k = k ? fmaf((float)k, a.w, t1) : t1;
            const float t2k = k ? fmaf((float)k, c.x, t2) : t2;
            const float qq = fmaf(t1k, t1k, t2k * t2k);
            bool in = (unsigned)(ib + k - i0) <= (unsigned)(i1 - i0);
            if (CUT) in = in && qq <= c.w;
            const float w = in ? fast_exp2(lw - qq) : 0.f;
            sa[k] += w;
            sc[k] = fmaf(w, c.z, sc[k]);
          }
        }
      }
    }
    if (j < tc.w) {
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const int i = ib + k;
        if (i < tc.h) {
          const int64_t px = tc.px_off + (int64_t)i * tc.w + j;
          const float al = sa[k] + abg;
          image[px] = (sc[k] + abg * cbg) / al;
          alpha[px] = al;
        }
      }
    }
  }
  if (lane == 0 && evaluated)
    atomicAdd(reinterpret_cast<unsigned long long*>(&v.hdr->st.evaluated_pairs),
              evaluated * (unsigned long long)(32 * PPT));
}

// Sum of 8 per-lane values over the warp; lane f (0 <= f < 7) returns the
// total of value f. Recursive halving: each exchange sends half of the
// remaining values, so the warp issues 4 + 2 + 1 + 1 + 1 shuffles.
__device__ __forceinline__ float warp_reduce8(float v[8], int lane) {
  float r4[4];
  const bool up16 = lane & 16;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float send = up16 ? v[k] : v[k + 4];
    const float keep = up16 ? v[k + 4] : v[k];
    r4[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float r2[2];
  const bool up8 = lane & 8;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = up8 ? r4[k] : r4[k + 2];
    const float keep = up8 ? r4[k + 2] : r4[k];
    r2[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const bool up4 = lane & 4;
  const float send = up4 ? r2[0] : r2[1];
  const float keep = up4 ? r2[1] : r2[0];
  float r1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  r1 += __shfl_xor_sync(0xffffffffu, r1, 2);
  r1 += __shfl_xor_sync(0xffffffffu, r1, 1);
  // value index held: 4*(lane>>4 & 1) + 2*(lane>>3 & 1) + (lane>>2 & 1)
  return r1;
}

template <int TILE, int WW, int PPT, int CUT>
__global__ void __launch_bounds__(Layout<TILE, WW, PPT>::NT)
    k_render_bwd(WsView v, const uint32_t* __restrict__ vals, int P, int total_tiles,
                 const float* __restrict__ image, const float* __restrict__ alpha,
                 const float* __restrict__ grad_image) {
  using Lay = Layout<TILE, WW, PPT>;
  constexpr int NT = Lay::NT;
  __shared__ Stage<NT, Lay::NW, true> S;
  if (dev_failed(v.hdr)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wx = warp % Lay::WPR, wy = warp / Lay::WPR;
  const int lx = lane % WW, ly = lane / WW;
  // lane -> reduced value index (see warp_reduce8); lanes with (lane & 3) == 0 write
  const int fidx = 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1);
  TileCtx tc;
  unsigned long long evaluated = 0;
  while (next_tile(v, 1, P, total_tiles, tc, &S.tile, &S.plane)) {
    const int fj0 = tc.tx * TILE + wx * WW, fi0 = tc.ty * TILE + wy * Lay::WH;
    const int j = fj0 + lx;
    const int ib = fi0 + ly * PPT;
    const float pxj = (float)j + 0.5f, pyi = (float)ib + 0.5f;
    float rr[PPT], rc[PPT];  // r = G / alpha, r C
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int i = ib + k;
      rr[k] = 0.f;
      rc[k] = 0.f;
      if (j < tc.w && i < tc.h) {
        const int64_t px = tc.px_off + (int64_t)i * tc.w + j;
        const float r = __ldg(grad_image + px) / __ldg(alpha + px);
        rr[k] = r;
        rc[k] = r * __ldg(image + px);
      }
    }
    const uint2 rg = v.ranges[tc.tile];
    for (uint32_t b = rg.x; b < rg.y; b += NT) {
      const int cnt = (int)min((uint32_t)NT, rg.y - b);
      const int nl = stage_batch<TILE, WW, PPT, CUT, true>(S, v, vals, b, cnt, tc.tx, tc.ty);
      evaluated += (unsigned long long)nl;
      for (int e = 0; e < nl; ++e) {
        const uint32_t ent = S.list[warp][e];
        const int r = ent & 0x7fff;
        const float4 a = S.a[r];
        const float4 c = S.b[r];
        const float dx = pxj - a.x, dy = pyi - a.y;
        const float t1 = fmaf(a.z, dx, a.w * dy);
        const float t2 = c.x * dy;
        // Per lane: S0 = sum r w, S1 = sum gww, U1 = sum gww t1, U2 = sum gww t2,
        // K1 = sum k gww t1, K2 = sum k gww t2 over its PPT pixels (row ib + k);
        // then sum u1 dx = dx U1, sum u1 dy = dy U1 + K1, sum u2 dy = dy U2 + K2.
        float s0 = 0.f, s1 = 0.f, U1 = 0.f, U2 = 0.f, K1 = 0.f, K2 = 0.f;
        if (ent & 0x8000u) {  // the box covers the footprint: no per-pixel tests
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            const float t1k = k ? fmaf((float)k, a.w, t1) : t1;
            const float t2k = k ? fmaf((float)k, c.x, t2) : t2;
            float w;
            if (CUT) {
              const float qq = fmaf(t1k, t1k, t2k * t2k);
              w = qq <= c.w ? fast_exp2(c.y - qq) : 0.f;
            } else {
              w = fast_exp2(fmaf(-t1k, t1k, fmaf(-t2k, t2k, c.y)));
            }
            const float gww = fmaf(rr[k], c.z, -rc[k]) * w;  // dL/dw * w
            s0 = fmaf(rr[k], w, s0);
            s1 += gww;
            const float u1 = gww * t1k, u2 = gww * t2k;
            U1 += u1;
            U2 += u2;
            if (k) {
              K1 = fmaf((float)k, u1, K1);
              K2 = fmaf((float)k, u2, K2);
            }
          }
        } else {
          const uint2 bx = S.box[r];
          const int j0 = bx.x & 0xffff, j1 = bx.x >> 16, i0 = bx.y & 0xffff, i1 = bx.y >> 16;
          const float lw = (unsigned)(j - j0) <= (unsigned)(j1 - j0) ? c.y : -INFINITY;
          const int klo = i0 - ib, khi = i1 - ib;
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            const float t1k = k ? fmaf((float)k, a.w, t1) : t1;
            const float t2k = k ? fmaf((float)k, c.x, t2) : t2;
            const float qq = fmaf(t1k, t1k, t2k * t2k);
            bool in = k >= klo && k <= khi;
            if (CUT) in = in && qq <= c.w;
            const float w = in ? fast_exp2(lw - qq) : 0.f;
            const float gww = fmaf(rr[k], c.z, -rc[k]) * w;
            s0 = fmaf(rr[k], w, s0);
            s1 += gww;
            const float u1 = gww * t1k, u2 = gww * t2k;
            U1 += u1;
            U2 += u2;
            if (k) {
              K1 = fmaf((float)k, u1, K1);
              K2 = fmaf((float)k, u2, K2);
            }
          }
        }
        float acc[8];
        acc[0] = s0;
        acc[1] = s1;
        acc[2] = U1;
        acc[3] = U2;
        acc[4] = dx * U1;
        acc[5] = fmaf(dy, U1, K1);
        acc[6] = fmaf(dy, U2, K2);
        acc[7] = 0.f;
        const float tot = warp_reduce8(acc, lane);
        if ((lane & 3) == 0 && fidx < 7) atomicAdd(v.rec_grad + (size_t)S.rid[r] * 8 + fidx, tot);
      }
    }
  }
  if (lane == 0 && evaluated)
    atomicAdd(reinterpret_cast<unsigned long long*>(&v.hdr->st.evaluated_pairs_bwd),
              evaluated * (unsigned long long)(32 * PPT));
}

__global__ void k_zero_rec_grad(WsView v, int64_t cap) {
  if (dev_failed(v.hdr)) return;
  const int64_t nrec = min((int64_t)v.hdr->slots, cap);
  float4* g = reinterpret_cast<float4*>(v.rec_grad);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrec * 2;
       i += (int64_t)gridDim.x * blockDim.x)
    g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ------------------------------------------------------------------ variants
template <int TILE, int WW, int PPT>
struct Variant {
  static constexpr int NT = Layout<TILE, WW, PPT>::NT;
  template <int CUT>
  static cudaError_t fwd(const ug_plan* plan, WsView v, const uint32_t* vals, float* image,
                         float* alpha, cudaStream_t s) {
    static int grid = 0;
    if (grid == 0) {
      int occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_render_fwd<TILE, WW, PPT, CUT>, NT, 0);
      grid = device_sms() * (occ > 0 ? occ : 1);
    }
    const int g = min(grid, max(plan->total_tiles, 1));
    k_render_fwd<TILE, WW, PPT, CUT><<<g, NT, 0, s>>>(v, vals, plan->num_planes, plan->total_tiles,
                                                      plan->cfg.alpha_bg, plan->cfg.c_bg, image,
                                                      alpha);
    return cudaGetLastError();
  }
  template <int CUT>
  static cudaError_t bwd(const ug_plan* plan, WsView v, const uint32_t* vals, const float* image,
                         const float* alpha, const float* grad, cudaStream_t s) {
    static int grid = 0;
    if (grid == 0) {
      int occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_render_bwd<TILE, WW, PPT, CUT>, NT, 0);
      grid = device_sms() * (occ > 0 ? occ : 1);
    }
    const int g = min(grid, max(plan->total_tiles, 1));
    k_render_bwd<TILE, WW, PPT, CUT><<<g, NT, 0, s>>>(v, vals, plan->num_planes,
                                                      plan->total_tiles, image, alpha, grad);
    return cudaGetLastError();
  }
};

// Variant tables. Tile 16: 0 = 8x8 footprints (2 px/lane), 1 = 16x4 (2 px/lane),
// 2 = 8x16 (4 px/lane), 3 = 16x8 (4 px/lane), 4 = one warp per tile (8 px/lane).
// Tile 8: 0 = 8x8 (2 px/lane), 1 = 8x4 (1 px/lane).
template <int CUT>
static cudaError_t dispatch_fwd(const ug_plan* plan, WsView v, const uint32_t* vals, float* image,
                                float* alpha, cudaStream_t s) {
  const int var = plan->cfg.variant;
  if (plan->cfg.tile == 16) {
    switch (var) {
      case 0: return Variant<16, 8, 2>::fwd<CUT>(plan, v, vals, image, alpha, s);
      case 1: return Variant<16, 16, 2>::fwd<CUT>(plan, v, vals, image, alpha, s);
      case 2: return Variant<16, 8, 4>::fwd<CUT>(plan, v, vals, image, alpha, s);
      case 3: return Variant<16, 16, 4>::fwd<CUT>(plan, v, vals, image, alpha, s);
      default: return Variant<16, 16, 8>::fwd<CUT>(plan, v, vals, image, alpha, s);
    }
  }
  switch (var) {
    case 0: return Variant<8, 8, 2>::fwd<CUT>(plan, v, vals, image, alpha, s);
    default: return Variant<8, 8, 1>::fwd<CUT>(plan, v, vals, image, alpha, s);
  }
}

template <int CUT>
static cudaError_t dispatch_bwd(const ug_plan* plan, WsView v, const uint32_t* vals,
                                const float* image, const float* alpha, const float* grad,
                                cudaStream_t s) {
  const int var = plan->cfg.variant_bwd;
  if (plan->cfg.tile == 16) {
    switch (var) {
      case 0: return Variant<16, 8, 2>::bwd<CUT>(plan, v, vals, image, alpha, grad, s);
      case 1: return Variant<16, 16, 2>::bwd<CUT>(plan, v, vals, image, alpha, grad, s);
      case 2: return Variant<16, 8, 4>::bwd<CUT>(plan, v, vals, image, alpha, grad, s);
      case 3: return Variant<16, 16, 4>::bwd<CUT>(plan, v, vals, image, alpha, grad, s);
      default: return Variant<16, 16, 8>::bwd<CUT>(plan, v, vals, image, alpha, grad, s);
    }
  }
  switch (var) {
    case 0: return Variant<8, 8, 2>::bwd<CUT>(plan, v, vals, image, alpha, grad, s);
    default: return Variant<8, 8, 1>::bwd<CUT>(plan, v, vals, image, alpha, grad, s);
  }
}

int num_render_variants(int tile) { return tile == 16 ? 5 : (tile == 8 ? 2 : 0); }

cudaError_t launch_render(const ug_plan* plan, WsView v, float* image, float* alpha,
                          cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&v.hdr->tile_counter[0], 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&v.hdr->st.evaluated_pairs, 0, sizeof(int64_t), s);
  if (e != cudaSuccess) return e;
  const uint32_t* vals = v.vals[plan->sort_passes & 1];
  return plan->cfg.cutoff ? dispatch_fwd<1>(plan, v, vals, image, alpha, s)
                          : dispatch_fwd<0>(plan, v, vals, image, alpha, s);
}

cudaError_t launch_render_backward_raster(const ug_plan* plan, WsView v, const float* image,
                                          const float* alpha, const float* grad_image,
                                          cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&v.hdr->tile_counter[1], 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&v.hdr->st.evaluated_pairs_bwd, 0, sizeof(int64_t), s);
  if (e != cudaSuccess) return e;
  k_zero_rec_grad<<<device_sms() * 4, 256, 0, s>>>(v, plan->record_capacity);
  const uint32_t* vals = v.vals[plan->sort_passes & 1];
  return plan->cfg.cutoff ? dispatch_bwd<1>(plan, v, vals, image, alpha, grad_image, s)
                          : dispatch_bwd<0>(plan, v, vals, image, alpha, grad_image, s);
}

cudaError_t launch_render_backward(const ug_plan* plan, const ug_gaussians* g, WsView v,
                                   const float* image, const float* alpha,
                                   const float* grad_image, const ug_gaussian_grads* grads,
                                   cudaStream_t s) {
  const cudaError_t e = launch_render_backward_raster(plan, v, image, alpha, grad_image, s);
  if (e != cudaSuccess) return e;
  return launch_pre_backward(plan, g, v, grads, s);
}

}  // namespace ug
