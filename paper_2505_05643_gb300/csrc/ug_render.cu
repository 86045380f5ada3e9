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
  static constexpr int NP = (PPT + 1) / 2; // pixel pairs per lane
  static_assert(NT % 32 == 0, "whole warps");
  static_assert(WPR * (TILE / WH) == NW, "warps tile the tile");
  static_assert(NW <= 16, "mask layout");
  static_assert(PPT % 2 == 0, "pixels are processed in pairs");
  // one bit per lane row: lanes ly * WW + lx of column lx = 0
  static constexpr uint32_t rep() {
    uint32_t r = 0;
    for (int i = 0; i < LH; ++i) r |= 1u << (i * WW);
    return r;
  }
};

// Per-lane box masks of one (record, warp footprint) work item: bit `lane` of
// m[k] set when pixel k of that lane lies inside the record's box.
template <int PPT>
struct alignas(PPT >= 4 ? 16 : 4 * PPT) Masks {
  uint32_t m[PPT];
};

// A warp's current chunk of up to 32 work items, one slot per lane of the
// builder, as a structure of arrays (the builder's stores are conflict-free,
// the consumers' loads are broadcasts). The values come in pairs so that the
// packed FP32x2 arithmetic reads them straight from the loaded registers.
template <int PPT>
struct Chunk {
  float4 nxy[32];   // -x*_j, -x*_j, -x*_i, -x*_i
  float4 r1[32];    // r11, r11, r12, r12
  float4 r2[32];    // r22, r22, -lw2, -lw2
  float4 cv[32];    // c, c, ellipsoid threshold, record id (bit pattern)
  Masks<PPT> m[32];
};

// Shared-memory staging of one batch of records, the per-warp lists of the
// records that reach each warp's footprint (records whose box covers the
// footprint from the front, the others from the back), and each warp's chunk.
template <int NT, int NW, int PPT>
struct Stage {
  float4 a[NT];
  float4 b[NT];
  uint2 box[NT];
  uint32_t rid[NT];
  uint32_t mask[NT];          // bit w: live for warp w; bit 16 + w: box covers its footprint
  uint16_t list[NW][NT];
  Chunk<PPT> ch[NW];
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
// for every warp footprint; then every warp compacts its own lists. Returns
// the number of full-box items (list[0, nf)) and sets np, the number of
// partial-box items (list[NT - np, NT), item i at NT - 1 - i).
template <int TILE, int WW, int PPT, int CUT>
__device__ __forceinline__ int stage_batch(
    Stage<Layout<TILE, WW, PPT>::NT, Layout<TILE, WW, PPT>::NW, PPT>& S, const WsView& v,
    const uint32_t* __restrict__ vals, uint32_t b, int cnt, int tx, int ty, int& np) {
  using Lay = Layout<TILE, WW, PPT>;
  constexpr int NT = Lay::NT;
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
    S.rid[tid] = rid;
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
  int nf = 0;
  np = 0;
  const uint32_t lt = lanemask_lt();
  for (int base = 0; base < cnt; base += 32) {
    const int r = base + lane;
    const uint32_t m = r < cnt ? S.mask[r] : 0u;
    const bool live = (m >> warp) & 1u;
    const bool full = (m >> (16 + warp)) & 1u;
    const uint32_t bf = __ballot_sync(0xffffffffu, live && full);
    const uint32_t bp = __ballot_sync(0xffffffffu, live && !full);
    if (live && full) S.list[warp][nf + __popc(bf & lt)] = (uint16_t)r;
    if (live && !full) S.list[warp][NT - 1 - (np + __popc(bp & lt))] = (uint16_t)r;
    nf += __popc(bf);
    np += __popc(bp);
  }
  __syncwarp();
  return nf;
}

// Lane `slot` of a warp fills chunk slot `slot` from list entry `li`: the
// record's data and, for a partial box, the lane masks of box ∩ footprint
// (footprint origin fj0, fi0; lane = ly * WW + lx holds pixels (fi0 + ly PPT + k,
// fj0 + lx), k < PPT).
template <int TILE, int WW, int PPT, bool PARTIAL>
__device__ __forceinline__ void build_entry(
    Stage<Layout<TILE, WW, PPT>::NT, Layout<TILE, WW, PPT>::NW, PPT>& S, int warp, int li,
    int slot, int fj0, int fi0) {
  using Lay = Layout<TILE, WW, PPT>;
  const int r = S.list[warp][li];
  Chunk<PPT>& C = S.ch[warp];
  const float4 a = S.a[r], b = S.b[r];
  C.nxy[slot] = make_float4(-a.x, -a.x, -a.y, -a.y);
  C.r1[slot] = make_float4(a.z, a.z, a.w, a.w);
  C.r2[slot] = make_float4(b.x, b.x, -b.y, -b.y);
  C.cv[slot] = make_float4(b.z, b.z, b.w, __uint_as_float(S.rid[r]));
  if (PARTIAL) {
    const uint2 bx = S.box[r];
    const int j0 = bx.x & 0xffff, j1 = bx.x >> 16, i0 = bx.y & 0xffff, i1 = bx.y >> 16;
    // box ∩ footprint in footprint coordinates (non-empty: the record is live)
    const int cx0 = max(j0 - fj0, 0), cx1 = min(j1 - fj0, WW - 1);
    const int ry0 = max(i0 - fi0, 0), ry1 = min(i1 - fi0, Lay::WH - 1);
    const uint32_t cols = ((2u << cx1) - (1u << cx0)) * Lay::rep();  // 2u << 31 wraps to 0
    Masks<PPT> mk;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      // lane rows ly with ly * PPT + k in [ry0, ry1]
      const int ly0 = ry0 - k <= 0 ? 0 : (ry0 - k + PPT - 1) / PPT;
      const int ly1 = ry1 - k < 0 ? -1 : (ry1 - k) / PPT;
      const uint32_t rows =
          ly0 <= ly1 ? (uint32_t)((1ull << ((ly1 + 1) * WW)) - (1ull << (ly0 * WW))) : 0u;
      mk.m[k] = cols & rows;
    }
    C.m[slot] = mk;
  }
}

// q - lw2 for one lane's pixel pair (rows of py, column of dxx = x - x*_j):
// t1 = r11 dx + r12 dy, t2 = r22 dy, q = t1^2 + t2^2, in packed FP32x2
// arithmetic; the weight is w = 2^-(q - lw2). Pixels outside the box (PARTIAL:
// mask bits m0, m1) or outside the ellipsoid (CUT) get +inf (w = +0).
template <int CUT, bool PARTIAL>
__device__ __forceinline__ float2 pair_qlw(const float4& r1, const float4& r2, const float4& cv,
                                           float2 ny, float2 dxx, float2 py, uint32_t m0,
                                           uint32_t m1, uint32_t lanebit, float2& t1, float2& t2,
                                           float2& dy) {
  dy = __fadd2_rn(py, ny);
  t1 = __ffma2_rn(make_float2(r1.x, r1.y), dxx, __fmul2_rn(make_float2(r1.z, r1.w), dy));
  t2 = __fmul2_rn(make_float2(r2.x, r2.y), dy);
  float2 e;
  if (CUT) {
    const float2 q = __ffma2_rn(t1, t1, __fmul2_rn(t2, t2));
    e = __fadd2_rn(q, make_float2(r2.z, r2.w));
    if (!(q.x <= cv.z)) e.x = INFINITY;
    if (!(q.y <= cv.z)) e.y = INFINITY;
  } else {
    e = __ffma2_rn(t1, t1, __ffma2_rn(t2, t2, make_float2(r2.z, r2.w)));
  }
  if (PARTIAL) {
    if (!(m0 & lanebit)) e.x = INFINITY;
    if (!(m1 & lanebit)) e.y = INFINITY;
  }
  return e;
}

template <int PPT, int CUT, bool PARTIAL>
__device__ __forceinline__ void fwd_item(const Chunk<PPT>& C, int e, float2 pxx, const float2* py,
                                         uint32_t lanebit, float2* sa, float2* sc) {
  const float4 nxy = C.nxy[e], r1 = C.r1[e], r2 = C.r2[e], cv = C.cv[e];
  Masks<PPT> mk;
  if (PARTIAL) mk = C.m[e];
  const float2 dxx = __fadd2_rn(pxx, make_float2(nxy.x, nxy.y));
  const float2 ny = make_float2(nxy.z, nxy.w);
#pragma unroll
  for (int p = 0; p < PPT / 2; ++p) {
    float2 t1, t2, dy;
    const float2 e2 = pair_qlw<CUT, PARTIAL>(r1, r2, cv, ny, dxx, py[p],
                                             PARTIAL ? mk.m[2 * p] : 0u,
                                             PARTIAL ? mk.m[2 * p + 1] : 0u, lanebit, t1, t2, dy);
    const float2 w = make_float2(fast_exp2(-e2.x), fast_exp2(-e2.y));
    sa[p] = __fadd2_rn(sa[p], w);
    sc[p] = __ffma2_rn(w, make_float2(cv.x, cv.y), sc[p]);
  }
}

template <int TILE, int WW, int PPT, int CUT>
__global__ void __launch_bounds__(Layout<TILE, WW, PPT>::NT)
    k_render_fwd(WsView v, const uint32_t* __restrict__ vals, int P, int total_tiles, float abg,
                 float cbg, float* __restrict__ image, float* __restrict__ alpha) {
  using Lay = Layout<TILE, WW, PPT>;
  constexpr int NT = Lay::NT, NP = Lay::NP;
  __shared__ Stage<NT, Lay::NW, PPT> S;
  if (dev_failed(v.hdr)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wx = warp % Lay::WPR, wy = warp / Lay::WPR;
  const int lx = lane % WW, ly = lane / WW;
  const uint32_t lanebit = 1u << lane;
  TileCtx tc;
  unsigned long long evaluated = 0;  // (record, footprint) evaluations of this warp
  while (next_tile(v, 0, P, total_tiles, tc, &S.tile, &S.plane)) {
    const int fj0 = tc.tx * TILE + wx * WW, fi0 = tc.ty * TILE + wy * Lay::WH;
    const int j = fj0 + lx;
    const int ib = fi0 + ly * PPT;
    const float2 pxx = make_float2((float)j + 0.5f, (float)j + 0.5f);
    float2 py[NP], sa[NP], sc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      py[p] = make_float2((float)(ib + 2 * p) + 0.5f, (float)(ib + 2 * p + 1) + 0.5f);
      sa[p] = sc[p] = make_float2(0.f, 0.f);
    }
    const Chunk<PPT>& C = S.ch[warp];
    const uint2 rg = v.ranges[tc.tile];
    for (uint32_t b = rg.x; b < rg.y; b += NT) {
      const int cnt = (int)min((uint32_t)NT, rg.y - b);
      int np;
      const int nf = stage_batch<TILE, WW, PPT, CUT>(S, v, vals, b, cnt, tc.tx, tc.ty, np);
      evaluated += (unsigned long long)(nf + np);
      for (int base = 0; base < nf; base += 32) {
        if (base + lane < nf) build_entry<TILE, WW, PPT, false>(S, warp, base + lane, lane, fj0, fi0);
        __syncwarp();
        const int ne = min(32, nf - base);
        int e = 0;
        for (; e + 2 <= ne; e += 2) {
          fwd_item<PPT, CUT, false>(C, e, pxx, py, lanebit, sa, sc);
          fwd_item<PPT, CUT, false>(C, e + 1, pxx, py, lanebit, sa, sc);
        }
        if (e < ne) fwd_item<PPT, CUT, false>(C, e, pxx, py, lanebit, sa, sc);
        __syncwarp();
      }
      for (int base = 0; base < np; base += 32) {
        if (base + lane < np)
          build_entry<TILE, WW, PPT, true>(S, warp, NT - 1 - (base + lane), lane, fj0, fi0);
        __syncwarp();
        const int ne = min(32, np - base);
        int e = 0;
        for (; e + 2 <= ne; e += 2) {
          fwd_item<PPT, CUT, true>(C, e, pxx, py, lanebit, sa, sc);
          fwd_item<PPT, CUT, true>(C, e + 1, pxx, py, lanebit, sa, sc);
        }
        if (e < ne) fwd_item<PPT, CUT, true>(C, e, pxx, py, lanebit, sa, sc);
        __syncwarp();
      }
    }
    if (j < tc.w) {
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const int i = ib + k;
        if (i < tc.h) {
          const int64_t px = tc.px_off + (int64_t)i * tc.w + j;
          const float sak = (k & 1) ? sa[k >> 1].y : sa[k >> 1].x;
          const float sck = (k & 1) ? sc[k >> 1].y : sc[k >> 1].x;
          const float al = sak + abg;
          image[px] = (sck + abg * cbg) / al;
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

// Per lane and work item (Eq. us-render differentiated, box fixed): with
// G = dL/dC, r = G / alpha and dL/dw = r (c - C) at each pixel,
//   acc0 = sum r w                (dL/dc),
//   acc1 = sum g,   g = w dL/dw   (dL/dlw2 / ln 2),
//   acc2 = sum g t1, acc3 = sum g t2,
//   acc4 = sum g t1 dx, acc5 = sum g t1 dy, acc6 = sum g t2 dy
// over the lane's pixels; the chain kernel turns the warp totals into the
// gradients of x*, r11, r12, r22. Returns the record id.
template <int PPT, int CUT, bool PARTIAL>
__device__ __forceinline__ uint32_t bwd_item(const Chunk<PPT>& C, int e, float2 pxx,
                                             const float2* py, const float2* rr,
                                             const float2* nrc, uint32_t lanebit, float acc[8]) {
  const float4 nxy = C.nxy[e], r1 = C.r1[e], r2 = C.r2[e], cv = C.cv[e];
  Masks<PPT> mk;
  if (PARTIAL) mk = C.m[e];
  const float2 dxx = __fadd2_rn(pxx, make_float2(nxy.x, nxy.y));
  const float2 ny = make_float2(nxy.z, nxy.w), cc = make_float2(cv.x, cv.y);
  float2 s0, s1, u1s, u2s, a5, a6;
#pragma unroll
  for (int p = 0; p < PPT / 2; ++p) {
    float2 t1, t2, dy;
    const float2 e2 = pair_qlw<CUT, PARTIAL>(r1, r2, cv, ny, dxx, py[p],
                                             PARTIAL ? mk.m[2 * p] : 0u,
                                             PARTIAL ? mk.m[2 * p + 1] : 0u, lanebit, t1, t2, dy);
    const float2 w = make_float2(fast_exp2(-e2.x), fast_exp2(-e2.y));
    const float2 g = __fmul2_rn(__ffma2_rn(rr[p], cc, nrc[p]), w);  // w dL/dw
    const float2 u1 = __fmul2_rn(g, t1), u2 = __fmul2_rn(g, t2);
    if (p == 0) {
      s0 = __fmul2_rn(rr[p], w);
      s1 = g;
      u1s = u1;
      u2s = u2;
      a5 = __fmul2_rn(u1, dy);
      a6 = __fmul2_rn(u2, dy);
    } else {
      s0 = __ffma2_rn(rr[p], w, s0);
      s1 = __fadd2_rn(s1, g);
      u1s = __fadd2_rn(u1s, u1);
      u2s = __fadd2_rn(u2s, u2);
      a5 = __ffma2_rn(u1, dy, a5);
      a6 = __ffma2_rn(u2, dy, a6);
    }
  }
  acc[0] = s0.x + s0.y;
  acc[1] = s1.x + s1.y;
  acc[2] = u1s.x + u1s.y;
  acc[3] = u2s.x + u2s.y;
  acc[4] = dxx.x * acc[2];
  acc[5] = a5.x + a5.y;
  acc[6] = a6.x + a6.y;
  acc[7] = 0.f;
  return __float_as_uint(cv.w);
}

// Work items e and e + 1 of the chunk, interleaved, each reduced over the
// warp and added to its record's accumulators.
template <int PPT, int CUT, bool PARTIAL, bool TWO>
__device__ __forceinline__ void bwd_items(const Chunk<PPT>& C, int e, float2 pxx,
                                          const float2* py, const float2* rr, const float2* nrc,
                                          uint32_t lanebit, int lane, int fidx, float* rec_grad) {
  float acc0[8], acc1[8];
  const uint32_t rid0 = bwd_item<PPT, CUT, PARTIAL>(C, e, pxx, py, rr, nrc, lanebit, acc0);
  uint32_t rid1 = 0;
  if (TWO) rid1 = bwd_item<PPT, CUT, PARTIAL>(C, e + 1, pxx, py, rr, nrc, lanebit, acc1);
  const float tot0 = warp_reduce8(acc0, lane);
  float tot1 = 0.f;
  if (TWO) tot1 = warp_reduce8(acc1, lane);
  if ((lane & 3) == 0 && fidx < 7) {
    atomicAdd(rec_grad + (size_t)rid0 * 8 + fidx, tot0);
    if (TWO) atomicAdd(rec_grad + (size_t)rid1 * 8 + fidx, tot1);
  }
}

template <int TILE, int WW, int PPT, int CUT>
__global__ void __launch_bounds__(Layout<TILE, WW, PPT>::NT)
    k_render_bwd(WsView v, const uint32_t* __restrict__ vals, int P, int total_tiles,
                 const float* __restrict__ image, const float* __restrict__ alpha,
                 const float* __restrict__ grad_image) {
  using Lay = Layout<TILE, WW, PPT>;
  constexpr int NT = Lay::NT, NP = Lay::NP;
  __shared__ Stage<NT, Lay::NW, PPT> S;
  if (dev_failed(v.hdr)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wx = warp % Lay::WPR, wy = warp / Lay::WPR;
  const int lx = lane % WW, ly = lane / WW;
  const uint32_t lanebit = 1u << lane;
  // lane -> reduced value index (see warp_reduce8); lanes with (lane & 3) == 0 write
  const int fidx = 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1);
  TileCtx tc;
  unsigned long long evaluated = 0;
  while (next_tile(v, 1, P, total_tiles, tc, &S.tile, &S.plane)) {
    const int fj0 = tc.tx * TILE + wx * WW, fi0 = tc.ty * TILE + wy * Lay::WH;
    const int j = fj0 + lx;
    const int ib = fi0 + ly * PPT;
    const float2 pxx = make_float2((float)j + 0.5f, (float)j + 0.5f);
    float2 py[NP], rr[NP], nrc[NP];  // row centres; r = G / alpha and -r C per pixel
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      py[p] = make_float2((float)(ib + 2 * p) + 0.5f, (float)(ib + 2 * p + 1) + 0.5f);
      float r2[2] = {0.f, 0.f}, c2[2] = {0.f, 0.f};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = ib + 2 * p + h;
        if (j < tc.w && i < tc.h) {
          const int64_t px = tc.px_off + (int64_t)i * tc.w + j;
          const float r = __ldg(grad_image + px) / __ldg(alpha + px);
          r2[h] = r;
          c2[h] = -r * __ldg(image + px);
        }
      }
      rr[p] = make_float2(r2[0], r2[1]);
      nrc[p] = make_float2(c2[0], c2[1]);
    }
    const Chunk<PPT>& C = S.ch[warp];
    const uint2 rg = v.ranges[tc.tile];
    for (uint32_t b = rg.x; b < rg.y; b += NT) {
      const int cnt = (int)min((uint32_t)NT, rg.y - b);
      int np;
      const int nf = stage_batch<TILE, WW, PPT, CUT>(S, v, vals, b, cnt, tc.tx, tc.ty, np);
      evaluated += (unsigned long long)(nf + np);
      for (int base = 0; base < nf; base += 32) {
        if (base + lane < nf) build_entry<TILE, WW, PPT, false>(S, warp, base + lane, lane, fj0, fi0);
        __syncwarp();
        const int ne = min(32, nf - base);
        int e = 0;
        for (; e + 2 <= ne; e += 2)
          bwd_items<PPT, CUT, false, true>(C, e, pxx, py, rr, nrc, lanebit, lane, fidx, v.rec_grad);
        if (e < ne)
          bwd_items<PPT, CUT, false, false>(C, e, pxx, py, rr, nrc, lanebit, lane, fidx, v.rec_grad);
        __syncwarp();
      }
      for (int base = 0; base < np; base += 32) {
        if (base + lane < np)
          build_entry<TILE, WW, PPT, true>(S, warp, NT - 1 - (base + lane), lane, fj0, fi0);
        __syncwarp();
        const int ne = min(32, np - base);
        int e = 0;
        for (; e + 2 <= ne; e += 2)
          bwd_items<PPT, CUT, true, true>(C, e, pxx, py, rr, nrc, lanebit, lane, fidx, v.rec_grad);
        if (e < ne)
          bwd_items<PPT, CUT, true, false>(C, e, pxx, py, rr, nrc, lanebit, lane, fidx, v.rec_grad);
        __syncwarp();
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
// Tile 8: 0 = one 8x8 footprint (2 px/lane).
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
  return Variant<8, 8, 2>::fwd<CUT>(plan, v, vals, image, alpha, s);
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
  return Variant<8, 8, 2>::bwd<CUT>(plan, v, vals, image, alpha, grad, s);
}

int num_render_variants(int tile) { return tile == 16 ? 5 : (tile == 8 ? 1 : 0); }

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
