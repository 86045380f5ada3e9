// Internal definitions shared by the CUDA translation units of libug:
// workspace layout, the device-side plane table, status handling and small
// warp/block primitives.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ug.h"

namespace ug {

constexpr int kChunk = 32;        // Gaussians per warp chunk in the preprocess passes
constexpr int kScanItems = 2048;  // entries per block of the count scan
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;    // keys per thread per sort block
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kMseBlocks = 1024;  // partial sums of the MSE loss
constexpr int kChainFloats = 16;  // per-record inputs of the backward chain

// Workspace sections (indices into ug_plan::off).
enum WsSection {
  kOffHeader = 0,
  kOffPlanes,
  kOffTileOff,
  kOffGFlag,     // per chunk: ballot of Gaussians whose covariance inverse runs in FP64
  kOffMask,      // per (chunk, plane): candidate record bits
  kOffSlotBase,  // per (chunk, plane): first record slot
  kOffF64Base,   // per (chunk, plane): first FP64 list entry
  kOffScanPart,  // partials of the (chunk, plane) scan
  kOffList,      // record work list: uint4 (gaussian, plane, slot, 0); FP32 part then FP64 part
  kOffRecA,
  kOffRecB,
  kOffRecC,
  kOffRecBox,
  kOffRecPlane,
  kOffInstOff,   // per record: tile count, scanned in place to the first instance
  kOffSlotPart,  // partials of the record scan
  kOffKeys0,
  kOffKeys1,
  kOffVals0,
  kOffVals1,
  kOffSortHist,
  kOffSortPart,
  kOffRanges,
  kOffRecGrad,   // per record: 8 accumulators of the backward rasterizer
  kOffRecPGrad,  // per record: gradient of the Gaussian's parameters (12 floats)
  kOffRecChain,  // per record: geometry the backward chain needs (kChainFloats floats)
  kOffEnd
};

// Header at the start of the workspace (256 bytes).
struct WsHeader {
  ug_ws_status st;            // 64 B, copied out by ug_read_status
  uint32_t tile_counter[2];   // persistent-kernel work queues (forward, backward)
  uint32_t slots, slots64;    // record slots and FP64 list entries of the last preprocess
  unsigned long long box_pixels;
  uint32_t holes;             // candidates rejected by the exact test (empty slots)
  uint32_t kept64;            // visible records of the FP64 list
  uint32_t pad0;
  uint32_t stall_test;        // non-zero: the rasterizers' producers issue nothing (test hook;
                              // cleared by the preprocess)
  float origin_reach;         // largest |o| over the planes (set by the plane set-up)
  uint32_t pad1[37];
};
static_assert(sizeof(WsHeader) == 256, "header size");

// Derived per-plane data (128 bytes), written by the plane set-up kernel.
struct PlaneDev {
  float o[3], u[3], v[3], n[3];
  float pu, pv, inv_pu, inv_pv;
  float half_w, half_h;       // width/2, height/2
  float jshift, ishift;       // width/2 - 1/2, height/2 - 1/2
  int32_t w, h, tiles_x, tiles_y;
  int32_t tile_off, pad;
  int64_t px_off;
  int32_t pad2[4];
};
static_assert(sizeof(PlaneDev) == 128, "plane size");

// Render-side record of one visible (plane, Gaussian) pair: three float4 and
// the pixel box. Pixel coordinates put the centre of pixel (i, j) at
// (j + 1/2, i + 1/2); X, Y below are relative to the box's first column j0 and
// row i0, so pixel (i, j) sits at (j - j0 + 1/2, i - i0 + 1/2).
//  a = (X, Y, r11, kappa)   high parts,
//  c = (X', Y', kappa', 0)  low parts (|low| <= ulp(high) / 2): the in-plane
//      peak x* = (X + X', Y + Y') and kappa + kappa' = r12 / r11 to double-word
//      accuracy;
//  b = (r22, lw2, c, e_thr): lw2 = log2(alpha) - (log2 e / 2) q0, intensity,
//      ellipsoid threshold (log2 e / 2)(chi2 - q0);
//  box = (j0 | j1 << 16, i0 | i1 << 16).
// (r11, r12, r22) is the upper Cholesky factor of (log2 e / 2) D A D, D =
// diag(pitch_u, pitch_v), A the in-plane precision. Weight at pixel (i, j):
//   w = exp2(lw2 - t1^2 - t2^2),  t1 = r11 (dx + kappa dy),  t2 = r22 dy,
//   dx = j - j0 + 1/2 - X,  dy = i - i0 + 1/2 - Y.
// For a thin Gaussian r11 dx and r11 kappa dy are far larger than t1 and
// cancel; the rasterizers therefore form t1 = r11 (x - S(y)) from the row's
// crossing S(y) = X - kappa (y - Y), which they hold to double-word accuracy
// (item_geo below).

struct WsView {
  WsHeader* hdr;
  PlaneDev* planes;
  int32_t* tile_off;
  uint32_t* gflag;
  uint32_t* mask;
  uint32_t* slot_base;
  uint32_t* f64_base;
  unsigned long long* scan_part;
  uint4* list;
  float4* rec_a;
  float4* rec_b;
  float4* rec_c;
  uint2* rec_box;
  uint32_t* rec_plane;
  uint32_t* inst_off;
  unsigned long long* slot_part;
  uint32_t* keys[2];
  uint32_t* vals[2];
  uint32_t* sort_hist;
  unsigned long long* sort_part;
  uint2* ranges;
  float* rec_grad;   // 8 floats per record
  float* rec_pgrad;  // 12 floats per record
  float* rec_chain;  // kChainFloats floats per record
};

inline WsView make_view(const ug_plan* plan, void* ws) {
  char* b = static_cast<char*>(ws);
  WsView v;
  v.hdr = reinterpret_cast<WsHeader*>(b + plan->off[kOffHeader]);
  v.planes = reinterpret_cast<PlaneDev*>(b + plan->off[kOffPlanes]);
  v.tile_off = reinterpret_cast<int32_t*>(b + plan->off[kOffTileOff]);
  v.gflag = reinterpret_cast<uint32_t*>(b + plan->off[kOffGFlag]);
  v.mask = reinterpret_cast<uint32_t*>(b + plan->off[kOffMask]);
  v.slot_base = reinterpret_cast<uint32_t*>(b + plan->off[kOffSlotBase]);
  v.f64_base = reinterpret_cast<uint32_t*>(b + plan->off[kOffF64Base]);
  v.scan_part = reinterpret_cast<unsigned long long*>(b + plan->off[kOffScanPart]);
  v.list = reinterpret_cast<uint4*>(b + plan->off[kOffList]);
  v.rec_a = reinterpret_cast<float4*>(b + plan->off[kOffRecA]);
  v.rec_b = reinterpret_cast<float4*>(b + plan->off[kOffRecB]);
  v.rec_c = reinterpret_cast<float4*>(b + plan->off[kOffRecC]);
  v.rec_box = reinterpret_cast<uint2*>(b + plan->off[kOffRecBox]);
  v.rec_plane = reinterpret_cast<uint32_t*>(b + plan->off[kOffRecPlane]);
  v.inst_off = reinterpret_cast<uint32_t*>(b + plan->off[kOffInstOff]);
  v.slot_part = reinterpret_cast<unsigned long long*>(b + plan->off[kOffSlotPart]);
  v.keys[0] = reinterpret_cast<uint32_t*>(b + plan->off[kOffKeys0]);
  v.keys[1] = reinterpret_cast<uint32_t*>(b + plan->off[kOffKeys1]);
  v.vals[0] = reinterpret_cast<uint32_t*>(b + plan->off[kOffVals0]);
  v.vals[1] = reinterpret_cast<uint32_t*>(b + plan->off[kOffVals1]);
  v.sort_hist = reinterpret_cast<uint32_t*>(b + plan->off[kOffSortHist]);
  v.sort_part = reinterpret_cast<unsigned long long*>(b + plan->off[kOffSortPart]);
  v.ranges = reinterpret_cast<uint2*>(b + plan->off[kOffRanges]);
  v.rec_grad = reinterpret_cast<float*>(b + plan->off[kOffRecGrad]);
  v.rec_pgrad = reinterpret_cast<float*>(b + plan->off[kOffRecPGrad]);
  v.rec_chain = reinterpret_cast<float*>(b + plan->off[kOffRecChain]);
  return v;
}

// Number of blocks of the count scan and of a sort pass.
__host__ __device__ inline int64_t scan_blocks(int64_t entries) { return (entries + kScanItems - 1) / kScanItems; }
inline int64_t sort_blocks(int64_t capacity) { return (capacity + kSortTile - 1) / kSortTile; }

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ void dev_fail(WsHeader* h, int code, int detail) {
  if (atomicCAS(&h->st.status, 0, code) == 0) h->st.detail = detail;
}

__device__ __forceinline__ bool dev_failed(const WsHeader* h) {
  return *(volatile const int32_t*)&h->st.status != 0;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Inclusive warp prefix sum.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// exp2 on the special-function unit (PTX ex2.approx.ftz.f32: relative error
// about 2^-22 over the range used here; exp2 of very negative numbers flushes
// to +0).
__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 2^-x on the special-function unit (the negation is exact; +inf gives +0).
__device__ __forceinline__ float fast_exp2_neg(float x) {
  float y;
  asm("{\n\t.reg .f32 t;\n\tneg.f32 t, %1;\n\tex2.approx.ftz.f32 %0, t;\n\t}"
      : "=f"(y)
      : "f"(x));
  return y;
}

// Lower bound of q = t1^2 + t2^2 over the pixel centres of the rectangle
// [xa, xb] x [ya, yb] (pixel indices) for a record (a = rec_a, r22) whose box
// starts at (j0, i0). Along a row y, t1 / r11 = x - S(y) with the crossing
// S(y) = X - kappa (y - Y); t1 is linear, so its range over the rectangle
// comes from the corners, and min |t2| from the first and last row. The FP32
// evaluation uses the high parts only; e1 and e2 bound its rounding errors and
// the omitted low parts (each at most 2^-24 of its high part), so the result
// is a lower bound for the exact record values, which the rasterizers
// reproduce to a few ulps. Explicit round-to-nearest intrinsics: the binning's
// passes and the rasterizers take the same decision from the same floats.
__device__ __forceinline__ float rect_q_lower_bound(const float4& a, float r22, int j0, int i0,
                                                    int xa, int xb, int ya, int yb) {
  const float eps = 5.9604645e-8f;  // 2^-24
  const float xlo = __fadd_rn((float)(xa - j0), 0.5f), xhi = __fadd_rn((float)(xb - j0), 0.5f);
  const float ylo = __fadd_rn((float)(ya - i0), 0.5f), yhi = __fadd_rn((float)(yb - i0), 0.5f);
  const float dylo = __fsub_rn(ylo, a.y), dyhi = __fsub_rn(yhi, a.y);
  const float slo = __fmaf_rn(-a.w, dylo, a.x), shi = __fmaf_rn(-a.w, dyhi, a.x);
  // the least and greatest of the four corner differences x - s: rounding is
  // monotone, so they are xlo - max(s) and xhi - min(s), rounded once
  const float umin = __fsub_rn(xlo, fmaxf(slo, shi)), umax = __fsub_rn(xhi, fminf(slo, shi));
  const float ady = fmaxf(fabsf(dylo), fabsf(dyhi)), ay = fabsf(a.y);
  const float e1 = __fmul_rn(
      4.f * eps, __fadd_rn(__fadd_rn(fmaxf(fabsf(umin), fabsf(umax)), fmaxf(fabsf(slo), fabsf(shi))),
                           __fadd_rn(fabsf(a.x), __fmul_rn(fabsf(a.w), __fadd_rn(2.f * ady, ay)))));
  const float e2 = __fmul_rn(4.f * eps, __fadd_rn(ady, ay));
  // distance of [umin, umax] from [-e1, e1]: umin - e1 above it, -umax - e1
  // below it (umin <= umax, so at most one is positive), else 0
  const float m1 = fmaxf(__fsub_rn(fmaxf(umin, -umax), e1), 0.f);
  const float m2 = fmaxf(__fsub_rn(fmaxf(dylo, -dyhi), e2), 0.f);  // likewise (dylo <= dyhi)
  const float t1 = __fmul_rn(a.z, m1), t2 = __fmul_rn(r22, m2);
  return __fmaf_rn(t1, t1, __fmul_rn(t2, t2));
}

// Whether a record (a = rec_a, b = rec_b, box origin (j0, i0)) can have a
// non-zero weight at any pixel of the rectangle. Below an exponent of -126,
// 2^e is subnormal and ex2.approx.ftz returns +0; the test uses -127, so the
// rounding of the rasterizers' q cannot bring a dropped pixel's weight above
// zero. With cut, pixels beyond the ellipsoid threshold b.w are zero as well.
__device__ __forceinline__ bool rect_live(const float4& a, const float4& b, int j0, int i0, int xa,
                                          int xb, int ya, int yb, int cut) {
  const float q = rect_q_lower_bound(a, b.x, j0, i0, xa, xb, ya, yb);
  // without branches (bitwise &): lanes of a warp test different records
  return !(__fsub_rn(b.y, q) < -127.f) & !((cut != 0) & (q > __fmaf_rn(b.w, 1.0001f, 1e-6f)));
}

// Sorted instance keys: the (plane, tile) id in the low kKeyTileBits bits;
// the top byte holds the instance's footprint tests, computed once by the
// binning for both rasterizers: for the f-th 8 x 8 footprint of the tile (row
// major), bit 2f says the record can have a non-zero weight there and bit
// 2f + 1 that its box covers the whole footprint. The sort's digits come from
// the low bits only, so the tests travel with their instance.
constexpr int kKeyTileBits = 24;
constexpr uint32_t kKeyTileMask = (1u << kKeyTileBits) - 1u;

// Work-item test of one record (a = rec_a, b = rec_b, pixel box bx) against
// the footprint [fj0, fj0 + 7] x [fi0, fi0 + fh - 1]: bit 0 live (the box
// overlaps it and not every weight there is an FP32 zero), bit 1 the box
// covers it. Branch-free: the lanes of a warp test different records.
__device__ __forceinline__ uint32_t footprint_bits(const float4& a, const float4& b, uint2 bx,
                                                   int fj0, int fi0, int fh, int cut) {
  const int j0 = bx.x & 0xffff, j1 = bx.x >> 16, i0 = bx.y & 0xffff, i1 = bx.y >> 16;
  const int fj1 = fj0 + 7, fi1 = fi0 + fh - 1;
  const int xa = max(fj0, j0), xb = min(fj1, j1), ya = max(fi0, i0), yb = min(fi1, i1);
  // overlap, and not every weight in it an FP32 zero (the bound of an empty
  // overlap is finite and ignored)
  const bool live = (xa <= xb) & (ya <= yb) & rect_live(a, b, j0, i0, xa, xb, ya, yb, cut);
  const bool full = (j0 <= fj0) & (j1 >= fj1) & (i0 <= fi0) & (i1 >= fi1);
  return (uint32_t)live | ((uint32_t)(live & full) << 1);
}

// footprint_bits for the four 8x8 footprints of the 16x16 tile whose first
// pixel is (tj, ti), bits 2f and 2f + 1 for footprint f (row major): the
// terms that depend only on a footprint row (the crossings S at its first and
// last row, t2, the rounding bounds) or column are computed once, and each
// footprint combines them with the operations of rect_q_lower_bound, in the
// same order, so every test gives footprint_bits' result.
__device__ __forceinline__ uint32_t tile_footprints16(const float4& a, const float4& b, uint2 bx,
                                                      int tj, int ti, int cut) {
  const float eps = 5.9604645e-8f;  // 2^-24
  const int j0 = bx.x & 0xffff, j1 = bx.x >> 16, i0 = bx.y & 0xffff, i1 = bx.y >> 16;
  const float ay = fabsf(a.y), ax = fabsf(a.x), aw = fabsf(a.w);
  const float thr = __fmaf_rn(b.w, 1.0001f, 1e-6f);
  float xlo[2], xhi[2];
  bool xok[2], xfull[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int f0 = tj + 8 * k, xa = max(f0, j0), xb = min(f0 + 7, j1);
    xok[k] = xa <= xb;
    xfull[k] = (j0 <= f0) & (j1 >= f0 + 7);
    xlo[k] = __fadd_rn((float)(xa - j0), 0.5f);
    xhi[k] = __fadd_rn((float)(xb - j0), 0.5f);
  }
  uint32_t fm = 0;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int f0 = ti + 8 * r, ya = max(f0, i0), yb = min(f0 + 7, i1);
    const bool yok = ya <= yb, yfull = (i0 <= f0) & (i1 >= f0 + 7);
    const float ylo = __fadd_rn((float)(ya - i0), 0.5f), yhi = __fadd_rn((float)(yb - i0), 0.5f);
    const float dylo = __fsub_rn(ylo, a.y), dyhi = __fsub_rn(yhi, a.y);
    const float slo = __fmaf_rn(-a.w, dylo, a.x), shi = __fmaf_rn(-a.w, dyhi, a.x);
    const float s_hi = fmaxf(slo, shi), s_lo = fminf(slo, shi);
    const float ady = fmaxf(fabsf(dylo), fabsf(dyhi));
    const float smax = fmaxf(fabsf(slo), fabsf(shi));
    const float es = __fadd_rn(ax, __fmul_rn(aw, __fadd_rn(2.f * ady, ay)));
    const float e2 = __fmul_rn(4.f * eps, __fadd_rn(ady, ay));
    const float m2 = fmaxf(__fsub_rn(fmaxf(dylo, -dyhi), e2), 0.f);
    const float t2 = __fmul_rn(b.x, m2);
    const float t2sq = __fmul_rn(t2, t2);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float umin = __fsub_rn(xlo[k], s_hi), umax = __fsub_rn(xhi[k], s_lo);
      const float e1 =
          __fmul_rn(4.f * eps, __fadd_rn(__fadd_rn(fmaxf(fabsf(umin), fabsf(umax)), smax), es));
      const float m1 = fmaxf(__fsub_rn(fmaxf(umin, -umax), e1), 0.f);
      const float t1 = __fmul_rn(a.z, m1);
      const float q = __fmaf_rn(t1, t1, t2sq);
      const bool live = xok[k] & yok & !(__fsub_rn(b.y, q) < -127.f) &
                        !((cut != 0) & (q > thr));
      const uint32_t bits = (uint32_t)live | ((uint32_t)(live & xfull[k] & yfull) << 1);
      fm |= bits << (2 * (2 * r + k));
    }
  }
  return fm;
}

// Constants of one record over a region of at most SPAN x SPAN pixels (a
// footprint or a whole tile) whose first pixel is (fi0, fj0). With col, row
// the pixel's offsets in the region:
//   t1 = r11 (col + nsh(row)) + nrs(row),  t2 = r22 dy(row),
//   nsh(row) = kq row - s0q,  nrs(row) = a1 row + a0,  dy(row) = (row + nyh) + nyl.
// S0 = s0q + s0l is the crossing at row 0 in double words (the region's
// anchor is subtracted first, so S0 stays small), and kappa = kq + kl. s0q and
// kq are rounded to the grid G = 2^(E - 21), E = floor(log2 B), B >= |S0| +
// SPAN |kappa| + SPAN: every nsh(row) and col + nsh(row) is then a multiple of
// G below 2^22 G, so both are exact in FP32, and the low parts (s0l, kl, at
// most G / 2 plus the double word's own) enter through nrs in FP32. t1 thus
// carries a few ulps of relative error whatever r11 dx and r11 kappa dy are
// (see the record comment above).
struct ItemGeo {
  float r11, kq, ns0q, a1, a0, nyh, nyl, r22;
};

template <int SPAN = 8>
__device__ __forceinline__ ItemGeo item_geo(const float4& a, const float4& b, const float4& c,
                                            uint2 bx, int fj0, int fi0) {
  static_assert(SPAN == 8 || SPAN == 16, "region edge");
  const int j0 = bx.x & 0xffff, i0 = bx.y & 0xffff;
  const float ox = __fadd_rn((float)(fj0 - j0), 0.5f), oy = __fadd_rn((float)(fi0 - i0), 0.5f);
  // Xf = X - ox, Yf = Y - oy in double words (Knuth's 2Sum)
  auto two_sum = [](float p, float q, float& s, float& e) {
    s = __fadd_rn(p, q);
    const float pp = __fsub_rn(s, q), qq = __fsub_rn(s, pp);
    e = __fadd_rn(__fsub_rn(p, pp), __fsub_rn(q, qq));
  };
  float xh, xe, yh, ye;
  two_sum(a.x, -ox, xh, xe);
  two_sum(a.y, -oy, yh, ye);
  const float xl = __fadd_rn(c.x, xe), yl = __fadd_rn(c.y, ye);
  // S0 = Xf + kappa Yf: 2Prod of the high parts, the cross terms in FP32
  const float ph = __fmul_rn(a.w, yh);
  float pl = __fmaf_rn(a.w, yh, -ph);
  pl = __fmaf_rn(a.w, yl, pl);
  pl = __fmaf_rn(c.z, yh, pl);
  float sh, se;
  two_sum(xh, ph, sh, se);
  const float sl = __fadd_rn(__fadd_rn(xl, pl), se);
  // the grid: M = 1.5 * 2^23 * G rounds a value below 2^22 G to a multiple of G
  const float B =
      __fadd_rn(__fadd_rn(fabsf(sh), __fmul_rn((float)SPAN, fabsf(a.w))), (float)SPAN);
  const uint32_t eb = min(__float_as_uint(B) >> 23, 250u);
  const float M = __uint_as_float(((eb + 2u) << 23) | (1u << 22));
  const float s0q = __fsub_rn(__fadd_rn(sh, M), M);
  const float kq = __fsub_rn(__fadd_rn(a.w, M), M);
  const float s0l = __fadd_rn(sl, __fsub_rn(sh, s0q));
  const float kl = __fadd_rn(c.z, __fsub_rn(a.w, kq));
  ItemGeo g;
  g.r11 = a.z;
  g.kq = kq;
  g.ns0q = -s0q;
  g.a1 = __fmul_rn(a.z, kl);
  g.a0 = -__fmul_rn(a.z, s0l);
  g.nyh = -yh;
  g.nyl = -yl;
  g.r22 = b.x;
  return g;
}

// ------------------------------------------------------------------ launchers
// Each translation unit exposes host launchers; all return cudaGetLastError().
cudaError_t launch_setup_planes(const ug_plan* plan, const ug_plane* d_planes, WsView v,
                                cudaStream_t s);
cudaError_t launch_preprocess(const ug_plan* plan, const ug_gaussians* g, WsView v,
                              cudaStream_t s);
cudaError_t launch_bin_sort(const ug_plan* plan, WsView v, cudaStream_t s);
cudaError_t launch_render(const ug_plan* plan, WsView v, float* image, float* alpha,
                          cudaStream_t s);
size_t ssim_scratch_floats(int32_t P, int32_t W, int32_t H);
size_t dssim_scratch_floats(int32_t P, int32_t W, int32_t H);
cudaError_t launch_l1_dssim(const float* image, const float* target, int32_t P, int32_t W,
                            int32_t H, float lam, float* scratch, float* grad, float* loss,
                            cudaStream_t s);
cudaError_t launch_ssim(const float* image, const float* target, int32_t P, int32_t W, int32_t H,
                        float* scratch, float* ssim, float* psnr, cudaStream_t s);
cudaError_t launch_render_scatter(const ug_plan* plan, WsView v, float* image, float* alpha,
                                  cudaStream_t s);
cudaError_t launch_render_backward_raster(const ug_plan* plan, WsView v, const float* image,
                                          const float* alpha, const float* grad_image,
                                          cudaStream_t s);
cudaError_t launch_render_backward(const ug_plan* plan, const ug_gaussians* g, WsView v,
                                   const float* image, const float* alpha,
                                   const float* grad_image, const ug_gaussian_grads* grads,
                                   cudaStream_t s);
cudaError_t launch_pre_backward(const ug_plan* plan, const ug_gaussians* g, WsView v,
                                const ug_gaussian_grads* grads, cudaStream_t s);
int device_sms();
cudaError_t launch_mse(const float* image, const float* target, int64_t n, int64_t denom,
                       float* grad, float* loss, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int32_t rows, int64_t n,
                        const ug_adam_row* d_rows, int32_t* d_step, float b1, float b2,
                        float eps, cudaStream_t s);
// Row f2 (ug_densify.cu). Decision thresholds in FP32, derived on the host.
struct DensifyThresholds {
  float logit_min;       // prune when logit < logit_min (sigmoid(logit) < min_opacity)
  float grad_threshold;  // densify when mean |dL/dmu| > grad_threshold
  float size2;           // TRI: split when trace Sigma > size2
  float log_size;        // SCALE_ROT: split when the largest log scale > log_size
  float beta, phi, log_phi;
};
size_t densify_scratch_bytes(int64_t n);
cudaError_t launch_sample(int cov, const float* params, int64_t n, float beta, const int32_t* idx,
                          int64_t m, const float* z, float* y, cudaStream_t s);
cudaError_t launch_densify_stats(const float* gmean, int64_t n, float* stats, cudaStream_t s);
cudaError_t launch_densify(int cov, const float* params, const float* m, const float* v,
                           int64_t n, const float* stats, const float* z,
                           const DensifyThresholds& t, int64_t cap, float* params_out,
                           float* m_out, float* v_out, int64_t* n_out, void* scratch,
                           cudaStream_t s);
int num_render_variants(int tile);
int num_render_variants_bwd(int tile);

}  // namespace ug
