// Rows a5 and a7: the forward tile rasterizer and its gradient.
//
// Both kernels are persistent and warp-specialised. One producer warp per CTA
// takes TILE x TILE pixel tiles from a device work counter (all tiles of all
// planes, so planes of different sizes share one launch) and gathers each
// tile's records, BATCH at a time, into a ring of shared-memory stages
// (ug_pipe.cuh); the other warps consume the stages. The tile is cut into
// footprints of 8 columns x FH rows. For every (record, footprint) of a stage
// a test decides whether the record can touch the footprint:
//   - its pixel box must overlap the footprint, and
//   - a lower bound on t1^2 + t2^2 over the overlap must leave the exponent
//     above -127: below that every weight in the overlap is exactly 0 in
//     FP32 (ex2 flushes results below 2^-126 to zero), so skipping the pair
//     changes no bit of the output or the gradient;
// and whether the box covers the whole footprint (then no per-pixel box test
// is needed). Each (record, footprint) that passes is one work item.
//
// Per pixel and record (see the record and item_geo in ug_internal.cuh):
//   t1 = r11 (col - S(row)) with the row's crossing S(row) held in two parts,
//   t2 = r22 dy(row),  w = 2^(lw2 - t1^2 - t2^2)  (= alpha exp(-q/2), Eq.
//   mahalanobis-3d),
// evaluated in packed FP32x2 arithmetic, two pixels per instruction; col and
// row are the pixel's offsets in its footprint.
//
// The binning computes every instance's tests against the tile's 8x8
// footprints (the key's top byte: live, box covers the footprint); the
// stages carry the keys, so neither pass tests 8x8 footprints again (the
// backward's 8x4-footprint variant tests its own).
// Forward: once a stage's copies have landed, the producer warp compacts each
// footprint's live records into lists. One consumer warp per footprint,
// otherwise independent of the other warps. The warp is split into G lane groups that each cover the whole
// footprint (2G pixels of one column per lane) and take every G-th work item;
// per pixel S_a += w, S_c += w c; at the end of the tile the groups' sums are
// reduce-scattered (every lane ends with two pixels' full sums), then C = (S_c
// + a_bg c_bg) / (S_a + a_bg) (Eq. alpha-combine, Eq. colour-combine). No
// atomics, fixed summation order.
//
// Backward: one lane per work item. The lane walks the 8 x FH pixels of its
// footprint and sums the seven per-record quantities of dL/dw over them in
// registers, so no cross-lane reduction is needed; it then adds them to the
// record's accumulators with two vector reductions.
#include "ug_pipe.cuh"

namespace ug {

template <int TILE, int FH>
struct Tiling {
  static constexpr int FW = 8;
  static constexpr int FX = TILE / FW;  // footprints per tile row
  static constexpr int FY = TILE / FH;  // footprint rows per tile
  static constexpr int NF = FX * FY;    // footprints per tile
  static_assert(NF <= 8, "footprint bits");
};

__device__ __forceinline__ void footprint_origin(int f, int fx_count, int fh, int tx, int ty,
                                                 int tile, int& fj0, int& fi0) {
  fj0 = tx * tile + (f % fx_count) * 8;
  fi0 = ty * tile + (f / fx_count) * fh;
}

// Work-item test of one record against the footprint [fj0, fj0 + 7] x [fi0,
// fi0 + fh - 1] (see footprint_bits): bit 0 live, bit 1 the box covers the
// footprint. The 8x8 footprints' tests come with the sorted keys; this is for
// the backward's 8x4 footprints.
template <int CUT>
__device__ __forceinline__ uint32_t classify(const float4& a, const float4& b, uint2 bx, int fj0,
                                             int fi0, int fh) {
  return footprint_bits(a, b, bx, fj0, fi0, fh, CUT);
}

// box ∩ footprint in footprint coordinates, packed cx0 | cx1 << 8 | ry0 << 16 |
// ry1 << 24 (non-empty for a live work item).
__device__ __forceinline__ uint32_t clip_box(uint2 bx, int fj0, int fi0, int fh) {
  const int j0 = bx.x & 0xffff, j1 = bx.x >> 16, i0 = bx.y & 0xffff, i1 = bx.y >> 16;
  const int cx0 = max(j0 - fj0, 0), cx1 = min(j1 - fj0, 7);
  const int ry0 = max(i0 - fi0, 0), ry1 = min(i1 - fi0, fh - 1);
  return (uint32_t)cx0 | ((uint32_t)cx1 << 8) | ((uint32_t)ry0 << 16) | ((uint32_t)ry1 << 24);
}

// ------------------------------------------------------------------ forward
// A warp's current chunk of up to 32 work items (structure of arrays, one
// slot per lane of the builder; the item_geo constants in pairs for the
// FP32x2 arithmetic). Slots past the last item, up to a multiple of the lane
// groups, hold inert items (-lw2 = +inf), so that every group runs the same
// number of items.
struct FwdChunk {
  float4 p0[32];     // r11, r11, kq, kq
  float4 p1[32];     // -s0q, -s0q, a1, a1
  float4 p2[32];     // a0, a0, nyh, nyh
  float4 p3[32];     // nyl, nyl, r22, r22
  float4 p4[32];     // -lw2, -lw2, c, c
  float4 lc[2][32];  // partial items: -lw2 in the box's columns, +inf outside
  uint32_t rows[32]; // partial items: bit y set for the box's rows
  float thr[32];     // ellipsoid threshold (cut-off by ellipsoid)
};

template <int TILE, int G, int MINB = 0>
struct FwdShape {
  using T = Tiling<TILE, 8>;
  static constexpr int NW = T::NF;        // one consumer warp per 8x8 footprint
  static constexpr int NCT = 32 * NW;     // consumer threads
  static constexpr int NT = NCT + 32;     // plus the producer warp
  static constexpr int LG = 32 / G;       // lanes per group: 8 rows x LG / 8 column blocks
  static constexpr int NP = G;            // column pairs per lane
  static_assert(G == 1 || G == 2 || G == 4, "groups");
  // resident blocks asked of the compiler (MINB, or by default 5 for the
  // 16x16 tile's 160 threads: at most 80 registers a thread, so that shared
  // memory, not registers, limits the blocks per SM)
  static constexpr int kMinBlocks = MINB > 0 ? MINB : (NT >= 160 ? 5 : 1);
};

template <int TILE, int NW, int NS, int BATCH>
struct FwdSmem {
  RecStage<TILE, false, BATCH> st[NS];
  PipeBars<NS> bars;
  FwdChunk ch[NW];
  PlaneTable T;
};

// The weight is w = 2^-n with n = t1^2 + (t2^2 - lw2) >= 0 formed by plain
// (un-negated) fused multiply-adds; the special-function unit takes the
// negation. Pixels outside the box (PARTIAL) or the ellipsoid (CUT), and inert
// items, get n = +inf, whose weight is +0.
__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }

// One lane, one work item: the lane's footprint row y, k2 = (its row in the
// tile) twice, column pairs cp0 .. cp0 + NP - 1 of the footprint (col2[p] =
// their two columns in the tile).
template <int CUT, bool PARTIAL, int NP>
__device__ __forceinline__ void fwd_item(const FwdChunk& C, int e, float2 k2, int y, int cp0,
                                         const float2* col2, float2* sa, float2* sc) {
  const float4 p0 = C.p0[e], p1 = C.p1[e], p2 = C.p2[e], p3 = C.p3[e], p4 = C.p4[e];
  const float2 r11 = lo2(p0), cc = hi2(p4);
  const float2 nsh = __ffma2_rn(hi2(p0), k2, lo2(p1));  // kq row - s0q (exact)
  const float2 nrs = __ffma2_rn(hi2(p1), k2, lo2(p2));  // a1 row + a0
  const float2 dy = __fadd2_rn(__fadd2_rn(k2, hi2(p2)), lo2(p3));
  const float2 t2 = __fmul2_rn(hi2(p3), dy);
  float2 c2[NP];  // t2^2 - lw2 per column pair
  if (PARTIAL) {
    float4 lw4[2];
    lw4[0] = C.lc[0][e];
    lw4[1] = C.lc[1][e];
    float2 t2sq = __fmul2_rn(t2, t2);
    if (!((C.rows[e] >> y) & 1u)) t2sq = make_float2(INFINITY, INFINITY);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int q = cp0 + p;
      const float4 l = lw4[q >> 1];
      c2[p] = __fadd2_rn((q & 1) ? hi2(l) : lo2(l), t2sq);
    }
  } else {
    const float2 c = __ffma2_rn(t2, t2, lo2(p4));
#pragma unroll
    for (int p = 0; p < NP; ++p) c2[p] = c;
  }
  float thr = 0.f;
  if (CUT) thr = C.thr[e];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const float2 d = __fadd2_rn(col2[p], nsh);  // col - S(row), exact
    const float2 t1 = __ffma2_rn(r11, d, nrs);
    float2 n2 = __ffma2_rn(t1, t1, c2[p]);  // q - lw2
    if (CUT) {
      const float2 q = __ffma2_rn(t1, t1, __fmul2_rn(t2, t2));
      if (!(q.x <= thr)) n2.x = INFINITY;
      if (!(q.y <= thr)) n2.y = INFINITY;
    }
    const float2 w = make_float2(fast_exp2_neg(n2.x), fast_exp2_neg(n2.y));
    sa[p] = __fadd2_rn(sa[p], w);
    sc[p] = __ffma2_rn(w, cc, sc[p]);
  }
}

// Chunk slot `lane` from the record's tile-anchored constants (g0 = r11, kq,
// -s0q, a1; g1 = a0, -yh, -yl, r22; see stage_tile_geo), b and box bx, with
// -lw2 where the weight's exponent needs it; real = false makes the slot inert
// (-lw2 = +inf: every weight is +0).
template <int CUT, bool PARTIAL>
__device__ __forceinline__ void fwd_build(FwdChunk& W, int lane, bool real, const float4& g0,
                                          const float4& b, const float4& g1, uint2 bx, int fj0,
                                          int fi0) {
  const float nlw = real ? -b.y : INFINITY;
  W.p0[lane] = make_float4(g0.x, g0.x, g0.y, g0.y);
  W.p1[lane] = make_float4(g0.z, g0.z, g0.w, g0.w);
  W.p2[lane] = make_float4(g1.x, g1.x, g1.y, g1.y);
  W.p3[lane] = make_float4(g1.z, g1.z, g1.w, g1.w);
  W.p4[lane] = make_float4(nlw, nlw, b.z, b.z);
  if (PARTIAL) {
    const uint32_t cl = clip_box(bx, fj0, fi0, 8);
    const int cx0 = cl & 0xff, cx1 = (cl >> 8) & 0xff, ry0 = (cl >> 16) & 0xff, ry1 = cl >> 24;
    float l[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) l[q] = ((q >= cx0) & (q <= cx1)) ? nlw : INFINITY;
    W.lc[0][lane] = make_float4(l[0], l[1], l[2], l[3]);
    W.lc[1][lane] = make_float4(l[4], l[5], l[6], l[7]);
    W.rows[lane] = (2u << ry1) - (1u << ry0);
  }
  if (CUT) W.thr[lane] = b.w;
}

// The record constants of a stage anchored at the tile's first pixel
// (item_geo over the whole TILE x TILE region), computed once per record by
// the producer warp for all of the tile's footprints and written over the
// record words that only they were derived from: a <- (r11, kq, -s0q, a1), c
// <- (a0, -yh, -yl, r22). A consumer adds its footprint's offset in the tile
// to the pixel's column and row.
template <int TILE, bool RAW, int BATCH>
__device__ __forceinline__ void stage_tile_geo(RecStage<TILE, RAW, BATCH>& S, int lane) {
  const int cnt = S.h.cnt, tj = S.h.tx * TILE, ti = S.h.ty * TILE;
#pragma unroll
  for (int q = 0; q < BATCH / 32; ++q) {
    const int r = lane + 32 * q;
    if (r < cnt) {
      const ItemGeo g = item_geo<TILE>(S.a[r], S.b[r], S.c[r], S.box[r], tj, ti);
      S.a[r] = make_float4(g.r11, g.kq, g.ns0q, g.a1);
      S.c[r] = make_float4(g.a0, g.nyh, g.nyl, g.r22);
    }
  }
}

// The producer's finishing step of a forward stage: per 8x8 footprint of the
// tile, the compacted lists of its live records (box covering the footprint
// from the front, the others from the back) and their counts, from the
// binning's footprint tests (the top byte of each instance's key), written to
// the stage for the consumers; then the records' tile-anchored constants.
template <int TILE, int BATCH>
struct FwdPrep {
  static constexpr bool kDefer = true;
  __device__ void operator()(RecStage<TILE, false, BATCH>& S, int lane) const {
    using T = Tiling<TILE, 8>;
    static_assert(T::NF <= kMaxFootprints, "a stage carries the lists of four footprints");
    const int cnt = S.h.cnt;
    uint32_t mq[BATCH / 32];
#pragma unroll
    for (int q = 0; q < BATCH / 32; ++q) {
      const int r = lane + 32 * q;
      mq[q] = r < cnt ? S.mask[r] >> kKeyTileBits : 0u;
    }
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int f = 0; f < T::NF; ++f) {
      int nf = 0, np = 0;
#pragma unroll
      for (int q = 0; q < BATCH / 32; ++q) {
        const uint32_t mf = mq[q] >> (2 * f);
        const bool live = mf & 1u, full = mf & 2u;
        const uint32_t bf = __ballot_sync(0xffffffffu, live && full);
        const uint32_t bp = __ballot_sync(0xffffffffu, live && !full);
        const int r = lane + 32 * q;
        if (live && full) S.list[f][nf + __popc(bf & lt)] = (uint8_t)r;
        if (live && !full) S.list[f][BATCH - 1 - (np + __popc(bp & lt))] = (uint8_t)r;
        nf += __popc(bf);
        np += __popc(bp);
      }
      if (lane == 0) {
        S.nfull[f] = (uint16_t)nf;
        S.npart[f] = (uint16_t)np;
      }
    }
    stage_tile_geo(S, lane);
  }
};

template <int TILE, int G, int CUT, int NS = kStages, int BATCH = kBatch, int MINB = 0>
__global__ void __launch_bounds__(FwdShape<TILE, G, MINB>::NT, FwdShape<TILE, G, MINB>::kMinBlocks)
    k_render_fwd(WsView v, const uint32_t* __restrict__ vals, int P, int total_tiles, float abg,
                 float cbg, float* __restrict__ image, float* __restrict__ alpha,
                 const uint32_t* __restrict__ sorted_keys) {
  using Sh = FwdShape<TILE, G, MINB>;
  constexpr int NW = Sh::NW, LG = Sh::LG, NP = Sh::NP;
  extern __shared__ __align__(16) unsigned char fwd_smem[];
  FwdSmem<TILE, NW, NS, BATCH>& S = *reinterpret_cast<FwdSmem<TILE, NW, NS, BATCH>*>(fwd_smem);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  pipe_init(S.T, S.bars, v, P, Sh::NCT, 32);
  if (__syncthreads_or(dev_failed(v.hdr))) return;  // the whole CTA leaves, or none of it
  if (warp == NW) {
    produce<TILE, false, false, true, FwdPrep<TILE, BATCH>, NS, BATCH>(
        S.st, S.bars, S.T, v, vals, 0, P, total_tiles, nullptr, nullptr, nullptr, sorted_keys,
        FwdPrep<TILE, BATCH>{});
    return;
  }
  const int grp = lane / LG, gl = lane % LG;
  const int y = gl & 7, cp0 = (gl >> 3) * NP;  // this lane's row and first column pair
  // the record constants are anchored at the tile: this footprint's offset in
  // it goes into the lane's row and columns
  const int dx0 = (warp % Tiling<TILE, 8>::FX) * 8, dy0 = (warp / Tiling<TILE, 8>::FX) * 8;
  const float2 k2 = make_float2((float)(y + dy0), (float)(y + dy0));
  float2 col2[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p)
    col2[p] = make_float2((float)(2 * (cp0 + p) + dx0), (float)(2 * (cp0 + p) + 1 + dx0));
  unsigned long long evaluated = 0;  // (record, footprint) items of this warp
  int fj0 = 0, fi0 = 0, tw = 0, th = 0;
  int64_t tpx = 0;
  float2 sa[NP], sc[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) sa[p] = sc[p] = make_float2(0.f, 0.f);
  const FwdChunk& C = S.ch[warp];
  for (uint32_t k = 0;; ++k) {
    const int s = (int)(k % NS);
    if (!mbar_wait(&S.bars.full[s], (k / NS) & 1u)) {
      dev_fail(v.hdr, UG_ERR_TIMEOUT, 1);
      break;
    }
    const RecStage<TILE, false, BATCH>& R = S.st[s];
    const StageHdr h = R.h;
    if (h.tile < 0) break;
    if (h.flags & kFirst) {
      footprint_origin(warp, Tiling<TILE, 8>::FX, 8, h.tx, h.ty, TILE, fj0, fi0);
      tw = h.w;
      th = h.h;
      tpx = h.px_off;
#pragma unroll
      for (int p = 0; p < NP; ++p) sa[p] = sc[p] = make_float2(0.f, 0.f);
    }
    // this warp's lists, compacted by the producer: full-box items from the
    // front, partial from the back
    const int nf = R.nfull[warp], np = R.npart[warp];
    evaluated += (unsigned long long)(nf + np);
    FwdChunk& W = S.ch[warp];
    for (int base = 0; base < nf; base += 32) {
      const int ne = min(32, nf - base), nr = (ne + G - 1) / G * G;
      if (lane < nr) {  // lane-parallel chunk build
        const bool real = lane < ne;
        const int r = real ? (int)R.list[warp][base + lane] : 0;
        fwd_build<CUT, false>(W, lane, real, R.a[r], R.b[r], R.c[r], R.box[r], fj0, fi0);
      }
      __syncwarp();
      for (int e = grp; e < nr; e += G) fwd_item<CUT, false, NP>(C, e, k2, y, cp0, col2, sa, sc);
      __syncwarp();
    }
    for (int base = 0; base < np; base += 32) {
      const int ne = min(32, np - base), nr = (ne + G - 1) / G * G;
      if (lane < nr) {
        const bool real = lane < ne;
        const int r = real ? (int)R.list[warp][BATCH - 1 - (base + lane)] : 0;
        fwd_build<CUT, true>(W, lane, real, R.a[r], R.b[r], R.c[r], R.box[r], fj0, fi0);
      }
      __syncwarp();
      for (int e = grp; e < nr; e += G) fwd_item<CUT, true, NP>(C, e, k2, y, cp0, col2, sa, sc);
      __syncwarp();
    }
    mbar_arrive(&S.bars.empty[s]);  // the stage is no longer read by this thread
    if (h.flags & kLast) {
      // Reduce-scatter the groups' sums (fixed order): at each level a lane
      // keeps half of its column pairs and adds the partner group's sums of
      // that half, so in the end every lane holds the full sums of one column
      // pair (two pixels) and forms those two pixels.
      int cpk = 0;  // the kept column pair, relative to this lane's first
#pragma unroll
      for (int l = 0; (LG << l) < 32; ++l) {
        const int o = LG << l, hh = NP >> (l + 1);
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int p = 0; p < hh; ++p) {
          const float2 ka = up ? sa[p + hh] : sa[p], kc = up ? sc[p + hh] : sc[p];
          const float2 ga = up ? sa[p] : sa[p + hh], gc = up ? sc[p] : sc[p + hh];
          sa[p] = make_float2(ka.x + __shfl_xor_sync(0xffffffffu, ga.x, o),
                              ka.y + __shfl_xor_sync(0xffffffffu, ga.y, o));
          sc[p] = make_float2(kc.x + __shfl_xor_sync(0xffffffffu, gc.x, o),
                              kc.y + __shfl_xor_sync(0xffffffffu, gc.y, o));
        }
        if (up) cpk += hh;
      }
      const int i = fi0 + y;
      if (i < th) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int j = fj0 + 2 * (cp0 + cpk) + q;
          if (j < tw) {
            const int64_t px = tpx + (int64_t)i * tw + j;
            const float al = (q ? sa[0].y : sa[0].x) + abg;
            image[px] = ((q ? sc[0].y : sc[0].x) + abg * cbg) / al;
            alpha[px] = al;
          }
        }
      }
    }
  }
  if (lane == 0 && evaluated)
    atomicAdd(reinterpret_cast<unsigned long long*>(&v.hdr->st.evaluated_pairs),
              evaluated * 64ull);
}

// ------------------------------------------------------------------ backward
template <int TILE, int FH>
struct BwdShape {
  using T = Tiling<TILE, FH>;
  static constexpr int NW = T::NF;     // one consumer warp per footprint
  static constexpr int NCT = 32 * NW;  // consumer threads
  static constexpr int NT = NCT + 32;  // plus the producer warp
};

// Stages in the backward's ring by default: one more than the forward's,
// because a consumer warp holds a stage until it has processed the stage's
// items.
constexpr int kBwdStages = 4;

// A consumer warp's queue of work items, in a ring of a power-of-two length
// above the items a warp can hold (31 left over from a round plus one stage's
// BATCH): (stage << 8) | record index. The items are read from the stages
// themselves, so a stage is released only once the warp has processed all of
// its items.
template <int BATCH>
struct BwdQueue {
  static constexpr int kLen = BATCH <= 128 ? 256 : 512;
  static_assert(kLen >= 31 + BATCH, "the queue holds a round's remainder and a whole stage");
  uint16_t idx[kLen];
};

template <int TILE, int FH, int NS, int BATCH>
struct BwdSmem {
  using Sh = BwdShape<TILE, FH>;
  RecStage<TILE, true, BATCH> st[NS];
  PipeBars<NS> bars;
  BwdQueue<BATCH> q[Sh::NW];
  // per footprint and tile parity, row pair rp and column c (index 8 rp + c):
  // r, r', -rC, -rC' of rows 2 rp and 2 rp + 1
  float4 pix[Sh::NW][2][FH * 4];
  PlaneTable Tb;
};

// Vector reduction of four floats into 16-byte aligned global memory.
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(__cvta_generic_to_global(p)),
               "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Column offset that stands for a column outside a partial item's box: t1 =
// r11 (kFarCol + nsh) + nrs is then so large that t1^2 overflows or the
// exponent is far below -127, so the weight is exactly +0, while t1 stays
// finite for any r11 below 2^88 (0 * t1 is 0, never a NaN).
constexpr float kFarCol = 1099511627776.f;  // 2^40

// One lane, one work item (or, with TAIL, nrows of its FH rows from row y0,
// in a rolled loop; nrows even): sums over the footprint's 8 x FH (8 x nrows)
// pixels of
//   acc0 = sum r w        (dL/dc),
//   acc1 = sum g,  g = w dL/dw   (dL/dlw2 / ln 2),
//   acc2 = sum g t1,    acc3 = sum g t2,
//   acc4 = sum g t1^2,  acc5 = sum g t1 t2,  acc6 = sum g t2^2,
// with r = G / alpha and dL/dw = r (c - C) at each pixel (Eq. us-render
// differentiated, box fixed), added to the record's accumulators; the chain
// kernel turns them into the gradients of the Gaussian's parameters. The
// FP32x2 arithmetic pairs two ROWS of one column, so the per-row terms (the
// row's crossing, t2, lw2 - t2^2 and the row sums) are computed once per row
// and not duplicated. Pixels outside the box (rows: lw2 - t2^2 = -inf, or a
// large finite exponent in the fast form; columns: kFarCol) or the ellipsoid
// (CUT) get w = 0, never a NaN: every factor that multiplies w stays finite.
// The fast form takes sum g t1^2 from the exponent n = t1^2 + t2^2 - lw2 the
// weight needs anyway (nine packed operations per column and row pair
// instead of ten); the roundings of n and of the row's sums then cost below
// 2^-19 (t2^2 - lw2) times the row's sum of |g|, and t2^2 - lw2 <= 150 in a
// row with a non-zero weight.
template <int FH, int CUT, bool TAIL = false>
__device__ __forceinline__ void bwd_item(const float4& a, const float4& bb, const float4& cr,
                                         uint2 bx, uint32_t cl, uint32_t rid,
                                         const float4* __restrict__ pix, int fj0, int fi0,
                                         float* __restrict__ rec_grad, int y0 = 0,
                                         int nrows = FH) {
  static_assert(FH % 2 == 0, "rows are processed in pairs");
  const ItemGeo ig = item_geo(a, bb, cr, bx, fj0, fi0);
  const float2 r11 = make_float2(ig.r11, ig.r11), kq = make_float2(ig.kq, ig.kq);
  const float2 ns0q = make_float2(ig.ns0q, ig.ns0q), a1 = make_float2(ig.a1, ig.a1);
  const float2 a0 = make_float2(ig.a0, ig.a0), nyh = make_float2(ig.nyh, ig.nyh);
  const float2 nyl = make_float2(ig.nyl, ig.nyl), r22 = make_float2(ig.r22, ig.r22);
  const float2 nlw = make_float2(-bb.y, -bb.y), cc = make_float2(bb.z, bb.z);
  const int cx0 = cl & 0xff, cx1 = (cl >> 8) & 0xff, ry0 = (cl >> 16) & 0xff, ry1 = cl >> 24;
  float2 colv[8];  // column offsets as FP32x2 pairs; columns outside the box far away
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float cv = (c >= cx0 && c <= cx1) ? (float)c : kFarCol;
    colv[c] = make_float2(cv, cv);
  }
  // packed sums over the footprint (.x even rows, .y odd rows, added at the end)
  float2 s0 = make_float2(0.f, 0.f), a4 = make_float2(0.f, 0.f);
  float2 s1p = make_float2(0.f, 0.f), u1p = make_float2(0.f, 0.f), u2p = make_float2(0.f, 0.f);
  float2 a5p = make_float2(0.f, 0.f), a6p = make_float2(0.f, 0.f);
  // pixel factors of row pair rp, column c: pix[8 rp + c] = (r, r', -rC, -rC')
  const float4* __restrict__ pxr = pix + 4 * y0;
  // Fast form (r11 <= 2^20, so every t1 and t1^2 of the footprint is finite):
  // sum g t1^2 per row as sum g n - (t2^2 - lw2) sum g with n = t1^2 + t2^2 -
  // lw2 the exponent already formed; pixels whose weight is zero get a large
  // finite n (never 0 * inf).
  constexpr float kBigN = 1.2676506e30f;  // 2^100
  auto row_pair_fast = [&](int j) {
    const int y = y0 + 2 * j;
    const float2 k2 = make_float2((float)y, (float)(y + 1));
    const float2 nsh = __ffma2_rn(kq, k2, ns0q);
    const float2 nrs = __ffma2_rn(a1, k2, a0);
    const float2 dy = __fadd2_rn(__fadd2_rn(k2, nyh), nyl);
    const float2 t2 = __fmul2_rn(r22, dy);
    const float2 t2sq = __fmul2_rn(t2, t2);
    float2 crow = __fadd2_rn(t2sq, nlw);
    if (y < ry0 || y > ry1) crow.x = kBigN;
    if (y + 1 < ry0 || y + 1 > ry1) crow.y = kBigN;
    float2 s1r = make_float2(0.f, 0.f), u1r = make_float2(0.f, 0.f), a4r = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float2 t1 = __ffma2_rn(r11, __fadd2_rn(colv[c], nsh), nrs);
      float2 n2 = __ffma2_rn(t1, t1, crow);
      if (CUT) {
        const float2 q = __ffma2_rn(t1, t1, t2sq);
        if (!(q.x <= bb.w)) n2.x = kBigN;
        if (!(q.y <= bb.w)) n2.y = kBigN;
      }
      const float2 w = make_float2(fast_exp2_neg(n2.x), fast_exp2_neg(n2.y));
      const float4 px = pxr[8 * j + c];
      const float2 rr = make_float2(px.x, px.y);
      const float2 g = __fmul2_rn(__ffma2_rn(rr, cc, make_float2(px.z, px.w)), w);
      s0 = __ffma2_rn(rr, w, s0);
      s1r = __fadd2_rn(s1r, g);
      u1r = __ffma2_rn(g, t1, u1r);
      a4r = __ffma2_rn(g, n2, a4r);
    }
    s1p = __fadd2_rn(s1p, s1r);
    u1p = __fadd2_rn(u1p, u1r);
    a4 = __ffma2_rn(make_float2(-crow.x, -crow.y), s1r, __fadd2_rn(a4, a4r));
    a5p = __ffma2_rn(t2, u1r, a5p);
    u2p = __ffma2_rn(t2, s1r, u2p);
    a6p = __ffma2_rn(t2sq, s1r, a6p);
  };
  auto row_pair = [&](int j) {
    const int y = y0 + 2 * j;
    const float2 k2 = make_float2((float)y, (float)(y + 1));
    const float2 nsh = __ffma2_rn(kq, k2, ns0q);  // kq row - s0q (exact)
    const float2 nrs = __ffma2_rn(a1, k2, a0);
    const float2 dy = __fadd2_rn(__fadd2_rn(k2, nyh), nyl);
    const float2 t2 = __fmul2_rn(r22, dy);
    const float2 t2sq = __fmul2_rn(t2, t2);
    float2 crow = __fadd2_rn(t2sq, nlw);  // t2^2 - lw2
    if (y < ry0 || y > ry1) crow.x = INFINITY;  // row outside the box
    if (y + 1 < ry0 || y + 1 > ry1) crow.y = INFINITY;
    float2 s1r = make_float2(0.f, 0.f), u1r = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float2 t1 = __ffma2_rn(r11, __fadd2_rn(colv[c], nsh), nrs);
      float2 n2 = __ffma2_rn(t1, t1, crow);  // t1^2 + t2^2 - lw2
      if (CUT) {
        const float2 q = __ffma2_rn(t1, t1, t2sq);
        if (!(q.x <= bb.w)) n2.x = INFINITY;
        if (!(q.y <= bb.w)) n2.y = INFINITY;
      }
      const float2 w = make_float2(fast_exp2_neg(n2.x), fast_exp2_neg(n2.y));
      const float4 px = pxr[8 * j + c];
      const float2 rr = make_float2(px.x, px.y);
      const float2 g = __fmul2_rn(__ffma2_rn(rr, cc, make_float2(px.z, px.w)), w);  // w dL/dw
      s0 = __ffma2_rn(rr, w, s0);
      s1r = __fadd2_rn(s1r, g);
      const float2 gu = __fmul2_rn(g, t1);
      u1r = __fadd2_rn(u1r, gu);
      a4 = __ffma2_rn(gu, t1, a4);
    }
    s1p = __fadd2_rn(s1p, s1r);
    u1p = __fadd2_rn(u1p, u1r);
    a5p = __ffma2_rn(t2, u1r, a5p);
    u2p = __ffma2_rn(t2, s1r, u2p);
    a6p = __ffma2_rn(t2sq, s1r, a6p);
  };
  if (TAIL) {
#pragma unroll 1
    for (int j = 0; j < nrows / 2; ++j) row_pair(j);
  } else if (ig.r11 <= 1048576.f) {
#pragma unroll
    for (int j = 0; j < FH / 2; ++j) row_pair_fast(j);
  } else {
#pragma unroll
    for (int j = 0; j < FH / 2; ++j) row_pair(j);
  }
  const float s1 = s1p.x + s1p.y, u1 = u1p.x + u1p.y, u2 = u2p.x + u2p.y;
  const float a5 = a5p.x + a5p.y, a6 = a6p.x + a6p.y;
  // the record's 8-float accumulator block (32-byte aligned): two vector
  // reductions instead of seven scalar atomics
  float* dst = rec_grad + (size_t)rid * 8;
  red_add_v4(dst, s0.x + s0.y, s1, u1, u2);
  red_add_v4(dst + 4, a4.x + a4.y, a5, a6, 0.f);
}

// Each consumer warp owns one footprint of the tile. It queues the indices of
// the stage's records that are live for its footprint and processes the queue
// 32 items at a time, one item per lane, reading each item's record from its
// stage. Items are carried across tiles (a round may hold the end of one tile
// and the start of the next): the pixel factors are kept for two tiles (by
// tile parity), each item names its parity, and before a tile writes its
// factors the items of the tile before the previous one are processed; only
// the queue's last items, at the kernel's end, run as a partial round. A
// stage is released when all of its items are processed, and at the latest
// before the wait that reuses its slot (the items still queued are processed
// first, so the producer never waits for a stage that a consumer holds). The
// warps share no barrier.
template <int TILE, int FH, int CUT, int NS = kBwdStages, int BATCH = kBatch, int MINB = 4>
__global__ void __launch_bounds__(BwdShape<TILE, FH>::NT, MINB)
    k_render_bwd(WsView v, const uint32_t* __restrict__ vals, int P, int total_tiles,
                 const float* __restrict__ image, const float* __restrict__ alpha,
                 const float* __restrict__ grad_image, const uint32_t* __restrict__ sorted_keys) {
  using Sh = BwdShape<TILE, FH>;
  using T = Tiling<TILE, FH>;
  constexpr int NW = Sh::NW;
  constexpr uint32_t QL = BwdQueue<BATCH>::kLen;
  static_assert(NS >= 2 && NS <= 4 && BATCH <= 256,
                "queue entries hold a stage (2 bits) and a record index (8 bits)");
  extern __shared__ __align__(16) unsigned char bwd_smem[];
  BwdSmem<TILE, FH, NS, BATCH>& S = *reinterpret_cast<BwdSmem<TILE, FH, NS, BATCH>*>(bwd_smem);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  pipe_init(S.Tb, S.bars, v, P, Sh::NCT);
  if (__syncthreads_or(dev_failed(v.hdr))) return;  // the whole CTA leaves, or none of it
  // the binning's footprint tests apply when the footprints are 8x8 (the
  // 8x4-footprint variant tests its own)
  constexpr bool use_masks = FH == 8;
  if (warp == NW) {
    produce<TILE, true, true, false, NoPrep, NS, BATCH>(S.st, S.bars, S.Tb, v, vals, 1, P,
                                                        total_tiles, grad_image, alpha, image,
                                                        use_masks ? sorted_keys : nullptr);
    return;
  }
  const uint32_t lt = lanemask_lt();
  uint16_t* Q = S.q[warp].idx;
  unsigned long long evaluated = 0;
  int fj0 = 0, fi0 = 0;           // this footprint's origin in the current tile
  uint32_t tpar = 1;              // parity of the current tile (of this warp's tiles)
  uint32_t qmark0 = 0, qmark1 = 0;  // queue end of the last tile of each parity
  uint32_t qhead = 0, qtail = 0;  // items processed / queued so far
  uint32_t qe0 = 0, qe1 = 0, qe2 = 0, qe3 = 0;  // qtail after each held stage's items, by slot
  auto qend = [&](uint32_t slot) {
    return slot == 0 ? qe0 : slot == 1 ? qe1 : slot == 2 ? qe2 : qe3;
  };
  uint32_t krel = 0;                    // the stages before krel are released
  // item i of the queue (0 = its oldest) from row y0: its record read from its
  // stage, its footprint's origin from the stage's tile; queue entries: record
  // index (bits 0-7), stage slot (8-9), tile parity (10)
  auto item = [&](uint32_t i, int y0, int rows, bool part) {
    const uint32_t e = Q[(qhead + i) % QL];
    const RecStage<TILE, true, BATCH>& Rs = S.st[(e >> 8) & 3u];
    const int r = (int)(e & 255u);
    const float4* pix = S.pix[warp][(e >> 10) & 1u];
    int ij0, ii0;
    footprint_origin(warp, T::FX, FH, Rs.h.tx, Rs.h.ty, TILE, ij0, ii0);
    const uint2 bx = Rs.box[r];
    const uint32_t cl = clip_box(bx, ij0, ii0, FH);
    if (part)
      bwd_item<FH, CUT, true>(Rs.a[r], Rs.b[r], Rs.c[r], bx, cl, Rs.rid[r], pix, ij0, ii0,
                              v.rec_grad, y0, rows);
    else
      bwd_item<FH, CUT>(Rs.a[r], Rs.b[r], Rs.c[r], bx, cl, Rs.rid[r], pix, ij0, ii0,
                        v.rec_grad);
  };
  // one round: the oldest min(queued, 32) items; fewer than 17 are split by
  // rows over 2 or 4 lanes each (each lane adds its rows' sums)
  auto round = [&]() {
    const uint32_t n = min(qtail - qhead, 32u);
    if (n > 16) {
      if (lane < (int)n) item(lane, 0, FH, false);
    } else {
      // log2 of the lanes per item (each lane an even number of rows)
      const int lg = (n > 8 || FH < 8) ? 1 : 2;
      const int it = lane & (31 >> lg), part = lane >> (5 - lg), rows = FH >> lg;
      if (it < (int)n) item(it, part * rows, rows, true);
    }
    qhead += n;
    __syncwarp();  // every lane has read its records
  };
  // release the held stages up to `last` whose items are all processed, in order
  auto release = [&](uint32_t last) {
    while (krel <= last && qend(krel % NS) <= qhead) {
      mbar_arrive(&S.bars.empty[krel % NS]);
      ++krel;
    }
  };
  bool failed = false;
  for (uint32_t k = 0;; ++k) {
    const int s = (int)(k % NS);
    if (k >= (uint32_t)NS && krel + NS <= k) {
      // this wait reuses the slot of stage k - NS: process its items
      while (qhead < qend(s)) round();
      release(k - 1);
    }
    if (!mbar_wait(&S.bars.full[s], (k / NS) & 1u)) {
      dev_fail(v.hdr, UG_ERR_TIMEOUT, 2);
      failed = true;
      break;
    }
    const RecStage<TILE, true, BATCH>& R = S.st[s];
    const StageHdr h = R.h;
    if (h.tile < 0) break;
    if (h.flags & kFirst) {
      // the current tile's items end here; the new tile takes the other
      // parity, whose factors the items of the tile before are still using
      if (tpar) qmark1 = qtail;
      else qmark0 = qtail;
      tpar ^= 1u;
      while (qhead < (tpar ? qmark1 : qmark0)) round();
      // per-pixel factors of this warp's footprint: r = G / alpha and -r C
      // (0 off the plane)
      footprint_origin(warp, T::FX, FH, h.tx, h.ty, TILE, fj0, fi0);
      // layout: entry 8 rp + c holds rows 2 rp and 2 rp + 1 of column c
      for (int q = lane; q < FH * 4; q += 32) {
        const int rp = q / 8, c = q % 8;
        const int p0 = ((warp / T::FX) * FH + 2 * rp) * TILE + (warp % T::FX) * 8 + c;
        float v4[4];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int pp = p0 + hh * TILE;
          const float rv = R.raw[0][pp] / R.raw[1][pp];
          v4[hh] = rv;
          v4[2 + hh] = -rv * R.raw[2][pp];
        }
        S.pix[warp][tpar][q] = make_float4(v4[0], v4[1], v4[2], v4[3]);
      }
      __syncwarp();
    }
    // queue the stage's live records for this footprint, in record order
    uint32_t m[BATCH / 32];
#pragma unroll
    for (int q = 0; q < BATCH / 32; ++q) {
      const int r = 32 * q + lane;
      m[q] = 0;
      if (r < h.cnt)
        m[q] = use_masks ? R.mask[r] >> (kKeyTileBits + 2 * warp)
                         : classify<CUT>(R.a[r], R.b[r], R.box[r], fj0, fi0, FH);
    }
    const uint32_t q0 = qtail;
#pragma unroll
    for (int q = 0; q < BATCH / 32; ++q) {
      const uint32_t bl = __ballot_sync(0xffffffffu, m[q] & 1u);
      if (m[q] & 1u)
        Q[(qtail + __popc(bl & lt)) % QL] = (uint16_t)((tpar << 10) | (s << 8) | (32 * q + lane));
      qtail += __popc(bl);
    }
    evaluated += qtail - q0;
    if (s == 0) qe0 = qtail;
    else if (s == 1) qe1 = qtail;
    else if (s == 2) qe2 = qtail;
    else qe3 = qtail;
    __syncwarp();
    while (qtail - qhead >= 32u) round();  // full rounds
    release(k);
  }
  if (!failed)
    while (qtail > qhead) round();  // the queue's last items
  if (lane == 0 && evaluated)
    atomicAdd(reinterpret_cast<unsigned long long*>(&v.hdr->st.evaluated_pairs_bwd),
              evaluated * (unsigned long long)(8 * FH));
}

// Zero the per-record accumulators of the backward rasterizer, and (block 0)
// its tile counter and evaluated-pair count.
__global__ void k_zero_rec_grad(WsView v, int64_t cap) {
  if (dev_failed(v.hdr)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    v.hdr->tile_counter[1] = 0;
    v.hdr->st.evaluated_pairs_bwd = 0;
  }
  const int64_t nrec = min((int64_t)v.hdr->slots, cap);
  float4* g = reinterpret_cast<float4*>(v.rec_grad);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrec * 2;
       i += (int64_t)gridDim.x * blockDim.x)
    g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ------------------------------------------------------------------ variants
// The sorted keys, whose top byte holds each instance's footprint tests.
static const uint32_t* sorted_keys(const ug_plan* plan, const WsView& v) {
  return v.keys[plan->sort_passes & 1];
}

template <typename K>
static int occupancy_grid(K kernel, int threads, size_t dyn_smem = 0) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, dyn_smem);
  return device_sms() * (occ > 0 ? occ : 1);
}

template <int TILE, int G, int CUT, int NS, int BATCH, int MINB>
static cudaError_t fwd_launch(const ug_plan* plan, WsView v, const uint32_t* vals, float* image,
                              float* alpha, cudaStream_t s) {
  constexpr int NT = FwdShape<TILE, G, MINB>::NT;
  constexpr size_t SM = sizeof(FwdSmem<TILE, FwdShape<TILE, G, MINB>::NW, NS, BATCH>);
  auto kern = k_render_fwd<TILE, G, CUT, NS, BATCH, MINB>;
  static const cudaError_t attr =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
  if (attr != cudaSuccess) return attr;
  static const int grid = occupancy_grid(kern, NT, SM);
  const int g = min(grid, max(plan->total_tiles, 1));
  kern<<<g, NT, SM, s>>>(v, vals, plan->num_planes, plan->total_tiles, plan->cfg.alpha_bg,
                         plan->cfg.c_bg, image, alpha, sorted_keys(plan, v));
  return cudaGetLastError();
}

template <int TILE, int FH, int CUT, int NS, int BATCH, int MINB>
static cudaError_t bwd_launch(const ug_plan* plan, WsView v, const uint32_t* vals,
                              const float* image, const float* alpha, const float* grad,
                              cudaStream_t s) {
  constexpr int NT = BwdShape<TILE, FH>::NT;
  constexpr size_t SM = sizeof(BwdSmem<TILE, FH, NS, BATCH>);
  auto kern = k_render_bwd<TILE, FH, CUT, NS, BATCH, MINB>;
  static const cudaError_t attr =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
  if (attr != cudaSuccess) return attr;
  static const int grid = occupancy_grid(kern, NT, SM);
  const int g = min(grid, max(plan->total_tiles, 1));
  kern<<<g, NT, SM, s>>>(v, vals, plan->num_planes, plan->total_tiles, image, alpha, grad,
                         sorted_keys(plan, v));
  return cudaGetLastError();
}

// Forward variants (G lane groups per 8x8 footprint, NS stages in the ring,
// BATCH records per stage, MINB resident blocks asked of the compiler, 0 =
// the default):
//   0: G 4 (8 pixels of one row per lane), NS 3, BATCH 128
//   1: G 2 (4 pixels), 2: G 1 (2 pixels)
//   3: G 4, BATCH 64, MINB 6     4: G 4, NS 2, BATCH 256     5: G 4, NS 4, MINB 4
// (3-5 for the 16 x 16 tile only).
template <int TILE, int CUT>
static cudaError_t dispatch_fwd(const ug_plan* plan, WsView v, const uint32_t* vals, float* image,
                                float* alpha, cudaStream_t s) {
  switch (plan->cfg.variant) {
    case 0: return fwd_launch<TILE, 4, CUT, 3, 128, 0>(plan, v, vals, image, alpha, s);
    case 1: return fwd_launch<TILE, 2, CUT, 3, 128, 0>(plan, v, vals, image, alpha, s);
    case 2: return fwd_launch<TILE, 1, CUT, 3, 128, 0>(plan, v, vals, image, alpha, s);
    default: break;
  }
  if constexpr (TILE == 16) {
    switch (plan->cfg.variant) {
      case 3: return fwd_launch<TILE, 4, CUT, 3, 64, 6>(plan, v, vals, image, alpha, s);
      case 4: return fwd_launch<TILE, 4, CUT, 2, 256, 0>(plan, v, vals, image, alpha, s);
      case 5: return fwd_launch<TILE, 4, CUT, 4, 128, 4>(plan, v, vals, image, alpha, s);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

// Backward variants (FH footprint rows, NS stages, BATCH records per stage,
// MINB resident blocks asked of the compiler, which bounds its registers):
//   0: FH 8, NS 4, BATCH 128, MINB 4     1: FH 4, NS 4, BATCH 128, MINB 2 (tile 16)
//   2: FH 8, NS 3, BATCH 128, MINB 5     3: FH 8, NS 4, BATCH 64, MINB 5
//   4: FH 8, NS 3, BATCH 256, MINB 3     5: FH 8, NS 4, BATCH 128, MINB 3 (128 registers a
//   thread, no spills)
// (2-5 for the 16 x 16 tile only).
template <int TILE, int CUT>
static cudaError_t dispatch_bwd(const ug_plan* plan, WsView v, const uint32_t* vals,
                                const float* image, const float* alpha, const float* grad,
                                cudaStream_t s) {
  switch (plan->cfg.variant_bwd) {
    case 0: return bwd_launch<TILE, 8, CUT, 4, 128, 4>(plan, v, vals, image, alpha, grad, s);
    case 1:  // twice the consumer warps per block: half the resident blocks
      return bwd_launch<TILE, 4, CUT, 4, 128, TILE == 16 ? 2 : 4>(plan, v, vals, image, alpha,
                                                                 grad, s);
    default: break;
  }
  if constexpr (TILE == 16) {
    switch (plan->cfg.variant_bwd) {
      case 2: return bwd_launch<TILE, 8, CUT, 3, 128, 5>(plan, v, vals, image, alpha, grad, s);
      case 3: return bwd_launch<TILE, 8, CUT, 4, 64, 5>(plan, v, vals, image, alpha, grad, s);
      case 4: return bwd_launch<TILE, 8, CUT, 3, 256, 3>(plan, v, vals, image, alpha, grad, s);
      case 5: return bwd_launch<TILE, 8, CUT, 4, 128, 3>(plan, v, vals, image, alpha, grad, s);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

int num_render_variants(int tile) { return tile == 16 ? 6 : tile == 8 ? 3 : 0; }
int num_render_variants_bwd(int tile) { return tile == 16 ? 6 : tile == 8 ? 2 : 0; }

cudaError_t launch_render(const ug_plan* plan, WsView v, float* image, float* alpha,
                          cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&v.hdr->tile_counter[0], 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&v.hdr->st.evaluated_pairs, 0, sizeof(int64_t), s);
  if (e != cudaSuccess) return e;
  const uint32_t* vals = v.vals[plan->sort_passes & 1];
  if (plan->cfg.tile == 16)
    e = plan->cfg.cutoff ? dispatch_fwd<16, 1>(plan, v, vals, image, alpha, s)
                         : dispatch_fwd<16, 0>(plan, v, vals, image, alpha, s);
  else
    e = plan->cfg.cutoff ? dispatch_fwd<8, 1>(plan, v, vals, image, alpha, s)
                         : dispatch_fwd<8, 0>(plan, v, vals, image, alpha, s);
  return e;
}

cudaError_t launch_render_backward_raster(const ug_plan* plan, WsView v, const float* image,
                                          const float* alpha, const float* grad_image,
                                          cudaStream_t s) {
  k_zero_rec_grad<<<device_sms() * 4, 256, 0, s>>>(v, plan->record_capacity);
  const uint32_t* vals = v.vals[plan->sort_passes & 1];
  if (plan->cfg.tile == 16)
    return plan->cfg.cutoff ? dispatch_bwd<16, 1>(plan, v, vals, image, alpha, grad_image, s)
                            : dispatch_bwd<16, 0>(plan, v, vals, image, alpha, grad_image, s);
  return plan->cfg.cutoff ? dispatch_bwd<8, 1>(plan, v, vals, image, alpha, grad_image, s)
                          : dispatch_bwd<8, 0>(plan, v, vals, image, alpha, grad_image, s);
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
