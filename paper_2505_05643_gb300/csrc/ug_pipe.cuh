// Record pipeline of the tile rasterizers: one producer warp per CTA takes
// tiles from the persistent work counter and gathers each tile's records
// (sorted instance -> record id -> rec_a, rec_b, rec_c, rec_box) into a ring of
// shared-memory stages; the CTA's other warps consume the stages. Full/empty
// handshakes are mbarriers (arrive: release, try_wait: acquire, CTA scope),
// so the gathers of the next batches overlap the arithmetic of the current
// one instead of stalling every warp on two dependent global loads per batch.
//
// Every wait is bounded in time: a wait that gives up records
// UG_ERR_TIMEOUT in the workspace status and the warp leaves the kernel; the
// waits of the other warps then run out as well, so the kernel always ends.
#pragma once

#include "ug_internal.cuh"

namespace ug {

constexpr int kBatch = 128;   // records per stage (default; a template parameter)
constexpr int kStages = 3;    // stages in the ring (default; a template parameter)
constexpr int kFirst = 1;     // stage flag: first batch of its tile
constexpr int kLast = 2;      // stage flag: last batch of its tile
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s
constexpr uint32_t kWaitLimitIters = 1u << 20;
// A waiting thread sleeps until the phase completes or this long (ns), so
// waiting warps take no issue slots from the working ones.
constexpr uint32_t kSuspendHintNs = 20000;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "n"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}

// Wait for the completion of the barrier phase with the given parity; false
// if it has not completed within kWaitLimitNs (or kWaitLimitIters polls).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < kWaitLimitIters; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) break;
  }
  return false;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)),
               "l"(__cvta_generic_to_global(gmem))
               : "memory");
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem)),
               "l"(__cvta_generic_to_global(gmem))
               : "memory");
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)),
               "l"(__cvta_generic_to_global(gmem))
               : "memory");
}

// Arrive on the barrier once all of this thread's earlier cp.async copies
// have completed (the arrival is counted in the barrier's expected count).
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Wait until at most one of this thread's committed copy groups is pending.
__device__ __forceinline__ void cp_async_wait_prev() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

struct StageHdr {
  int32_t tile;   // -1: no more tiles
  int32_t tx, ty, w, h;
  int32_t cnt;    // records in this stage
  int32_t flags;  // kFirst | kLast
  uint32_t inst0; // sorted instance of the stage's first record
  int64_t px_off;
};

// 8x8 footprints of a tile whose item lists a forward stage carries.
constexpr int kMaxFootprints = 4;

// One stage: up to BATCH records of one tile, with each instance's sorted key
// (the binning's footprint tests in its top byte). Forward (not RAW): per 8x8
// footprint, the indices of the records live there (those whose box covers
// the footprint from the front, the others from the back) and their counts,
// written by the producer's finishing step. Backward (RAW): with the first
// stage of a tile the tile's pixel inputs (dL/dC, alpha, C; pixels off the
// plane hold 0, 1, 0).
template <int TILE, bool RAW, int BATCH = kBatch>
struct RecStage {
  static_assert(BATCH % 32 == 0 && BATCH <= 256, "records per stage: a multiple of 32, <= 256");
  float4 a[BATCH];
  float4 b[BATCH];
  float4 c[BATCH];
  uint2 box[BATCH];
  uint32_t rid[BATCH];
  uint32_t mask[BATCH];  // the instances' sorted keys (footprint tests in the top byte)
  uint8_t list[RAW ? 1 : kMaxFootprints][RAW ? 1 : BATCH];  // record indices (< 256)
  uint16_t nfull[RAW ? 1 : kMaxFootprints], npart[RAW ? 1 : kMaxFootprints];
  StageHdr h;
  float raw[RAW ? 3 : 1][RAW ? TILE * TILE : 1];
};

template <int NS = kStages>
struct PipeBars {
  static constexpr int kN = NS;  // stages in the ring
  uint64_t full[NS];
  uint64_t empty[NS];
};

// Planes whose tile data a CTA keeps in shared memory (more planes: looked up
// in global memory).
constexpr int kSmemPlanes = 64;

struct TilePlane {
  int32_t tile_off, tiles_x, w, h;
  int64_t px_off;
};

struct PlaneTable {
  TilePlane pl[kSmemPlanes];
  int32_t tile_off[kSmemPlanes];
};

__device__ __forceinline__ int find_plane(const int32_t* tile_off, int P, int t) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_off[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Fill the plane table and the barriers; the caller follows with __syncthreads.
template <class Bars>
__device__ __forceinline__ void pipe_init(PlaneTable& T, Bars& bars, const WsView& v, int P,
                                          uint32_t consumer_threads, uint32_t full_arrivals = 64) {
  for (int p = threadIdx.x; p < min(P, kSmemPlanes); p += blockDim.x) {
    const PlaneDev& d = v.planes[p];
    T.pl[p] = TilePlane{d.tile_off, d.tiles_x, d.w, d.h, d.px_off};
    T.tile_off[p] = d.tile_off;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < Bars::kN; ++s) {
      // per producer lane: one plain arrival, and one cp.async arrival unless
      // the producer finishes the stage itself (then 32)
      mbar_init(&bars.full[s], full_arrivals);
      mbar_init(&bars.empty[s], consumer_threads);
    }
  }
}

// The producer warp. Stage k of the stream goes to slot k % NS (NS stages in
// the ring); from k = NS on, the slot is reused once its consumers have
// released stage k - NS. The record ids are read into registers, the records themselves
// (and the backward's pixel inputs) are copied with cp.async, whose completion
// arrives on the stage's full barrier, so up to NS batches of gathers
// are in flight. RID: the stage also keeps the record ids. inst_mask (may be
// null): per sorted instance (the sorted keys), copied into the stage. EMPTY_TILES: tiles
// without records still get one stage (the forward pass writes their
// background pixels).
struct TileCtx {
  int tx, ty, w, h;
  int64_t px_off;
};

__device__ __forceinline__ TileCtx tile_ctx(const PlaneTable& T, const WsView& v, int P, int t) {
  int local, tiles_x;
  TileCtx c;
  if (P <= kSmemPlanes) {
    const TilePlane& pl = T.pl[find_plane(T.tile_off, P, t)];
    local = t - pl.tile_off;
    tiles_x = pl.tiles_x;
    c.w = pl.w;
    c.h = pl.h;
    c.px_off = pl.px_off;
  } else {
    const PlaneDev& pl = v.planes[find_plane(v.tile_off, P, t)];
    local = t - pl.tile_off;
    tiles_x = pl.tiles_x;
    c.w = pl.w;
    c.h = pl.h;
    c.px_off = pl.px_off;
  }
  c.tx = local % tiles_x;
  c.ty = local / tiles_x;
  return c;
}

// No finishing step: the stage is complete when its copies have landed.
struct NoPrep {
  static constexpr bool kDefer = false;
  template <class S>
  __device__ void operator()(S&, int) const {}
};

template <int TILE, bool RAW, bool RID, bool EMPTY_TILES, class Prep = NoPrep, int NS = kStages,
          int BATCH = kBatch>
__device__ __forceinline__ void produce(RecStage<TILE, RAW, BATCH>* st, PipeBars<NS>& bars,
                                        const PlaneTable& T, const WsView& v,
                                        const uint32_t* __restrict__ vals, int which, int P,
                                        int total_tiles, const float* __restrict__ grad,
                                        const float* __restrict__ alpha,
                                        const float* __restrict__ image,
                                        const uint32_t* __restrict__ inst_mask,
                                        Prep prep = Prep()) {
  const int lane = threadIdx.x & 31;
  constexpr int PER = BATCH / 32;
  // test hook: issue nothing, so that the consumers' bounded waits run out
  if (*(volatile const uint32_t*)&v.hdr->stall_test != 0) return;
  const uint32_t total = (uint32_t)total_tiles;
  uint32_t* counter = &v.hdr->tile_counter[which];
  // Tile look-ahead: A is the tile being issued, B the next one (its range
  // load in flight), C the one after (its queue reservation in flight), so
  // neither the queue's atomic nor the range load stalls a tile change.
  uint32_t c_pending = 0;
  if (lane == 0) c_pending = atomicAdd(counter, 1u);
  uint32_t tA = __shfl_sync(0xffffffffu, c_pending, 0);
  uint2 rA = tA < total ? v.ranges[tA] : make_uint2(0u, 0u);
  if (lane == 0) c_pending = atomicAdd(counter, 1u);
  uint32_t tB = __shfl_sync(0xffffffffu, c_pending, 0);
  uint2 rB = tB < total ? v.ranges[tB] : make_uint2(0u, 0u);
  if (lane == 0) c_pending = atomicAdd(counter, 1u);
  auto next_tile = [&]() {
    tA = tB;
    rA = rB;
    tB = __shfl_sync(0xffffffffu, c_pending, 0);
    rB = tB < total ? v.ranges[tB] : make_uint2(0u, 0u);
    if (lane == 0 && tB < total) c_pending = atomicAdd(counter, 1u);
    if (tB >= total) c_pending = total;
  };
  if (!EMPTY_TILES)
    while (tA < total && rA.y == rA.x) next_tile();
  TileCtx cA = tA < total ? tile_ctx(T, v, P, (int)tA) : TileCtx{};
  uint32_t b = rA.x;
  // record ids of the batch to issue, read one batch ahead
  uint32_t rid[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const uint32_t r = b + lane + 32 * q;
    rid[q] = (tA < total && r < rA.y) ? __ldg(vals + r) : 0u;
  }
  uint32_t k = 0;
  while (tA < total) {
    // the batch to issue now
    const uint32_t t = tA, b0 = b;
    const uint2 rg = rA;
    const TileCtx c = cA;
    const int cnt = (int)min((uint32_t)BATCH, rg.y - b0);
    const bool first = b0 == rg.x, last = b0 + BATCH >= rg.y;
    // advance the cursor and start reading the next batch's record ids
    if (!last) {
      b += BATCH;
    } else {
      next_tile();
      if (!EMPTY_TILES)
        while (tA < total && rA.y == rA.x) next_tile();
      if (tA < total) cA = tile_ctx(T, v, P, (int)tA);
      b = rA.x;
    }
    uint32_t rid_next[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const uint32_t r = b + lane + 32 * q;
      rid_next[q] = (tA < total && r < rA.y) ? __ldg(vals + r) : 0u;
    }
    const int s = (int)(k % NS);
    if (k >= (uint32_t)NS && !mbar_wait(&bars.empty[s], ((k / NS) - 1) & 1u)) {
      dev_fail(v.hdr, UG_ERR_TIMEOUT, 100 + which);
      cp_async_wait_all();
      return;
    }
    RecStage<TILE, RAW, BATCH>& S = st[s];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int r = lane + 32 * q;
      if (r < cnt) {
        cp_async16(&S.a[r], v.rec_a + rid[q]);
        cp_async16(&S.b[r], v.rec_b + rid[q]);
        cp_async16(&S.c[r], v.rec_c + rid[q]);
        cp_async8(&S.box[r], v.rec_box + rid[q]);
        if (RID) S.rid[r] = rid[q];
        if (inst_mask) cp_async4(&S.mask[r], inst_mask + b0 + r);
      }
    }
    if constexpr (RAW) {
      if (first) {
        for (int p = lane; p < TILE * TILE; p += 32) {
          const int i = c.ty * TILE + p / TILE, j = c.tx * TILE + p % TILE;
          if (i < c.h && j < c.w) {
            const int64_t px = c.px_off + (int64_t)i * c.w + j;
            cp_async4(&S.raw[0][p], grad + px);
            cp_async4(&S.raw[1][p], alpha + px);
            cp_async4(&S.raw[2][p], image + px);
          } else {
            S.raw[0][p] = 0.f;
            S.raw[1][p] = 1.f;
            S.raw[2][p] = 0.f;
          }
        }
      }
    }
    if (lane == 0) {
      StageHdr hd;
      hd.tile = (int32_t)t;
      hd.tx = c.tx;
      hd.ty = c.ty;
      hd.w = c.w;
      hd.h = c.h;
      hd.cnt = cnt;
      hd.flags = (first ? kFirst : 0) | (last ? kLast : 0);
      hd.inst0 = b0;
      hd.px_off = c.px_off;
      S.h = hd;
    }
    if constexpr (Prep::kDefer) {
      // finish the previous stage (its copies, issued by this lane for the
      // records this lane finishes, have landed) and hand it over
      cp_async_commit();
      if (k > 0) {
        cp_async_wait_prev();
        __syncwarp();
        const int sp = (int)((k - 1) % NS);
        prep(st[sp], lane);
        mbar_arrive(&bars.full[sp]);
      }
    } else {
      mbar_arrive(&bars.full[s]);      // the plain shared-memory stores above
      cp_async_arrive(&bars.full[s]);  // this lane's copies, once they have landed
    }
    ++k;
#pragma unroll
    for (int q = 0; q < PER; ++q) rid[q] = rid_next[q];
  }
  if constexpr (Prep::kDefer) {
    if (k > 0) {
      cp_async_wait_all();
      __syncwarp();
      const int sp = (int)((k - 1) % NS);
      prep(st[sp], lane);
      mbar_arrive(&bars.full[sp]);
    }
  }
  const int s = (int)(k % NS);
  if (k >= (uint32_t)NS && !mbar_wait(&bars.empty[s], ((k / NS) - 1) & 1u)) {
    dev_fail(v.hdr, UG_ERR_TIMEOUT, 100 + which);
    cp_async_wait_all();
    return;
  }
  if (lane == 0) st[s].h.tile = -1;
  mbar_arrive(&bars.full[s]);
  if constexpr (!Prep::kDefer) cp_async_arrive(&bars.full[s]);
  cp_async_wait_all();
}

}  // namespace ug
