// Row a4: stable LSD radix sort of the (tile key, record id) instances and
// the [start, end) range of every tile.
//
// Each 8-bit pass: (1) every block of kSortTile keys counts its digits in
// shared memory and writes them digit-major, (2) one exclusive scan over
// (digit, block) gives every block the output base of each digit, (3) every
// block ranks its keys stably (warps in order, each warp's items in element
// order, the lanes with equal digits found by one ballot per digit bit) and
// scatters keys and values. Instances arrive in (Gaussian chunk, plane,
// Gaussian) order, so the stable sort leaves each tile's records in ascending
// Gaussian order.
#include "ug_scan.cuh"

namespace ug {

__global__ void __launch_bounds__(kSortThreads)
    k_sort_hist(const uint32_t* __restrict__ keys, int shift, int64_t nblk, WsView v) {
  __shared__ uint32_t hist[256];
  if (dev_failed(v.hdr)) return;
  const int64_t n = v.hdr->st.instances;
  hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base < n) {
    // all loads first (in flight together), then the counts
    uint32_t d[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      const int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
      d[k] = i < n ? (__ldg(keys + i) >> shift) & 0xffu : 256u;
    }
#pragma unroll
    for (int k = 0; k < kSortItems; ++k)
      if (d[k] < 256u) atomicAdd(&hist[d[k]], 1u);
  }
  __syncthreads();
  v.sort_hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = hist[threadIdx.x];
}

// Warp w of block b holds elements b*kSortTile + w*32*kSortItems + k*32 + lane
// (item k of lane `lane`): each warp ranks its 32*kSortItems keys in element
// order with per-warp digit counters in shared memory (items in order, lanes in
// order, equal digits found by ballots). The block then places its
// keys in shared memory in digit order and writes them out so that consecutive
// threads write consecutive addresses of each digit's output run.
__global__ void __launch_bounds__(kSortThreads, 3)
    k_sort_scatter(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                   uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int shift,
                   int64_t nblk, WsView v) {
  constexpr int NW = kSortThreads / 32;
  __shared__ uint32_t cnt[NW][256];
  __shared__ uint32_t dstart[256];
  __shared__ uint32_t gb[256];
  __shared__ uint32_t sk[kSortTile];
  __shared__ uint32_t sv[kSortTile];
  if (dev_failed(v.hdr)) return;
  const int64_t n = v.hdr->st.instances;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base >= n) return;
  const int count = (int)min((int64_t)kSortTile, n - base);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int w = 0; w < NW; ++w) cnt[w][tid] = 0;
  gb[tid] = v.sort_hist[(int64_t)tid * nblk + blockIdx.x];
  const int wbase = warp * 32 * kSortItems + lane;
  uint32_t kreg[kSortItems], vreg[kSortItems], rank[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const int i = wbase + k * 32;
    kreg[k] = i < count ? __ldg(keys_in + base + i) : 0u;
    vreg[k] = i < count ? __ldg(vals_in + base + i) : 0u;
  }
  __syncthreads();
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const bool valid = wbase + k * 32 < count;
    const uint32_t d = valid ? (kreg[k] >> shift) & 0xffu : 256u;
    // the lanes with the same digit: one ballot per digit bit (faster here
    // than __match_any_sync)
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const uint32_t bit = (d >> b) & 1u;
      const uint32_t bal = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? bal : ~bal;
    }
    if (count < kSortTile) {  // the last block: its missing items carry digit 256
      const uint32_t bit = d >> 8;
      const uint32_t bal = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? bal : ~bal;
    }
    const uint32_t before = valid ? cnt[warp][d] : 0u;
    __syncwarp();
    if (valid && (peers & lt) == 0) cnt[warp][d] = before + __popc(peers);
    __syncwarp();
    rank[k] = before + __popc(peers & lt);
  }
  __syncthreads();
  uint32_t total = 0;  // thread tid owns digit tid: exclusive prefix over the warps
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint32_t c = cnt[w][tid];
    cnt[w][tid] = total;
    total += c;
  }
  uint32_t all;
  dstart[tid] = block_excl_scan<uint32_t>(total, &all);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    if (wbase + k * 32 < count) {
      const uint32_t d = (kreg[k] >> shift) & 0xffu;
      const uint32_t lpos = dstart[d] + cnt[warp][d] + rank[k];
      sk[lpos] = kreg[k];
      sv[lpos] = vreg[k];
    }
  }
  __syncthreads();
  for (int i = tid; i < count; i += kSortThreads) {
    const uint32_t key = sk[i];
    const uint32_t d = (key >> shift) & 0xffu;
    const uint32_t pos = gb[d] + (uint32_t)i - dstart[d];
    keys_out[pos] = key;
    vals_out[pos] = sv[i];
  }
}

// A warp takes 32 x kRangeItems consecutive sorted instances (coalesced
// loads, all issued before the comparisons); each key's neighbours come from
// the next and previous lane, or from the warp's neighbouring items. A tile's
// range starts where the key differs from the one before and ends where it
// differs from the one after.
constexpr int kRangeItems = 8;

__global__ void __launch_bounds__(256) k_tile_ranges(const uint32_t* __restrict__ keys, WsView v) {
  if (dev_failed(v.hdr)) return;
  const int64_t n = v.hdr->st.instances;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  constexpr int64_t span = 32 * kRangeItems;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * span < n;
       w += nwarps) {
    const int64_t base = w * span;
    uint32_t k[kRangeItems];
#pragma unroll
    for (int u = 0; u < kRangeItems; ++u) {
      const int64_t i = base + u * 32 + lane;
      k[u] = i < n ? __ldg(keys + i) & kKeyTileMask : ~0u;  // ~0u: no tile
    }
    const uint32_t before = base > 0 ? __ldg(keys + base - 1) & kKeyTileMask : ~0u;
    const uint32_t after = base + span < n ? __ldg(keys + base + span) & kKeyTileMask : ~0u;
#pragma unroll
    for (int u = 0; u < kRangeItems; ++u) {
      // the keys just before lane 0 and just after lane 31 of this item
      const uint32_t edge_prev =
          u > 0 ? __shfl_sync(0xffffffffu, k[u > 0 ? u - 1 : 0], 31) : before;
      const uint32_t edge_next =
          u + 1 < kRangeItems ? __shfl_sync(0xffffffffu, k[u + 1 < kRangeItems ? u + 1 : u], 0)
                              : after;
      uint32_t kp = __shfl_up_sync(0xffffffffu, k[u], 1);
      uint32_t kn = __shfl_down_sync(0xffffffffu, k[u], 1);
      if (lane == 0) kp = edge_prev;
      if (lane == 31) kn = edge_next;
      const int64_t i = base + u * 32 + lane;
      if (i < n) {
        if (kp != k[u]) v.ranges[k[u]].x = (uint32_t)i;
        if (kn != k[u]) v.ranges[k[u]].y = (uint32_t)(i + 1);
      }
    }
  }
}

struct HistLoad {
  const uint32_t* h;
  __device__ void operator()(int64_t e, uint32_t out[1]) const { out[0] = h[e]; }
};
struct HistStore {
  uint32_t* h;
  __device__ void operator()(int64_t e, const uint32_t ex[1]) const { h[e] = ex[0]; }
};

cudaError_t launch_bin_sort(const ug_plan* plan, WsView v, cudaStream_t s) {
  const int64_t nblk = sort_blocks(plan->instance_capacity);
  const int64_t entries = 256 * nblk;
  const int64_t sblk = scan_blocks(entries);
  HistLoad ld{v.sort_hist};
  HistStore st{v.sort_hist};
  for (int pass = 0; pass < plan->sort_passes; ++pass) {
    const int shift = 8 * pass;
    const int src = pass & 1, dst = src ^ 1;
    k_sort_hist<<<(unsigned)nblk, kSortThreads, 0, s>>>(v.keys[src], shift, nblk, v);
    // block partials, then each down-sweep block sums those before its own
    k_scan_partial<1, HistLoad><<<(unsigned)sblk, kScanThreads, 0, s>>>(ld, entries, v.sort_part,
                                                                        v.hdr);
    k_scan_down<1, HistLoad, HistStore, true><<<(unsigned)sblk, kScanThreads, 0, s>>>(
        ld, st, entries, v.sort_part, v.hdr, sblk, 0, 0);
    k_sort_scatter<<<(unsigned)nblk, kSortThreads, 0, s>>>(v.keys[src], v.vals[src], v.keys[dst],
                                                           v.vals[dst], shift, nblk, v);
  }
  cudaError_t e = cudaMemsetAsync(v.ranges, 0, sizeof(uint2) * (size_t)plan->total_tiles, s);
  if (e != cudaSuccess) return e;
  k_tile_ranges<<<(unsigned)(device_sms() * 8), 256, 0, s>>>(v.keys[plan->sort_passes & 1], v);
  return cudaGetLastError();
}

}  // namespace ug
