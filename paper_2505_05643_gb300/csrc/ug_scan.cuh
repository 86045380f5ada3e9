// Exclusive prefix sums over large arrays: partial sum per block of
// kScanItems entries -> scan of the block partials -> down-sweep. No
// inter-block waiting, deterministic. Either k_scan_partial and k_scan_top
// give the down-sweep each block's exclusive prefix, or the kernel that
// produces the counts adds them to the block partials (atomic integer sums:
// the result does not depend on their order) and every down-sweep block sums
// the partials before its own (RAW_PARTS), which saves both launches.
#pragma once

#include "ug_internal.cuh"

namespace ug {

constexpr int kScanThreads = 256;
constexpr int kScanPerThread = kScanItems / kScanThreads;  // 8
static_assert(kScanPerThread * kScanThreads == kScanItems, "scan tiling");

// Block-wide exclusive scan of one value per thread (256 threads); returns the
// exclusive prefix and writes the block total to *total.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T x, T* total) {
  __shared__ T warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  T base = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kScanThreads / 32; ++w) {
    if (w < warp) base += warp_tot[w];
    tot += warp_tot[w];
  }
  __syncthreads();
  *total = tot;
  return base + incl - x;
}

// Partial sums of NV values per block of kScanItems entries (integer sums:
// the order of the additions does not matter, so the loads are coalesced).
template <int NV, class Load>
__global__ void __launch_bounds__(kScanThreads)
    k_scan_partial(Load ld, int64_t entries, unsigned long long* part, const WsHeader* hdr) {
  if (hdr && dev_failed(hdr)) return;
  const int64_t base = (int64_t)blockIdx.x * kScanItems + threadIdx.x;
  unsigned long long s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k] = 0;
#pragma unroll
  for (int it = 0; it < kScanPerThread; ++it) {
    const int64_t e = base + (int64_t)it * kScanThreads;
    if (e < entries) {
      uint32_t val[NV];
      ld(e, val);
#pragma unroll
      for (int k = 0; k < NV; ++k) s[k] += val[k];
    }
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    unsigned long long tot;
    block_excl_scan<unsigned long long>(s[k], &tot);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NV + k] = tot;
  }
}

// The totals of a scan: mode 1 (candidate scan, NV = 2): the record slots
// and the FP64 entries; mode 2 (record scan, NV = 1): the instance count.
// Both write them to the header and flag capacity overflow (cap0).
template <int NV>
__device__ __forceinline__ void scan_totals(WsHeader* hdr, int mode,
                                            const unsigned long long tot[NV], int64_t cap0) {
  if (mode == 1) {
    hdr->st.records = (int64_t)tot[0];
    hdr->slots = (uint32_t)min(tot[0], (unsigned long long)cap0);
    hdr->slots64 = NV > 1 ? (uint32_t)min(tot[NV - 1], (unsigned long long)cap0) : 0u;
    if ((int64_t)tot[0] > cap0) dev_fail(hdr, UG_ERR_CAPACITY, 0);
  }
  if (mode == 2) {
    hdr->st.instances = (int64_t)tot[0];
    if ((int64_t)tot[0] > cap0) dev_fail(hdr, UG_ERR_CAPACITY, 1);
  }
}

// Exclusive scan of the block partials in place (one block of 1024 threads),
// then the totals by mode (scan_totals).
template <int NV>
__global__ void __launch_bounds__(1024)
    k_scan_top(unsigned long long* part, int64_t nblk, WsHeader* hdr, int mode, int64_t cap0,
               int64_t cap1) {
  if (hdr && dev_failed(hdr)) return;
  __shared__ unsigned long long sh[32][NV];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t per = (nblk + 1023) / 1024;
  const int64_t b0 = (int64_t)tid * per;
  unsigned long long loc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) loc[k] = 0;
  for (int64_t b = b0; b < b0 + per && b < nblk; ++b)
#pragma unroll
    for (int k = 0; k < NV; ++k) loc[k] += part[b * NV + k];
  unsigned long long excl[NV], tot[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    unsigned long long incl = loc[k];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) sh[warp][k] = incl;
    excl[k] = incl - loc[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    unsigned long long base = 0, t = 0;
    for (int w = 0; w < 32; ++w) {
      if (w < warp) base += sh[w][k];
      t += sh[w][k];
    }
    excl[k] += base;
    tot[k] = t;
  }
  __syncthreads();
  unsigned long long run[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) run[k] = excl[k];
  for (int64_t b = b0; b < b0 + per && b < nblk; ++b)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      unsigned long long v = part[b * NV + k];
      part[b * NV + k] = run[k];
      run[k] += v;
    }
  if (tid == 0) scan_totals<NV>(hdr, mode, tot, cap0);
}

// Down-sweep: exclusive prefix of every entry, passed to st(e, excl[NV]).
// The block's entries go through shared memory, so that the loads and the
// stores are coalesced while every thread scans kScanPerThread consecutive
// entries (shared index i + i / 32: the threads' runs start in different
// banks). part holds the blocks' exclusive prefixes, or with RAW_PARTS the
// nblk blocks' own sums: each block then adds those before it, and block 0
// adds them all and writes the totals by mode (scan_totals).
__device__ __forceinline__ int scan_smem_index(int i) { return i + (i >> 5); }

template <int NV, class Load, class Store, bool RAW_PARTS = false>
__global__ void __launch_bounds__(kScanThreads)
    k_scan_down(Load ld, Store st, int64_t entries, const unsigned long long* part,
                WsHeader* hdr, int64_t nblk = 0, int mode = 0, int64_t cap0 = 0) {
  __shared__ uint32_t sv[NV][kScanItems + kScanItems / 32];
  if (hdr && dev_failed(hdr)) return;
  const int64_t base = (int64_t)blockIdx.x * kScanItems;
  unsigned long long bpre[NV];
  if (RAW_PARTS) {
    const int64_t lim = blockIdx.x == 0 ? nblk : (int64_t)blockIdx.x;
    unsigned long long x[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) x[k] = 0;
    for (int64_t b = threadIdx.x; b < lim; b += kScanThreads)
#pragma unroll
      for (int k = 0; k < NV; ++k) x[k] += part[b * NV + k];
#pragma unroll
    for (int k = 0; k < NV; ++k) block_excl_scan<unsigned long long>(x[k], &bpre[k]);
    if (blockIdx.x == 0) {
      if (threadIdx.x == 0) scan_totals<NV>(hdr, mode, bpre, cap0);
#pragma unroll
      for (int k = 0; k < NV; ++k) bpre[k] = 0;
    }
  } else {
#pragma unroll
    for (int k = 0; k < NV; ++k) bpre[k] = part[(int64_t)blockIdx.x * NV + k];
  }
#pragma unroll
  for (int it = 0; it < kScanPerThread; ++it) {
    const int i = it * kScanThreads + (int)threadIdx.x;
    const int64_t e = base + i;
    uint32_t val[NV];
    if (e < entries) {
      ld(e, val);
    } else {
#pragma unroll
      for (int k = 0; k < NV; ++k) val[k] = 0;
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) sv[k][scan_smem_index(i)] = val[k];
  }
  __syncthreads();
  const int t0 = (int)threadIdx.x * kScanPerThread;
  uint32_t loc[kScanPerThread][NV];
  unsigned long long s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k] = 0;
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      loc[j][k] = sv[k][scan_smem_index(t0 + j)];
      s[k] += loc[j][k];
    }
  unsigned long long run[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    unsigned long long tot;
    run[k] = block_excl_scan<unsigned long long>(s[k], &tot) + bpre[k];
  }
  // each thread overwrites only the entries it read
#pragma unroll
  for (int j = 0; j < kScanPerThread; ++j)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      sv[k][scan_smem_index(t0 + j)] = (uint32_t)run[k];
      run[k] += loc[j][k];
    }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kScanPerThread; ++it) {
    const int i = it * kScanThreads + (int)threadIdx.x;
    const int64_t e = base + i;
    if (e < entries) {
      uint32_t ex[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) ex[k] = sv[k][scan_smem_index(i)];
      st(e, ex);
    }
  }
}

}  // namespace ug
