// Rows a1-a3 and a8: plane set-up, the per-(plane, Gaussian) preprocess, the
// tile instances, and the chain rule from per-record gradients back to the
// Gaussian parameters.
//
// Record-parallel pipeline (every heavy kernel runs with full warps):
//  1. cull     one warp per chunk of 32 consecutive Gaussians (coalesced
//              structure-of-arrays loads) walks all planes (staged in shared
//              memory) and sets one candidate bit per (plane, Gaussian) with a
//              conservative FP32 test that carries a rigorous rounding bound:
//              it only drops pairs that the exact test would drop too. It adds
//              the candidate counts to the next scan's block partials.
//  2. scan     of the candidate counts in (chunk, plane) order: every
//              candidate gets its record slot, so for any plane the records,
//              and after the stable sort the tile lists, are in ascending
//              Gaussian order.
//  3. list     writes the candidates into a work list, FP32 part first, then
//              the extended-precision part.
//  4. records  one thread per list entry: the exact FP32 or double-word
//              geometry (phase 1, box, in-plane conic, peak weight) and the
//              record; candidates that the exact test rejects become empty
//              slots.
//  5. live     one warp per 32 record slots counts each record's box tiles
//              that can hold a non-zero weight (adding them to the next scan's
//              block partials); the scan gives every record its first instance,
//              and the emit writes the (tile, record) instances, a warp's 32
//              records' instances spread over its lanes.
// The backward chain is one thread per record (per-record parameter
// gradients), then a per-Gaussian gather in the same slot order: no atomics,
// deterministic.
#include <algorithm>

#include "ug_geometry.cuh"
#include "ug_scan.cuh"

namespace ug {

int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// ------------------------------------------------------------------ warp helpers
// Transpose of a 32 x 32 bit matrix held one row per lane (bit c of lane r's
// word is element (r, c)): afterwards lane c holds column c. Five butterfly
// steps swap the off-diagonal blocks of ever smaller block pairs.
__device__ __forceinline__ uint32_t warp_bit_transpose(uint32_t x, int lane) {
  const uint32_t m[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int j = 16 >> k;
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? (x & ~m[k]) | ((y >> j) & m[k]) : (x & m[k]) | ((y & m[k]) << j);
  }
  return x;
}

// Largest lane l whose non-decreasing per-lane value pre[l] is <= o.
__device__ __forceinline__ int warp_search(uint32_t pre, uint32_t o) {
  int l = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const uint32_t p = __shfl_sync(0xffffffffu, pre, l + step);
    if (p <= o) l += step;
  }
  return l;
}

// Position of the n-th (0-based) set bit of m (which has more than n set bits).
__device__ __forceinline__ uint32_t nth_set_bit(unsigned long long m, uint32_t n) {
  uint32_t pos = 0;
#pragma unroll
  for (int w = 32; w >= 1; w >>= 1) {
    const uint32_t c = (uint32_t)__popcll(m & ((1ull << w) - 1ull));
    if (n >= c) {
      n -= c;
      m >>= w;
      pos += (uint32_t)w;
    }
  }
  return pos;
}

// ------------------------------------------------------------------ planes
__global__ void __launch_bounds__(256)
    k_setup_planes(const ug_plane* planes, int P, int tile, int total_tiles,
                   int64_t total_px, int64_t cand_blocks, int64_t rec_blocks, WsView v) {
  __shared__ int s_run;
  const int tid = threadIdx.x;
  if (tid == 0) {
    WsHeader* h = v.hdr;
    h->st.status = 0;
    h->st.detail = 0;
    h->st.records = 0;
    h->st.instances = 0;
    h->st.fp64_records = 0;
    h->st.box_pixels = 0;
    h->tile_counter[0] = 0;
    h->tile_counter[1] = 0;
    h->slots = 0;
    h->slots64 = 0;
    h->box_pixels = 0;
    h->holes = 0;
    h->stall_test = 0;
    h->kept64 = 0;
    h->origin_reach = 0.f;
    s_run = 0;
  }
  // the count scans' block partials, added to by the cull and the live-tile pass
  for (int64_t k = tid; k < 2 * cand_blocks; k += blockDim.x) v.scan_part[k] = 0;
  for (int64_t k = tid; k < rec_blocks; k += blockDim.x) v.slot_part[k] = 0;
  __syncthreads();
  for (int base = 0; base < P; base += 256) {
    const int p = base + tid;
    int ntiles = 0;
    if (p < P) {
      const ug_plane q = planes[p];
      bool ok = true;
      float nu = 0.f, nv = 0.f, uv = 0.f;
      for (int k = 0; k < 3; ++k) {
        ok = ok && isfinite(q.origin[k]) && isfinite(q.u[k]) && isfinite(q.v[k]);
        nu += q.u[k] * q.u[k];
        nv += q.v[k] * q.v[k];
        uv += q.u[k] * q.v[k];
      }
      ok = ok && fabsf(sqrtf(nu) - 1.f) <= 1e-4f && fabsf(sqrtf(nv) - 1.f) <= 1e-4f &&
           fabsf(uv) <= 1e-4f;
      ok = ok && isfinite(q.pitch_u) && isfinite(q.pitch_v) && q.pitch_u > 0.f && q.pitch_v > 0.f;
      ok = ok && q.width >= 1 && q.height >= 1 && q.width <= 16384 && q.height <= 16384;
      ok = ok && q.pixel_offset >= 0 && q.pixel_offset + (int64_t)q.width * q.height <= total_px;
      if (!ok) dev_fail(v.hdr, UG_ERR_INVALID_PLANE, p);
      if (ok) {  // |o| rounded up (non-negative floats order like their bits)
        const float r = __fsqrt_ru(__fmaf_ru(q.origin[2], q.origin[2],
                                             __fmaf_ru(q.origin[1], q.origin[1],
                                                       __fmul_ru(q.origin[0], q.origin[0]))));
        atomicMax(reinterpret_cast<int*>(&v.hdr->origin_reach), __float_as_int(r));
      }
      PlaneDev d;
      for (int k = 0; k < 3; ++k) {
        d.o[k] = q.origin[k];
        d.u[k] = q.u[k];
        d.v[k] = q.v[k];
      }
      d.n[0] = __fmaf_rn(q.u[1], q.v[2], -__fmul_rn(q.u[2], q.v[1]));
      d.n[1] = __fmaf_rn(q.u[2], q.v[0], -__fmul_rn(q.u[0], q.v[2]));
      d.n[2] = __fmaf_rn(q.u[0], q.v[1], -__fmul_rn(q.u[1], q.v[0]));
      d.pu = q.pitch_u;
      d.pv = q.pitch_v;
      d.inv_pu = __fdiv_rn(1.f, q.pitch_u);
      d.inv_pv = __fdiv_rn(1.f, q.pitch_v);
      d.half_w = 0.5f * (float)q.width;
      d.half_h = 0.5f * (float)q.height;
      d.jshift = d.half_w - 0.5f;
      d.ishift = d.half_h - 0.5f;
      d.w = q.width;
      d.h = q.height;
      d.tiles_x = (q.width + tile - 1) / tile;
      d.tiles_y = (q.height + tile - 1) / tile;
      d.px_off = q.pixel_offset;
      d.pad = 0;
      d.pad2[0] = d.pad2[1] = d.pad2[2] = d.pad2[3] = 0;
      ntiles = d.tiles_x * d.tiles_y;
      d.tile_off = 0;
      v.planes[p] = d;
    }
    int tot;
    const int excl = block_excl_scan<int>(ntiles, &tot);
    if (p < P) {
      v.planes[p].tile_off = s_run + excl;
      v.tile_off[p] = s_run + excl;
    }
    __syncthreads();
    if (tid == 0) s_run += tot;
    __syncthreads();
  }
  if (tid == 0) {
    v.tile_off[P] = s_run;
    if (s_run != total_tiles) dev_fail(v.hdr, UG_ERR_INVALID_PLANE, -1);
  }
}

// ------------------------------------------------------------------ 1. cull
// A conservative FP32 test per (plane, Gaussian), the same arithmetic for every
// lane (no sqrt, no divergent branch): it keeps every pair that the exact
// test in the record kernels can accept, and drops the rest.
//   phase 1:  (|m3| - Bm)^2 <= chi2 (S33 + B33) (1 + 2e-3)
//   image:    the pixel box with half-extent sqrt(chi2) ||Fi||_F >= sqrt(chi2
//             Sigma3D_kk) (plus one pixel) overlaps the image.
// Fi is the inverse factor (FP64-computed and rounded for ill-conditioned
// Gaussians). With z = Fi r computed in FP32 (|r_k| <= 1), rs[i] = sum_k
// |Fi_ik| and R2 = sum_i rs[i]^2:
//   |z_i - z_i*| <= 5 eps rs[i],  |S - S*| <= 10 eps sqrt(S R2) + 25 eps^2 R2 + 3 eps S,
//   |m - m*| <= 8 eps sum_k |mu_k - o_k|   (eps = 2^-24);
// the factor 1 + 2e-3 also covers the FP32 forward substitution of ordinary
// Gaussians (axis-ratio proxy <= fp64_ratio).
struct CullGauss {
  float mu[3];
  float Fi[3][3];
  float R2;
  float hb;  // sqrt(chi2) ||Fi||_F: bound of every half-extent
};

template <typename PL>
__device__ __forceinline__ bool cull_pair(const CullGauss& c, const PL& pl, float chi2) {
  const float eps = 5.9604645e-8f;
  float d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = c.mu[k] - pl.o[k];
  const float Bm = 8.f * eps * (fabsf(d[0]) + fabsf(d[1]) + fabsf(d[2])) * 1.001f + 1e-30f;
  const float m3 = fmaf(pl.n[2], d[2], fmaf(pl.n[1], d[1], pl.n[0] * d[0]));
  float S = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float z = fmaf(c.Fi[i][2], pl.n[2], fmaf(c.Fi[i][1], pl.n[1], c.Fi[i][0] * pl.n[0]));
    S = fmaf(z, z, S);
  }
  // sqrt(S R2) <= (S + R2) / 2 keeps the bound free of a square root
  const float B = 5.f * eps * (S + c.R2) + 25.f * eps * eps * c.R2 + 3.f * eps * S;
  const float lo = fmaxf(fabsf(m3) - Bm, 0.f);
  const bool ph1 = lo * lo <= chi2 * (S + B) * 1.002f;
  const float m1 = fmaf(pl.u[2], d[2], fmaf(pl.u[1], d[1], pl.u[0] * d[0]));
  const float m2 = fmaf(pl.v[2], d[2], fmaf(pl.v[1], d[1], pl.v[0] * d[0]));
  const float h = c.hb + Bm;
  const float cj = fmaf(m1, pl.inv_pu, pl.jshift), hj = fmaf(h, pl.inv_pu, 1.f);
  const float ci = fmaf(m2, pl.inv_pv, pl.ishift), hi = fmaf(h, pl.inv_pv, 1.f);
  const bool img = cj + hj >= 0.f && cj - hj <= (float)(pl.w - 1) && ci + hi >= 0.f &&
                   ci - hi <= (float)(pl.h - 1);  // (w - 1, h - 1 exact in FP32)
  return ph1 && img;
}

struct LaneGauss {
  GaussParams prm;
  Factor<float> ff;
  bool active, use64;
};

// The extended-precision branch takes a Gaussian when its axis-ratio proxy
// exceeds `ratio`, or when ||F||_F (|mu| + the planes' largest |o|) exceeds
// `reach`: the latter bounds, in units of the Gaussian's smallest scale, how
// far the FP32 difference mu - o and the products F^T (mu - o) are from the
// numbers they cancel to near the Gaussian, so it bounds the FP32 geometry's
// error in t (a few 1e-7 times the bound).
template <int COV>
__device__ __forceinline__ void lane_setup(const ug_gaussians& g, int64_t n, int64_t i, float beta,
                                           float ratio, float reach, float oreach, LaneGauss& L) {
  L.active = i < n;
  L.use64 = false;
  if (!L.active) return;
  load_params(g, n, i, COV, L.prm);
  make_factor<float, COV>(L.prm, beta, L.ff);
  float fro = 0.f;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) fro = fmaf(L.ff.F[r][k], L.ff.F[r][k], fro);
  const float mu = sqrtf(fmaf(L.prm.mu[2], L.prm.mu[2],
                              fmaf(L.prm.mu[1], L.prm.mu[1], L.prm.mu[0] * L.prm.mu[0])));
  const float size = sqrtf(fro) * (mu + oreach) * 1.001f;
  L.use64 = !(axis_ratio_proxy<COV>(L.ff) <= ratio) || !(size <= reach);
}

constexpr int kCullPlanesSmem = 64;  // planes staged in shared memory per pass

// The plane fields the cull reads, 19 words (odd: lanes reading different
// planes hit different banks).
struct CullPlane {
  float o[3], u[3], v[3], n[3];
  float inv_pu, inv_pv, jshift, ishift;
  int32_t w, h, pad;
};

// A warp's Gaussians for the second test, structure of arrays.
struct CullWarp {
  float mu[3][32];
  float Fi[9][32];
  float R2[32], hb[32];
  uint32_t bits[kCullPlanesSmem];  // candidate bits of the current plane group
};

// Two tests per (Gaussian, plane). The first is the plane distance against the
// Gaussian's largest extent, |m3| - Bm <= sqrt(chi2 smax) with smax >= S + B:
// S = |Fi n|^2 <= ||Fi||_F^2 |n|^2 and |n|^2 <= 1.0004 for a valid plane, so it
// passes every pair that cull_pair passes. It is evaluated as m3' = n.mu - n.o
// with n.o per plane: three roundings in n.mu and in n.o (|n_k| <= 1.0001) and
// one in the difference keep |m3' - n.(mu - o)| below 4.01 eps (|mu|_1 + |o|_1).
// cull_pair passes only if |m3| <= sqrt(thr1) + Bm with its own m3 within Bm =
// 8.008 eps |mu - o|_1 of n.(mu - o), so |m3'| <= sqrt(thr1) + 2 Bm + 4.01 eps
// (|mu|_1 + |o|_1) <= sqrt(thr1) + 20.03 eps (|mu|_1 + |o|_1): the test |m3'| <=
// sqrt(thr1) + 24 eps (|mu|_1 + sqrt(3) max|o|) (one threshold per Gaussian,
// rounded up) passes every pair that cull_pair passes. Pairs that pass it
// take the full test 32 at a time, every lane busy.
template <int COV>
__global__ void __launch_bounds__(256)
    k_cull(ug_gaussians g, int64_t n, int P, float chi2, float beta, float ratio, float reach,
           int64_t chunks, WsView v) {
  __shared__ CullPlane s_pl[kCullPlanesSmem];
  __shared__ float4 s_no[kCullPlanesSmem];  // (n, n.o) of each plane, for the first test
  __shared__ CullWarp s_w[256 / 32];
  if (dev_failed(v.hdr)) return;
  const int64_t chunk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  CullWarp& W = s_w[threadIdx.x >> 5];
  const bool live_warp = chunk < chunks;
  LaneGauss L;
  L.active = false;
  L.use64 = false;
  if (live_warp)
    lane_setup<COV>(g, n, chunk * kChunk + lane, beta, ratio, reach, v.hdr->origin_reach, L);
  float thr1;  // first test: lo^2 <= thr1
  {
    float Fi[3][3];
    if (L.use64) {
      Factor<dd> fd;
      make_factor<dd, COV>(L.prm, beta, fd);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) Fi[i][k] = (float)fd.Fi[i][k];
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) Fi[i][k] = L.active ? L.ff.Fi[i][k] : 0.f;
    }
    float R2 = 0.f, fro = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      W.mu[i][lane] = L.active ? L.prm.mu[i] : 0.f;
      float rs = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        W.Fi[3 * i + k][lane] = Fi[i][k];
        rs += fabsf(Fi[i][k]);
        fro = fmaf(Fi[i][k], Fi[i][k], fro);
      }
      R2 = fmaf(rs, rs, R2);
    }
    R2 *= 1.001f;
    W.R2[lane] = R2;
    W.hb[lane] = sqrtf(chi2 * fro) * 1.001f;
    const float eps = 5.9604645e-8f;
    const float smax = fro * 1.001f;
    const float bmax = 5.f * eps * (smax + R2) + 25.f * eps * eps * R2 + 3.f * eps * smax;
    thr1 = L.active ? chi2 * (smax + bmax) * 1.0021f : -1.f;
  }
  // first test |m3| <= T (inactive lanes: T < 0, never passes)
  float T = -1.f;
  if (L.active) {
    const float eps = 5.9604645e-8f;
    const float mu1 = __fadd_ru(__fadd_ru(fabsf(L.prm.mu[0]), fabsf(L.prm.mu[1])),
                                fabsf(L.prm.mu[2]));
    const float o1 = __fmul_ru(1.7320509f, v.hdr->origin_reach);
    const float Bm = __fadd_ru(__fmul_ru(__fmul_ru(24.f * eps, __fadd_ru(mu1, o1)), 1.001f), 1e-30f);
    T = __fadd_ru(__fsqrt_ru(thr1), Bm);
  }
  uint32_t fl = 0;  // the chunk's Gaussians on the extended branch
  if (live_warp) {
    fl = __ballot_sync(0xffffffffu, L.use64);
    if (lane == 0) v.gflag[chunk] = fl;
  }
  const float mx = W.mu[0][lane], my = W.mu[1][lane], mz = W.mu[2][lane];
  for (int p0 = 0; p0 < P; p0 += kCullPlanesSmem) {
    const int np = min(kCullPlanesSmem, P - p0);
    __syncthreads();
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
      const PlaneDev& d = v.planes[p0 + q];
      CullPlane c;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        c.o[k] = d.o[k];
        c.u[k] = d.u[k];
        c.v[k] = d.v[k];
        c.n[k] = d.n[k];
      }
      c.inv_pu = d.inv_pu;
      c.inv_pv = d.inv_pv;
      c.jshift = d.jshift;
      c.ishift = d.ishift;
      c.w = d.w;
      c.h = d.h;
      c.pad = 0;
      s_pl[q] = c;
      s_no[q] = make_float4(d.n[0], d.n[1], d.n[2],
                            fmaf(d.n[2], d.o[2], fmaf(d.n[1], d.o[1], d.n[0] * d.o[0])));
    }
    __syncthreads();
    if (!live_warp) continue;
    for (int q = lane; q < kCullPlanesSmem; q += 32) W.bits[q] = 0u;
    // 32 planes at a time: every lane tests its Gaussian against each plane
    // (bit j of `pass`), the bits are transposed so that lane j holds plane
    // j's passing Gaussians, and the pairs, numbered plane by plane, take the
    // full test 32 at a time (every lane busy)
    for (int g0 = 0; g0 < np; g0 += 32) {
      const int ng = min(32, np - g0);
      uint32_t pass = 0;
#pragma unroll 8
      for (int j = 0; j < 32; ++j) {
        const float4 nq = s_no[g0 + j];
        const float m3 = __fsub_rn(
            __fmaf_rn(nq.z, mz, __fmaf_rn(nq.y, my, __fmul_rn(nq.x, mx))), nq.w);
        pass |= (uint32_t)((fabsf(m3) <= T) & (j < ng)) << j;
      }
      const uint32_t pm = warp_bit_transpose(pass, lane);  // plane g0 + lane's Gaussians
      const uint32_t cnt = (uint32_t)__popc(pm);
      const uint32_t incl = warp_incl_scan(cnt);
      const uint32_t excl = incl - cnt;
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      for (uint32_t rb = 0; rb < total; rb += 32u) {
        const uint32_t e = rb + (uint32_t)lane;
        const int j = warp_search(excl, e);  // the plane of pair e
        const uint32_t mj = __shfl_sync(0xffffffffu, pm, j);
        const uint32_t ej = __shfl_sync(0xffffffffu, excl, j);
        if (e < total) {
          const int el = (int)nth_set_bit(mj, e - ej);
          const int eq = g0 + j;
          CullGauss c;
#pragma unroll
          for (int k = 0; k < 3; ++k) c.mu[k] = W.mu[k][el];
#pragma unroll
          for (int k = 0; k < 9; ++k) c.Fi[k / 3][k % 3] = W.Fi[k][el];
          c.R2 = W.R2[el];
          c.hb = W.hb[el];
          if (cull_pair(c, s_pl[eq], chi2)) atomicOr(&W.bits[eq], 1u << el);
        }
      }
    }
    __syncwarp();
    for (int q = lane; q < np; q += 32) v.mask[chunk * P + p0 + q] = W.bits[q];
    // the candidate scan's block partials (records, FP64 records): this
    // group's entries are consecutive, so they fall into at most two scan
    // blocks; the counts (at most 64 x 32 each) travel as 16-bit halves
    {
      const int64_t e0 = chunk * P + p0, b0 = e0 / kScanItems;
      const int split = (int)min((int64_t)np, (b0 + 1) * kScanItems - e0);
      uint32_t c_all = 0, c_64 = 0;
      for (int q = lane; q < np; q += 32) {
        const uint32_t m = W.bits[q], sh = q < split ? 0u : 16u;
        c_all += (uint32_t)__popc(m) << sh;
        c_64 += (uint32_t)__popc(m & fl) << sh;
      }
      c_all = warp_sum(c_all);
      c_64 = warp_sum(c_64);
      if (lane < 4) {
        const uint32_t x = ((lane & 1) ? c_64 : c_all) >> (lane < 2 ? 0 : 16) & 0xffffu;
        if (x) atomicAdd(&v.scan_part[(b0 + (lane >> 1)) * 2 + (lane & 1)], (unsigned long long)x);
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ 2. scan
struct CandLoad {
  const uint32_t* mask;
  const uint32_t* gflag;
  int P;
  __device__ void operator()(int64_t e, uint32_t out[2]) const {
    const uint32_t m = mask[e];
    out[0] = __popc(m);
    out[1] = __popc(m & gflag[e / P]);
  }
};
struct CandStore {
  uint32_t* slot_base;
  uint32_t* f64_base;
  __device__ void operator()(int64_t e, const uint32_t ex[2]) const {
    slot_base[e] = ex[0];
    f64_base[e] = ex[1];
  }
};

// ------------------------------------------------------------------ 3. list
// One warp per chunk of 32 Gaussians, 32 planes at a time: the lanes load the
// planes' candidate masks and bases (one plane per lane, coalesced), the
// masks are transposed so that every lane holds its own Gaussian's planes, and
// each lane writes the list entries of its candidates (its record slot and its
// place in the FP32 or the FP64 part) with the planes' data from shared memory.
__global__ void __launch_bounds__(256) k_list(int P, int64_t chunks, WsView v) {
  __shared__ uint32_t s_m[8][32], s_b[8][32], s_f[8][32];
  if (dev_failed(v.hdr)) return;
  const int64_t chunk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (chunk >= chunks) return;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const uint32_t fl = v.gflag[chunk];
  const uint32_t n32 = v.hdr->slots - v.hdr->slots64;
  const uint32_t lt = lanemask_lt();
  const bool ext = (fl >> lane) & 1u;
  const uint32_t g = (uint32_t)(chunk * kChunk + lane);
  for (int p0 = 0; p0 < P; p0 += 32) {
    const int pl = p0 + lane;
    const int64_t e = chunk * P + pl;
    const uint32_t mq = pl < P ? __ldg(v.mask + e) : 0u;
    __syncwarp();  // the previous group's planes are read
    s_m[wl][lane] = mq;
    s_b[wl][lane] = pl < P ? __ldg(v.slot_base + e) : 0u;
    s_f[wl][lane] = pl < P ? __ldg(v.f64_base + e) : 0u;
    uint32_t mine = warp_bit_transpose(mq, lane);  // bit q: candidate on plane p0 + q
    __syncwarp();
    while (mine) {
      const int q = __ffs(mine) - 1;
      mine &= mine - 1u;
      const uint32_t mask = s_m[wl][q], base = s_b[wl][q], b64 = s_f[wl][q];
      const uint32_t slot = base + __popc(mask & lt);
      const uint32_t idx = ext ? n32 + b64 + __popc(mask & fl & lt)
                               : (base - b64) + __popc(mask & ~fl & lt);
      v.list[idx] = make_uint4(g, (uint32_t)(p0 + q), slot, 0u);
    }
  }
}

// ------------------------------------------------------------------ 4. records

// Split of x - n (n an integer) into a high part and the remainder.
__device__ __forceinline__ void split_rel(float x, int n, float& h, float& l) {
  const float b = -(float)n;
  h = __fadd_rn(x, b);
  const float xp = __fsub_rn(h, b), bp = __fsub_rn(h, xp);
  l = __fadd_rn(__fsub_rn(x, xp), __fsub_rn(b, bp));
}
__device__ __forceinline__ void split_rel(dd x, int n, float& h, float& l) {
  // a double word plus an FP32 number (DWPlusFP of Joldes, Muller and Popescu)
  const dd s = two_sum(x.hi, (float)(-n));
  const dd r = fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
  h = r.hi;
  l = r.lo;
}
__device__ __forceinline__ void split_hl(float x, float& h, float& l) {
  h = x;
  l = 0.f;
}
__device__ __forceinline__ void split_hl(dd x, float& h, float& l) {
  h = x.hi;
  l = x.lo;
}

// The record (see ug_internal.cuh) and the inputs of the backward chain
// (kChainFloats floats: q1[3], q2[3], nh[3], rho3, ew[3], r11, r12, r22, with
// r12 = r11 kappa formed in FP32 from the record's high parts, so the chain
// reads the pixel-unit factor from here instead of the render words).
template <typename T>
__device__ __forceinline__ void write_record(const PairLsq<T>& L, const PairBox& pb,
                                             const GaussParams& prm, float chi2, WsView& v,
                                             uint32_t slot) {
  float xh, xl, yh, yl, kh, kl;
  split_rel(L.X, pb.j0, xh, xl);
  split_rel(L.Y, pb.i0, yh, yl);
  split_hl(L.kappa, kh, kl);
  const float q0 = __fmul_rn(L.rho3, L.rho3);
  const float lw2 = log2_sigmoid(prm.logit) - kHalfLog2e * q0;
  const float ethr = kHalfLog2e * (chi2 - q0);
  v.rec_a[slot] = make_float4(xh, yh, L.r11, kh);
  v.rec_b[slot] = make_float4(L.r22, lw2, prm.c, ethr);
  v.rec_c[slot] = make_float4(xl, yl, kl, 0.f);
  v.rec_box[slot] = make_uint2((uint32_t)pb.j0 | ((uint32_t)pb.j1 << 16),
                               (uint32_t)pb.i0 | ((uint32_t)pb.i1 << 16));
  float4* d4 = reinterpret_cast<float4*>(v.rec_chain + (size_t)slot * kChainFloats);
  d4[0] = make_float4(L.q1[0], L.q1[1], L.q1[2], L.q2[0]);
  d4[1] = make_float4(L.q2[1], L.q2[2], L.nh[0], L.nh[1]);
  d4[2] = make_float4(L.nh[2], L.rho3, L.ew[0], L.ew[1]);
  d4[3] = make_float4(L.ew[2], L.r11, __fmul_rn(L.r11, kh), L.r22);
}

__device__ __forceinline__ bool box_empty(uint2 b) {
  return (b.x & 0xffffu) > (b.x >> 16) || (b.y & 0xffffu) > (b.y >> 16);
}

template <typename T, int COV>
__global__ void __launch_bounds__(256)
    k_records(ug_gaussians g, int64_t n, int ts, int cut, float chi2, float beta, WsView v,
              int part) {
  if (dev_failed(v.hdr)) return;
  const uint32_t slots = v.hdr->slots, n64 = v.hdr->slots64;
  const uint32_t begin = part == 0 ? 0u : slots - n64;
  const uint32_t end = part == 0 ? slots - n64 : slots;
  unsigned long long npx = 0;
  uint32_t holes = 0, kept = 0;
  // the next entry of the list is read one iteration ahead
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t k = begin + blockIdx.x * blockDim.x + threadIdx.x;
  uint4 e_next = k < end ? v.list[k] : make_uint4(0u, 0u, 0u, 0u);
  for (; k < end; k += stride) {
    const uint4 e = e_next;
    if (k + stride < end) e_next = v.list[k + stride];
    const uint32_t slot = e.z;
    const PlaneDev pl = v.planes[e.y];
    GaussParams prm;
    load_params(g, n, e.x, COV, prm);
    Factor<T> f;
    make_factor<T, COV>(prm, beta, f);
    // the decisions (phase 1, pixel box) in FP32 for both branches; the render
    // geometry in T from the exact mean offset
    const PairBox pb = pair_box_f32<T, COV>(f, pl, chi2);
    v.rec_plane[slot] = e.y;
    if (pb.visible) {
      PairGeo<T> gg;
      mean_offset(prm.mu, pl.o, gg.d);
      PairLsq<T> L;
      pair_lsq<T, COV>(f, pl, gg, L);
      write_record<T>(L, pb, prm, chi2, v, slot);
      npx += (unsigned long long)(pb.j1 - pb.j0 + 1) * (unsigned long long)(pb.i1 - pb.i0 + 1);
      kept++;
    } else {
      v.rec_box[slot] = make_uint2(1u, 1u);  // empty: j0 = 1 > j1 = 0
      holes++;
    }
  }
  npx = warp_sum(npx);
  holes = warp_sum(holes);
  kept = warp_sum(kept);
  if ((threadIdx.x & 31) == 0) {
    if (npx) atomicAdd(&v.hdr->box_pixels, npx);
    if (holes) atomicAdd(&v.hdr->holes, holes);
    if (part == 1 && kept) atomicAdd(&v.hdr->kept64, kept);
  }
}

struct SlotLoad {
  const uint32_t* cnt;
  const WsHeader* hdr;
  __device__ void operator()(int64_t e, uint32_t out[1]) const {
    out[0] = e < (int64_t)hdr->slots ? cnt[e] : 0u;
  }
};
struct SlotStore {
  uint32_t* off;
  const WsHeader* hdr;
  __device__ void operator()(int64_t e, const uint32_t ex[1]) const {
    if (e < (int64_t)hdr->slots) off[e] = ex[0];
  }
};

// ------------------------------------------------------------------ 5. emit
// Box-tile geometry of one record slot, for the live-tile pass and the emit.
struct SlotTiles {
  uint32_t nt, nx, tx0, ty0;  // box tiles, tiles per box row, first tile column and row
  uint2 bx;                   // pixel box
};

__device__ __forceinline__ SlotTiles slot_tiles(uint2 bx, int ts) {
  SlotTiles q{0u, 1u, 0u, 0u, bx};
  if (!box_empty(bx)) {
    const int j0 = bx.x & 0xffff, j1 = bx.x >> 16, i0 = bx.y & 0xffff, i1 = bx.y >> 16;
    q.tx0 = (uint32_t)(j0 >> ts);
    q.ty0 = (uint32_t)(i0 >> ts);
    q.nx = (uint32_t)(j1 >> ts) - q.tx0 + 1;
    q.nt = q.nx * ((uint32_t)(i1 >> ts) - q.ty0 + 1);
  }
  return q;
}

// Whether box tile k (row-major within the record's box) can hold a non-zero
// weight of the record.
__device__ __forceinline__ bool box_tile_live(const float4& a, const float4& b, uint2 bx,
                                              uint32_t nx, uint32_t tx0, uint32_t ty0, uint32_t k,
                                              int ts, int cut) {
  const uint32_t dy = k / nx, dx = k - dy * nx;
  const int tile = 1 << ts, tx = (int)(tx0 + dx), ty = (int)(ty0 + dy);
  const int j0 = bx.x & 0xffff, j1 = bx.x >> 16, i0 = bx.y & 0xffff, i1 = bx.y >> 16;
  return rect_live(a, b, j0, i0, max(j0, tx * tile), min(j1, tx * tile + tile - 1),
                   max(i0, ty * tile), min(i1, ty * tile + tile - 1), cut);
}

constexpr uint32_t kMaskTiles = 64;  // boxes up to this many tiles keep their live-tile mask

// Live-tile pass, one warp per 32 consecutive record slots. The box tiles of
// those records form one sequence (record by record, row-major within a
// record); lane k tests tiles k, k + 32, ... of it (no lane waits for a record
// with many tiles), and every record's lane collects the ballot bits of its own
// tiles: the count of its live tiles (inst_off, scanned next into the first
// instance) and, for a box of at most 64 tiles, which ones (kept in the
// per-record gradient scratch, unused until the backward, for the emit).
__global__ void __launch_bounds__(256) k_live(int ts, int cut, WsView v) {
  __shared__ float4 s_a[8][32], s_b[8][32];
  __shared__ uint4 s_t[8][32];
  if (dev_failed(v.hdr)) return;
  const uint32_t slots = v.hdr->slots;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long* live_mask = reinterpret_cast<unsigned long long*>(v.rec_pgrad);
  for (uint32_t w0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32u; w0 < slots;
       w0 += warps * 32u) {
    const uint32_t slot = w0 + lane;
    SlotTiles q = slot_tiles(make_uint2(1u, 1u), ts);
    if (slot < slots) {  // the render data loaded with the box (read only for box tiles)
      const uint2 bx = v.rec_box[slot];
      s_a[wl][lane] = v.rec_a[slot];
      s_b[wl][lane] = v.rec_b[slot];
      q = slot_tiles(bx, ts);
    }
    s_t[wl][lane] = make_uint4(q.bx.x, q.bx.y, q.nx | (q.tx0 << 16), q.ty0);
    uint32_t incl = q.nt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const uint32_t bpre = incl - q.nt;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    uint32_t cnt = 0;
    unsigned long long mask = 0;
    for (uint32_t kb = 0; kb < total; kb += 32u) {
      const uint32_t k = kb + (uint32_t)lane;
      const int l = warp_search(bpre, k);
      const uint32_t lpre = __shfl_sync(0xffffffffu, bpre, l);
      bool live = false;
      if (k < total) {
        const uint4 t4 = s_t[wl][l];
        live = box_tile_live(s_a[wl][l], s_b[wl][l], make_uint2(t4.x, t4.y), t4.z & 0xffffu,
                             t4.z >> 16, t4.w, k - lpre, ts, cut);
      }
      const uint32_t bal = __ballot_sync(0xffffffffu, live);
      // this lane's record: its tiles in this window, [lo, hi) of the sequence
      const uint32_t lo = max(bpre, kb), hi = min(bpre + q.nt, kb + 32u);
      if (lo < hi) {
        const uint32_t len = hi - lo;
        const uint32_t bits = (bal >> (lo - kb)) & (len == 32u ? 0xffffffffu : ((1u << len) - 1u));
        cnt += (uint32_t)__popc(bits);
        if (q.nt <= kMaskTiles) mask |= (unsigned long long)bits << (lo - bpre);
      }
    }
    if (slot < slots) {
      v.inst_off[slot] = cnt;
      live_mask[slot] = mask;
    }
    // the record scan's block partial (the 32 slots lie in one scan block)
    const uint32_t wsum = warp_sum(cnt);
    if (lane == 0 && wsum) atomicAdd(&v.slot_part[w0 / kScanItems], (unsigned long long)wsum);
    __syncwarp();
  }
}

// The footprint tests of one (record, tile) instance (the key's top byte):
// every 8 x 8 footprint of the tile (tx, ty) in row-major order.
__device__ __forceinline__ uint32_t instance_footprints(const float4& a, const float4& b,
                                                       uint2 bx, int tx, int ty, int ts,
                                                       int cut) {
  const int tile = 1 << ts, fx = tile >> 3;
  if (tile == 16) return tile_footprints16(a, b, bx, tx * 16, ty * 16, cut);
  uint32_t fm = 0;
  for (int f = 0; f < fx * fx; ++f)
    fm |= footprint_bits(a, b, bx, tx * tile + (f % fx) * 8, ty * tile + (f / fx) * 8, 8, cut)
          << (2 * f);
  return fm;
}

// A warp emits the instances of 32 consecutive record slots together: their
// instances form one contiguous range (the slot scan), so lane k writes
// instances k, k + 32, ... of the range (coalesced stores, no lane waits for
// a record with many tiles); a record's live tiles come from its mask. The
// few records with more than 64 box tiles are emitted after, one at a time, by
// the whole warp re-testing their box tiles 32 at a time.
__global__ void __launch_bounds__(256, 4) k_emit(int ts, int cut, uint32_t inst_cap, WsView v) {
  // the warp's 32 records' render data, read once (coalesced) for the
  // footprint tests of all their instances
  __shared__ float4 s_a[8][32], s_b[8][32];
  __shared__ uint2 s_bx[8][32];
  // the record kernels' counts into the status (they have all finished)
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    v.hdr->st.fp64_records = (int64_t)v.hdr->kept64;
    v.hdr->st.box_pixels = (int64_t)v.hdr->box_pixels;
  }
  if (dev_failed(v.hdr)) return;
  const uint32_t slots = v.hdr->slots;
  const uint32_t n_inst = (uint32_t)v.hdr->st.instances;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const unsigned long long* live_mask = reinterpret_cast<const unsigned long long*>(v.rec_pgrad);
  for (uint32_t w0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32u; w0 < slots;
       w0 += warps * 32u) {
    const uint32_t slot = w0 + lane;
    // per lane: first instance (UINT32_MAX past the last slot, so the search
    // never picks it), live count, box tiles, key of the first box tile
    uint32_t pre = 0xffffffffu, cnt = 0, key0 = 0, tiles_x = 0;
    SlotTiles q = slot_tiles(make_uint2(1u, 1u), ts);
    unsigned long long mask = 0;
    if (slot < slots) {
      // every input of the slot loaded at once (used only when it has instances)
      pre = v.inst_off[slot];
      const uint32_t nxt = slot + 1 < slots ? v.inst_off[slot + 1] : n_inst;
      const uint2 bx = v.rec_box[slot];
      const uint32_t plane = v.rec_plane[slot];
      const unsigned long long lm = live_mask[slot];
      const float4 ra = v.rec_a[slot], rb = v.rec_b[slot];
      cnt = nxt - pre;
      if (cnt) {
        q = slot_tiles(bx, ts);
        const PlaneDev& pl = v.planes[plane];
        tiles_x = (uint32_t)pl.tiles_x;
        key0 = (uint32_t)pl.tile_off + q.ty0 * tiles_x + q.tx0;
        mask = lm;
        s_a[wl][lane] = ra;
        s_b[wl][lane] = rb;
        s_bx[wl][lane] = q.bx;
      }
    }
    __syncwarp();
    const int last = (int)min(31u, slots - 1u - w0);
    const uint32_t base = __shfl_sync(0xffffffffu, pre, 0);
    const uint32_t end = __shfl_sync(0xffffffffu, pre + cnt, last);
    for (uint32_t kb = base; kb < end; kb += 32u) {
      const uint32_t o = kb + (uint32_t)lane;
      const int l = warp_search(pre, o);
      const uint32_t l_pre = __shfl_sync(0xffffffffu, pre, l);
      const uint32_t l_nt = __shfl_sync(0xffffffffu, q.nt, l);
      const uint32_t l_nx = __shfl_sync(0xffffffffu, q.nx, l);
      const uint32_t l_key0 = __shfl_sync(0xffffffffu, key0, l);
      const uint32_t l_tx = __shfl_sync(0xffffffffu, tiles_x, l);
      const unsigned long long l_mask = __shfl_sync(0xffffffffu, mask, l);
      const uint32_t l_tx0 = __shfl_sync(0xffffffffu, q.tx0, l);
      const uint32_t l_ty0 = __shfl_sync(0xffffffffu, q.ty0, l);
      if (o < end && l_nt <= kMaskTiles && o < inst_cap) {
        const uint32_t pos = nth_set_bit(l_mask, o - l_pre);
        const uint32_t dy = pos / l_nx, dx = pos - dy * l_nx;
        const uint32_t l_slot = w0 + (uint32_t)l;
        const uint32_t fm = instance_footprints(s_a[wl][l], s_b[wl][l], s_bx[wl][l],
                                                (int)(l_tx0 + dx), (int)(l_ty0 + dy), ts, cut);
        v.keys[0][o] = (l_key0 + dy * l_tx + dx) | (fm << kKeyTileBits);
        v.vals[0][o] = l_slot;
      }
    }
    // records with more boxes tiles than a mask holds
    uint32_t big = __ballot_sync(0xffffffffu, cnt > 0 && q.nt > kMaskTiles);
    while (big) {
      const int r = __ffs(big) - 1;
      big &= big - 1;
      const uint32_t r_slot = w0 + (uint32_t)r;
      const uint32_t r_nt = __shfl_sync(0xffffffffu, q.nt, r);
      const uint32_t r_nx = __shfl_sync(0xffffffffu, q.nx, r);
      const uint32_t r_tx0 = __shfl_sync(0xffffffffu, q.tx0, r);
      const uint32_t r_ty0 = __shfl_sync(0xffffffffu, q.ty0, r);
      const uint32_t r_key0 = __shfl_sync(0xffffffffu, key0, r);
      const uint32_t r_tx = __shfl_sync(0xffffffffu, tiles_x, r);
      const uint2 r_bx = make_uint2(__shfl_sync(0xffffffffu, q.bx.x, r),
                                    __shfl_sync(0xffffffffu, q.bx.y, r));
      const float4 a = s_a[wl][r], b = s_b[wl][r];
      uint32_t out = __shfl_sync(0xffffffffu, pre, r);
      for (uint32_t kb = 0; kb < r_nt; kb += 32u) {
        const uint32_t k = kb + (uint32_t)lane;
        const bool live = k < r_nt && box_tile_live(a, b, r_bx, r_nx, r_tx0, r_ty0, k, ts, cut);
        const uint32_t bal = __ballot_sync(0xffffffffu, live);
        if (live) {
          const uint32_t o = out + (uint32_t)__popc(bal & lt);
          if (o < inst_cap) {
            const uint32_t dy = k / r_nx, dx = k - dy * r_nx;
            const uint32_t fm = instance_footprints(a, b, r_bx, (int)(r_tx0 + dx),
                                                    (int)(r_ty0 + dy), ts, cut);
            v.keys[0][o] = (r_key0 + dy * r_tx + dx) | (fm << kKeyTileBits);
            v.vals[0][o] = r_slot;
          }
        }
        out += (uint32_t)__popc(bal);
      }
    }
    __syncwarp();  // the shared records are read; the next slots may overwrite them
  }
}


static int tile_shift(int tile) { return tile == 8 ? 3 : 4; }

cudaError_t launch_setup_planes(const ug_plan* plan, const ug_plane* d_planes, WsView v,
                                cudaStream_t s) {
  k_setup_planes<<<1, 256, 0, s>>>(d_planes, plan->num_planes, plan->cfg.tile, plan->total_tiles,
                                    plan->total_pixels,
                                    scan_blocks(plan->chunks * plan->num_planes),
                                    scan_blocks(plan->record_capacity), v);
  return cudaGetLastError();
}

static unsigned list_grid(int64_t cap) {
  const int64_t want = (cap + 255) / 256;
  const int64_t most = (int64_t)device_sms() * 8;
  return (unsigned)std::max<int64_t>(1, std::min(want, most));
}

template <int COV>
static void launch_pre_cov(const ug_plan* plan, const ug_gaussians* g, WsView v, cudaStream_t s) {
  const int P = plan->num_planes;
  const int64_t chunks = plan->chunks;
  const int ts = tile_shift(plan->cfg.tile);
  const ug_config& c = plan->cfg;
  const int64_t wblocks = (chunks * 32 + 255) / 256;
  // the cull adds the candidate scan's block partials, the down-sweep scans
  // them (no cull without Gaussians: the header's counts stay zero)
  if (chunks > 0)
    k_cull<COV><<<(unsigned)wblocks, 256, 0, s>>>(*g, plan->n, P, c.chi2, c.beta, c.fp64_ratio,
                                                  c.fp32_reach, chunks, v);
  const int64_t entries = chunks * P;
  const int64_t nblk = scan_blocks(entries);
  CandLoad ld{v.mask, v.gflag, P};
  CandStore st{v.slot_base, v.f64_base};
  if (nblk > 0)
    k_scan_down<2, CandLoad, CandStore, true><<<(unsigned)nblk, kScanThreads, 0, s>>>(
        ld, st, entries, v.scan_part, v.hdr, nblk, 1, plan->record_capacity);
  if (chunks > 0) k_list<<<(unsigned)wblocks, 256, 0, s>>>(P, chunks, v);
  const unsigned lg = list_grid(plan->record_capacity);
  k_records<float, COV><<<lg, 256, 0, s>>>(*g, plan->n, ts, c.cutoff, c.chi2, c.beta, v, 0);
  k_records<dd, COV><<<lg, 256, 0, s>>>(*g, plan->n, ts, c.cutoff, c.chi2, c.beta, v, 1);
  // the live-tile pass adds the record scan's block partials, the down-sweep
  // scans them
  k_live<<<lg, 256, 0, s>>>(ts, c.cutoff, v);
  const int64_t rblk = scan_blocks(plan->record_capacity);
  SlotLoad sl{v.inst_off, v.hdr};
  SlotStore ss{v.inst_off, v.hdr};
  k_scan_down<1, SlotLoad, SlotStore, true><<<(unsigned)rblk, kScanThreads, 0, s>>>(
      sl, ss, plan->record_capacity, v.slot_part, v.hdr, rblk, 2, plan->instance_capacity);
  k_emit<<<lg, 256, 0, s>>>(ts, c.cutoff, (uint32_t)plan->instance_capacity, v);
}

cudaError_t launch_preprocess(const ug_plan* plan, const ug_gaussians* g, WsView v,
                              cudaStream_t s) {
  if (plan->cfg.cov_param == UG_COV_TRI) launch_pre_cov<UG_COV_TRI>(plan, g, v, s);
  else launch_pre_cov<UG_COV_SCALE_ROT>(plan, g, v, s);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ backward chain
// Per-record accumulators written by the backward rasterizer (8 floats), with
// g = w dL/dw at each pixel (dL/dw = r (c - C)):
//   [0] sum r w  (dL/dc)   [1] sum g   [2] sum g t1   [3] sum g t2
//   [4] sum g t1^2         [5] sum g t1 t2            [6] sum g t2^2
// In the record's least-squares frame (ug_geometry.cuh) the residual of a
// pixel is rho = F^T (X_w - mu) = (q1 t1 + q2 t2) / sc - rho3 nh, sc =
// sqrt(log2(e) / 2), and w = alpha exp(-|rho|^2 / 2), so
//   dL/dmu = F sum g rho,
//   dL/dF  = -sum g (X_w - mu) rho^T,  X_w - mu = pu dx u + pv dy v + ew,
// with (dx, dy) = R^-1 (t1, t2) for the pixel-unit factor R = [[r11, r12],
// [0, r22]]; every sum is a combination of the seven above.
struct ChainOut {
  float gmu[3];
  float gF[3][3];
  float glw2;
};

__device__ __forceinline__ void chain_record(const float* ch, float r11, float r12, float r22,
                                             const PlaneDev& pl, const float* F, const float* acc,
                                             ChainOut& o) {
  const float isc = 1.17741002251547469101f;  // 1 / sqrt(log2(e) / 2)
  const float q1[3] = {ch[0], ch[1], ch[2]}, q2[3] = {ch[3], ch[4], ch[5]};
  const float nh[3] = {ch[6], ch[7], ch[8]}, rho3 = ch[9];
  const float ew[3] = {ch[10], ch[11], ch[12]};
  const float Sg = acc[1], S1 = acc[2], S2 = acc[3], S11 = acc[4], S12 = acc[5], S22 = acc[6];
  float G[3], G1[3], G2[3], Gx[3], Gy[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    G[a] = fmaf(isc, fmaf(q1[a], S1, q2[a] * S2), -rho3 * nh[a] * Sg);    // sum g rho
    G1[a] = fmaf(isc, fmaf(q1[a], S11, q2[a] * S12), -rho3 * nh[a] * S1);  // sum g rho t1
    G2[a] = fmaf(isc, fmaf(q1[a], S12, q2[a] * S22), -rho3 * nh[a] * S2);  // sum g rho t2
    Gy[a] = G2[a] / r22;                                                    // sum g rho dy
    Gx[a] = (G1[a] - r12 * Gy[a]) / r11;                                    // sum g rho dx
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    o.gmu[k] = fmaf(F[3 * k + 2], G[2], fmaf(F[3 * k + 1], G[1], F[3 * k] * G[0]));
    const float pu_u = pl.pu * pl.u[k], pv_v = pl.pv * pl.v[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) o.gF[k][a] = -fmaf(pu_u, Gx[a], fmaf(pv_v, Gy[a], ew[k] * G[a]));
  }
  o.glw2 = kLn2 * Sg;
}

// Parameter gradient of one record (12 floats: mean[3], tri[6] or
// log_scale[3] + quat[4], logit, intensity; unused entries zero).
template <typename T, int COV>
__device__ __forceinline__ void record_param_grad(const ChainOut& o, const Factor<T>& f,
                                                  const GaussParams& prm, float gc, float* out) {
#pragma unroll
  for (int k = 0; k < 3; ++k) out[k] = o.gmu[k];
  const float alpha = sigmoidf(prm.logit);
  if (COV == UG_COV_TRI) {
    const float* t = prm.cp;
    out[3] = 2.f * t[0] * o.gF[0][0];
    out[4] = o.gF[1][0];
    out[5] = o.gF[2][0];
    out[6] = 2.f * t[3] * o.gF[1][1];
    out[7] = o.gF[2][1];
    out[8] = 2.f * t[5] * o.gF[2][2];
    out[9] = o.glw2 * (1.f - alpha) * kLog2e;
    out[10] = gc;
    out[11] = 0.f;
  } else {
    // F = R diag(1/s): dL/dR_ka = gF_ka / s_a, dL/dlog s_a = -sum_k gF_ka F_ka
    float gR[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float sinv = expf(-prm.cp[a]);
      float sacc = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        gR[k][a] = o.gF[k][a] * sinv;
        sacc += o.gF[k][a] * (float)f.F[k][a];
      }
      out[3 + a] = -sacc;
    }
    const float w = (float)f.qn[0], x = (float)f.qn[1], y = (float)f.qn[2], z = (float)f.qn[3];
    const float gw = 2.f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] -
                            y * gR[2][0] + x * gR[2][1]);
    const float gx = 2.f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2.f * x * gR[1][1] -
                            w * gR[1][2] + z * gR[2][0] + w * gR[2][1] - 2.f * x * gR[2][2]);
    const float gy = 2.f * (-2.f * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] +
                            z * gR[1][2] - w * gR[2][0] + z * gR[2][1] - 2.f * y * gR[2][2]);
    const float gz = 2.f * (-2.f * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] -
                            2.f * z * gR[1][1] + y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
    const float dot = gw * w + gx * x + gy * y + gz * z;
    const float inv = 1.f / (float)f.qnorm;
    out[6] = (gw - w * dot) * inv;
    out[7] = (gx - x * dot) * inv;
    out[8] = (gy - y * dot) * inv;
    out[9] = (gz - z * dot) * inv;
    out[10] = o.glw2 * (1.f - alpha) * kLog2e;
    out[11] = gc;
  }
}

// One thread per record (both parts of the work list), from the chain inputs
// the record kernels stored.
template <int COV>
__global__ void __launch_bounds__(256)
    k_chain(ug_gaussians g, int64_t n, float beta, WsView v) {
  if (dev_failed(v.hdr)) return;
  const uint32_t slots = v.hdr->slots;
  // the next entry of the list is read one iteration ahead, and every input
  // of a record is loaded before its box is tested (one round trip)
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  uint4 e_next = k < slots ? v.list[k] : make_uint4(0u, 0u, 0u, 0u);
  for (; k < slots; k += stride) {
    const uint4 e = e_next;
    if (k + stride < slots) e_next = v.list[k + stride];
    const uint32_t slot = e.z;
    const uint2 box = v.rec_box[slot];
    const float4 a0 = *reinterpret_cast<const float4*>(v.rec_grad + (size_t)slot * 8);
    const float4 a1 = *reinterpret_cast<const float4*>(v.rec_grad + (size_t)slot * 8 + 4);
    GaussParams prm;
    load_params(g, n, e.x, COV, prm);
    float ch[kChainFloats];
    const float4* c4 = reinterpret_cast<const float4*>(v.rec_chain + (size_t)slot * kChainFloats);
#pragma unroll
    for (int q = 0; q < kChainFloats / 4; ++q) {
      const float4 t = c4[q];
      ch[4 * q] = t.x;
      ch[4 * q + 1] = t.y;
      ch[4 * q + 2] = t.z;
      ch[4 * q + 3] = t.w;
    }
    float out[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) out[q] = 0.f;
    if (!box_empty(box)) {
      const float acc[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const PlaneDev& pl = v.planes[e.y];
      Factor<float> f;
      make_factor<float, COV>(prm, beta, f);
      float F[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) F[q] = f.F[q / 3][q % 3];
      ChainOut o;
      chain_record(ch, ch[13], ch[14], ch[15], pl, F, acc, o);
      record_param_grad<float, COV>(o, f, prm, acc[0], out);
    }
    float4* dst = reinterpret_cast<float4*>(v.rec_pgrad + (size_t)slot * 12);
    dst[0] = make_float4(out[0], out[1], out[2], out[3]);
    dst[1] = make_float4(out[4], out[5], out[6], out[7]);
    dst[2] = make_float4(out[8], out[9], out[10], out[11]);
  }
}

// Sum of the per-record parameter gradients of every Gaussian, in plane
// order (deterministic), written to the gradient rows. A chunk's records of a
// group of 32 planes occupy consecutive slots (the scan runs in (chunk, plane)
// order), so the warp reads them with full-width coalesced loads into a
// shared-memory window, kGatherWin records at a time. Every lane holds its own
// Gaussian's planes (the group's candidate masks transposed) and adds its
// records from each window, planes in ascending order: its slots ascend with
// the plane, so it stops at the first record beyond the window.
constexpr int kGatherWin = 96;

template <int COV>
__global__ void __launch_bounds__(256)
    k_gather(int64_t n, int P, int64_t chunks, WsView v, ug_gaussian_grads out) {
  __shared__ float4 win[256 / 32][kGatherWin * 3];
  __shared__ uint32_t s_m[256 / 32][32], s_b[256 / 32][32];
  if (dev_failed(v.hdr)) return;
  const int64_t chunk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (chunk >= chunks) return;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  float4* W = win[wl];
  const int64_t i = chunk * kChunk + lane;
  const uint32_t lt = lanemask_lt();
  float acc[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) acc[q] = 0.f;
  const float4* pg = reinterpret_cast<const float4*>(v.rec_pgrad);
  for (int p0 = 0; p0 < P; p0 += 32) {
    const int pl = p0 + lane, np = min(32, P - p0);
    const uint32_t mq = pl < P ? __ldg(v.mask + chunk * P + pl) : 0u;
    const uint32_t bq = pl < P ? __ldg(v.slot_base + chunk * P + pl) : 0u;
    // this plane group's slots: [first, last)
    const uint32_t first = __shfl_sync(0xffffffffu, bq, 0);
    const uint32_t last = __shfl_sync(0xffffffffu, bq + __popc(mq), np - 1);
    __syncwarp();  // the previous group's planes are read
    s_m[wl][lane] = mq;
    s_b[wl][lane] = bq;
    uint32_t mine = warp_bit_transpose(mq, lane);  // bit q: a record on plane p0 + q
    for (uint32_t w0 = first; w0 < last; w0 += kGatherWin) {
      const int cnt = (int)min((uint32_t)kGatherWin, last - w0);
      __syncwarp();  // the previous window is consumed
      for (int k = lane; k < cnt * 3; k += 32) W[k] = __ldg(pg + (size_t)w0 * 3 + k);
      __syncwarp();
      while (mine) {
        const int q = __ffs(mine) - 1;
        const uint32_t r = s_b[wl][q] + __popc(s_m[wl][q] & lt) - w0;
        if (r >= (uint32_t)cnt) break;  // this record and the later ones: a later window
        mine &= mine - 1u;
        const float4 x0 = W[3 * r], x1 = W[3 * r + 1], x2 = W[3 * r + 2];
        acc[0] += x0.x; acc[1] += x0.y; acc[2] += x0.z; acc[3] += x0.w;
        acc[4] += x1.x; acc[5] += x1.y; acc[6] += x1.z; acc[7] += x1.w;
        acc[8] += x2.x; acc[9] += x2.y; acc[10] += x2.z; acc[11] += x2.w;
      }
    }
  }
  if (i >= n) return;
#pragma unroll
  for (int k = 0; k < 3; ++k) out.mean[k * n + i] = acc[k];
  if (COV == UG_COV_TRI) {
#pragma unroll
    for (int k = 0; k < 6; ++k) out.tri[k * n + i] = acc[3 + k];
    out.opacity_logit[i] = acc[9];
    out.intensity[i] = acc[10];
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) out.log_scale[k * n + i] = acc[3 + k];
#pragma unroll
    for (int k = 0; k < 4; ++k) out.quat[k * n + i] = acc[6 + k];
    out.opacity_logit[i] = acc[10];
    out.intensity[i] = acc[11];
  }
}

template <int COV>
static void launch_chain_cov(const ug_plan* plan, const ug_gaussians* g, WsView v,
                             const ug_gaussian_grads* grads, cudaStream_t s) {
  const ug_config& c = plan->cfg;
  const unsigned lg = list_grid(plan->record_capacity);
  k_chain<COV><<<lg, 256, 0, s>>>(*g, plan->n, c.beta, v);
  const int64_t chunks = plan->chunks;
  if (chunks > 0)
    k_gather<COV><<<(unsigned)((chunks * 32 + 255) / 256), 256, 0, s>>>(plan->n, plan->num_planes,
                                                                         chunks, v, *grads);
}

cudaError_t launch_pre_backward(const ug_plan* plan, const ug_gaussians* g, WsView v,
                                const ug_gaussian_grads* grads, cudaStream_t s) {
  if (plan->cfg.cov_param == UG_COV_TRI) launch_chain_cov<UG_COV_TRI>(plan, g, v, grads, s);
  else launch_chain_cov<UG_COV_SCALE_ROT>(plan, g, v, grads, s);
  return cudaGetLastError();
}

}  // namespace ug
