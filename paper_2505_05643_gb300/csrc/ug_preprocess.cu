// Rows a1-a3 and a8: plane set-up, per-(plane, Gaussian) preprocess in two
// passes (count, then emit records and tile instances), and the chain rule
// from per-record gradients back to the Gaussian parameters.
//
// Work decomposition: one warp owns a chunk of 32 consecutive Gaussians
// (one per lane, structure-of-arrays loads are coalesced) and walks all
// planes, so the per-Gaussian factor (a1) is built once per step. Counts are
// kept per (chunk, plane); their exclusive scan in (chunk, plane) order gives
// every record its slot, so for any plane the records - and after the stable
// sort the tile lists - are in ascending Gaussian order.
#include "ug_geometry.cuh"
#include "ug_scan.cuh"

namespace ug {

// ------------------------------------------------------------------ planes
__global__ void __launch_bounds__(256)
    k_setup_planes(const ug_plane* planes, int P, int tile, int total_tiles,
                   int64_t total_px, WsView v) {
  __shared__ int s_run;
  const int tid = threadIdx.x;
  if (tid == 0) {
    WsHeader* h = v.hdr;
    h->st.status = 0;
    h->st.detail = 0;
    h->st.records = 0;
    h->st.instances = 0;
    h->st.fp64_records = 0;
    h->tile_counter[0] = 0;
    h->tile_counter[1] = 0;
    h->fp64_count = 0;
    h->box_pixels = 0;
    h->st.box_pixels = 0;
    s_run = 0;
  }
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
      PlaneDev d;
      for (int k = 0; k < 3; ++k) {
        d.o[k] = q.origin[k];
        d.u[k] = q.u[k];
        d.v[k] = q.v[k];
      }
      d.n[0] = q.u[1] * q.v[2] - q.u[2] * q.v[1];
      d.n[1] = q.u[2] * q.v[0] - q.u[0] * q.v[2];
      d.n[2] = q.u[0] * q.v[1] - q.u[1] * q.v[0];
      d.pu = q.pitch_u;
      d.pv = q.pitch_v;
      d.inv_pu = 1.f / q.pitch_u;
      d.inv_pv = 1.f / q.pitch_v;
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

// ------------------------------------------------------------------ passes
struct LaneGauss {
  GaussParams prm;
  Factor<float> ff;
  Factor<double> fd;
  bool active, use64;
};

template <int COV>
__device__ __forceinline__ void lane_setup(const ug_gaussians& g, int64_t n, int64_t i, float beta,
                                           float ratio, LaneGauss& L) {
  L.active = i < n;
  L.use64 = false;
  if (!L.active) return;
  load_params(g, n, i, COV, L.prm);
  make_factor<float, COV>(L.prm, beta, L.ff);
  L.use64 = !(axis_ratio_proxy<COV>(L.ff) <= ratio);
  if (L.use64) make_factor<double, COV>(L.prm, beta, L.fd);
}

__device__ __forceinline__ uint32_t tile_count(const PairBox& pb, int ts) {
  if (!pb.visible) return 0u;
  return (uint32_t)(((pb.j1 >> ts) - (pb.j0 >> ts) + 1) * ((pb.i1 >> ts) - (pb.i0 >> ts) + 1));
}

template <int COV>
__global__ void __launch_bounds__(256)
    k_pre_count(ug_gaussians g, int64_t n, int P, int ts, float chi2, float beta, float ratio,
                int64_t chunks, WsView v) {
  if (dev_failed(v.hdr)) return;
  const int64_t chunk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (chunk >= chunks) return;
  const int lane = threadIdx.x & 31;
  LaneGauss L;
  lane_setup<COV>(g, n, chunk * kChunk + lane, beta, ratio, L);
  for (int p = 0; p < P; ++p) {
    const PlaneDev pl = v.planes[p];
    PairBox pb;
    pb.visible = false;
    if (L.active) {
      if (L.use64) {
        PairGeo<double> gg;
        pb = pair_box<double, COV>(L.fd, pl, chi2, gg);
      } else {
        PairGeo<float> gg;
        pb = pair_box<float, COV>(L.ff, pl, chi2, gg);
      }
    }
    const uint32_t mask = __ballot_sync(0xffffffffu, pb.visible);
    const uint32_t tot = warp_sum(tile_count(pb, ts));
    if (lane == 0) {
      v.mask[chunk * P + p] = mask;
      v.inst_cnt[chunk * P + p] = tot;
    }
  }
}

template <typename T>
__device__ __forceinline__ void write_record(const PairRec<T>& rc, const PairGeo<T>& gg,
                                             const PlaneDev& pl, const PairBox& pb,
                                             const LaneGauss& L, float chi2, WsView& v,
                                             uint32_t rid) {
  const float xs_j = (float)(rc.xs1 * (T)pl.inv_pu + (T)pl.half_w);
  const float xs_i = (float)(rc.xs2 * (T)pl.inv_pv + (T)pl.half_h);
  const float q0 = (float)rc.q0;
  const float lw2 = log2_sigmoid(L.prm.logit) - kHalfLog2e * q0;
  const float ethr = kHalfLog2e * (chi2 - q0);
  v.rec_a[rid] = make_float4(xs_j, xs_i, (float)rc.r11, (float)rc.r12);
  v.rec_b[rid] = make_float4((float)rc.r22, lw2, L.prm.c, ethr);
  v.rec_box[rid] = make_uint2((uint32_t)pb.j0 | ((uint32_t)pb.j1 << 16),
                              (uint32_t)pb.i0 | ((uint32_t)pb.i1 << 16));
}

template <int COV>
__global__ void __launch_bounds__(256)
    k_pre_emit(ug_gaussians g, int64_t n, int P, int ts, float chi2, float beta, float ratio,
               int64_t chunks, WsView v, uint32_t rec_cap, uint32_t inst_cap) {
  if (dev_failed(v.hdr)) return;
  const int64_t chunk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (chunk >= chunks) return;
  const int lane = threadIdx.x & 31;
  LaneGauss L;
  lane_setup<COV>(g, n, chunk * kChunk + lane, beta, ratio, L);
  uint32_t n64 = 0;
  unsigned long long npx = 0;
  for (int p = 0; p < P; ++p) {
    const int64_t e = chunk * P + p;
    const uint32_t mask = v.mask[e];
    if (mask == 0u) continue;
    const bool mine = (mask >> lane) & 1u;
    const PlaneDev pl = v.planes[p];
    PairBox pb;
    pb.visible = false;
    const uint32_t rid = v.rec_base[e] + __popc(mask & lanemask_lt());
    const bool rid_ok = rid < rec_cap;  // always true after a successful count scan
    if (mine && !rid_ok) dev_fail(v.hdr, UG_ERR_INTERNAL, 3);
    if (mine && rid_ok) {
      if (L.use64) {
        PairGeo<double> gg;
        pb = pair_box<double, COV>(L.fd, pl, chi2, gg);
        if (pb.visible) {
          PairRec<double> rc;
          pair_record<double, COV>(L.fd, pl, gg, rc);
          write_record<double>(rc, gg, pl, pb, L, chi2, v, rid);
        }
        n64++;
      } else {
        PairGeo<float> gg;
        pb = pair_box<float, COV>(L.ff, pl, chi2, gg);
        if (pb.visible) {
          PairRec<float> rc;
          pair_record<float, COV>(L.ff, pl, gg, rc);
          write_record<float>(rc, gg, pl, pb, L, chi2, v, rid);
        }
      }
      if (!pb.visible) dev_fail(v.hdr, UG_ERR_INTERNAL, 1);
    }
    const uint32_t cnt = tile_count(pb, ts);
    const uint32_t incl = warp_incl_scan(cnt);
    const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 0 && tot != v.inst_cnt[e]) dev_fail(v.hdr, UG_ERR_INTERNAL, 2);
    if (mine && pb.visible) {
      npx += (unsigned long long)(pb.j1 - pb.j0 + 1) * (unsigned long long)(pb.i1 - pb.i0 + 1);
      uint32_t o = v.inst_base[e] + incl - cnt;
      const int tx0 = pb.j0 >> ts, tx1 = pb.j1 >> ts, ty0 = pb.i0 >> ts, ty1 = pb.i1 >> ts;
      uint32_t* keys = v.keys[0];
      uint32_t* vals = v.vals[0];
      for (int ty = ty0; ty <= ty1; ++ty) {
        const uint32_t row = (uint32_t)(pl.tile_off + ty * pl.tiles_x);
        for (int tx = tx0; tx <= tx1; ++tx) {
          if (o < inst_cap) {  // guards a count/emit disagreement (flagged above)
            keys[o] = row + (uint32_t)tx;
            vals[o] = rid;
          }
          ++o;
        }
      }
    }
  }
  const uint32_t w64 = warp_sum(n64);
  if (lane == 0 && w64) atomicAdd(&v.hdr->fp64_count, (unsigned long long)w64);
  const unsigned long long wpx = warp_sum(npx);
  if (lane == 0 && wpx) atomicAdd(&v.hdr->box_pixels, wpx);
}

__global__ void k_finish_pre(WsView v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    v.hdr->st.fp64_records = (int64_t)v.hdr->fp64_count;
    v.hdr->st.box_pixels = (int64_t)v.hdr->box_pixels;
  }
}

struct CountLoad {
  const uint32_t* mask;
  const uint32_t* cnt;
  __device__ void operator()(int64_t e, uint32_t out[2]) const {
    out[0] = __popc(mask[e]);
    out[1] = cnt[e];
  }
};
struct CountStore {
  uint32_t* rec_base;
  uint32_t* inst_base;
  __device__ void operator()(int64_t e, const uint32_t ex[2]) const {
    rec_base[e] = ex[0];
    inst_base[e] = ex[1];
  }
};

static int tile_shift(int tile) { return tile == 8 ? 3 : 4; }

cudaError_t launch_setup_planes(const ug_plan* plan, const ug_plane* d_planes, WsView v,
                                cudaStream_t s) {
  k_setup_planes<<<1, 256, 0, s>>>(d_planes, plan->num_planes, plan->cfg.tile, plan->total_tiles,
                                    plan->total_pixels, v);
  return cudaGetLastError();
}

cudaError_t launch_preprocess(const ug_plan* plan, const ug_gaussians* g, WsView v,
                              cudaStream_t s) {
  const int P = plan->num_planes;
  const int64_t chunks = plan->chunks;
  const int ts = tile_shift(plan->cfg.tile);
  const ug_config& c = plan->cfg;
  if (chunks > 0) {
    const int64_t blocks = (chunks * 32 + 255) / 256;
    if (c.cov_param == UG_COV_TRI)
      k_pre_count<UG_COV_TRI><<<(unsigned)blocks, 256, 0, s>>>(*g, plan->n, P, ts, c.chi2, c.beta,
                                                               c.fp64_ratio, chunks, v);
    else
      k_pre_count<UG_COV_SCALE_ROT><<<(unsigned)blocks, 256, 0, s>>>(
          *g, plan->n, P, ts, c.chi2, c.beta, c.fp64_ratio, chunks, v);
  }
  const int64_t entries = chunks * P;
  const int64_t nblk = scan_blocks(entries);
  CountLoad ld{v.mask, v.inst_cnt};
  CountStore st{v.rec_base, v.inst_base};
  if (nblk > 0) k_scan_partial<2, CountLoad><<<(unsigned)nblk, kScanThreads, 0, s>>>(ld, entries, v.scan_part, v.hdr);
  k_scan_top<2><<<1, 1024, 0, s>>>(v.scan_part, nblk, v.hdr, 1, plan->record_capacity,
                                   plan->instance_capacity);
  if (nblk > 0)
    k_scan_down<2, CountLoad, CountStore><<<(unsigned)nblk, kScanThreads, 0, s>>>(ld, st, entries, v.scan_part, v.hdr);
  if (chunks > 0) {
    const int64_t blocks = (chunks * 32 + 255) / 256;
    if (c.cov_param == UG_COV_TRI)
      k_pre_emit<UG_COV_TRI><<<(unsigned)blocks, 256, 0, s>>>(
          *g, plan->n, P, ts, c.chi2, c.beta, c.fp64_ratio, chunks, v,
          (uint32_t)plan->record_capacity, (uint32_t)plan->instance_capacity);
    else
      k_pre_emit<UG_COV_SCALE_ROT><<<(unsigned)blocks, 256, 0, s>>>(
          *g, plan->n, P, ts, c.chi2, c.beta, c.fp64_ratio, chunks, v,
          (uint32_t)plan->record_capacity, (uint32_t)plan->instance_capacity);
  }
  k_finish_pre<<<1, 32, 0, s>>>(v);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ backward chain
// Per-record accumulators written by the backward rasterizer (8 floats):
//   [0] sum r w        (dL/dc)
//   [1] sum gw w       (gw = dL/dw = r (c - C))
//   [2] sum gw w t1    [3] sum gw w t2
//   [4] sum gw w t1 dx [5] sum gw w t1 dy [6] sum gw w t2 dy
// With w = 2^(lw2 - t1^2 - t2^2) these give
//   dL/dlw2 = ln2 [1];  dL/dr11 = -2 ln2 [4];  dL/dr12 = -2 ln2 [5];
//   dL/dr22 = -2 ln2 [6];  dL/dxs_j = 2 ln2 r11 [2];
//   dL/dxs_i = 2 ln2 (r12 [2] + r22 [3]).
template <typename T>
struct ChainOut {
  T gmu[3];
  T gF[3][3];
  T glw2;  // for the logit
};

template <typename T>
__device__ __forceinline__ void chain_record(const PairRec<T>& rc, const PairGeo<T>& gg,
                                             const PlaneDev& pl, const float* acc, ChainOut<T>& o) {
  const T ln2 = (T)kLn2;
  const T a_p = (T)acc[1], a_t1 = (T)acc[2], a_t2 = (T)acc[3];
  const T a_t1dx = (T)acc[4], a_t1dy = (T)acc[5], a_t2dy = (T)acc[6];
  const T g_r11 = -2 * ln2 * a_t1dx;
  const T g_r12 = -2 * ln2 * a_t1dy;
  const T g_r22 = -2 * ln2 * a_t2dy;
  const T g_xsj = 2 * ln2 * rc.r11 * a_t1;
  const T g_xsi = 2 * ln2 * (rc.r12 * a_t1 + rc.r22 * a_t2);
  const T g_lw2 = ln2 * a_p;
  const T pu = (T)pl.pu, pv = (T)pl.pv;
  const T gx1 = g_xsj * (T)pl.inv_pu, gx2 = g_xsi * (T)pl.inv_pv;
  const T c = (T)kHalfLog2e;
  const T g_q0 = -c * g_lw2;
  // Cholesky backward of M = c D A D (M11 = r11^2, M12 = r11 r12, M22 = r12^2 + r22^2)
  const T gM22 = g_r22 / (2 * rc.r22);
  const T gr12 = g_r12 - g_r22 * rc.r12 / rc.r22;
  const T gM12 = gr12 / rc.r11;
  const T gr11 = g_r11 - gr12 * rc.r12 / rc.r11;
  const T gM11 = gr11 / (2 * rc.r11);
  T gA11 = c * pu * pu * gM11, gA12 = c * pu * pv * gM12, gA22 = c * pv * pv * gM22;
  // x* = m12 + m3 kappa, kappa = A^-1 s;  q0 = m3^2 (P33 - s^T A^-1 s)
  const T* b1 = rc.b[0];
  const T* b2 = rc.b[1];
  const T* b3 = rc.b[2];
  const T A11 = rc.nb1 * rc.nb1, A12 = b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2];
  const T A22 = b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2];
  const T det = rc.cr * rc.cr;
  const T gam0 = (A22 * gx1 - A12 * gx2) / det;
  const T gam1 = (A11 * gx2 - A12 * gx1) / det;
  const T m3 = gg.m[2];
  const T kp0 = rc.kappa[0], kp1 = rc.kappa[1];
  const T gm1 = gx1, gm2 = gx2;
  const T gm3 = gx1 * kp0 + gx2 * kp1 + 2 * rc.k * g_q0;
  const T m3sq_gq0 = m3 * m3 * g_q0;
  const T gs0 = m3 * gam0 - 2 * m3sq_gq0 * kp0;
  const T gs1 = m3 * gam1 - 2 * m3sq_gq0 * kp1;
  const T gP33 = m3sq_gq0;
  gA11 += -m3 * gam0 * kp0 + m3sq_gq0 * kp0 * kp0;
  gA12 += -m3 * (gam0 * kp1 + gam1 * kp0) + 2 * m3sq_gq0 * kp0 * kp1;
  gA22 += -m3 * gam1 * kp1 + m3sq_gq0 * kp1 * kp1;
  T gb1[3], gb2[3], gb3[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gb1[a] = 2 * gA11 * b1[a] + gA12 * b2[a] + gs0 * b3[a];
    gb2[a] = gA12 * b1[a] + 2 * gA22 * b2[a] + gs1 * b3[a];
    gb3[a] = gs0 * b1[a] + gs1 * b2[a] + 2 * gP33 * b3[a];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T u = (T)pl.u[k], vv = (T)pl.v[k], nn = (T)pl.n[k];
    o.gmu[k] += gm1 * u + gm2 * vv + gm3 * nn;
#pragma unroll
    for (int a = 0; a < 3; ++a) o.gF[k][a] += u * gb1[a] + vv * gb2[a] + nn * gb3[a];
  }
  o.glw2 += g_lw2;
}

template <int COV>
__global__ void __launch_bounds__(256)
    k_pre_bwd(ug_gaussians g, int64_t n, int P, float chi2, float beta, float ratio,
              int64_t chunks, WsView v, ug_gaussian_grads out) {
  if (dev_failed(v.hdr)) return;
  const int64_t chunk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (chunk >= chunks) return;
  const int lane = threadIdx.x & 31;
  const int64_t i = chunk * kChunk + lane;
  LaneGauss L;
  lane_setup<COV>(g, n, i, beta, ratio, L);
  ChainOut<float> of;
  ChainOut<double> od;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    of.gmu[k] = 0.f;
    od.gmu[k] = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      of.gF[k][a] = 0.f;
      od.gF[k][a] = 0.0;
    }
  }
  of.glw2 = 0.f;
  od.glw2 = 0.0;
  float gc = 0.f;
  for (int p = 0; p < P; ++p) {
    const int64_t e = chunk * P + p;
    const uint32_t mask = v.mask[e];
    if (!((mask >> lane) & 1u)) continue;
    const uint32_t rid = v.rec_base[e] + __popc(mask & lanemask_lt());
    const float4 a0 = *reinterpret_cast<const float4*>(v.rec_grad + (size_t)rid * 8);
    const float4 a1 = *reinterpret_cast<const float4*>(v.rec_grad + (size_t)rid * 8 + 4);
    const float acc[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    gc += acc[0];
    const PlaneDev pl = v.planes[p];
    if (L.use64) {
      PairGeo<double> gg;
      pair_box<double, COV>(L.fd, pl, chi2, gg);
      PairRec<double> rc;
      pair_record<double, COV>(L.fd, pl, gg, rc);
      chain_record<double>(rc, gg, pl, acc, od);
    } else {
      PairGeo<float> gg;
      pair_box<float, COV>(L.ff, pl, chi2, gg);
      PairRec<float> rc;
      pair_record<float, COV>(L.ff, pl, gg, rc);
      chain_record<float>(rc, gg, pl, acc, of);
    }
  }
  if (!L.active) return;
  float gmu[3], gF[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gmu[k] = of.gmu[k] + (float)od.gmu[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) gF[k][a] = of.gF[k][a] + (float)od.gF[k][a];
  }
  const float glw2 = of.glw2 + (float)od.glw2;
  const float alpha = sigmoidf(L.prm.logit);
#pragma unroll
  for (int k = 0; k < 3; ++k) out.mean[k * n + i] = gmu[k];
  out.opacity_logit[i] = glw2 * (1.f - alpha) * kLog2e;
  out.intensity[i] = gc;
  if (COV == UG_COV_TRI) {
    const float* t = L.prm.cp;
    out.tri[0 * n + i] = 2.f * t[0] * gF[0][0];
    out.tri[1 * n + i] = gF[1][0];
    out.tri[2 * n + i] = gF[2][0];
    out.tri[3 * n + i] = 2.f * t[3] * gF[1][1];
    out.tri[4 * n + i] = gF[2][1];
    out.tri[5 * n + i] = 2.f * t[5] * gF[2][2];
  } else {
    // F = R diag(1/s): dL/dR_ka = gF_ka / s_a, dL/dlog s_a = -sum_k gF_ka F_ka
    const Factor<float>& f = L.ff;
    float gR[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float sacc = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        gR[k][a] = gF[k][a] / f.s[a];
        sacc += gF[k][a] * f.F[k][a];
      }
      out.log_scale[a * n + i] = -sacc;
    }
    const float w = f.qn[0], x = f.qn[1], y = f.qn[2], z = f.qn[3];
    const float gw = 2.f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] -
                            y * gR[2][0] + x * gR[2][1]);
    const float gx = 2.f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2.f * x * gR[1][1] -
                            w * gR[1][2] + z * gR[2][0] + w * gR[2][1] - 2.f * x * gR[2][2]);
    const float gy = 2.f * (-2.f * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] +
                            z * gR[1][2] - w * gR[2][0] + z * gR[2][1] - 2.f * y * gR[2][2]);
    const float gz = 2.f * (-2.f * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] -
                            2.f * z * gR[1][1] + y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
    const float dot = gw * w + gx * x + gy * y + gz * z;
    const float inv = 1.f / f.qnorm;
    out.quat[0 * n + i] = (gw - w * dot) * inv;
    out.quat[1 * n + i] = (gx - x * dot) * inv;
    out.quat[2 * n + i] = (gy - y * dot) * inv;
    out.quat[3 * n + i] = (gz - z * dot) * inv;
  }
}

cudaError_t launch_pre_backward(const ug_plan* plan, const ug_gaussians* g, WsView v,
                                const ug_gaussian_grads* grads, cudaStream_t s) {
  const int64_t chunks = plan->chunks;
  if (chunks == 0) return cudaGetLastError();
  const ug_config& c = plan->cfg;
  const int64_t blocks = (chunks * 32 + 255) / 256;
  if (c.cov_param == UG_COV_TRI)
    k_pre_bwd<UG_COV_TRI><<<(unsigned)blocks, 256, 0, s>>>(*g, plan->n, plan->num_planes, c.chi2,
                                                           c.beta, c.fp64_ratio, chunks, v, *grads);
  else
    k_pre_bwd<UG_COV_SCALE_ROT><<<(unsigned)blocks, 256, 0, s>>>(
        *g, plan->n, plan->num_planes, c.chi2, c.beta, c.fp64_ratio, chunks, v, *grads);
  return cudaGetLastError();
}

}  // namespace ug
