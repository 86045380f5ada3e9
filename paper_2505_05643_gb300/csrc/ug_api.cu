// The C ABI entry points (include/ug.h): argument validation, the workspace
// plan, and the launch sequences of each hot-path row.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cmath>

#include "ug_internal.cuh"

using namespace ug;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool finite3(const float* a) { return isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]); }

ug_status check_config(const ug_config* c) {
  if (!c) return UG_ERR_INVALID_ARGUMENT;
  if (!(isfinite(c->chi2) && c->chi2 > 0.f)) return UG_ERR_INVALID_ARGUMENT;
  if (!(isfinite(c->beta) && c->beta > 0.f)) return UG_ERR_INVALID_ARGUMENT;
  if (!(isfinite(c->alpha_bg) && c->alpha_bg > 0.f)) return UG_ERR_INVALID_ARGUMENT;
  if (!isfinite(c->c_bg)) return UG_ERR_INVALID_ARGUMENT;
  if (c->cutoff != UG_CUTOFF_BOX && c->cutoff != UG_CUTOFF_BOX_AND_ELLIPSOID)
    return UG_ERR_INVALID_ARGUMENT;
  if (c->cov_param != UG_COV_TRI && c->cov_param != UG_COV_SCALE_ROT)
    return UG_ERR_INVALID_ARGUMENT;
  if (c->tile != 8 && c->tile != 16) return UG_ERR_NOT_SUPPORTED;
  if (c->variant < 0 || c->variant >= num_render_variants(c->tile)) return UG_ERR_NOT_SUPPORTED;
  if (c->variant_bwd < 0 || c->variant_bwd >= num_render_variants_bwd(c->tile))
    return UG_ERR_NOT_SUPPORTED;
  if (!(c->fp64_ratio > 0.f)) return UG_ERR_INVALID_ARGUMENT;
  if (!(c->fp32_reach > 0.f)) return UG_ERR_INVALID_ARGUMENT;  // both +inf: FP32 only
  return UG_OK;
}

ug_status check_plan(const ug_plan* p) {
  if (!p) return UG_ERR_INVALID_ARGUMENT;
  ug_status s = check_config(&p->cfg);
  if (s != UG_OK) return s;
  if (p->n < 0 || p->num_planes < 1 || p->total_tiles < 1 || p->workspace_bytes == 0)
    return UG_ERR_INVALID_ARGUMENT;
  return UG_OK;
}

ug_status check_ws(const ug_plan* p, const void* ws, size_t ws_bytes) {
  if (!ws) return UG_ERR_INVALID_ARGUMENT;
  if ((uintptr_t)ws % kAlign != 0) return UG_ERR_INVALID_ARGUMENT;
  if (ws_bytes < p->workspace_bytes) return UG_ERR_WORKSPACE_TOO_SMALL;
  return UG_OK;
}

ug_status check_gaussians(const ug_plan* p, const ug_gaussians* g) {
  if (!g) return UG_ERR_INVALID_ARGUMENT;
  if (p->n == 0) return UG_OK;
  if (!g->mean || !g->opacity_logit || !g->intensity) return UG_ERR_INVALID_ARGUMENT;
  if (p->cfg.cov_param == UG_COV_TRI && !g->tri) return UG_ERR_INVALID_ARGUMENT;
  if (p->cfg.cov_param == UG_COV_SCALE_ROT && (!g->log_scale || !g->quat))
    return UG_ERR_INVALID_ARGUMENT;
  return UG_OK;
}

ug_status cuda_status(cudaError_t e) { return e == cudaSuccess ? UG_OK : UG_ERR_CUDA; }

}  // namespace

extern "C" {

int32_t ug_version(void) { return 100; }

const char* ug_status_string(ug_status s) {
  switch (s) {
    case UG_OK: return "ok";
    case UG_ERR_INVALID_ARGUMENT: return "invalid argument";
    case UG_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case UG_ERR_CAPACITY: return "record or instance capacity exceeded";
    case UG_ERR_CUDA: return "CUDA error";
    case UG_ERR_TIMEOUT: return "bounded device wait gave up";
    case UG_ERR_NOT_SUPPORTED: return "not supported";
    case UG_ERR_INVALID_PLANE: return "invalid plane in device memory";
    case UG_ERR_INTERNAL: return "internal inconsistency";
  }
  return "unknown status";
}

int32_t ug_num_variants(int32_t tile) { return num_render_variants(tile); }
int32_t ug_num_variants_bwd(int32_t tile) { return num_render_variants_bwd(tile); }

ug_status ug_config_default(ug_config* cfg) {
  if (!cfg) return UG_ERR_INVALID_ARGUMENT;
  memset(cfg, 0, sizeof(*cfg));
  cfg->chi2 = 7.815f;
  cfg->beta = 1e-4f;
  cfg->alpha_bg = 1e-3f;
  cfg->c_bg = 0.f;
  cfg->cutoff = UG_CUTOFF_BOX;
  cfg->cov_param = UG_COV_TRI;
  cfg->tile = 16;
  cfg->variant = 0;
  cfg->variant_bwd = 0;
  cfg->fp64_ratio = 1e3f;
  cfg->fp32_reach = 20.f;
  return UG_OK;
}

ug_status ug_plan_init(const ug_config* cfg, int64_t n, const ug_plane* host_planes,
                       int32_t num_planes, int64_t record_capacity, int64_t instance_capacity,
                       ug_plan* plan) {
  if (!plan || !host_planes) return UG_ERR_INVALID_ARGUMENT;
  ug_status s = check_config(cfg);
  if (s != UG_OK) return s;
  if (n < 0 || n > ((int64_t)1 << 34) || num_planes < 1 || num_planes > (1 << 20))
    return UG_ERR_INVALID_ARGUMENT;
  if (record_capacity < 1 || record_capacity >= ((int64_t)1 << 31)) return UG_ERR_INVALID_ARGUMENT;
  if (instance_capacity < 1 || instance_capacity >= ((int64_t)1 << 31))
    return UG_ERR_INVALID_ARGUMENT;
  const int tile = cfg->tile;
  int64_t total_tiles = 0, total_px = 0;
  std::vector<std::pair<int64_t, int64_t>> spans;
  for (int p = 0; p < num_planes; ++p) {
    const ug_plane& q = host_planes[p];
    if (!finite3(q.origin) || !finite3(q.u) || !finite3(q.v)) return UG_ERR_INVALID_ARGUMENT;
    const double nu = sqrt((double)q.u[0] * q.u[0] + (double)q.u[1] * q.u[1] + (double)q.u[2] * q.u[2]);
    const double nv = sqrt((double)q.v[0] * q.v[0] + (double)q.v[1] * q.v[1] + (double)q.v[2] * q.v[2]);
    const double uv = (double)q.u[0] * q.v[0] + (double)q.u[1] * q.v[1] + (double)q.u[2] * q.v[2];
    if (fabs(nu - 1.0) > 1e-4 || fabs(nv - 1.0) > 1e-4 || fabs(uv) > 1e-4)
      return UG_ERR_INVALID_ARGUMENT;
    if (!(isfinite(q.pitch_u) && isfinite(q.pitch_v) && q.pitch_u > 0.f && q.pitch_v > 0.f))
      return UG_ERR_INVALID_ARGUMENT;
    if (q.width < 1 || q.height < 1 || q.width > 16384 || q.height > 16384 || q.reserved != 0)
      return UG_ERR_INVALID_ARGUMENT;
    if (q.pixel_offset < 0) return UG_ERR_INVALID_ARGUMENT;
    const int64_t npx = (int64_t)q.width * q.height;
    spans.push_back({q.pixel_offset, q.pixel_offset + npx});
    total_px = std::max(total_px, q.pixel_offset + npx);
    total_tiles += (int64_t)((q.width + tile - 1) / tile) * ((q.height + tile - 1) / tile);
  }
  std::sort(spans.begin(), spans.end());
  for (size_t k = 1; k < spans.size(); ++k)
    if (spans[k].first < spans[k - 1].second) return UG_ERR_INVALID_ARGUMENT;  // planes overlap
  if (total_tiles >= ((int64_t)1 << 31)) return UG_ERR_INVALID_ARGUMENT;

  memset(plan, 0, sizeof(*plan));
  plan->cfg = *cfg;
  plan->n = n;
  plan->num_planes = num_planes;
  plan->total_tiles = (int32_t)total_tiles;
  plan->total_pixels = total_px;
  plan->record_capacity = record_capacity;
  plan->instance_capacity = instance_capacity;
  int bits = 1;
  while (((int64_t)1 << bits) < total_tiles) ++bits;
  if (bits > kKeyTileBits) return UG_ERR_NOT_SUPPORTED;  // the key's top byte is taken
  plan->key_bits = bits;
  plan->sort_passes = (bits + 7) / 8;
  plan->chunks = (n + kChunk - 1) / kChunk;

  const int64_t P = num_planes;
  const int64_t entries = plan->chunks * P;
  const int64_t nblk_sort = sort_blocks(instance_capacity);
  const int64_t hist_entries = 256 * nblk_sort;
  size_t sz[kOffEnd];
  const int64_t rc = record_capacity, ic = instance_capacity;
  sz[kOffHeader] = sizeof(WsHeader);
  sz[kOffPlanes] = sizeof(PlaneDev) * (size_t)P;
  sz[kOffTileOff] = sizeof(int32_t) * (size_t)(P + 1);
  sz[kOffGFlag] = sizeof(uint32_t) * (size_t)plan->chunks;
  sz[kOffMask] = sizeof(uint32_t) * (size_t)entries;
  sz[kOffSlotBase] = sz[kOffMask];
  sz[kOffF64Base] = sz[kOffMask];
  sz[kOffScanPart] = 2 * sizeof(unsigned long long) * (size_t)(scan_blocks(entries) + 1);
  sz[kOffList] = sizeof(uint4) * (size_t)rc;
  sz[kOffRecA] = sizeof(float4) * (size_t)rc;
  sz[kOffRecB] = sizeof(float4) * (size_t)rc;
  sz[kOffRecC] = sizeof(float4) * (size_t)rc;
  sz[kOffRecBox] = sizeof(uint2) * (size_t)rc;
  sz[kOffRecPlane] = sizeof(uint32_t) * (size_t)rc;
  sz[kOffInstOff] = sizeof(uint32_t) * (size_t)rc;
  sz[kOffSlotPart] = sizeof(unsigned long long) * (size_t)(scan_blocks(rc) + 1);
  sz[kOffKeys0] = sizeof(uint32_t) * (size_t)ic;
  sz[kOffKeys1] = sz[kOffKeys0];
  sz[kOffVals0] = sz[kOffKeys0];
  sz[kOffVals1] = sz[kOffKeys0];
  sz[kOffSortHist] = sizeof(uint32_t) * (size_t)hist_entries;
  sz[kOffSortPart] = sizeof(unsigned long long) * (size_t)(scan_blocks(hist_entries) + 1);
  sz[kOffRanges] = sizeof(uint2) * (size_t)total_tiles;
  sz[kOffRecGrad] = 8 * sizeof(float) * (size_t)rc;
  sz[kOffRecPGrad] = 12 * sizeof(float) * (size_t)rc;
  sz[kOffRecChain] = kChainFloats * sizeof(float) * (size_t)rc;
  static_assert(kOffEnd <= 32, "ug_plan::off holds 32 sections");
  size_t off = 0;
  for (int k = 0; k < kOffEnd; ++k) {
    plan->off[k] = off;
    off = align_up(off + sz[k]);
  }
  plan->workspace_bytes = off;
  return UG_OK;
}

ug_status ug_preprocess(const ug_plan* plan, const ug_gaussians* gaussians,
                        const ug_plane* d_planes, void* ws, size_t ws_bytes, ug_stream stream) {
  ug_status s = check_plan(plan);
  if (s == UG_OK) s = check_ws(plan, ws, ws_bytes);
  if (s == UG_OK) s = check_gaussians(plan, gaussians);
  if (s != UG_OK) return s;
  if (!d_planes) return UG_ERR_INVALID_ARGUMENT;
  WsView v = make_view(plan, ws);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  s = cuda_status(launch_setup_planes(plan, d_planes, v, st));
  if (s != UG_OK) return s;
  return cuda_status(launch_preprocess(plan, gaussians, v, st));
}

ug_status ug_bin_sort(const ug_plan* plan, void* ws, size_t ws_bytes, ug_stream stream) {
  ug_status s = check_plan(plan);
  if (s == UG_OK) s = check_ws(plan, ws, ws_bytes);
  if (s != UG_OK) return s;
  return cuda_status(launch_bin_sort(plan, make_view(plan, ws), reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_render(const ug_plan* plan, void* ws, size_t ws_bytes, float* image, float* alpha,
                    ug_stream stream) {
  ug_status s = check_plan(plan);
  if (s == UG_OK) s = check_ws(plan, ws, ws_bytes);
  if (s != UG_OK) return s;
  if (!image || !alpha) return UG_ERR_INVALID_ARGUMENT;
  return cuda_status(launch_render(plan, make_view(plan, ws), image, alpha,
                                   reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_mse_loss_grad(const float* image, const float* target, int64_t n, float* grad_image,
                           float* loss, ug_stream stream) {
  if (!image || !target || !loss || n < 1) return UG_ERR_INVALID_ARGUMENT;
  return cuda_status(launch_mse(image, target, n, n, grad_image, loss,
                                reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_mse_loss_grad_part(const float* image, const float* target, int64_t n,
                                int64_t n_total, float* grad_image, float* loss,
                                ug_stream stream) {
  if (!image || !target || !loss || n < 1 || n_total < n) return UG_ERR_INVALID_ARGUMENT;
  return cuda_status(launch_mse(image, target, n, n_total, grad_image, loss,
                                reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_render_backward(const ug_plan* plan, const ug_gaussians* gaussians,
                             const ug_plane* d_planes, void* ws, size_t ws_bytes,
                             const float* image, const float* alpha, const float* grad_image,
                             const ug_gaussian_grads* grads, ug_stream stream) {
  ug_status s = check_plan(plan);
  if (s == UG_OK) s = check_ws(plan, ws, ws_bytes);
  if (s == UG_OK) s = check_gaussians(plan, gaussians);
  if (s != UG_OK) return s;
  if (!d_planes || !image || !alpha || !grad_image || !grads) return UG_ERR_INVALID_ARGUMENT;
  if (plan->n > 0) {
    if (!grads->mean || !grads->opacity_logit || !grads->intensity) return UG_ERR_INVALID_ARGUMENT;
    if (plan->cfg.cov_param == UG_COV_TRI && !grads->tri) return UG_ERR_INVALID_ARGUMENT;
    if (plan->cfg.cov_param == UG_COV_SCALE_ROT && (!grads->log_scale || !grads->quat))
      return UG_ERR_INVALID_ARGUMENT;
  }
  (void)d_planes;  // the plane table was derived into the workspace by ug_preprocess
  return cuda_status(launch_render_backward(plan, gaussians, make_view(plan, ws), image, alpha,
                                            grad_image, grads,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

size_t ug_ssim_scratch_floats(int32_t P, int32_t W, int32_t H) {
  if (P < 1 || W < 11 || H < 11) return 0;
  return ssim_scratch_floats(P, W, H);
}

ug_status ug_ssim(const float* image, const float* target, int32_t P, int32_t W, int32_t H,
                  float* scratch, size_t scratch_floats, float* ssim, float* psnr,
                  ug_stream stream) {
  if (!image || !target || !scratch || (!ssim && !psnr)) return UG_ERR_INVALID_ARGUMENT;
  if (P < 1 || W < 11 || H < 11 || W > 16384 || H > 16384) return UG_ERR_INVALID_ARGUMENT;
  if (scratch_floats < ssim_scratch_floats(P, W, H)) return UG_ERR_WORKSPACE_TOO_SMALL;
  return cuda_status(launch_ssim(image, target, P, W, H, scratch, ssim, psnr,
                                 reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_render_scatter(const ug_plan* plan, void* ws, size_t ws_bytes, float* image,
                            float* alpha, ug_stream stream) {
  ug_status s = check_plan(plan);
  if (s == UG_OK) s = check_ws(plan, ws, ws_bytes);
  if (s != UG_OK) return s;
  if (!image || !alpha) return UG_ERR_INVALID_ARGUMENT;
  return cuda_status(launch_render_scatter(plan, make_view(plan, ws), image, alpha,
                                           reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_render_backward_raster(const ug_plan* plan, void* ws, size_t ws_bytes,
                                    const float* image, const float* alpha,
                                    const float* grad_image, ug_stream stream) {
  ug_status s = check_plan(plan);
  if (s == UG_OK) s = check_ws(plan, ws, ws_bytes);
  if (s != UG_OK) return s;
  if (!image || !alpha || !grad_image) return UG_ERR_INVALID_ARGUMENT;
  return cuda_status(launch_render_backward_raster(plan, make_view(plan, ws), image, alpha,
                                                   grad_image,
                                                   reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_preprocess_backward(const ug_plan* plan, const ug_gaussians* gaussians, void* ws,
                                 size_t ws_bytes, const ug_gaussian_grads* grads,
                                 ug_stream stream) {
  ug_status s = check_plan(plan);
  if (s == UG_OK) s = check_ws(plan, ws, ws_bytes);
  if (s == UG_OK) s = check_gaussians(plan, gaussians);
  if (s != UG_OK) return s;
  if (!grads) return UG_ERR_INVALID_ARGUMENT;
  if (plan->n > 0) {
    if (!grads->mean || !grads->opacity_logit || !grads->intensity) return UG_ERR_INVALID_ARGUMENT;
    if (plan->cfg.cov_param == UG_COV_TRI && !grads->tri) return UG_ERR_INVALID_ARGUMENT;
    if (plan->cfg.cov_param == UG_COV_SCALE_ROT && (!grads->log_scale || !grads->quat))
      return UG_ERR_INVALID_ARGUMENT;
  }
  return cuda_status(launch_pre_backward(plan, gaussians, make_view(plan, ws), grads,
                                         reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_adam_step(float* param, const float* grad, float* exp_avg, float* exp_avg_sq,
                       int32_t rows, int64_t n, const ug_adam_row* d_rows, int32_t* d_step,
                       float beta1, float beta2, float eps, ug_stream stream) {
  if (!param || !grad || !exp_avg || !exp_avg_sq || !d_rows || !d_step) return UG_ERR_INVALID_ARGUMENT;
  if (rows < 1 || rows > 65535 || n < 1) return UG_ERR_INVALID_ARGUMENT;
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f))
    return UG_ERR_INVALID_ARGUMENT;
  return cuda_status(launch_adam(param, grad, exp_avg, exp_avg_sq, rows, n, d_rows, d_step, beta1,
                                 beta2, eps, reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_read_status(const ug_plan* plan, const void* ws, size_t ws_bytes, ug_ws_status* out,
                         ug_stream stream) {
  ug_status s = check_plan(plan);
  if (s == UG_OK) s = check_ws(plan, ws, ws_bytes);
  if (s != UG_OK) return s;
  if (!out) return UG_ERR_INVALID_ARGUMENT;
  const char* src = static_cast<const char*>(ws) + plan->off[kOffHeader];
  return cuda_status(cudaMemcpyAsync(out, src, sizeof(ug_ws_status), cudaMemcpyDefault,
                                     reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_debug_views(const ug_plan* plan, void* ws, size_t ws_bytes, uint32_t** sorted_keys,
                         uint32_t** sorted_records, uint32_t** tile_ranges,
                         uint32_t** record_boxes, float** record_a, float** record_b,
                         float** record_c, uint32_t** record_planes) {
  ug_status s = check_plan(plan);
  if (s == UG_OK) s = check_ws(plan, ws, ws_bytes);
  if (s != UG_OK) return s;
  WsView v = make_view(plan, ws);
  const int fin = plan->sort_passes & 1;
  if (sorted_keys) *sorted_keys = v.keys[fin];
  if (sorted_records) *sorted_records = v.vals[fin];
  if (tile_ranges) *tile_ranges = reinterpret_cast<uint32_t*>(v.ranges);
  if (record_boxes) *record_boxes = reinterpret_cast<uint32_t*>(v.rec_box);
  if (record_a) *record_a = reinterpret_cast<float*>(v.rec_a);
  if (record_b) *record_b = reinterpret_cast<float*>(v.rec_b);
  if (record_c) *record_c = reinterpret_cast<float*>(v.rec_c);
  if (record_planes) *record_planes = v.rec_plane;
  return UG_OK;
}

size_t ug_l1_dssim_scratch_floats(int32_t P, int32_t W, int32_t H) {
  if (P < 1 || W < 11 || H < 11) return 0;
  return dssim_scratch_floats(P, W, H);
}

ug_status ug_l1_dssim_loss_grad(const float* image, const float* target, int32_t P, int32_t W,
                                int32_t H, float lambda, float* scratch, size_t scratch_floats,
                                float* grad, float* loss, ug_stream stream) {
  if (!image || !target || !scratch || !grad || !loss) return UG_ERR_INVALID_ARGUMENT;
  if (P < 1 || W < 11 || H < 11 || W > 16384 || H > 16384) return UG_ERR_INVALID_ARGUMENT;
  if (!(lambda >= 0.f && lambda <= 1.f)) return UG_ERR_INVALID_ARGUMENT;
  if (scratch_floats < dssim_scratch_floats(P, W, H)) return UG_ERR_WORKSPACE_TOO_SMALL;
  return cuda_status(launch_l1_dssim(image, target, P, W, H, lambda, scratch, grad, loss,
                                     reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_densify_config_default(ug_densify_config* dc) {
  if (!dc) return UG_ERR_INVALID_ARGUMENT;
  *dc = ug_densify_config{};
  dc->grad_threshold = 2e-4f;
  dc->min_opacity = 0.005f;
  dc->size_threshold = 0.01f;
  dc->split_factor = 1.6f;
  return UG_OK;
}

static bool cov_ok(const ug_config* cfg) {
  return cfg && (cfg->cov_param == UG_COV_TRI || cfg->cov_param == UG_COV_SCALE_ROT) &&
         cfg->beta > 0.f && std::isfinite(cfg->beta);
}

ug_status ug_sample(const ug_config* cfg, const float* params, int64_t n, const int32_t* idx,
                    int64_t m, const float* z, float* y, ug_stream stream) {
  if (!cov_ok(cfg) || n < 1 || m < 0) return UG_ERR_INVALID_ARGUMENT;
  if (m > 0 && (!params || !idx || !z || !y)) return UG_ERR_INVALID_ARGUMENT;
  return cuda_status(launch_sample(cfg->cov_param, params, n, cfg->beta, idx, m, z, y,
                                   reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_densify_stats(const float* grad_mean, int64_t n, float* stats, ug_stream stream) {
  if (n < 1 || !grad_mean || !stats) return UG_ERR_INVALID_ARGUMENT;
  return cuda_status(launch_densify_stats(grad_mean, n, stats,
                                          reinterpret_cast<cudaStream_t>(stream)));
}

size_t ug_densify_scratch_bytes(int64_t n) { return n < 1 ? 0 : densify_scratch_bytes(n); }

ug_status ug_densify(const ug_config* cfg, const ug_densify_config* dc, const float* params,
                     const float* exp_avg, const float* exp_avg_sq, int64_t n, const float* stats,
                     const float* z, int64_t capacity, float* params_out, float* exp_avg_out,
                     float* exp_avg_sq_out, int64_t* n_out, void* scratch, size_t scratch_bytes,
                     ug_stream stream) {
  if (!cov_ok(cfg) || !dc || n < 1 || n >= ((int64_t)1 << 31) || capacity < 1)
    return UG_ERR_INVALID_ARGUMENT;
  if (!params || !exp_avg || !exp_avg_sq || !stats || !z || !params_out || !exp_avg_out ||
      !exp_avg_sq_out || !n_out || !scratch)
    return UG_ERR_INVALID_ARGUMENT;
  if (!(dc->min_opacity > 0.f && dc->min_opacity < 1.f) || !(dc->split_factor > 1.f) ||
      !(dc->size_threshold > 0.f) || !std::isfinite(dc->grad_threshold) ||
      !std::isfinite(dc->size_threshold) || !std::isfinite(dc->split_factor))
    return UG_ERR_INVALID_ARGUMENT;
  if (scratch_bytes < densify_scratch_bytes(n)) return UG_ERR_WORKSPACE_TOO_SMALL;
  const double p = dc->min_opacity, sz = dc->size_threshold;
  DensifyThresholds t;
  t.logit_min = (float)std::log(p / (1.0 - p));
  t.grad_threshold = dc->grad_threshold;
  t.size2 = (float)(sz * sz);
  t.log_size = (float)std::log(sz);
  t.beta = cfg->beta;
  t.phi = dc->split_factor;
  t.log_phi = (float)std::log((double)dc->split_factor);
  return cuda_status(launch_densify(cfg->cov_param, params, exp_avg, exp_avg_sq, n, stats, z, t,
                                    capacity, params_out, exp_avg_out, exp_avg_sq_out, n_out,
                                    scratch, reinterpret_cast<cudaStream_t>(stream)));
}

ug_status ug_debug_stall_pipeline(const ug_plan* plan, void* ws, size_t ws_bytes, int32_t on,
                                  ug_stream stream) {
  ug_status s = check_plan(plan);
  if (s == UG_OK) s = check_ws(plan, ws, ws_bytes);
  if (s != UG_OK) return s;
  WsView v = make_view(plan, ws);
  return cuda_status(cudaMemsetAsync(&v.hdr->stall_test, on ? 0xff : 0, sizeof(uint32_t),
                                     reinterpret_cast<cudaStream_t>(stream)));
}

}  // extern "C"
