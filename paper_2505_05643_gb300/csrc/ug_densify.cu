// Row f2: resampling and the densify / prune step.
//
// Resampling draws a point of a Gaussian as y = mu + L^-T z with z standard
// normal (Sec. 4.2: the triangular precision factor makes this one back
// substitution with L^T); for the scale/rotation front-end y = mu + R S z.
//
// The densify / prune step follows the heuristics the paper takes over from
// Kerbl et al. (Sec. 4.5), with the decision quantities read as stated in the
// ug_densify_config documentation: prune when the opacity is below a minimum;
// densify when the mean norm of dL/dmu over the counted steps exceeds a
// threshold; a densified Gaussian whose extent is at most the size threshold is
// cloned (the original and an identical copy), a larger one is split into two
// children drawn from it (y = mu + L^-T z, two draws) with the covariance
// divided by phi^2. Kept Gaussians keep their Adam moments; clones and
// children start from zero moments. The output keeps the input order (each
// Gaussian's outputs at its exclusive prefix of the output counts), so the step
// is deterministic.
//
// Every decision is taken on FP32 quantities formed with explicitly rounded
// operations (no contraction into FMA), so a reader can replay it exactly.
#include "ug_scan.cuh"

namespace ug {

// Offset L^-T z (TRI: L from the parameters with L_kk = l_kk^2 + beta; back
// substitution with the upper-triangular L^T) or R S z (SCALE_ROT).
__device__ __forceinline__ void sample_offset(int cov, const float* p, int64_t stride, float beta,
                                              const float z[3], float w[3]) {
  if (cov == UG_COV_TRI) {
    const float l11 = p[3 * stride], l21 = p[4 * stride], l31 = p[5 * stride];
    const float l22 = p[6 * stride], l32 = p[7 * stride], l33 = p[8 * stride];
    const float L11 = __fadd_rn(__fmul_rn(l11, l11), beta);
    const float L22 = __fadd_rn(__fmul_rn(l22, l22), beta);
    const float L33 = __fadd_rn(__fmul_rn(l33, l33), beta);
    w[2] = __fdiv_rn(z[2], L33);
    w[1] = __fdiv_rn(__fsub_rn(z[1], __fmul_rn(l32, w[2])), L22);
    w[0] = __fdiv_rn(__fsub_rn(__fsub_rn(z[0], __fmul_rn(l21, w[1])), __fmul_rn(l31, w[2])), L11);
  } else {
    const float s0 = expf(p[3 * stride]), s1 = expf(p[4 * stride]), s2 = expf(p[5 * stride]);
    float qw = p[6 * stride], qx = p[7 * stride], qy = p[8 * stride], qz = p[9 * stride];
    const float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= inv;
    qx *= inv;
    qy *= inv;
    qz *= inv;
    const float R[3][3] = {
        {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
        {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
        {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
    const float sz[3] = {s0 * z[0], s1 * z[1], s2 * z[2]};
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = R[k][0] * sz[0] + R[k][1] * sz[1] + R[k][2] * sz[2];
  }
}

__global__ void __launch_bounds__(256)
    k_sample(int cov, const float* __restrict__ params, int64_t n, float beta,
             const int32_t* __restrict__ idx, int64_t m, const float* __restrict__ z,
             float* __restrict__ y) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx[k];
    const float zz[3] = {z[k], z[m + k], z[2 * m + k]};
    float w[3];
    sample_offset(cov, params + i, n, beta, zz, w);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c * m + k] = __fadd_rn(params[c * n + i], w[c]);
  }
}

// Trace of Sigma = L^-T L^-1 = sum of the squares of L^-1 (TRI), by forward
// substitution with explicitly rounded operations.
__device__ __forceinline__ float tri_trace(const float* p, int64_t stride, float beta) {
  const float l11 = p[3 * stride], l21 = p[4 * stride], l31 = p[5 * stride];
  const float l22 = p[6 * stride], l32 = p[7 * stride], l33 = p[8 * stride];
  const float i00 = __fdiv_rn(1.f, __fadd_rn(__fmul_rn(l11, l11), beta));
  const float i11 = __fdiv_rn(1.f, __fadd_rn(__fmul_rn(l22, l22), beta));
  const float i22 = __fdiv_rn(1.f, __fadd_rn(__fmul_rn(l33, l33), beta));
  const float i10 = -__fmul_rn(__fmul_rn(l21, i00), i11);
  const float i21 = -__fmul_rn(__fmul_rn(l32, i11), i22);
  const float i20 = -__fmul_rn(__fadd_rn(__fmul_rn(l31, i00), __fmul_rn(l32, i10)), i22);
  float t = __fmul_rn(i00, i00);
  t = __fadd_rn(t, __fmul_rn(i10, i10));
  t = __fadd_rn(t, __fmul_rn(i11, i11));
  t = __fadd_rn(t, __fmul_rn(i20, i20));
  t = __fadd_rn(t, __fmul_rn(i21, i21));
  t = __fadd_rn(t, __fmul_rn(i22, i22));
  return t;
}

// Output count of Gaussian i: 0 prune, 1 keep, 2 clone or split; action 0 prune,
// 1 keep, 2 clone, 3 split.
__device__ __forceinline__ uint32_t densify_action(int cov, const float* params, int64_t n,
                                                   int64_t i, const float* stats,
                                                   const DensifyThresholds& t) {
  const float* p = params + i;
  const int row_logit = cov == UG_COV_TRI ? 9 : 10;
  if (p[row_logit * n] < t.logit_min) return 0u;
  const float cnt = stats[n + i];
  const float avg = cnt > 0.f ? __fdiv_rn(stats[i], cnt) : 0.f;
  if (!(avg > t.grad_threshold)) return 1u;
  bool large;
  if (cov == UG_COV_TRI) {
    large = tri_trace(p, n, t.beta) > t.size2;
  } else {
    large = fmaxf(p[3 * n], fmaxf(p[4 * n], p[5 * n])) > t.log_size;
  }
  return large ? 3u : 2u;
}

__global__ void __launch_bounds__(256)
    k_densify_classify(int cov, const float* __restrict__ params, int64_t n,
                       const float* __restrict__ stats, DensifyThresholds t,
                       uint32_t* __restrict__ action) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    action[i] = densify_action(cov, params, n, i, stats, t);
}

struct ActLoad {
  const uint32_t* action;
  __device__ void operator()(int64_t e, uint32_t out[1]) const {
    const uint32_t a = action[e];
    out[0] = a == 0u ? 0u : (a == 1u ? 1u : 2u);
  }
};
struct PosStore {
  uint32_t* pos;
  __device__ void operator()(int64_t e, const uint32_t ex[1]) const { pos[e] = ex[0]; }
};

// The rows of one parameter set are a compile-time count (11 TRI, 12
// SCALE_ROT), so that a thread's loads of its Gaussian's rows are all in
// flight together.
template <int COV>
__global__ void __launch_bounds__(256)
    k_densify_emit(const float* __restrict__ params, const float* __restrict__ m,
                   const float* __restrict__ v, int64_t n, const float* __restrict__ z,
                   const uint32_t* __restrict__ action, const uint32_t* __restrict__ pos,
                   DensifyThresholds t, int64_t cap, float* __restrict__ params_out,
                   float* __restrict__ m_out, float* __restrict__ v_out,
                   int64_t* __restrict__ n_out) {
  constexpr int cov = COV;
  constexpr int rows = COV == UG_COV_TRI ? 11 : 12;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t a = action[i];
    const int64_t o = pos[i];
    const uint32_t cnt = a == 0u ? 0u : (a == 1u ? 1u : 2u);
    if (i == n - 1) *n_out = o + cnt;
    if (cnt == 0u || o + cnt > cap) continue;
    if (a == 1u || a == 2u) {  // the original, with its moments
      float pr[rows], mr[rows], vr[rows];
#pragma unroll
      for (int r = 0; r < rows; ++r) {
        pr[r] = params[r * n + i];
        mr[r] = m[r * n + i];
        vr[r] = v[r * n + i];
      }
#pragma unroll
      for (int r = 0; r < rows; ++r) {
        params_out[r * cap + o] = pr[r];
        m_out[r * cap + o] = mr[r];
        v_out[r * cap + o] = vr[r];
      }
      if (a == 2u) {  // an identical copy with zero moments
#pragma unroll
        for (int r = 0; r < rows; ++r) {
          params_out[r * cap + o + 1] = pr[r];
          m_out[r * cap + o + 1] = 0.f;
          v_out[r * cap + o + 1] = 0.f;
        }
      }
    }
    if (a == 3u) {  // two children drawn from the parent, covariance / phi^2
      for (int c = 0; c < 2; ++c) {
        const int64_t oc = o + c;
        const float zz[3] = {z[(3 * c) * n + i], z[(3 * c + 1) * n + i], z[(3 * c + 2) * n + i]};
        float w[3];
        sample_offset(cov, params + i, n, t.beta, zz, w);
        for (int k = 0; k < 3; ++k) params_out[k * cap + oc] = __fadd_rn(params[k * n + i], w[k]);
        if constexpr (cov == UG_COV_TRI) {
          // L' = phi L: L'_kk = phi (l_kk^2 + beta) = l'_kk^2 + beta, l'_jk = phi l_jk
          const int diag[3] = {3, 6, 8};
          for (int d = 0; d < 3; ++d) {
            const float l = params[diag[d] * n + i];
            const float Lk = __fmul_rn(t.phi, __fadd_rn(__fmul_rn(l, l), t.beta));
            const float lp = sqrtf(fmaxf(__fsub_rn(Lk, t.beta), 0.f));
            params_out[diag[d] * cap + oc] = l < 0.f ? -lp : lp;
          }
          const int off[3] = {4, 5, 7};
          for (int d = 0; d < 3; ++d)
            params_out[off[d] * cap + oc] = __fmul_rn(t.phi, params[off[d] * n + i]);
        } else {
          for (int k = 3; k < 6; ++k)
            params_out[k * cap + oc] = __fsub_rn(params[k * n + i], t.log_phi);
          for (int k = 6; k < 10; ++k) params_out[k * cap + oc] = params[k * n + i];
        }
#pragma unroll
        for (int r = rows - 2; r < rows; ++r) params_out[r * cap + oc] = params[r * n + i];
#pragma unroll
        for (int r = 0; r < rows; ++r) {
          m_out[r * cap + oc] = 0.f;
          v_out[r * cap + oc] = 0.f;
        }
      }
    }
  }
}

// Statistics of the densify step: stats[0][i] += |dL/dmu_i|, stats[1][i] += 1
// when the gradient is non-zero (the Gaussian was seen in the step).
__global__ void __launch_bounds__(256)
    k_densify_stats(const float* __restrict__ gmean, int64_t n, float* __restrict__ stats) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gx = gmean[i], gy = gmean[n + i], gz = gmean[2 * n + i];
    const float s = __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
    if (s > 0.f) {
      stats[i] = __fadd_rn(stats[i], sqrtf(s));
      stats[n + i] = __fadd_rn(stats[n + i], 1.f);
    }
  }
}

size_t densify_scratch_bytes(int64_t n) {
  const int64_t nblk = scan_blocks(n);
  return 2 * sizeof(uint32_t) * (size_t)n + sizeof(unsigned long long) * (size_t)(nblk + 1) + 256;
}

static unsigned grid_of(int64_t work) {
  const int64_t b = (work + 255) / 256;
  const int64_t cap = (int64_t)device_sms() * 8;
  return (unsigned)max((int64_t)1, min(b, cap));
}

cudaError_t launch_sample(int cov, const float* params, int64_t n, float beta, const int32_t* idx,
                          int64_t m, const float* z, float* y, cudaStream_t s) {
  if (m > 0) k_sample<<<grid_of(m), 256, 0, s>>>(cov, params, n, beta, idx, m, z, y);
  return cudaGetLastError();
}

cudaError_t launch_densify_stats(const float* gmean, int64_t n, float* stats, cudaStream_t s) {
  if (n > 0) k_densify_stats<<<grid_of(n), 256, 0, s>>>(gmean, n, stats);
  return cudaGetLastError();
}

cudaError_t launch_densify(int cov, const float* params, const float* m, const float* v,
                           int64_t n, const float* stats, const float* z,
                           const DensifyThresholds& t, int64_t cap, float* params_out,
                           float* m_out, float* v_out, int64_t* n_out, void* scratch,
                           cudaStream_t s) {
  uint32_t* action = static_cast<uint32_t*>(scratch);
  uint32_t* pos = action + n;
  unsigned long long* part = reinterpret_cast<unsigned long long*>(
      (reinterpret_cast<uintptr_t>(pos + n) + 255) & ~uintptr_t(255));
  const unsigned g = grid_of(n);
  k_densify_classify<<<g, 256, 0, s>>>(cov, params, n, stats, t, action);
  const int64_t nblk = scan_blocks(n);
  ActLoad ld{action};
  PosStore st{pos};
  k_scan_partial<1, ActLoad><<<(unsigned)nblk, kScanThreads, 0, s>>>(ld, n, part, nullptr);
  k_scan_top<1><<<1, 1024, 0, s>>>(part, nblk, nullptr, 0, 0, 0);
  k_scan_down<1, ActLoad, PosStore><<<(unsigned)nblk, kScanThreads, 0, s>>>(ld, st, n, part,
                                                                              nullptr);
  if (cov == UG_COV_TRI)
    k_densify_emit<UG_COV_TRI><<<g, 256, 0, s>>>(params, m, v, n, z, action, pos, t, cap,
                                                 params_out, m_out, v_out, n_out);
  else
    k_densify_emit<UG_COV_SCALE_ROT><<<g, 256, 0, s>>>(params, m, v, n, z, action, pos, t, cap,
                                                       params_out, m_out, v_out, n_out);
  return cudaGetLastError();
}

}  // namespace ug
