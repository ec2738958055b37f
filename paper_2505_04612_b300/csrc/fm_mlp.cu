// Learned per-pair inlier weights: the per-image-pair feature tables, the
// features alone, and the optimiser of the 8-64-64-1 GELU network: the
// fixed-order sum of the training kernel's per-CTA partials and Adam.  The
// network itself runs on the tcgen05 tensor cores (fm_mlp_tc.cu): inference
// (k_mlp_forward_tc) and the binary cross-entropy gradient (k_mlp_grad_tc).
// The paper down-weights outliers with IRLS and a periodic filter (Sec. 3.3,
// Eq. 9); the network replaces the filter by a predicted inlier probability.
// Feature and network definitions (readings) are those of the problem-level
// documentation in include/fastmap.h.
#include <cuda_bf16.h>

#include "fm_device.cuh"
#include "fm_internal.h"
#include "fm_mlp.cuh"

namespace fm {
namespace {

constexpr int kIn = 8;
constexpr int kWarps = 4;

// ------------------------------------------------------------ features

// per image pair: E (9), R_i (9), R_j (9), mean |r|, log Z_n, fbar, 0
constexpr int kTab = kMlpTab;

// params: epipolar-stage [N][9]; or, with rel_t, rotation-stage [N][6] and
// E_n = [t^{i->j}]_x R_j R_i^T from the relative translation of the pair
__global__ void __launch_bounds__(128) k_mlp_pair_tables(const float* params, const float* rel_t,
                                                         const int* __restrict__ pi, const int* __restrict__ pj,
                                                         const int* __restrict__ seg_off,
                                                         const float4* __restrict__ kp,
                                                         const float* __restrict__ focal, int P,
                                                         float* __restrict__ tab) {
  const int lane = threadIdx.x & 31;
  const int n = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (n >= P) return;
  const int ci = pi[n], cj = pj[n];
  // the keypoints do not depend on the geometry: the first loads go out now,
  // four per lane in flight (pairs b + lane + 32 u; the sum keeps that order)
  const int b = seg_off[n], e = seg_off[n + 1];
  constexpr int kAhead = 4;
  float4 xs[kAhead];
#pragma unroll
  for (int u = 0; u < kAhead; ++u) {
    const int m = b + lane + 32 * u;
    xs[u] = m < e ? __ldg(kp + m) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  PairGeo g;
  float E[9];
  if (rel_t) {
    float qi[6], qj[6];
    load_plain(params + 6 * ci, qi, 6);
    load_plain(params + 6 * cj, qj, 6);
    Rot6 si, sj;
    rot6_forward(qi, si);
    rot6_forward(qj, sj);
    rot6_matrix(si, g.Ri);
    rot6_matrix(sj, g.Rj);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        g.Rij[r * 3 + c] = fmaf(g.Rj[r * 3 + 0], g.Ri[c * 3 + 0],
                           fmaf(g.Rj[r * 3 + 1], g.Ri[c * 3 + 1], g.Rj[r * 3 + 2] * g.Ri[c * 3 + 2]));
    float t[3];
    load_plain(rel_t + 3 * n, t, 3);
    const float inv = rsqrtf(fmaxf(dot3(t, t), 1e-30f));
    for (int k = 0; k < 3; ++k) g.that[k] = t[k] * inv;
    essential(g, E);
  } else {
    float qi[9], qj[9];
    load_plain(params + 9 * ci, qi, 9);
    load_plain(params + 9 * cj, qj, 9);
    pair_geometry(qi, qj, g);
    essential(g, E);
  }
  float s = 0.f;
  for (int m0 = b; m0 < e; m0 += 32 * kAhead) {
    float4 cur[kAhead];
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      cur[u] = xs[u];
      const int m = m0 + 32 * kAhead + lane + 32 * u;
      xs[u] = m < e ? __ldg(kp + m) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      if (m0 + lane + 32 * u >= e) break;
      const float4 x = cur[u];
      const float a0 = fmaf(E[0], x.x, fmaf(E[1], x.y, E[2]));
      const float a1 = fmaf(E[3], x.x, fmaf(E[4], x.y, E[5]));
      const float a2 = fmaf(E[6], x.x, fmaf(E[7], x.y, E[8]));
      s += fabsf(fmaf(x.z, a0, fmaf(x.w, a1, a2)));
    }
  }
  s = warp_sum(s);
  float* o = tab + (size_t)kTab * n;
  if (lane < 9) {
    float ev = E[0], ri = g.Ri[0], rj = g.Rj[0];
#pragma unroll
    for (int k = 1; k < 9; ++k)
      if (lane == k) { ev = E[k]; ri = g.Ri[k]; rj = g.Rj[k]; }
    o[lane] = ev;
    o[9 + lane] = ri;
    o[18 + lane] = rj;
  }
  if (lane == 0) {
    const int zn = e - b;
    o[27] = zn > 0 ? s / (float)zn : 0.f;
    o[28] = zn > 0 ? logf((float)zn) : 0.f;
    o[29] = 0.5f * (focal[ci] + focal[cj]);
    o[30] = 0.f;
    o[31] = 0.f;
  }
}

// features (and residuals) only; the network runs in k_mlp_forward_tc
__global__ void __launch_bounds__(kWarps * 32) k_mlp_infer(InferArgs a) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < a.Z; m += (int64_t)gridDim.x * blockDim.x) {
    float f[kIn];
    float r = 0.f;
    pair_features(a, m, f, r);
    if (a.feat)
#pragma unroll
      for (int k = 0; k < kIn; ++k) a.feat[m * kIn + k] = f[k];
    if (a.resid) a.resid[m] = r;
  }
}

// w = 1 for pairs with p >= p_min, else 0
__global__ void k_mask_from_prob(const float* __restrict__ prob, int64_t Z, float p_min, float* __restrict__ w) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m < Z) w[m] = prob[m] >= p_min ? 1.f : 0.f;
}

// fixed-order sum of the CTA partials (stride entries each): grad [4801], loss
__global__ void k_mlp_reduce(const float* __restrict__ partial, int parts, int stride, float* __restrict__ grad,
                             float* __restrict__ loss) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > kMlpParams) return;
  float s = 0.f;
  for (int c = 0; c < parts; ++c) s += partial[(size_t)c * stride + k];
  if (k < kMlpParams) {
    if (grad) grad[k] = s;
  } else if (loss) {
    *loss = s;
  }
}

__global__ void k_mlp_adam(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                           float* __restrict__ v, int step, float lr, float b1, float b2, float eps) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kMlpParams) return;
  const float gk = grad[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  theta[k] -= lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
}

int grid_for_pairs(int64_t n, int per_block) {
  int64_t g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > 148 * 8) g = 148 * 8;
  return (int)g;
}

}  // namespace


void launch_mlp_pair_tables(const fm_problem* pr, const float* params, const float* rel_t, float* tab,
                            cudaStream_t s) {
  k_mlp_pair_tables<<<(pr->P + 3) / 4, 128, 0, s>>>(params, rel_t, pr->pair_i, pr->pair_j, pr->seg_off, pr->kp,
                                                   pr->focal, pr->P, tab);
}

void launch_mask_from_prob(const float* prob, int64_t Z, float p_min, float* w, cudaStream_t s) {
  if (Z == 0) return;
  k_mask_from_prob<<<(unsigned)((Z + 255) / 256), 256, 0, s>>>(prob, Z, p_min, w);
}

void launch_mlp_infer(const fm_problem* pr, const float* tab, const float* theta, const float* w, float iter_frac,
                      float delta, float* prob, float* logit, float* feat, float* resid, cudaStream_t s) {
  if (pr->Z == 0) return;
  InferArgs a;
  a.kp = pr->kp;
  a.kp_seg = pr->kp_seg;
  a.tab = tab;
  a.kp_track = pr->track_off ? pr->kp_track : nullptr;
  a.track_off = pr->track_off;
  a.w = w;
  a.iter_frac = iter_frac;
  a.inv_log_delta = 1.f / log1pf(1.f / delta);
  a.theta = theta;
  a.x = nullptr;
  a.Z = pr->Z;
  a.prob = prob;
  a.logit = logit;
  a.feat = feat;
  a.resid = resid;
  if (theta)
    launch_mlp_infer_tc(a, pr->d_err, pr->sm_count, s);
  else
    k_mlp_infer<<<grid_for_pairs(pr->Z, kWarps * 32), kWarps * 32, 0, s>>>(a);
}

void launch_mlp_grad(const float* theta, const float* x, const float* y, int64_t B, float* partial, float* grad,
                     float* loss, int* err, cudaStream_t s) {
  launch_mlp_grad_tc(theta, x, y, B, partial, err, s);
  k_mlp_reduce<<<(kMlpParams + 1 + 255) / 256, 256, 0, s>>>(partial, mlp_grad_parts(B), mlp_part_stride(), grad, loss);
}

void launch_mlp_adam(float* theta, const float* grad, float* m, float* v, int step, float lr, float b1, float b2,
                     float eps, cudaStream_t s) {
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(theta, grad, m, v, step, lr, b1, b2, eps);
}

}  // namespace fm
