// IRLS reweighting, outlier filtering and the compact quadratic form of the
// epipolar objective (Sec. 3.3, Eqs. 8-9; Appendix "Epipolar Adjustment",
// Eqs. 15-17).
//
//   k_ea_reweight  per keypoint pair: eps^ = x~2^T E_n x~1 at the current
//                  poses; the pair is kept if |eps^| < tau (the periodic
//                  filtering with a decreasing threshold) and weighted
//                  1/max(|eps^|, delta) (IRLS), or 1 (mask only);
//   k_w_build      per image pair: W_n = sum_m w_m vec(x~2 x~1^T) vec(...)^T,
//                  the 45 unique entries of the symmetric 9x9 matrix, plus the
//                  quadratic form's value and gradient at the reference
//                  essential matrix e0 of the current poses:
//                  b_n = W_n e0 = sum_m w_m r0_m v_m, c_n = e0^T W_n e0 = sum_m w_m r0_m^2
//                  with r0_m = v_m . e0 the pair's residual, and e0 itself;
//   k_ea_compact   per image pair: e = e0 + d, and
//                      e^T W e = c + 2 d.b + d^T W d,   W e = b + W d,
//                  loss inv_z e^T W e, dL/dE = 2 inv_z W e, then the chain rule
//                  to the two cameras -- the per-iteration cost is independent
//                  of the keypoint pairs.
//
// Why the centred form: near convergence e lies close to the null space of W,
// so e^T W e (= sum w r^2, tiny) is a difference of terms of size |W| |e|^2.
// Rounding W to float32 perturbs it by ~1e-7 |W| |e|^2, which can exceed the
// value itself.  Expanding around e0 is an exact identity; b and c are sums of
// the small, accurately computed residuals, and the only term that still sees
// W's rounding is d^T W d with d = e - e0 small while the poses stay near the
// ones of the last reweighting.
#include <algorithm>

#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

// one thread per run of kReweightRun consecutive keypoint pairs; the image
// pair of each pair comes from kp_seg (E reloaded when it changes)
constexpr int kReweightRun = 8;

__global__ void k_ea_reweight(const float4* __restrict__ kp, const int* __restrict__ kp_seg,
                              const float4* __restrict__ seg_tab, const int* __restrict__ pair_scene,
                              int Z, int n_runs, float tau, float delta, int irls, float* __restrict__ w,
                              unsigned long long* __restrict__ kept, const float* __restrict__ prob, float p_min) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  int my_kept = 0;
  int scene = -1;     // scene of the pairs counted in my_kept
  if (q < n_runs) {
    const int p0 = q * kReweightRun;
    const int pend = min(p0 + kReweightRun, Z);
    int s = -1;
    float4 e0 = make_float4(0.f, 0.f, 0.f, 0.f), e1 = e0, e2 = e0;
    for (int p = p0; p < pend; ++p) {
      const int sp = __ldg(kp_seg + p);
      if (sp != s) {
        s = sp;
        e0 = seg_tab[3 * s];
        e1 = seg_tab[3 * s + 1];
        e2 = seg_tab[3 * s + 2];
      }
      const int sc = __ldg(pair_scene + s);
      if (sc != scene) {   // a run crossing a scene boundary (rare): flush the count
        if (my_kept) atomicAdd(kept + scene, (unsigned long long)my_kept);
        my_kept = 0;
        scene = sc;
      }
      const float4 x = __ldg(kp + p);
      const float ex = fmaf(e0.x, x.x, fmaf(e0.y, x.y, e0.z));
      const float ey = fmaf(e0.w, x.x, fmaf(e1.x, x.y, e1.y));
      const float ez = fmaf(e1.z, x.x, fmaf(e1.w, x.y, e2.x));
      const float r = fabsf(fmaf(x.z, ex, fmaf(x.w, ey, ez)));
      const bool keep = prob ? (prob[p] >= p_min) : (r < tau);
      float wt = 0.f;
      if (keep) wt = irls ? 1.f / fmaxf(r, delta) : 1.f;
      w[p] = wt;
      my_kept += keep;
    }
  }
  // integer counts: the totals do not depend on the order of the atomics.
  // Lanes of one scene are summed with a warp reduction (the usual case);
  // otherwise every lane adds its own count.
  const unsigned FULL = 0xffffffffu;
  const int s0 = __shfl_sync(FULL, scene, 0);
  if (__all_sync(FULL, scene == s0 || my_kept == 0)) {
    for (int d = 16; d > 0; d >>= 1) my_kept += __shfl_xor_sync(FULL, my_kept, d);
    if ((threadIdx.x & 31) == 0 && my_kept) atomicAdd(kept + s0, (unsigned long long)my_kept);
  } else if (my_kept) {
    atomicAdd(kept + scene, (unsigned long long)my_kept);
  }
}

// count[s] += number of keypoint pairs with w > 0 in scene s (integer
// atomics: order-independent)
__global__ void k_count_positive(const float* __restrict__ w, const long long* __restrict__ sc_kp_off,
                                 unsigned long long* __restrict__ count) {
  // one CTA per (scene, chunk of 8192 pairs)
  const int s = blockIdx.y;
  const long long b = sc_kp_off[s] + (long long)blockIdx.x * 8192, e = min(b + 8192, sc_kp_off[s + 1]);
  int c = 0;
  for (long long m = b + threadIdx.x; m < e; m += blockDim.x) c += (w[m] > 0.f);
  for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count + s, (unsigned long long)c);
}

__global__ void k_pair_inv_from_counts(const unsigned long long* __restrict__ count,
                                       const int* __restrict__ pair_scene, int P, float* __restrict__ inv) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= P) return;
  const unsigned long long c = count[pair_scene[n]];
  inv[n] = c > 0 ? (float)(1.0 / (double)c) : 0.f;
}

// position of entry k (of 64) of image pair n in the tiled W
__host__ __device__ __forceinline__ size_t w_index(int n, int k) {
  return ((size_t)(n >> 5) * 64 + k) * 32 + (n & 31);
}

// one warp per image pair; lanes stride over its keypoint pairs, then a
// butterfly reduction in fixed order.  Output per image pair (64 floats):
// [0,45) W upper triangle, [45,54) b, [54] c, [55,64) e0, stored tiled by 32
// image pairs (w_index): entry k of the 32 pairs of a tile is one contiguous
// 128-byte row, so k_ea_compact's warps read W with coalesced loads.
__global__ void __launch_bounds__(128) k_w_build(const float4* __restrict__ kp, const float* __restrict__ w,
                                                 const int* __restrict__ seg_off,
                                                 const float4* __restrict__ seg_tab, int P,
                                                 float* __restrict__ W) {
  const int lane = threadIdx.x & 31;
  const int n = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (n >= P) return;
  const float4 t0 = __ldg(seg_tab + 3 * n), t1 = __ldg(seg_tab + 3 * n + 1), t2 = __ldg(seg_tab + 3 * n + 2);
  const float e0[9] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, t2.x};
  float acc[55];
#pragma unroll
  for (int k = 0; k < 55; ++k) acc[k] = 0.f;
  const int b = seg_off[n], e = seg_off[n + 1];
  for (int m = b + lane; m < e; m += 32) {
    const float4 x = __ldg(kp + m);
    const float wt = w ? __ldg(w + m) : 1.f;
    // vec(x~2 x~1^T), row-major: (x2 x1, x2 y1, x2, y2 x1, y2 y1, y2, x1, y1, 1)
    const float v[9] = {x.z * x.x, x.z * x.y, x.z, x.w * x.x, x.w * x.y, x.w, x.x, x.y, 1.f};
    // the residual at e0, as the direct kernel forms it
    const float ex = fmaf(e0[0], x.x, fmaf(e0[1], x.y, e0[2]));
    const float ey = fmaf(e0[3], x.x, fmaf(e0[4], x.y, e0[5]));
    const float ez = fmaf(e0[6], x.x, fmaf(e0[7], x.y, e0[8]));
    const float r0 = fmaf(x.z, ex, fmaf(x.w, ey, ez));
    int k = 0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const float wa = wt * v[a];
#pragma unroll
      for (int c = a; c < 9; ++c) {
        acc[k] = fmaf(wa, v[c], acc[k]);
        ++k;
      }
    }
    const float wr = wt * r0;
#pragma unroll
    for (int a = 0; a < 9; ++a) acc[45 + a] = fmaf(wr, v[a], acc[45 + a]);
    acc[54] = fmaf(wr, r0, acc[54]);
  }
#pragma unroll
  for (int k = 0; k < 55; ++k) acc[k] = warp_sum(acc[k]);
  // lanes write in parallel: lane l writes entries l and l + 32
  for (int k = lane; k < 64; k += 32) {
    float v = 0.f;
#pragma unroll
    for (int j = 0; j < 55; ++j)
      if (j == k) v = acc[j];
    if (k >= 55) v = e0[k - 55];
    W[w_index(n, k)] = v;
  }
}

__device__ __forceinline__ int tri(int a, int c) {   // index of (a, c), a <= c, in the packed upper triangle
  return a * 9 - (a * (a - 1)) / 2 + (c - a);
}

// one thread per image pair; a warp's 32 image pairs form one tile of W
// (64 coalesced 128-byte rows).  The two 12-float parts of the chain rule go
// to their positions in the camera CSR (cam_pos), so that k_cam reads each
// camera's parts as one contiguous block instead of gathering them.
template <bool STEP>
__global__ void __launch_bounds__(128) k_ea_compact(const float* __restrict__ W, const float* __restrict__ params,
                                                    const int* __restrict__ pi, const int* __restrict__ pj, int P,
                                                    const float* __restrict__ pair_inv_z,
                                                    const int* __restrict__ cam_pos,
                                                    float* __restrict__ seg_grad, float* __restrict__ seg_loss,
                                                    int* step_counter) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int n0 = n - lane;   // the warp's first image pair
  if (STEP && step_counter && n == 0) *step_counter += 1;
  if (n0 >= P) return;
  const bool mine = n < P;
  const int nn = mine ? n : n0;   // lanes past the end repeat the first pair; nothing of theirs is stored
  const float inv_z = pair_inv_z[nn];   // normaliser of the image pair's scene
  // W is read once per iteration: streaming loads (evict-first), so that it
  // does not push the chain-rule outputs, which k_cam gathers next, out of L2
  float Wn[64];
  const float* Wt = W + w_index(nn, 0);
#pragma unroll
  for (int k = 0; k < 64; ++k) Wn[k] = __ldcs(Wt + 32 * k);
  PairGeo g;
  pair_geometry(params + 9 * pi[nn], params + 9 * pj[nn], g);
  float e[9];
  essential(g, e);
  float d[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) d[a] = e[a] - Wn[55 + a];
  float Wd[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 9; ++c) s = fmaf(Wn[a <= c ? tri(a, c) : tri(c, a)], d[c], s);
    Wd[a] = s;
  }
  // e^T W e = c + 2 d.b + d^T W d ;  W e = b + W d
  float q = 0.f, lb = 0.f;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    q = fmaf(d[a], Wd[a], q);
    lb = fmaf(d[a], Wn[45 + a], lb);
  }
  if (mine) seg_loss[n] = (Wn[54] + 2.f * lb + q) * inv_z;
  float G[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) G[a] = 2.f * inv_z * (Wn[45 + a] + Wd[a]);
  float o[kSegGradEa];
  pair_backward(g, G, o);
  if (mine) {
    constexpr int kPart = kSegGradEa / 2;   // 48 B: 16-byte aligned parts
    float4* oi = reinterpret_cast<float4*>(seg_grad + (size_t)kPart * cam_pos[2 * n]);
    float4* oj = reinterpret_cast<float4*>(seg_grad + (size_t)kPart * cam_pos[2 * n + 1]);
#pragma unroll
    for (int q = 0; q < kPart / 4; ++q) {
      oi[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
      oj[q] = make_float4(o[kPart + 4 * q], o[kPart + 4 * q + 1], o[kPart + 4 * q + 2], o[kPart + 4 * q + 3]);
    }
  }
}

}  // namespace

void launch_ea_reweight(const fm_problem* pr, float tau, float delta, int irls, float* w,
                        unsigned long long* kept, cudaStream_t s, const float* prob, float p_min) {
  const int n_runs = (int)((pr->Z + kReweightRun - 1) / kReweightRun);
  if (n_runs == 0) return;
  k_ea_reweight<<<(n_runs + 255) / 256, 256, 0, s>>>(pr->kp, pr->kp_seg, pr->seg_tab, pr->pair_scene, (int)pr->Z,
                                                     n_runs, tau, delta, irls, w, kept, prob, p_min);
}

void launch_w_build(const fm_problem* pr, const float* w, float* W, cudaStream_t s) {
  k_w_build<<<(pr->P + 3) / 4, 128, 0, s>>>(pr->kp, w, pr->seg_off, pr->seg_tab, pr->P, W);
}

void launch_ea_compact(const fm_problem* pr, const float* params, int* step_counter, cudaStream_t s) {
  k_ea_compact<true><<<(pr->P + 127) / 128, 128, 0, s>>>(pr->W, params, pr->pair_i, pr->pair_j, pr->P,
                                                         pr->pair_inv_z, pr->cam_pos, pr->seg_grad, pr->seg_loss,
                                                         step_counter);
}

void launch_count_positive(const fm_problem* pr, const float* w, unsigned long long* count, cudaStream_t s) {
  int64_t most = 0;
  for (int q = 0; q < pr->S; ++q) most = std::max<int64_t>(most, pr->h_sc_kp_off[q + 1] - pr->h_sc_kp_off[q]);
  if (most == 0) return;
  dim3 grid((unsigned)((most + 8191) / 8192), pr->S);
  k_count_positive<<<grid, 256, 0, s>>>(w, reinterpret_cast<const long long*>(pr->sc_kp_off), count);
}

void launch_pair_inv_from_counts(const fm_problem* pr, const unsigned long long* count, cudaStream_t s) {
  k_pair_inv_from_counts<<<(pr->P + 127) / 128, 128, 0, s>>>(count, pr->pair_scene, pr->P, pr->pair_inv_z);
}

}  // namespace fm
