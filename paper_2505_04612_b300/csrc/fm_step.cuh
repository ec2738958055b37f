// Device functions of the per-image-pair pass (k_ea_segments) and the
// per-camera pass (k_cam).
#pragma once
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace step {

constexpr int kSegLanes = 8;      // lanes that share one image pair
constexpr int kThreads = 128;     // CTA size of the per-image-pair and per-camera passes

// Static inputs of image pair n's pass, loaded before the dependency wait.
struct SegStatic {
  int r0 = 0, cnt = 0, ci = 0, cj = 0;
};

__device__ __forceinline__ SegStatic seg_static(const SegArgs& a, int n) {
  SegStatic s;
  if (n < a.P) {
    s.r0 = a.seg_rec[2 * n];
    s.cnt = a.seg_rec[2 * n + 1];
    s.ci = a.pi[n];
    s.cj = a.pj[n];
  }
  return s;
}

// Image pair n, shared by kSegLanes lanes (sub = lane index in the group):
// the lanes sum its records with a stride of kSegLanes and combine them with
// a butterfly inside the group (a fixed order), the group's first lane
// scales the sum by the normalisers and applies the chain rule through
// E_n = [t^]_x R_ij to the two cameras (Sec. 3.3).  Returns true on the lane
// that wrote image pair n's outputs.  Every lane of the warp must call it.
__device__ __forceinline__ bool segment_pair(const SegArgs& a, int n, int sub, const SegStatic& st) {
  const bool valid = n < a.P;
  // the cameras' parameters are needed by the chain rule after the sum:
  // loaded now, with the records, rather than after the butterfly
  const bool chain = valid && sub == 0 && a.seg_grad != nullptr && st.cnt > 0;
  float qi[9], qj[9];
  if (chain) {
    load_plain(a.params + 9 * st.ci, qi, 9);
    load_plain(a.params + 9 * st.cj, qj, 9);
  }
  float G[10];
  for (int k = 0; k < 10; ++k) G[k] = 0.f;
  if (valid && !a.dlde_in) {
    for (int r = st.r0 + sub; r < st.r0 + st.cnt; r += kSegLanes) {
      const float4 v0 = a.rec[3 * r], v1 = a.rec[3 * r + 1], v2 = a.rec[3 * r + 2];
      G[0] += v0.x; G[1] += v0.y; G[2] += v0.z; G[3] += v0.w;
      G[4] += v1.x; G[5] += v1.y; G[6] += v1.z; G[7] += v1.w;
      G[8] += v2.x; G[9] += v2.y;
    }
  }
#pragma unroll
  for (int d = kSegLanes / 2; d > 0; d >>= 1)
#pragma unroll
    for (int k = 0; k < 10; ++k) G[k] += __shfl_xor_sync(0xffffffffu, G[k], d);
  if (!valid || sub != 0) return false;
  const float ps = a.pair_scale ? a.pair_scale[n] : 1.f;
  if (a.dlde_in) {
    for (int k = 0; k < 9; ++k) G[k] = a.dlde_in[9 * (size_t)n + k];
  } else {
    const float gs = a.g_scale * ps;
    for (int k = 0; k < 9; ++k) G[k] *= gs;
  }
  if (a.seg_loss) a.seg_loss[n] = G[9] * (a.l_scale * ps);
  if (a.dlde_out)
    for (int k = 0; k < 9; ++k) a.dlde_out[9 * (size_t)n + k] = G[k];
  if (!a.seg_grad) return true;
  float* out = a.seg_grad + (size_t)kSegGradEa * n;
  if (st.cnt == 0) {   // an image pair without keypoint pairs (its geometry may be degenerate)
    for (int k = 0; k < kSegGradEa; ++k) out[k] = 0.f;
    return true;
  }
  if (a.grad_loss) {
    const float gl = a.grad_loss[a.pair_scene ? a.pair_scene[n] : 0];
    for (int k = 0; k < 9; ++k) G[k] *= gl;
  }
  PairGeo g;
  pair_geometry(qi, qj, g);
  float o[kSegGradEa];
  pair_backward(g, G, o);
  if ((reinterpret_cast<uintptr_t>(out) & 15u) == 0) {   // library buffers: 96-B rows, 16-B aligned
    float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll
    for (int k = 0; k < kSegGradEa / 4; ++k) o4[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
  } else {
    for (int k = 0; k < kSegGradEa; ++k) out[k] = o[k];
  }
  return true;
}

// Per-stage layout of the per-camera pass.  STAGE 0 rotation (part 9: dR,
// params 6D), 1 translation (part 3: do, params o), 2 epipolar (part 12: dR,
// dt; params 6D + t)
template <int STAGE>
struct Layout;
template <> struct Layout<0> { static constexpr int PART = 9, PDIM = 6; static constexpr bool ROT = true; };
template <> struct Layout<1> { static constexpr int PART = 3, PDIM = 3; static constexpr bool ROT = false; };
template <> struct Layout<2> { static constexpr int PART = 12, PDIM = 9; static constexpr bool ROT = true; };

// The first kCamPre incident image pairs of a lane (camera CSR entries b +
// lane + 32 k, -1 past e): static, loaded before the dependency wait.
constexpr int kCamPre = 4;
__device__ __forceinline__ void cam_prefetch(const int* __restrict__ cam_seg, int b, int e, int lane, int* v) {
#pragma unroll
  for (int u = 0; u < kCamPre; ++u) v[u] = (b + lane + 32 * u < e) ? __ldg(cam_seg + b + lane + 32 * u) : -1;
}

template <int PART>
__device__ __forceinline__ void cam_add(const float* sg, int entry, float* acc) {
  const unsigned w = (unsigned)entry;
  const int n = (int)(w & 0x7fffffffu);
  const int role = (int)(w >> 31);
  const float* g = sg + ((size_t)n * 2 + role) * PART;
  if (PART % 4 == 0) {   // 48-B parts of a cudaMalloc'd buffer: 16-B aligned
#pragma unroll
    for (int q = 0; q < PART / 4; ++q) {
      const float4 t = *reinterpret_cast<const float4*>(g + 4 * q);
      acc[4 * q] += t.x;
      acc[4 * q + 1] += t.y;
      acc[4 * q + 2] += t.z;
      acc[4 * q + 3] += t.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < PART; ++k) acc[k] += g[k];
  }
}

// Sum of a camera's parts over its incident image pairs [b, e) of the camera
// CSR, by one warp: lane l adds the entries b + l, b + l + 32, ... in that
// order (the first kCamPre of them prefetched in pre), then a butterfly gives
// every lane the total.
template <int PART>
__device__ __forceinline__ void cam_gather(const float* sg, const int* __restrict__ cam_seg, int b, int e, int lane,
                                           const int* pre, float* acc) {
#pragma unroll
  for (int k = 0; k < PART; ++k) acc[k] = 0.f;
#pragma unroll
  for (int u = 0; u < kCamPre; ++u)
    if (pre[u] != -1) cam_add<PART>(sg, pre[u], acc);
  for (int i0 = b + lane + 32 * kCamPre; i0 < e; i0 += 32 * kCamPre) {
    int v[kCamPre];
#pragma unroll
    for (int u = 0; u < kCamPre; ++u) v[u] = (i0 + 32 * u < e) ? __ldg(cam_seg + i0 + 32 * u) : -1;
#pragma unroll
    for (int u = 0; u < kCamPre; ++u)
      if (v[u] != -1) cam_add<PART>(sg, v[u], acc);
  }
#pragma unroll
  for (int k = 0; k < PART; ++k) acc[k] = warp_sum(acc[k]);
}

// Camera c of run `run` from its summed parts, its parameters p and (Adam)
// its moments m, v of lane's entry (all loaded beforehand): the 6D adjoint
// for rotations, then either the gradient or Adam (bias-corrected; the step
// counter was advanced by this step's first kernel), by lanes < PDIM.
template <int STAGE, bool ADAM>
__device__ __forceinline__ void cam_apply(const CamUpdate& u, size_t off, const float* p, float m, float v,
                                          const float* acc, int lane) {
  using L = Layout<STAGE>;
  float g[L::PDIM];
  if (L::ROT) {
    Rot6 s;
    rot6_forward(p, s);
    rot6_adjoint(p, s, acc, g);
    if (STAGE == 2) {
      g[6] = acc[9];
      g[7] = acc[10];
      g[8] = acc[11];
    }
  } else {
#pragma unroll
    for (int k = 0; k < L::PDIM; ++k) g[k] = acc[k];
  }
  if (lane >= L::PDIM) return;
  float gv = g[0], pv = p[0];
#pragma unroll
  for (int k = 1; k < L::PDIM; ++k)
    if (lane == k) { gv = g[k]; pv = p[k]; }
  if (!ADAM) {
    u.grad_out[off + lane] = gv;
    return;
  }
  if (u.grad_out) u.grad_out[off + lane] = gv;
  const float t = (float)*u.step;
  const float bc1 = 1.f - powf(u.b1, t);
  const float bc2 = 1.f - powf(u.b2, t);
  m = u.b1 * m + (1.f - u.b1) * gv;
  v = u.b2 * v + (1.f - u.b2) * gv * gv;
  u.m[off + lane] = m;
  u.v[off + lane] = v;
  u.params_out[off + lane] = pv - u.lr * (m / bc1) / (sqrtf(v / bc2) + u.eps);
}

// Fixed-order sum of n per-image-pair loss terms by one CTA of T threads.
// The order depends on n only -- not on where x starts, so that a scene's
// loss inside a batch adds exactly as the same scene alone: chunks of four
// consecutive terms, chunk c summed as (x0 + x1) + (x2 + x3) into thread
// c % T's accumulator (c / T) % 8, the n % 4 last terms one per thread, then
// the accumulators in a fixed order and a tree over the threads.  A chunk is
// one float4 load when x is 16-B aligned, four scalar loads otherwise; eight
// chunks per thread are in flight.  Every thread of the CTA must call it.
__device__ __forceinline__ float4 load_chunk(const float* x, int c, bool aligned) {
  if (aligned) return reinterpret_cast<const float4*>(x)[c];
  return make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
}

template <int T>
__device__ __forceinline__ float loss_sum_cta(const float* x, int n, float* part) {
  const int t = threadIdx.x;
  const bool aligned = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
  const int n4 = n >> 2;
  float acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = 0.f;
  int k = t;
  for (; k + 7 * T < n4; k += 8 * T) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = load_chunk(x, k + u * T, aligned);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] += (v[u].x + v[u].y) + (v[u].z + v[u].w);
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if (k < n4) {
      const float4 v = load_chunk(x, k, aligned);
      acc[u] += (v.x + v.y) + (v.z + v.w);
    }
    k += T;
  }
  if (t < n - 4 * n4) acc[0] += x[4 * n4 + t];
  part[t] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  __syncthreads();
  for (int d = T / 2; d > 0; d >>= 1) {
    if (t < d) part[t] += part[t + d];
    __syncthreads();
  }
  const float r = part[0];
  __syncthreads();
  return r;
}

}  // namespace step
}  // namespace fm
