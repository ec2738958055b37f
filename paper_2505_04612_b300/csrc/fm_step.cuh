// Device functions of the passes that follow the per-keypoint-pair kernels:
// the per-image-pair pass (k_ea_segments), the per-camera pass (k_cam), the
// epipolar step's per-camera pass with the image pairs' chain rule folded in
// (k_cam_ea) and the loss reductions.  Every quantity is formed in one fixed
// order wherever it is computed, so that all paths of the library give
// bit-identical results.
#pragma once
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace step {

constexpr int kSegLanes = 8;      // lanes that share one image pair in k_ea_segments
constexpr int kThreads = 128;     // CTA size of the per-camera passes and the loss slices
                                  // (256-thread CTAs of k_cam_ea need 32k registers: two
                                  // per SM, a second wave on 300 cameras, measured slower)

// ------------------------------------------------------------------ records
// An image pair's records (one per warp run it touches; 10 values: the nine
// terms of dL/dE_n and the loss) are added in a fixed order: blocks of eight
// records q0..q7 (zero past the last), each block combined as
// ((q0 + q4) + (q2 + q6)) + ((q1 + q5) + (q3 + q7)), the blocks added to a
// running sum that starts at 0, in order.  Eight lanes form a block with a
// xor butterfly; one thread with the same three pairwise steps.

// record r's 10 values, or zeros when !ok (a predicated load, no branch: the
// loads of several records can be in flight together)
__device__ __forceinline__ void rec_load(const float4* rec, int r, bool ok, float* v) {
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 a = ok ? rec[3 * r] : z;
  const float4 b = ok ? rec[3 * r + 1] : z;
  const float4 c = ok ? rec[3 * r + 2] : z;
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  v[8] = c.x; v[9] = c.y;
}

// eight lanes of one group (sub = 0..7; mask: the group's lanes); every lane
// of the group ends with the sum
__device__ __forceinline__ void rec_sum_lanes(const float4* rec, int r0, int cnt, int sub, unsigned mask, float* G) {
#pragma unroll
  for (int k = 0; k < 10; ++k) G[k] = 0.f;
  for (int b0 = 0; b0 < cnt; b0 += kSegLanes) {
    float v[10];
    rec_load(rec, r0 + b0 + sub, b0 + sub < cnt, v);
#pragma unroll
    for (int d = kSegLanes / 2; d > 0; d >>= 1)
#pragma unroll
      for (int k = 0; k < 10; ++k) v[k] += __shfl_xor_sync(mask, v[k], d);
#pragma unroll
    for (int k = 0; k < 10; ++k) G[k] += v[k];
  }
}

__device__ __forceinline__ void add10(float* a, const float* b) {
#pragma unroll
  for (int k = 0; k < 10; ++k) a[k] += b[k];
}

// one thread, the same order
__device__ __forceinline__ void rec_sum_serial(const float4* rec, int r0, int cnt, float* G) {
#pragma unroll
  for (int k = 0; k < 10; ++k) G[k] = 0.f;
  for (int b0 = 0; b0 < cnt; b0 += kSegLanes) {
    const int r = r0 + b0, left = cnt - b0;
    float a[10], b[10], c[10], d[10];
    rec_load(rec, r + 0, 0 < left, a);
    rec_load(rec, r + 4, 4 < left, b);
    add10(a, b);                        // q0 + q4
    rec_load(rec, r + 2, 2 < left, c);
    rec_load(rec, r + 6, 6 < left, b);
    add10(c, b);                        // q2 + q6
    add10(a, c);
    rec_load(rec, r + 1, 1 < left, c);
    rec_load(rec, r + 5, 5 < left, b);
    add10(c, b);                        // q1 + q5
    rec_load(rec, r + 3, 3 < left, d);
    rec_load(rec, r + 7, 7 < left, b);
    add10(d, b);                        // q3 + q7
    add10(c, d);
    add10(a, c);
    add10(G, a);
  }
}

// the loss terms (value 9) of one block of eight records, the same order
__device__ __forceinline__ float rec_loss_block(const float* q) {
  return ((q[0] + q[4]) + (q[2] + q[6])) + ((q[1] + q[5]) + (q[3] + q[7]));
}

__device__ __forceinline__ void rec_loss_load(const float4* rec, int r, int left, float* q) {
#pragma unroll
  for (int s = 0; s < kSegLanes; ++s) q[s] = (s < left) ? rec[3 * (r + s) + 2].y : 0.f;
}

// ------------------------------------------------------------- image pairs

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

// dL/dE_n from its summed records G (scaled in place by the normalisers), and
// the chain rule through E_n = [t^]_x R_ij to the two cameras (Sec. 3.3):
// o = (dL/dR_i, dL/dt_i, dL/dR_j, dL/dt_j).  An image pair without keypoint
// pairs (cnt 0; its geometry may be degenerate) gets zeros.
__device__ __forceinline__ void pair_grad(const SegArgs& a, int n, int cnt, float* G, const float* qi,
                                          const float* qj, float* o) {
  if (cnt == 0) {
#pragma unroll
    for (int k = 0; k < kSegGradEa; ++k) o[k] = 0.f;
    return;
  }
  if (a.grad_loss) {
    const float gl = a.grad_loss[a.pair_scene ? a.pair_scene[n] : 0];
    for (int k = 0; k < 9; ++k) G[k] *= gl;
  }
  PairGeo g;
  pair_geometry(qi, qj, g);
  pair_backward(g, G, o);
}

// Image pair n, shared by kSegLanes lanes (sub = lane index in the group):
// the records' sum in the fixed order, the normalisers, the loss term, and
// the chain rule by the group's first lane.  Every lane of the warp must
// call it.
__device__ __forceinline__ void segment_pair(const SegArgs& a, int n, int sub, const SegStatic& st) {
  const bool valid = n < a.P;
  // the cameras' parameters are needed by the chain rule after the sum:
  // loaded now, with the records, rather than after the butterfly
  const bool chain = valid && sub == 0 && a.seg_grad != nullptr && st.cnt > 0;
  float qi[9], qj[9];
  if (chain) {
    load_plain(a.params + 9 * st.ci, qi, 9);
    load_plain(a.params + 9 * st.cj, qj, 9);
  }
  const int lane = threadIdx.x & 31;
  const unsigned mask = 0xffu << (lane & ~(kSegLanes - 1));
  float G[10];
  rec_sum_lanes(a.rec, st.r0, (valid && !a.dlde_in) ? st.cnt : 0, sub, mask, G);
  if (!valid || sub != 0) return;
  const float ps = a.pair_scale ? a.pair_scale[n] : 1.f;
  if (a.dlde_in) {
    for (int k = 0; k < 9; ++k) G[k] = a.dlde_in[9 * (size_t)n + k];
  } else {
    const float gs = a.g_scale * ps;
    for (int k = 0; k < 9; ++k) G[k] *= gs;
  }
  if (a.seg_loss) a.seg_loss[n] = __fmul_rn(G[9], a.l_scale * ps);
  if (a.dlde_out)
    for (int k = 0; k < 9; ++k) a.dlde_out[9 * (size_t)n + k] = G[k];
  if (!a.seg_grad) return;
  float o[kSegGradEa];
  pair_grad(a, n, st.cnt, G, qi, qj, o);
  float* out = a.seg_grad + (size_t)kSegGradEa * n;
  if ((reinterpret_cast<uintptr_t>(out) & 15u) == 0) {   // library buffers: 96-B rows, 16-B aligned
    float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll
    for (int k = 0; k < kSegGradEa / 4; ++k) o4[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
  } else {
    for (int k = 0; k < kSegGradEa; ++k) out[k] = o[k];
  }
}

// ---------------------------------------------------------------- cameras

// Per-stage layout of the per-camera pass.  STAGE 0 rotation (part 9: dR,
// params 6D), 1 translation (part 3: do, params o), 2 epipolar (part 12: dR,
// dt; params 6D + t)
template <int STAGE>
struct Layout;
// PART floats of a camera's part, stored in a slot of STRIDE floats (a
// multiple of 4: 16-byte loads)
template <> struct Layout<0> { static constexpr int PART = 9, STRIDE = 12, PDIM = 6; static constexpr bool ROT = true; };
template <> struct Layout<1> { static constexpr int PART = 3, STRIDE = 4, PDIM = 3; static constexpr bool ROT = false; };
template <> struct Layout<2> { static constexpr int PART = 12, STRIDE = 12, PDIM = 9; static constexpr bool ROT = true; };

// adds the part at g (PART floats of a slot of STRIDE floats, 16-byte
// aligned in a cudaMalloc'd buffer)
template <int PART, int STRIDE>
__device__ __forceinline__ void cam_add_part(const float* g, float* acc) {
  static_assert(STRIDE % 4 == 0 && PART <= STRIDE, "16-byte slots");
  float v[STRIDE];
#pragma unroll
  for (int q = 0; q < STRIDE / 4; ++q) {
    const float4 t = *reinterpret_cast<const float4*>(g + 4 * q);
    v[4 * q] = t.x;
    v[4 * q + 1] = t.y;
    v[4 * q + 2] = t.z;
    v[4 * q + 3] = t.w;
  }
#pragma unroll
  for (int k = 0; k < PART; ++k) acc[k] += v[k];
}

// adds the part of camera-CSR entry `entry` (image pair | role << 31) of the
// per-image-pair gradients sg
template <int PART, int STRIDE>
__device__ __forceinline__ void cam_add(const float* sg, int entry, float* acc) {
  const unsigned w = (unsigned)entry;
  const int n = (int)(w & 0x7fffffffu);
  const int role = (int)(w >> 31);
  cam_add_part<PART, STRIDE>(sg + ((size_t)n * 2 + role) * STRIDE, acc);
}

// A camera's parts over its incident image pairs [b, e) of the camera CSR are
// added in a fixed order by one CTA of kThreads: thread t adds the entries
// b + t, b + t + kThreads, ... in that order, a xor butterfly combines each
// warp, and the warps' sums are added in warp order.  cam_reduce does the
// last two steps; warp 0 holds the total.
template <int PART>
__device__ __forceinline__ void cam_reduce(float* acc, float (*red)[PART]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < PART; ++k) acc[k] = warp_sum(acc[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < PART; ++k) red[warp][k] = acc[k];
  __syncthreads();
  if (warp == 0)
#pragma unroll
    for (int k = 0; k < PART; ++k) {
      float t = red[0][k];
      for (int w = 1; w < kThreads / 32; ++w) t += red[w][k];
      acc[k] = t;
    }
}

// What cam_apply needs besides the summed parts, formed from the camera's
// parameters p as soon as they are loaded (off the critical path of the
// gather and the reduction): the 6D map's forward state and Adam's bias
// corrections (the step counter was advanced by this step's first kernel).
struct CamPre {
  Rot6 s;
  float bc1, bc2;
};

template <int STAGE, bool ADAM>
__device__ __forceinline__ void cam_pre(const CamUpdate& u, const float* p, CamPre& pre) {
  if (Layout<STAGE>::ROT) rot6_forward(p, pre.s);
  if (ADAM) {
    const float t = (float)*u.step;
    pre.bc1 = 1.f - powf(u.b1, t);
    pre.bc2 = 1.f - powf(u.b2, t);
  }
}

// Camera c of run `run` from its summed parts, its parameters p, cam_pre's
// state and (Adam) its moments m, v of lane's entry (all loaded beforehand):
// the 6D adjoint for rotations, then either the gradient or Adam
// (bias-corrected), by lanes < PDIM of warp 0.
template <int STAGE, bool ADAM>
__device__ __forceinline__ void cam_apply(const CamUpdate& u, size_t off, const float* p, float m, float v,
                                          const float* acc, int lane, const CamPre& pre) {
  using L = Layout<STAGE>;
  float g[L::PDIM];
  if (L::ROT) {
    rot6_adjoint(p, pre.s, acc, g);
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
  m = u.b1 * m + (1.f - u.b1) * gv;
  v = u.b2 * v + (1.f - u.b2) * gv * gv;
  u.m[off + lane] = m;
  u.v[off + lane] = v;
  u.params_out[off + lane] = pv - u.lr * (m / pre.bc1) / (sqrtf(v / pre.bc2) + u.eps);
}

// ------------------------------------------------------------------- losses
// A scene's loss, the sum of its image pairs' loss terms x_0 .. x_{n-1}, is
// added in slices of kSlice terms: slice k (terms kSlice k ..) by one CTA,
// thread t adding the terms t, t + kThreads, ... of the slice in order, xor
// butterflies in each warp and the warps in order; then the slices' sums the
// same way (thread-strided over the slices, butterflies, warps in order).  One CTA per slice; the last to finish (an
// arrival counter per (scene, run) on a line of its own, reset by it) adds
// the slices.  The order depends on n only.
constexpr int kSlice = kLossSlice;

// the scene of global slice g: the largest s with sc_slice_off[s] <= g
__device__ __forceinline__ int slice_scene(const int* sc_slice_off, int S, int g) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sc_slice_off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Global slice g of run `run` (scene sc): the slice's sum, then the
// combination.  fill(j, k, v) puts the thread's terms j, j + kThreads, ...
// (k of them; the rest 0) into v, so that their loads can be issued
// together.  Every thread of the CTA calls it.
constexpr int kPerThread = kSlice / kThreads;

// the CTA's sum of one value per thread: xor butterflies in each warp, then
// the warps' sums in warp order (thread 0 returns it; every thread calls it)
__device__ __forceinline__ float cta_sum(float v, float* wpart) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) wpart[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0)
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += wpart[w];
  return s;
}

template <typename Fill>
__device__ __forceinline__ void loss_slice(const LossArgs& L, int sc, int g, int run, Fill fill) {
  __shared__ float wpart[2][kThreads / 32];
  __shared__ int last;
  const int t = threadIdx.x;
  const int n = L.sc_pair_off[sc + 1] - L.sc_pair_off[sc];
  const int j0 = (g - L.sc_slice_off[sc]) * kSlice, j1 = min(n, j0 + kSlice);
  const int k = (j1 - j0 - t + kThreads - 1) / kThreads;   // this thread's terms
  float v[kPerThread];
  fill(j0 + t, k > 0 ? k : 0, v);
  float acc = 0.f;
#pragma unroll
  for (int u = 0; u < kPerThread; ++u) acc += v[u];   // terms past the slice are +0 (terms are >= 0)
  const float slice = cta_sum(acc, wpart[0]);
  const int n_slices = L.sc_slice_off[sc + 1] - L.sc_slice_off[sc];
  float* partial = L.partial + (size_t)run * L.n_slices;
  int* cnt = L.cnt + ((size_t)run * L.S + sc) * kLossCntStride;
  if (t == 0) {
    partial[g] = slice;
    __threadfence();   // this slice's sum before its count
    last = atomicAdd(cnt, 1) == n_slices - 1;
    if (last) __threadfence();
  }
  __syncthreads();
  if (last) {   // the same value in every thread: the whole CTA adds the slices
    const float* ps = partial + L.sc_slice_off[sc];
    float q = 0.f;
    for (int i = t; i < n_slices; i += kThreads) q += __ldcg(ps + i);
    const float total = cta_sum(q, wpart[1]);
    if (t == 0) {
      const size_t o = (size_t)run * L.S + sc;
      L.out[o] = total;
      if (L.out2) L.out2[o] = total;
      *cnt = 0;   // ready for the next launch
    }
  }
}

// fill of loss terms stored in x
__device__ __forceinline__ void fill_stored(const float* x, int j, int k, float* v) {
#pragma unroll
  for (int u = 0; u < kPerThread; ++u) v[u] = (u < k) ? x[j + u * kThreads] : 0.f;
}

// Loss terms formed from records, as segment_pair forms seg_loss (the record
// sum's order, then an uncontracted product with the normalisers), in two
// parts: rec_ranges reads the static range and normaliser of each of the
// thread's k image pairs (before the dependency wait), fill_from_records the
// records: the first block of every image pair with predicated loads and no
// branch between them, so that they are all in flight together, then any
// further blocks (image pairs of more than eight records).
struct RecRanges {
  int r0[kPerThread], cnt[kPerThread];
  float scale[kPerThread];
};

__device__ __forceinline__ void rec_ranges(const SegArgs& s, int n0, int j, int k, RecRanges& R) {
#pragma unroll
  for (int u = 0; u < kPerThread; ++u) {
    const int n = n0 + j + u * kThreads;
    R.r0[u] = (u < k) ? s.seg_rec[2 * n] : 0;
    R.cnt[u] = (u < k) ? s.seg_rec[2 * n + 1] : 0;
    R.scale[u] = s.l_scale * ((u < k && s.pair_scale) ? s.pair_scale[n] : 1.f);
  }
}

__device__ __forceinline__ void fill_from_records(const SegArgs& s, const RecRanges& R, int k, float* v) {
  float q[kPerThread][kSegLanes];
#pragma unroll
  for (int u = 0; u < kPerThread; ++u) rec_loss_load(s.rec, R.r0[u], R.cnt[u], q[u]);
#pragma unroll
  for (int u = 0; u < kPerThread; ++u) {
    float G = 0.f;
    G += rec_loss_block(q[u]);
    for (int b0 = kSegLanes; b0 < R.cnt[u]; b0 += kSegLanes) {
      float w[kSegLanes];
      rec_loss_load(s.rec, R.r0[u] + b0, R.cnt[u] - b0, w);
      G += rec_loss_block(w);
    }
    v[u] = (u < k) ? __fmul_rn(G, R.scale[u]) : 0.f;
  }
}

// the terms of global slice g held by this thread: first term j, count k
__device__ __forceinline__ void slice_terms(const LossArgs& L, int sc, int g, int& j, int& k) {
  const int n = L.sc_pair_off[sc + 1] - L.sc_pair_off[sc];
  const int j0 = (g - L.sc_slice_off[sc]) * kSlice, j1 = min(n, j0 + kSlice);
  j = j0 + (int)threadIdx.x;
  k = max(0, (j1 - j + kThreads - 1) / kThreads);
}

}  // namespace step
}  // namespace fm
