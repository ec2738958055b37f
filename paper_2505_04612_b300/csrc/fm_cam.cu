// Per-camera assembly and optimiser step: a camera's gradient is the sum,
// over the image pairs it belongs to (camera CSR, fixed order), of the
// per-image-pair gradients; rotations then go through the adjoint of the 6D
// map (Sec. 3.3), and Adam updates the camera's parameters in place.
// One CTA per camera; threads stride over the incident image pairs, a
// butterfly inside each warp and a fixed-order sum over the warps combine
// them, so the order of additions is fixed.
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

// STAGE 0 rotation (part 9: dR, params 6D), 1 translation (part 3: do,
// params o), 2 epipolar (part 12: dR, dt; params 6D + t)
template <int STAGE>
struct Layout;
template <> struct Layout<0> { static constexpr int PART = 9, PDIM = 6; static constexpr bool ROT = true; };
template <> struct Layout<1> { static constexpr int PART = 3, PDIM = 3; static constexpr bool ROT = false; };
template <> struct Layout<2> { static constexpr int PART = 12, PDIM = 9; static constexpr bool ROT = true; };

constexpr int kCamThreads = 128;
constexpr int kCamWarps = kCamThreads / 32;

// fixed-order sum of n per-image-pair loss terms (one CTA of kCamThreads):
// scalar loads up to the first 16-B boundary, then float4 loads with eight in
// flight per thread, then the scalar tail; per-thread partials in a fixed
// order and a tree over the threads.  The order depends only on n and on the
// address of x, so every launch over the same range adds in the same order.
__device__ void loss_sum_cta(const float* x, int n, float* out) {
  __shared__ float part[kCamThreads];
  constexpr int T = kCamThreads;
  const int t = threadIdx.x;
  const int head = min(n, (int)(((16u - (unsigned)(reinterpret_cast<uintptr_t>(x) & 15u)) & 15u) >> 2));
  const float4* x4 = reinterpret_cast<const float4*>(x + head);
  const int n4 = (n - head) >> 2;
  float acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = 0.f;
  int k = t;
  for (; k + 7 * T < n4; k += 8 * T) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = x4[k + u * T];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] += (v[u].x + v[u].y) + (v[u].z + v[u].w);
  }
  for (; k < n4; k += T) {
    const float4 v = x4[k];
    acc[0] += (v.x + v.y) + (v.z + v.w);
  }
  if (t < head) acc[1] += x[t];
  for (int q = head + 4 * n4 + t; q < n; q += T) acc[2] += x[q];
  part[t] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  __syncthreads();
  for (int d = T / 2; d > 0; d >>= 1) {
    if (t < d) part[t] += part[t + d];
    __syncthreads();
  }
  if (t == 0) *out = part[0];
}

template <int STAGE, bool ADAM>
__global__ void __launch_bounds__(kCamThreads) k_cam(CamUpdate u) {
  using L = Layout<STAGE>;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int run = blockIdx.y;
  pdl_trigger();
  if (u.loss_out && (int)blockIdx.x >= u.N) {
    // the S extra CTAs of the grid reduce the loss of each scene
    const int sc = blockIdx.x - u.N;
    const int b = u.sc_pair_off[sc], e = u.sc_pair_off[sc + 1];
    pdl_wait();
    loss_sum_cta(u.seg_loss + (size_t)run * u.P + b, e - b, u.loss_out + (size_t)run * u.S + sc);
    return;
  }
  const int c = blockIdx.x;                                    // one CTA per camera
  const int b = u.cam_seg_off[c], e = u.cam_seg_off[c + 1];   // static: before the wait
  pdl_wait();
  float acc[L::PART];
#pragma unroll
  for (int k = 0; k < L::PART; ++k) acc[k] = 0.f;
  const float* sg = u.seg_grad + (size_t)run * u.P * 2 * L::PART;
  for (int idx = b + (int)threadIdx.x; idx < e; idx += kCamThreads) {
    const unsigned v = (unsigned)u.cam_seg[idx];
    const int n = (int)(v & 0x7fffffffu);
    const int role = (int)(v >> 31);
    const float* g = sg + ((size_t)n * 2 + role) * L::PART;
    if (L::PART % 4 == 0) {
      // 48-B parts of a cudaMalloc'd buffer: 16-B aligned
#pragma unroll
      for (int q = 0; q < L::PART / 4; ++q) {
        const float4 t = reinterpret_cast<const float4*>(g)[q];
        acc[4 * q] += t.x;
        acc[4 * q + 1] += t.y;
        acc[4 * q + 2] += t.z;
        acc[4 * q + 3] += t.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < L::PART; ++k) acc[k] += g[k];
    }
  }
  __shared__ float red[kCamWarps][L::PART];
#pragma unroll
  for (int k = 0; k < L::PART; ++k) acc[k] = warp_sum(acc[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < L::PART; ++k) red[warp][k] = acc[k];
  __syncthreads();
  if (warp != 0) return;
#pragma unroll
  for (int k = 0; k < L::PART; ++k) {
    float t = red[0][k];
    for (int w = 1; w < kCamWarps; ++w) t += red[w][k];
    acc[k] = t;
  }
  const float* prm = u.params + ((size_t)run * u.N + c) * L::PDIM;
  float p[L::PDIM];
#pragma unroll
  for (int k = 0; k < L::PDIM; ++k) p[k] = prm[k];
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
  __syncwarp();
  const size_t off = ((size_t)run * u.N + c) * L::PDIM;
  if (!ADAM) {
    if (lane < L::PDIM) {
      float gv = g[0];
#pragma unroll
      for (int k = 1; k < L::PDIM; ++k)
        if (lane == k) gv = g[k];
      u.grad_out[off + lane] = gv;
    }
    return;
  }
  if (lane < L::PDIM) {
    float gv = g[0], pv = p[0];
#pragma unroll
    for (int k = 1; k < L::PDIM; ++k)
      if (lane == k) { gv = g[k]; pv = p[k]; }
    if (u.grad_out) u.grad_out[off + lane] = gv;
    const float t = (float)*u.step;
    const float bc1 = 1.f - powf(u.b1, t);
    const float bc2 = 1.f - powf(u.b2, t);
    float m = u.m[off + lane], v = u.v[off + lane];
    m = u.b1 * m + (1.f - u.b1) * gv;
    v = u.b2 * v + (1.f - u.b2) * gv * gv;
    u.m[off + lane] = m;
    u.v[off + lane] = v;
    u.params_out[off + lane] = pv - u.lr * (m / bc1) / (sqrtf(v / bc2) + u.eps);
  }
}

// fixed-order sum of each scene's range of values per run (one CTA per
// (scene, run)); the same order as the loss CTAs of k_cam
__global__ void __launch_bounds__(kCamThreads) k_sum_fixed(const float* __restrict__ x, int P,
                                                           const int* __restrict__ sc_pair_off,
                                                           float* __restrict__ out) {
  const int sc = blockIdx.x, run = blockIdx.y;
  const int b = sc_pair_off ? sc_pair_off[sc] : 0, e = sc_pair_off ? sc_pair_off[sc + 1] : P;
  loss_sum_cta(x + (size_t)run * P + b, e - b, out + (size_t)run * gridDim.x + sc);
}

template <int STAGE>
void launch_stage(const CamUpdate& u, cudaStream_t s) {
  dim3 grid(u.N + (u.loss_out ? u.S : 0), u.runs);
  if (u.params_out) launch_pdl(k_cam<STAGE, true>, grid, dim3(kCamThreads), 0, s, u);
  else launch_pdl(k_cam<STAGE, false>, grid, dim3(kCamThreads), 0, s, u);
}

}  // namespace

void launch_cam_update(int stage, const CamUpdate& u, cudaStream_t s) {
  if (stage == FM_STAGE_ROTATION) launch_stage<0>(u, s);
  else if (stage == FM_STAGE_TRANSLATION) launch_stage<1>(u, s);
  else launch_stage<2>(u, s);
}

void launch_sum_fixed(const float* x, int P, int runs, const int* sc_pair_off, int S, float* out,
                      cudaStream_t s) {
  k_sum_fixed<<<dim3(S, runs), kCamThreads, 0, s>>>(x, P, sc_pair_off, out);
}

}  // namespace fm
