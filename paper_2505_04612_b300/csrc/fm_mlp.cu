// Learned per-pair inlier weights: the per-image-pair feature tables, the
// features alone, and the training of the 8-64-64-1 GELU network on the
// tensor cores (bfloat16 operands, float32 accumulation, mma.sync m16n8k16):
// its binary cross-entropy gradient and Adam.  Inference runs on tcgen05
// (fm_mlp_tc.cu).  The paper down-weights outliers with IRLS and a periodic filter
// (Sec. 3.3, Eq. 9); the network replaces the filter by a predicted inlier
// probability.  Feature and network definitions (readings) are those of the
// problem-level documentation in include/fastmap.h.
//
// Tensor-core layout: a warp runs the network on 16 pairs at a time (one
// m-tile).  Layer 1 is one k-step (8 features padded to 16) over 8 n-tiles,
// layer 2 four k-steps over 8 n-tiles.  The float32 accumulator fragments of
// one layer, rounded to bfloat16 pairwise, are exactly the A fragments of the
// next, so activations never leave registers.  Weights are staged once per
// CTA in shared memory in fragment order (one 8-byte load per lane per mma).
//
// Training (k_mlp_grad): per 64-pair chunk each warp runs the forward pass of
// 16 pairs, the output gradient, dz2 = dlogit w3 * GELU'(z2), dh1 = dz2 W2^T
// (tensor cores, W2^T fragments staged), dz1 = dh1 * GELU'(z1); x, h1, dz2
// and dz1 go to shared memory as bfloat16 and the weight gradients are
// contractions over the chunk's pairs: warp w owns rows 16w..16w+15 of dW2
// (h1 units) and n-tiles 2w, 2w+1 of dW1, so every entry is accumulated by
// one thread in a fixed order.  Per-CTA partial sums are reduced across CTAs
// in CTA order: the gradient is deterministic.
#include <cuda_bf16.h>

#include "fm_device.cuh"
#include "fm_internal.h"
#include "fm_mlp.cuh"

namespace fm {
namespace {

constexpr int kIn = 8, kHid = 64;
constexpr int kOffW1 = 0, kOffB1 = 512, kOffW2 = 576, kOffB2 = 4672, kOffW3 = 4736, kOffB3 = 4800;
static_assert(kOffB3 + 1 == kMlpParams, "parameter layout");
constexpr int kPartStride = kMlpParams + 3;   // + loss, padded to a multiple of 4
constexpr int kWarps = 4;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
  return *reinterpret_cast<uint32_t*>(&v);
}

// D += A B, A 16x16 (row), B 16x8 (col), bfloat16 in, float32 accumulate
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}
__device__ __forceinline__ float sigmoid_f(float o) { return 1.f / (1.f + expf(-o)); }
__device__ __forceinline__ float softplus_f(float o) { return fmaxf(o, 0.f) + log1pf(expf(-fabsf(o))); }

// weights of one CTA, B operands in fragment order: [k-tile][n-tile][lane][2]
struct MlpWeights {
  uint32_t w1f[8][32][2];       // W1 (k: feature, padded to 16; n: layer-1 unit)
  uint32_t w2f[4][8][32][2];    // W2 (k: layer-1 unit; n: layer-2 unit)
  uint32_t w2tf[4][8][32][2];   // W2^T (k: layer-2 unit; n: layer-1 unit), training only
  float b1[kHid], b2[kHid], w3[kHid], b3;
};

// B fragment (k, n) of lane l, register j: k = 2 (l % 4) + 8 j + {0, 1},
// n = l / 4 (PTX ISA, mma.m16n8k16 .bf16 fragment layout)
__device__ void stage_weights(const float* theta, MlpWeights& s, bool transposed) {
  for (int idx = threadIdx.x; idx < 8 * 32 * 2; idx += blockDim.x) {
    const int nt = idx >> 6, lane = (idx >> 1) & 31, j = idx & 1;
    const int k = 2 * (lane & 3) + 8 * j, n = nt * 8 + (lane >> 2);
    const float lo = k < kIn ? theta[kOffW1 + k * kHid + n] : 0.f;
    const float hi = k + 1 < kIn ? theta[kOffW1 + (k + 1) * kHid + n] : 0.f;
    s.w1f[nt][lane][j] = pack_bf16(lo, hi);
  }
  for (int idx = threadIdx.x; idx < 4 * 8 * 32 * 2; idx += blockDim.x) {
    const int kt = idx >> 9, nt = (idx >> 6) & 7, lane = (idx >> 1) & 31, j = idx & 1;
    const int k = kt * 16 + 2 * (lane & 3) + 8 * j, n = nt * 8 + (lane >> 2);
    s.w2f[kt][nt][lane][j] = pack_bf16(theta[kOffW2 + k * kHid + n], theta[kOffW2 + (k + 1) * kHid + n]);
    if (transposed)
      s.w2tf[kt][nt][lane][j] = pack_bf16(theta[kOffW2 + n * kHid + k], theta[kOffW2 + n * kHid + k + 1]);
  }
  for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
    s.b1[k] = theta[kOffB1 + k];
    s.b2[k] = theta[kOffB2 + k];
    s.w3[k] = theta[kOffW3 + k];
  }
  if (threadIdx.x == 0) s.b3 = theta[kOffB3];
}

// accumulators (n-tile nt: c0, c1 at row g, cols 8 nt + 2t + {0,1}; c2, c3 at
// row g + 8) initialised with a bias
__device__ __forceinline__ void init_bias(const float* b, int t, float (&z)[8][4]) {
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    z[nt][0] = z[nt][2] = b[nt * 8 + 2 * t];
    z[nt][1] = z[nt][3] = b[nt * 8 + 2 * t + 1];
  }
}

// the accumulator fragments of n-tiles 2kt, 2kt+1, rounded to bfloat16, are
// the A fragment of k-tile kt of the next product
__device__ __forceinline__ void to_a(const float (&h)[8][4], uint32_t (&a)[4][4]) {
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) {
    a[kt][0] = pack_bf16(h[2 * kt][0], h[2 * kt][1]);
    a[kt][1] = pack_bf16(h[2 * kt][2], h[2 * kt][3]);
    a[kt][2] = pack_bf16(h[2 * kt + 1][0], h[2 * kt + 1][1]);
    a[kt][3] = pack_bf16(h[2 * kt + 1][2], h[2 * kt + 1][3]);
  }
}

// forward pass of one m-tile; ax: A fragment of the features
__device__ __forceinline__ void mlp_forward(const MlpWeights& s, const uint32_t (&ax)[4], int lane,
                                            float (&z1)[8][4], uint32_t (&a1)[4][4], float (&z2)[8][4],
                                            float& o_g, float& o_g8) {
  const int t = lane & 3;
  init_bias(s.b1, t, z1);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) mma16816(z1[nt], ax, s.w1f[nt][lane]);
  float h1[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int c = 0; c < 4; ++c) h1[nt][c] = gelu_f(z1[nt][c]);
  to_a(h1, a1);
  init_bias(s.b2, t, z2);
#pragma unroll
  for (int kt = 0; kt < 4; ++kt)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) mma16816(z2[nt], a1[kt], s.w2f[kt][nt][lane]);
  float lo = 0.f, hi = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float w0 = s.w3[nt * 8 + 2 * t], w1 = s.w3[nt * 8 + 2 * t + 1];
    lo = fmaf(gelu_f(z2[nt][0]), w0, fmaf(gelu_f(z2[nt][1]), w1, lo));
    hi = fmaf(gelu_f(z2[nt][2]), w0, fmaf(gelu_f(z2[nt][3]), w1, hi));
  }
  // the four lanes of a row group hold disjoint columns: a fixed butterfly
  lo += __shfl_xor_sync(FULL, lo, 1);
  lo += __shfl_xor_sync(FULL, lo, 2);
  hi += __shfl_xor_sync(FULL, hi, 1);
  hi += __shfl_xor_sync(FULL, hi, 2);
  o_g = lo + s.b3;
  o_g8 = hi + s.b3;
}

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

// ------------------------------------------------------------ training

struct GradArgs {
  const float* theta;
  const float* x;   // [B][8]
  const float* y;   // [B]
  int64_t B;
  float inv_b;
  float* partial;   // [gridDim.x][kPartStride]
};

constexpr int kChunk = 16 * kWarps;   // pairs per chunk

struct GradSmem {
  MlpWeights w;
  __nv_bfloat16 xs[kChunk][16];       // x, features 8..15 zero
  __nv_bfloat16 h1s[kChunk][kHid];
  __nv_bfloat16 dz2s[kChunk][kHid];
  __nv_bfloat16 dz1s[kChunk][kHid];
  float red[kWarps][3][kHid];
  float red1[kWarps][2];
};

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p0, const __nv_bfloat16* p1) {
  __nv_bfloat162 v;
  v.x = *p0;
  v.y = *p1;
  return *reinterpret_cast<uint32_t*>(&v);
}

__global__ void __launch_bounds__(kWarps * 32) k_mlp_grad(GradArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  GradSmem& S = *reinterpret_cast<GradSmem*>(smraw);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  stage_weights(a.theta, S.w, true);
  __syncthreads();
  const MlpWeights& s = S.w;
  float dW2[8][4], dW1[2][4];
  float db1[8][2], db2[8][2], dw3[8][2];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int c = 0; c < 4; ++c) dW2[nt][c] = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) dW1[j][c] = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) db1[nt][0] = db1[nt][1] = db2[nt][0] = db2[nt][1] = dw3[nt][0] = dw3[nt][1] = 0.f;
  float db3 = 0.f, lsum = 0.f;

  for (int64_t chunk = blockIdx.x; chunk * kChunk < a.B; chunk += gridDim.x) {
    const int row0 = 16 * w;                      // the warp's rows inside the chunk
    const int64_t p0 = chunk * kChunk + row0;
    const int64_t pg = p0 + g, pg8 = p0 + g + 8;
    const bool vg = pg < a.B, vg8 = pg8 < a.B;
    float x0 = 0.f, x1 = 0.f, y0 = 0.f, y1 = 0.f;
    if (vg) { x0 = a.x[pg * kIn + 2 * t]; x1 = a.x[pg * kIn + 2 * t + 1]; }
    if (vg8) { y0 = a.x[pg8 * kIn + 2 * t]; y1 = a.x[pg8 * kIn + 2 * t + 1]; }
    const uint32_t ax[4] = {pack_bf16(x0, x1), pack_bf16(y0, y1), 0u, 0u};
    *reinterpret_cast<uint32_t*>(&S.xs[row0 + g][2 * t]) = ax[0];
    *reinterpret_cast<uint32_t*>(&S.xs[row0 + g + 8][2 * t]) = ax[1];
    *reinterpret_cast<uint32_t*>(&S.xs[row0 + g][8 + 2 * t]) = 0u;
    *reinterpret_cast<uint32_t*>(&S.xs[row0 + g + 8][8 + 2 * t]) = 0u;
    float z1[8][4], z2[8][4];
    uint32_t a1[4][4];
    float o_g, o_g8;
    mlp_forward(s, ax, lane, z1, a1, z2, o_g, o_g8);
    // h1 (bfloat16, as the A fragments hold it) into shared memory
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      *reinterpret_cast<uint32_t*>(&S.h1s[row0 + g][16 * kt + 2 * t]) = a1[kt][0];
      *reinterpret_cast<uint32_t*>(&S.h1s[row0 + g + 8][16 * kt + 2 * t]) = a1[kt][1];
      *reinterpret_cast<uint32_t*>(&S.h1s[row0 + g][16 * kt + 8 + 2 * t]) = a1[kt][2];
      *reinterpret_cast<uint32_t*>(&S.h1s[row0 + g + 8][16 * kt + 8 + 2 * t]) = a1[kt][3];
    }
    const float yg = vg ? a.y[pg] : 0.f, yg8 = vg8 ? a.y[pg8] : 0.f;
    const float dl_g = vg ? (sigmoid_f(o_g) - yg) * a.inv_b : 0.f;
    const float dl_g8 = vg8 ? (sigmoid_f(o_g8) - yg8) * a.inv_b : 0.f;
    if (t == 0) {
      if (vg) lsum += softplus_f(o_g) - yg * o_g;
      if (vg8) lsum += softplus_f(o_g8) - yg8 * o_g8;
      db3 += dl_g + dl_g8;
    }
    float dz2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float w0 = s.w3[nt * 8 + 2 * t], w1 = s.w3[nt * 8 + 2 * t + 1];
      dw3[nt][0] += gelu_f(z2[nt][0]) * dl_g + gelu_f(z2[nt][2]) * dl_g8;
      dw3[nt][1] += gelu_f(z2[nt][1]) * dl_g + gelu_f(z2[nt][3]) * dl_g8;
      dz2[nt][0] = dl_g * w0 * gelu_grad_f(z2[nt][0]);
      dz2[nt][1] = dl_g * w1 * gelu_grad_f(z2[nt][1]);
      dz2[nt][2] = dl_g8 * w0 * gelu_grad_f(z2[nt][2]);
      dz2[nt][3] = dl_g8 * w1 * gelu_grad_f(z2[nt][3]);
      db2[nt][0] += dz2[nt][0] + dz2[nt][2];
      db2[nt][1] += dz2[nt][1] + dz2[nt][3];
    }
    uint32_t adz2[4][4];
    to_a(dz2, adz2);
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      *reinterpret_cast<uint32_t*>(&S.dz2s[row0 + g][16 * kt + 2 * t]) = adz2[kt][0];
      *reinterpret_cast<uint32_t*>(&S.dz2s[row0 + g + 8][16 * kt + 2 * t]) = adz2[kt][1];
      *reinterpret_cast<uint32_t*>(&S.dz2s[row0 + g][16 * kt + 8 + 2 * t]) = adz2[kt][2];
      *reinterpret_cast<uint32_t*>(&S.dz2s[row0 + g + 8][16 * kt + 8 + 2 * t]) = adz2[kt][3];
    }
    // dh1 = dz2 W2^T, dz1 = dh1 * GELU'(z1)
    float dz1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) dz1[nt][0] = dz1[nt][1] = dz1[nt][2] = dz1[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) mma16816(dz1[nt], adz2[kt], s.w2tf[kt][nt][lane]);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
      for (int c = 0; c < 4; ++c) dz1[nt][c] *= gelu_grad_f(z1[nt][c]);
      db1[nt][0] += dz1[nt][0] + dz1[nt][2];
      db1[nt][1] += dz1[nt][1] + dz1[nt][3];
    }
    uint32_t adz1[4][4];
    to_a(dz1, adz1);
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      *reinterpret_cast<uint32_t*>(&S.dz1s[row0 + g][16 * kt + 2 * t]) = adz1[kt][0];
      *reinterpret_cast<uint32_t*>(&S.dz1s[row0 + g + 8][16 * kt + 2 * t]) = adz1[kt][1];
      *reinterpret_cast<uint32_t*>(&S.dz1s[row0 + g][16 * kt + 8 + 2 * t]) = adz1[kt][2];
      *reinterpret_cast<uint32_t*>(&S.dz1s[row0 + g + 8][16 * kt + 8 + 2 * t]) = adz1[kt][3];
    }
    __syncthreads();
    // dW2 rows 16w..16w+15 (layer-1 units) += h1^T dz2 over the chunk's pairs
#pragma unroll
    for (int ks = 0; ks < kChunk / 16; ++ks) {
      const int k0 = 16 * ks;
      const int u = 16 * w + g;
      const uint32_t A[4] = {ld_pair(&S.h1s[k0 + 2 * t][u], &S.h1s[k0 + 2 * t + 1][u]),
                             ld_pair(&S.h1s[k0 + 2 * t][u + 8], &S.h1s[k0 + 2 * t + 1][u + 8]),
                             ld_pair(&S.h1s[k0 + 2 * t + 8][u], &S.h1s[k0 + 2 * t + 9][u]),
                             ld_pair(&S.h1s[k0 + 2 * t + 8][u + 8], &S.h1s[k0 + 2 * t + 9][u + 8])};
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int v = nt * 8 + g;
        const uint32_t Bf[2] = {ld_pair(&S.dz2s[k0 + 2 * t][v], &S.dz2s[k0 + 2 * t + 1][v]),
                                ld_pair(&S.dz2s[k0 + 2 * t + 8][v], &S.dz2s[k0 + 2 * t + 9][v])};
        mma16816(dW2[nt], A, Bf);
      }
      // dW1 (features x layer-1 units), n-tiles 2w, 2w+1 += x^T dz1
      const uint32_t Ax[4] = {ld_pair(&S.xs[k0 + 2 * t][g], &S.xs[k0 + 2 * t + 1][g]),
                              ld_pair(&S.xs[k0 + 2 * t][g + 8], &S.xs[k0 + 2 * t + 1][g + 8]),
                              ld_pair(&S.xs[k0 + 2 * t + 8][g], &S.xs[k0 + 2 * t + 9][g]),
                              ld_pair(&S.xs[k0 + 2 * t + 8][g + 8], &S.xs[k0 + 2 * t + 9][g + 8])};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int v = (2 * w + j) * 8 + g;
        const uint32_t Bf[2] = {ld_pair(&S.dz1s[k0 + 2 * t][v], &S.dz1s[k0 + 2 * t + 1][v]),
                                ld_pair(&S.dz1s[k0 + 2 * t + 8][v], &S.dz1s[k0 + 2 * t + 9][v])};
        mma16816(dW1[j], Ax, Bf);
      }
    }
    __syncthreads();   // the staging buffers are refilled by the next chunk
  }

  // ---- this CTA's partial sums
  float* P = a.partial + (size_t)blockIdx.x * kPartStride;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int col = nt * 8 + 2 * t, r0 = 16 * w + g;
    P[kOffW2 + r0 * kHid + col] = dW2[nt][0];
    P[kOffW2 + r0 * kHid + col + 1] = dW2[nt][1];
    P[kOffW2 + (r0 + 8) * kHid + col] = dW2[nt][2];
    P[kOffW2 + (r0 + 8) * kHid + col + 1] = dW2[nt][3];
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {   // rows g < 8 are the features; rows g + 8 are padding
    const int col = (2 * w + j) * 8 + 2 * t;
    P[kOffW1 + g * kHid + col] = dW1[j][0];
    P[kOffW1 + g * kHid + col + 1] = dW1[j][1];
  }
  // column sums over the warp's row groups (fixed butterfly), then over warps
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int d = 4; d < 32; d <<= 1) {
        db1[nt][c] += __shfl_xor_sync(FULL, db1[nt][c], d);
        db2[nt][c] += __shfl_xor_sync(FULL, db2[nt][c], d);
        dw3[nt][c] += __shfl_xor_sync(FULL, dw3[nt][c], d);
      }
  if (g == 0) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        S.red[w][0][nt * 8 + 2 * t + c] = db1[nt][c];
        S.red[w][1][nt * 8 + 2 * t + c] = db2[nt][c];
        S.red[w][2][nt * 8 + 2 * t + c] = dw3[nt][c];
      }
  }
  db3 = warp_sum(db3);
  lsum = warp_sum(lsum);
  if (lane == 0) {
    S.red1[w][0] = db3;
    S.red1[w][1] = lsum;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kHid; k += blockDim.x) {
    float v0 = 0.f, v1 = 0.f, v2 = 0.f;
    for (int q = 0; q < kWarps; ++q) {
      v0 += S.red[q][0][k];
      v1 += S.red[q][1][k];
      v2 += S.red[q][2][k];
    }
    P[kOffB1 + k] = v0;
    P[kOffB2 + k] = v1;
    P[kOffW3 + k] = v2;
  }
  if (threadIdx.x == 0) {
    float v0 = 0.f, v1 = 0.f;
    for (int q = 0; q < kWarps; ++q) {
      v0 += S.red1[q][0];
      v1 += S.red1[q][1];
    }
    P[kOffB3] = v0;
    P[kMlpParams] = v1 * a.inv_b;
  }
}

// fixed-order sum of the CTA partials: grad [4801], loss
__global__ void k_mlp_reduce(const float* __restrict__ partial, int parts, float* __restrict__ grad,
                             float* __restrict__ loss) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > kMlpParams) return;
  float s = 0.f;
  for (int c = 0; c < parts; ++c) s += partial[(size_t)c * kPartStride + k];
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

size_t mlp_grad_smem() { return sizeof(GradSmem); }
int mlp_grad_parts(int64_t B) { return grid_for_pairs(B, kChunk); }
int mlp_part_stride() { return kPartStride; }

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
                     float* loss, cudaStream_t s) {
  GradArgs a;
  a.theta = theta;
  a.x = x;
  a.y = y;
  a.B = B;
  a.inv_b = B > 0 ? (float)(1.0 / (double)B) : 0.f;
  a.partial = partial;
  const int parts = grid_for_pairs(B, kChunk);
  const size_t smem = sizeof(GradSmem);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  k_mlp_grad<<<parts, kWarps * 32, smem, s>>>(a);
  k_mlp_reduce<<<(kMlpParams + 1 + 255) / 256, 256, 0, s>>>(partial, parts, grad, loss);
}

void launch_mlp_adam(float* theta, const float* grad, float* m, float* v, int step, float lr, float b1, float b2,
                     float eps, cudaStream_t s) {
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(theta, grad, m, v, step, lr, b1, b2, eps);
}

}  // namespace fm
