// Distortion interval search (Sec. 3.1 "Distortion Estimation", Eq. 1;
// Appendix "Distortion Estimation") and undistortion of the stored keypoints.
//
// Division model about the image centre: x_u = x_d / (1 + alpha r_d^2), x_d
// in half-diagonal units.  The stored keypoints are calibrated at f0
// (x_c = (pixel - centre) / f0), so x_d = s x_c with s = f0 / h per image.
//
// k_dist_errors: one warp per listed image pair, one lane per candidate
// alpha (up to 32 per launch).
//   * a provisional frame per image, the Hartley map of the observed points
//     (centroid to the origin, RMS distance sqrt(2)), the same for all
//     candidates: the lanes split the keypoint pairs (coalesced loads);
//   * pass 1, every lane reading the same keypoint pair (one broadcast request
//     per warp): the lane's moment matrix W0 = sum a a^T of its undistorted
//     points in the provisional frame (a = y0_2 (x) y0_1, packed upper
//     triangle in registers);
//   * the exact Hartley frame of the undistorted points (y = A y0) is read off
//     W0 (count, sums and sums of squares are entries of it), and a
//     per-thread Cholesky factorisation of W0 with inverse iteration on
//     W = K W0 K^T (K = A2 (x) A1, applied as x <- K^-T W0^-1 K^-1 x) gives
//     the smallest eigenvector F^, projected to rank 2 at unit Frobenius norm;
//   * pass 2: the epipolar errors |y_2^T F^ y_1| in the exact frame
//     (scale-free: a candidate that shrinks the points does not shrink the
//     error).  One read of the keypoints
// serves all candidates, so the kernel is bound by FP32 issue, not by HBM.
// A listed pair may fix one side's alpha (its camera is already estimated).
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

constexpr int kDistWarps = 4;
constexpr int kBigWarps = 8;          // warps per image pair of more than kDistSplit keypoint pairs
constexpr int kInvIters = 40;         // inverse-iteration steps at most
constexpr float kInvTol = 2e-7f;      // max-norm change of the unit vector that ends them
constexpr float kPivotFloor = 1e-9f;  // Cholesky pivots floored at this fraction of their diagonal

__host__ __device__ constexpr int sym9(int i, int j) {
  return i <= j ? i * 9 - (i * (i - 1)) / 2 + (j - i) : j * 9 - (j * (j - 1)) / 2 + (i - j);
}

// y = B y' for the homogeneous points of one image, B = [[s, 0, cx], [0, s,
// cy], [0, 0, 1]] (the inverse of a Hartley map y' = k (y - c): s = 1/k)
struct Inv {
  float s, cx, cy;
};

// x <- (B2 (x) B1) x and x <- (B2 (x) B1)^T x for a 9-vector x = vec(X),
// X[p][q] = x[3p + q] (p: image 2, q: image 1): B2 X B1^T and B2^T X B1
__device__ __forceinline__ void kron_apply(const Inv& b2, const Inv& b1, float (&x)[9]) {
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const float x2 = x[3 * p + 2];
    x[3 * p] = fmaf(b1.s, x[3 * p], b1.cx * x2);
    x[3 * p + 1] = fmaf(b1.s, x[3 * p + 1], b1.cy * x2);
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float y2 = x[6 + q];
    x[q] = fmaf(b2.s, x[q], b2.cx * y2);
    x[3 + q] = fmaf(b2.s, x[3 + q], b2.cy * y2);
  }
}
__device__ __forceinline__ void kron_apply_t(const Inv& b2, const Inv& b1, float (&x)[9]) {
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const float x0 = x[3 * p], x1 = x[3 * p + 1];
    x[3 * p + 2] = fmaf(b1.cx, x0, fmaf(b1.cy, x1, x[3 * p + 2]));
    x[3 * p] = b1.s * x0;
    x[3 * p + 1] = b1.s * x1;
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float y0 = x[q], y1 = x[3 + q];
    x[6 + q] = fmaf(b2.cx, y0, fmaf(b2.cy, y1, x[6 + q]));
    x[q] = b2.s * y0;
    x[3 + q] = b2.s * y1;
  }
}

// Eigenvector of the smallest eigenvalue of W = K W0 K^T, K^-1 = B2 (x) B1,
// for a symmetric positive semi-definite 9 x 9 W0 held by one thread (packed
// upper triangle, overwritten): Cholesky factor W0 = U^T U (pivots floored at
// kPivotFloor of their diagonal, so that a singular W0 still factors), then
// inverse iteration x <- W^-1 x = K^-T W0^-1 K^-1 x from x = (1, ..., 1)/3
// until no component moves by more than kInvTol or kInvIters steps
// (warp-uniform loop).  Converges as (lambda1 / lambda2)^k; where the two
// smallest eigenvalues nearly coincide the eigenvector is not determined at
// float32 precision anyway.  Every index is a compile-time constant after
// unrolling, so W0 stays in registers.
__device__ __forceinline__ void smallest_eigenvector(float (&W)[45], const Inv& b2, const Inv& b1, float (&x)[9]) {
  float id[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float wii = W[sym9(i, i)];
    float d = wii;
#pragma unroll
    for (int k = 0; k < i; ++k) d = fmaf(-W[sym9(k, i)], W[sym9(k, i)], d);
    d = fmaxf(d, fmaxf(kPivotFloor * wii, 1e-30f));
    const float r = rsqrtf(d);
    id[i] = r;
    W[sym9(i, i)] = d * r;
#pragma unroll
    for (int j = i + 1; j < 9; ++j) {
      float v = W[sym9(i, j)];
#pragma unroll
      for (int k = 0; k < i; ++k) v = fmaf(-W[sym9(k, i)], W[sym9(k, j)], v);
      W[sym9(i, j)] = v * r;
    }
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) x[i] = 1.f / 3.f;
  bool active = true;
#pragma unroll 1
  for (int it = 0; it < kInvIters; ++it) {
    if (active) {
      float z[9], y[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) y[i] = x[i];
      kron_apply(b2, b1, y);
      float mz = 0.f;
#pragma unroll
      for (int i = 0; i < 9; ++i) {   // U^T z = K^-1 x
        float v = y[i];
#pragma unroll
        for (int k = 0; k < i; ++k) v = fmaf(-W[sym9(k, i)], z[k], v);
        z[i] = v * id[i];
        mz = fmaxf(mz, fabsf(z[i]));
      }
      const float sz = 1.f / mz;      // rescaled so that no solve overflows
#pragma unroll
      for (int i = 8; i >= 0; --i) {  // U v = z
        float v = z[i] * sz;
#pragma unroll
        for (int j = i + 1; j < 9; ++j) v = fmaf(-W[sym9(i, j)], y[j], v);
        y[i] = v * id[i];
      }
      kron_apply_t(b2, b1, y);        // K^-T v
      float my = 0.f;
#pragma unroll
      for (int i = 0; i < 9; ++i) my = fmaxf(my, fabsf(y[i]));
      const float sy = 1.f / my;
      float nrm = 0.f, dot = 0.f;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        y[i] *= sy;
        nrm = fmaf(y[i], y[i], nrm);
        dot = fmaf(y[i], x[i], dot);
      }
      const float sn = copysignf(rsqrtf(nrm), dot);
      float delta = 0.f;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const float v = y[i] * sn;
        delta = fmaxf(delta, fabsf(v - x[i]));
        x[i] = v;
      }
      active = delta > kInvTol;
    }
    if (!__any_sync(0xffffffffu, active)) break;
  }
}

// x_u of a calibrated point (x, y) with image scale s and distortion alpha
// (the reciprocal by the fast intrinsic: ~2 ulp)
__device__ __forceinline__ float2 undistorted(float x, float y, float s, float alpha) {
  const float xd = x * s, yd = y * s;
  const float g = __fdividef(1.f, fmaf(alpha, fmaf(xd, xd, yd * yd), 1.f));
  return make_float2(xd * g, yd * g);
}

__device__ __forceinline__ void accumulate(float (&W)[45], float2 u1, float2 u2) {
  const float a[9] = {u2.x * u1.x, u2.x * u1.y, u2.x, u2.y * u1.x, u2.y * u1.y, u2.y, u1.x, u1.y, 1.f};
#pragma unroll
  for (int p = 0; p < 9; ++p)
#pragma unroll
    for (int q = p; q < 9; ++q) W[sym9(p, q)] = fmaf(a[p], a[q], W[sym9(p, q)]);
}

struct DistArgs {
  const float4* kp;
  const int* seg_off;
  const int* pi;
  const int* pj;
  const float* scale;   // [N] f0 / h
  const int* idx;       // [M] image pair of each work item, or null: item q is pair q
  const int* row;       // [M] output row of each work item, or null: row q
  const float* fix_i;   // [rows] alpha of image i when known (NaN: the candidate), or null
  const float* fix_j;
  const float* cand;    // [K]
  int M, K;
  float* err;           // [rows*K] sum of |y_2^T F^ y_1| per (row, candidate)
};

// one image pair seen by one lane (candidate)
struct PairCtx {
  int b, e;
  float ai, aj, si, sj;
};

struct Norm {   // y = k (x_u - c) per image
  float c1x, c1y, k1, c2x, c2y, k2;
};

__device__ __forceinline__ PairCtx pair_ctx(const DistArgs& a, int n, int r, int lane) {
  PairCtx p;
  p.b = a.seg_off[n];
  p.e = a.seg_off[n + 1];
  const float alpha = a.cand[min(lane, a.K - 1)];
  p.ai = alpha;
  p.aj = alpha;
  if (a.fix_i && !isnan(a.fix_i[r])) p.ai = a.fix_i[r];
  if (a.fix_j && !isnan(a.fix_j[r])) p.aj = a.fix_j[r];
  p.si = a.scale[a.pi[n]];
  p.sj = a.scale[a.pj[n]];
  return p;
}

// f(x) for keypoint pairs [lo, hi), loads issued four at a time
template <typename Fn>
__device__ __forceinline__ void for_range(const float4* __restrict__ kp, int lo, int hi, Fn&& f) {
  int m = lo;
  for (; m + 4 <= hi; m += 4) {
    float4 x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = __ldg(kp + m + u);
#pragma unroll
    for (int u = 0; u < 4; ++u) f(x[u]);
  }
  for (; m < hi; ++m) f(__ldg(kp + m));
}

// sums of x, y and x^2 + y^2 of the observed points x_d of each image over
// keypoint pairs lo + lane, lo + lane + 32, ... < hi (the lanes split them:
// coalesced loads), reduced over the warp by a fixed xor tree
__device__ __forceinline__ void observed_sums(const float4* kp, const PairCtx& p, int lo, int hi, int lane,
                                              float (&st)[6]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) st[k] = 0.f;
  for (int m = lo + lane; m < hi; m += 32) {
    const float4 x = __ldg(kp + m);
    const float a = x.x * p.si, b = x.y * p.si, c = x.z * p.sj, d = x.w * p.sj;
    st[0] += a;
    st[1] += b;
    st[2] = fmaf(a, a, fmaf(b, b, st[2]));
    st[3] += c;
    st[4] += d;
    st[5] = fmaf(c, c, fmaf(d, d, st[5]));
  }
#pragma unroll
  for (int k = 0; k < 6; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) st[k] += __shfl_xor_sync(0xffffffffu, st[k], o);
}

// Hartley normalisation from the sums over the pair's m keypoint pairs:
// centroid to the origin, RMS distance sqrt(2)
__device__ __forceinline__ Norm norm_from(const float (&st)[6], int m) {
  Norm z;
  const float inv_m = 1.f / (float)m;
  z.c1x = st[0] * inv_m;
  z.c1y = st[1] * inv_m;
  z.c2x = st[3] * inv_m;
  z.c2y = st[4] * inv_m;
  const float v1 = fmaf(st[2], inv_m, -fmaf(z.c1x, z.c1x, z.c1y * z.c1y));
  const float v2 = fmaf(st[5], inv_m, -fmaf(z.c2x, z.c2x, z.c2y * z.c2y));
  z.k1 = 1.41421356f * rsqrtf(fmaxf(v1, 1e-30f));
  z.k2 = 1.41421356f * rsqrtf(fmaxf(v2, 1e-30f));
  return z;
}

// The exact Hartley normalisation of the points y0 (provisional frame) read
// off their moments: W0[8][8] = m, W0[6][8], W0[7][8] = sums of image 1's
// coordinates, W0[6][6] + W0[7][7] = sum of their squares, W0[2][8],
// W0[5][8], W0[2][2] + W0[5][5] the same for image 2
__device__ __forceinline__ Norm exact_frame(const float (&W)[45]) {
  const float st[6] = {W[sym9(6, 8)], W[sym9(7, 8)], W[sym9(6, 6)] + W[sym9(7, 7)],
                       W[sym9(2, 8)], W[sym9(5, 8)], W[sym9(2, 2)] + W[sym9(5, 5)]};
  return norm_from(st, (int)W[sym9(8, 8)]);
}

// y = k1 (k0 (x_u - c0) - c1) = (k1 k0) (x_u - (c0 + c1 / k0)) per image
__device__ __forceinline__ Norm compose(const Norm& z0, const Norm& z1) {
  Norm z;
  z.k1 = z1.k1 * z0.k1;
  z.c1x = z0.c1x + z1.c1x / z0.k1;
  z.c1y = z0.c1y + z1.c1y / z0.k1;
  z.k2 = z1.k2 * z0.k2;
  z.c2x = z0.c2x + z1.c2x / z0.k2;
  z.c2y = z0.c2y + z1.c2y / z0.k2;
  return z;
}

// pass 1: moments of the provisionally normalised points
__device__ __forceinline__ void moments_range(const float4* kp, const PairCtx& p, const Norm& z, int lo, int hi,
                                              float (&W)[45]) {
#pragma unroll
  for (int k = 0; k < 45; ++k) W[k] = 0.f;
  const float o1x = -z.c1x * z.k1, o1y = -z.c1y * z.k1, o2x = -z.c2x * z.k2, o2y = -z.c2y * z.k2;
  for_range(kp, lo, hi, [&](const float4& x) {
    const float2 u1 = undistorted(x.x, x.y, p.si, p.ai), u2 = undistorted(x.z, x.w, p.sj, p.aj);
    accumulate(W, make_float2(fmaf(u1.x, z.k1, o1x), fmaf(u1.y, z.k1, o1y)),
               make_float2(fmaf(u2.x, z.k2, o2x), fmaf(u2.y, z.k2, o2y)));
  });
}

// F^ from the moments W0 of the provisionally normalised points (the exact
// frame is y = B^-1 y0 per image): smallest eigenvector, rank 2 (F <- F - (F u) u^T with
// u the right singular vector of the smallest singular value, the
// eigenvector of F^T F), unit Frobenius norm
__device__ __forceinline__ void fundamental(float (&W)[45], const Inv& b2, const Inv& b1, float (&F)[9]) {
  smallest_eigenvector(W, b2, b1, F);
  float S[9], Q[9];
#pragma unroll
  for (int c0 = 0; c0 < 3; ++c0)
#pragma unroll
    for (int c1 = 0; c1 < 3; ++c1)
      S[c0 * 3 + c1] = F[c0] * F[c1] + F[3 + c0] * F[3 + c1] + F[6 + c0] * F[6 + c1];
  jacobi3(S, Q);
  float u0 = Q[0], u1 = Q[3], u2 = Q[6], lo = S[0];
  if (S[4] < lo) {
    lo = S[4];
    u0 = Q[1];
    u1 = Q[4];
    u2 = Q[7];
  }
  if (S[8] < lo) {
    u0 = Q[2];
    u1 = Q[5];
    u2 = Q[8];
  }
  float nrm = 0.f;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float fu = F[3 * r] * u0 + F[3 * r + 1] * u1 + F[3 * r + 2] * u2;
    F[3 * r] -= fu * u0;
    F[3 * r + 1] -= fu * u1;
    F[3 * r + 2] -= fu * u2;
    nrm = fmaf(F[3 * r], F[3 * r], fmaf(F[3 * r + 1], F[3 * r + 1], fmaf(F[3 * r + 2], F[3 * r + 2], nrm)));
  }
  const float inv = rsqrtf(nrm);
#pragma unroll
  for (int k = 0; k < 9; ++k) F[k] *= inv;
}

// pass 2: sum of |y_2^T F^ y_1| in the normalised frame
__device__ __forceinline__ float error_range(const float4* kp, const PairCtx& p, const Norm& z, const float (&F)[9],
                                             int lo, int hi) {
  float sum = 0.f;
  const float o1x = -z.c1x * z.k1, o1y = -z.c1y * z.k1, o2x = -z.c2x * z.k2, o2y = -z.c2y * z.k2;
  for_range(kp, lo, hi, [&](const float4& x) {
    const float2 u1 = undistorted(x.x, x.y, p.si, p.ai), u2 = undistorted(x.z, x.w, p.sj, p.aj);
    const float y1x = fmaf(u1.x, z.k1, o1x), y1y = fmaf(u1.y, z.k1, o1y);
    const float y2x = fmaf(u2.x, z.k2, o2x), y2y = fmaf(u2.y, z.k2, o2y);
    const float l0 = fmaf(F[0], y1x, fmaf(F[1], y1y, F[2]));
    const float l1 = fmaf(F[3], y1x, fmaf(F[4], y1y, F[5]));
    const float l2 = fmaf(F[6], y1x, fmaf(F[7], y1y, F[8]));
    sum += fabsf(fmaf(y2x, l0, fmaf(y2y, l1, l2)));
  });
  return sum;
}

// One warp per work item (image pairs of up to kDistSplit keypoint pairs).
__global__ void __launch_bounds__(kDistWarps * 32) k_dist_errors(DistArgs a) {
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * kDistWarps + (threadIdx.x >> 5);
  if (q >= a.M) return;   // warp-uniform
  const int n = a.idx ? a.idx[q] : q;
  const int r = a.row ? a.row[q] : q;
  const PairCtx p = pair_ctx(a, n, r, lane);
  const int m = p.e - p.b;
  if (m < 8) {
    if (lane < a.K) a.err[(size_t)r * a.K + lane] = 0.f;
    return;
  }
  float st[6];
  observed_sums(a.kp, p, p.b, p.e, lane, st);
  const Norm z0 = norm_from(st, m);   // provisional frame: the observed points' Hartley map
  float W[45];
  moments_range(a.kp, p, z0, p.b, p.e, W);
  const Norm z1 = exact_frame(W);
  float F[9];
  fundamental(W, Inv{1.f / z1.k2, z1.c2x, z1.c2y}, Inv{1.f / z1.k1, z1.c1x, z1.c1y}, F);
  const float sum = error_range(a.kp, p, compose(z0, z1), F, p.b, p.e);
  if (lane < a.K) a.err[(size_t)r * a.K + lane] = sum;
}

// One CTA of kBigWarps warps per work item (image pairs of more than
// kDistSplit keypoint pairs): warp w takes the w-th of kBigWarps contiguous
// slices of the pair's keypoint pairs in every pass; the slices' sums meet
// in shared memory in a fixed order; warp 0 solves for F^ and hands F^ and
// the exact frame of every lane (candidate) to the other warps.
__global__ void __launch_bounds__(kBigWarps * 32) k_dist_errors_big(DistArgs a) {
  __shared__ float red[kBigWarps * 45 * 32];   // per-warp moments (first: the observed sums)
  __shared__ float Fs[9 * 32];
  __shared__ float Zs[6 * 32];                 // exact frame (c1x, c1y, k1, c2x, c2y, k2) per lane
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int q = blockIdx.x;
  const int n = a.idx ? a.idx[q] : q;
  const int r = a.row ? a.row[q] : q;
  const PairCtx p = pair_ctx(a, n, r, lane);
  const int m = p.e - p.b;
  const int L = (m + kBigWarps - 1) / kBigWarps;
  const int lo = min(p.b + wid * L, p.e), hi = min(lo + L, p.e);

  float st[6];
  observed_sums(a.kp, p, lo, hi, lane, st);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) red[wid * 6 + k] = st[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float t = 0.f;
    for (int w = 0; w < kBigWarps; ++w) t += red[w * 6 + k];
    st[k] = t;
  }
  const Norm z0 = norm_from(st, m);   // provisional frame, the same for every lane
  __syncthreads();   // the sums are read before the moments overwrite them

  float W[45];
  moments_range(a.kp, p, z0, lo, hi, W);
#pragma unroll
  for (int k = 0; k < 45; ++k) red[(wid * 45 + k) * 32 + lane] = W[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < 45; ++k) {
      float t = 0.f;
      for (int w = 0; w < kBigWarps; ++w) t += red[(w * 45 + k) * 32 + lane];
      W[k] = t;
    }
    const Norm z1 = exact_frame(W);
    float F[9];
    fundamental(W, Inv{1.f / z1.k2, z1.c2x, z1.c2y}, Inv{1.f / z1.k1, z1.c1x, z1.c1y}, F);
#pragma unroll
    for (int k = 0; k < 9; ++k) Fs[k * 32 + lane] = F[k];
    Zs[0 * 32 + lane] = z1.c1x;
    Zs[1 * 32 + lane] = z1.c1y;
    Zs[2 * 32 + lane] = z1.k1;
    Zs[3 * 32 + lane] = z1.c2x;
    Zs[4 * 32 + lane] = z1.c2y;
    Zs[5 * 32 + lane] = z1.k2;
  }
  __syncthreads();
  float F[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) F[k] = Fs[k * 32 + lane];
  Norm z1;
  z1.c1x = Zs[0 * 32 + lane];
  z1.c1y = Zs[1 * 32 + lane];
  z1.k1 = Zs[2 * 32 + lane];
  z1.c2x = Zs[3 * 32 + lane];
  z1.c2y = Zs[4 * 32 + lane];
  z1.k2 = Zs[5 * 32 + lane];
  const float sum = error_range(a.kp, p, compose(z0, z1), F, lo, hi);
  red[wid * 32 + lane] = sum;   // the moments were consumed before the last barrier
  __syncthreads();
  if (wid == 0) {
    float t = 0.f;
    for (int w = 0; w < kBigWarps; ++w) t += red[w * 32 + lane];
    if (lane < a.K) a.err[(size_t)r * a.K + lane] = t;
  }
}

// out[k] = sum over the listed pairs of err[q*K + k], in a fixed order
__global__ void __launch_bounds__(256) k_dist_reduce(const float* __restrict__ err, int M, int K,
                                                      float* __restrict__ out) {
  __shared__ float part[256];
  const int k = blockIdx.x;
  float s = 0.f;
  for (int q = threadIdx.x; q < M; q += 256) s += err[(size_t)q * K + k];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) part[threadIdx.x] += part[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] = part[0];
}

// x_c <- x_c / (1 + alpha (s |x_c|)^2) for both images of every keypoint pair;
// a denominator <= 0 (the model has no undistorted point) leaves the point
// and sets *bad
__global__ void k_undistort(float4* __restrict__ kp, const int* __restrict__ kp_seg, const int* __restrict__ pi,
                            const int* __restrict__ pj, const float* __restrict__ scale,
                            const float* __restrict__ alpha, int64_t Z, int* __restrict__ bad) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < Z; m += (int64_t)gridDim.x * blockDim.x) {
    const int n = kp_seg[m];
    const int i = pi[n], j = pj[n];
    float4 x = kp[m];
    const float si = scale[i], sj = scale[j];
    const float di = fmaf(alpha[i] * si * si, fmaf(x.x, x.x, x.y * x.y), 1.f);
    const float dj = fmaf(alpha[j] * sj * sj, fmaf(x.z, x.z, x.w * x.w), 1.f);
    if (!(di > 0.f) || !(dj > 0.f)) {
      atomicOr(bad, 1);
      continue;
    }
    x.x /= di;
    x.y /= di;
    x.z /= dj;
    x.w /= dj;
    kp[m] = x;
  }
}

}  // namespace

void launch_dist_errors(const fm_problem* pr, const float* scale, const int* idx, const int* row,
                        const float* fix_i, const float* fix_j, int M, bool big, const float* cand, int K,
                        float* err, cudaStream_t s) {
  if (M == 0) return;
  DistArgs a{pr->kp, pr->seg_off, pr->pair_i, pr->pair_j, scale, idx, row, fix_i, fix_j, cand, M, K, err};
  if (big)
    k_dist_errors_big<<<M, kBigWarps * 32, 0, s>>>(a);
  else
    k_dist_errors<<<(M + kDistWarps - 1) / kDistWarps, kDistWarps * 32, 0, s>>>(a);
}

void launch_dist_reduce(const float* err, int M, int K, float* out, cudaStream_t s) {
  if (K == 0) return;
  k_dist_reduce<<<K, 256, 0, s>>>(err, M, K, out);
}

void launch_undistort(const fm_problem* pr, const float* scale, const float* alpha, int* bad, cudaStream_t s) {
  if (pr->Z == 0) return;
  int64_t g = (pr->Z + 255) / 256;
  if (g > 148 * 32) g = 148 * 32;
  k_undistort<<<(unsigned)g, 256, 0, s>>>(pr->kp, pr->kp_seg, pr->pair_i, pr->pair_j, scale, alpha, pr->Z, bad);
}

}  // namespace fm
