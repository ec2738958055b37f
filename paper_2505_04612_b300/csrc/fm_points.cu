// Sparse reconstruction (Appendix "Sparse Reconstruction"): triangulate every
// keypoint pair of a completed track, average per track, reject keypoints by
// reprojection error, keep points with >= 3 inlier keypoints (distinct
// cameras) and a large enough triangulation angle.  Readings (the paper names
// no method or thresholds): two-ray midpoint (rays within ~0.057 deg of
// parallel give no point); an observation is an inlier if
// its reprojection error is <= max_err_px; the triangulation angle of a pair
// is the angle at the averaged point between the rays to the two camera
// centres, and the largest over pairs whose two keypoints are inliers must be
// >= min_angle.
//
// Track table (built once): keypoint pairs grouped by track id, in increasing
// pair index inside a track (per-track counts, a multi-CTA scan and a stable
// radix sort of the pair indices by track, so the order -- and every sum --
// is deterministic).  One thread per track.
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

__global__ void k_track_max(const int* __restrict__ track, int Z, int* out_max, int* err) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  int v = -1;
  if (m < Z) {
    v = track[m];
    if (v < 0) atomicOr(err, kErrKpRange);
  }
  for (int d = 16; d > 0; d >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, d));
  if ((threadIdx.x & 31) == 0) atomicMax(out_max, v);
}

__global__ void k_track_count(const int* __restrict__ track, int Z, int* __restrict__ cnt) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < Z) atomicAdd(cnt + track[m], 1);
}

struct Cam {
  float R[9], t[3], o[3];
};

__device__ __forceinline__ void load_cam(const float* params, int c, Cam& k) {
  Rot6 s;
  rot6_forward(params + 9 * c, s);
  rot6_matrix(s, k.R);
  for (int a = 0; a < 3; ++a) k.t[a] = params[9 * c + 6 + a];
  for (int a = 0; a < 3; ++a) k.o[a] = -(k.R[a] * k.t[0] + k.R[3 + a] * k.t[1] + k.R[6 + a] * k.t[2]);
}

// R^T x for homogeneous x = (u, v, 1)
__device__ __forceinline__ void ray(const Cam& k, float u, float v, float* d) {
  for (int a = 0; a < 3; ++a) d[a] = k.R[a] * u + k.R[3 + a] * v + k.R[6 + a];
}

// Midpoint of the shortest segment between rays o1 + s d1 and o2 + u d2.  The
// determinant of the normal equations, |d1|^2 |d2|^2 - (d1.d2)^2, is taken in
// the equal form |d1 x d2|^2 with rounded (uncontracted) products, so that
// parallel directions give exactly 0 (a fused a*c - b*b leaves the rounding
// error of b*b); rays closer than kParallelSin2 to parallel give no point.
constexpr float kParallelSin2 = 1e-6f;
__device__ __forceinline__ bool midpoint(const float* o1, const float* d1, const float* o2, const float* d2,
                                         float* X) {
  float w0[3];
  for (int a = 0; a < 3; ++a) w0[a] = o1[a] - o2[a];
  const float a = dot3(d1, d1), b = dot3(d1, d2), c = dot3(d2, d2);
  const float d = dot3(d1, w0), e = dot3(d2, w0);
  const float k0 = __fsub_rn(__fmul_rn(d1[1], d2[2]), __fmul_rn(d1[2], d2[1]));
  const float k1 = __fsub_rn(__fmul_rn(d1[2], d2[0]), __fmul_rn(d1[0], d2[2]));
  const float k2 = __fsub_rn(__fmul_rn(d1[0], d2[1]), __fmul_rn(d1[1], d2[0]));
  const float den = k0 * k0 + k1 * k1 + k2 * k2;
  if (!(den > kParallelSin2 * a * c)) return false;
  const float s = (b * e - c * d) / den, u = (a * e - b * d) / den;
  for (int k = 0; k < 3; ++k) X[k] = 0.5f * (o1[k] + s * d1[k] + o2[k] + u * d2[k]);
  return true;
}

// reprojection error in pixels (infinite behind the camera)
__device__ __forceinline__ float reproj(const Cam& k, const float* X, float u, float v, float f) {
  const float xc = k.R[0] * X[0] + k.R[1] * X[1] + k.R[2] * X[2] + k.t[0];
  const float yc = k.R[3] * X[0] + k.R[4] * X[1] + k.R[5] * X[2] + k.t[1];
  const float zc = k.R[6] * X[0] + k.R[7] * X[1] + k.R[8] * X[2] + k.t[2];
  if (!(zc > 0.f)) return 3.4e38f;
  const float du = xc / zc - u, dv = yc / zc - v;
  return f * sqrtf(du * du + dv * dv);
}

constexpr int kMaxCams = 64;   // distinct inlier cameras tracked per point

__global__ void k_triangulate(const float4* __restrict__ kp, const int* __restrict__ kp_seg,
                              const int* __restrict__ pi, const int* __restrict__ pj,
                              const float* __restrict__ focal, const float* __restrict__ params,
                              const int* __restrict__ off, const int* __restrict__ idx, int T,
                              float max_err_px, float min_cos, float* __restrict__ pts,
                              int* __restrict__ valid, int* __restrict__ ncam_out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int b = off[t], e = off[t + 1];
  float S[3] = {0.f, 0.f, 0.f};
  int cnt = 0;
  for (int q = b; q < e; ++q) {
    const int m = idx[q];
    const int n = kp_seg[m];
    Cam ci, cj;
    load_cam(params, pi[n], ci);
    load_cam(params, pj[n], cj);
    const float4 x = kp[m];
    float d1[3], d2[3], X[3];
    ray(ci, x.x, x.y, d1);
    ray(cj, x.z, x.w, d2);
    if (midpoint(ci.o, d1, cj.o, d2, X)) {
      for (int a = 0; a < 3; ++a) S[a] += X[a];
      ++cnt;
    }
  }
  float P[3];
  const float inv = cnt > 0 ? 1.f / (float)cnt : 0.f;
  for (int a = 0; a < 3; ++a) P[a] = S[a] * inv;
  int cams[kMaxCams];
  int nc = 0;
  float max_cos = 2.f;   // the smallest cosine = the largest angle
  for (int q = b; q < e; ++q) {
    const int m = idx[q];
    const int n = kp_seg[m];
    const int i = pi[n], j = pj[n];
    Cam ci, cj;
    load_cam(params, i, ci);
    load_cam(params, j, cj);
    const float4 x = kp[m];
    const bool in1 = reproj(ci, P, x.x, x.y, focal[i]) <= max_err_px;
    const bool in2 = reproj(cj, P, x.z, x.w, focal[j]) <= max_err_px;
    for (int side = 0; side < 2; ++side) {
      if (!(side == 0 ? in1 : in2)) continue;
      const int c = side == 0 ? i : j;
      bool seen = false;
      for (int k = 0; k < nc; ++k) seen |= (cams[k] == c);
      if (!seen && nc < kMaxCams) cams[nc++] = c;
    }
    if (in1 && in2) {
      float r1[3], r2[3];
      for (int a = 0; a < 3; ++a) {
        r1[a] = ci.o[a] - P[a];
        r2[a] = cj.o[a] - P[a];
      }
      const float den = sqrtf(dot3(r1, r1) * dot3(r2, r2));
      const float cs = den > 0.f ? dot3(r1, r2) / den : 1.f;
      max_cos = fminf(max_cos, cs);
    }
  }
  for (int a = 0; a < 3; ++a) pts[3 * t + a] = P[a];
  ncam_out[t] = nc;
  valid[t] = (cnt > 0 && nc >= 3 && max_cos <= min_cos) ? 1 : 0;
}

}  // namespace

// Builds the track table; returns the number of tracks in *T_out (host).
cudaError_t build_track_table(fm_problem* pr, int* T_out) {
  cudaStream_t s = pr->stream;
  const int Z = (int)pr->Z;
  int* d_max = nullptr;
  cudaError_t e = cudaMalloc((void**)&d_max, 2 * sizeof(int));
  if (e != cudaSuccess) return e;
  int init = -1;
  cudaMemcpyAsync(d_max, &init, sizeof(int), cudaMemcpyHostToDevice, s);
  if (Z > 0) k_track_max<<<(Z + 255) / 256, 256, 0, s>>>(pr->kp_track, Z, d_max, pr->d_err);
  int mx = -1, bits = 0;
  cudaMemcpyAsync(&mx, d_max, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&bits, pr->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { cudaFree(d_max); return e; }
  if (bits & kErrKpRange) {   // a negative track id: reported by the caller, nothing indexed with it
    cudaFree(d_max);
    *T_out = 0;
    return cudaSuccess;
  }
  const int T = mx + 1;
  *T_out = T;
  pr->n_tracks = T;
  e = cudaMalloc((void**)&pr->track_off, sizeof(int) * (size_t)(T + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&pr->track_idx, sizeof(int) * (size_t)(Z > 0 ? Z : 1));
  if (e != cudaSuccess) { cudaFree(d_max); return e; }
  pr->device_bytes += (int64_t)sizeof(int) * (T + 1 + (Z > 0 ? Z : 1));
  cudaMemsetAsync(pr->track_off, 0, sizeof(int) * (size_t)(T + 1), s);
  if (Z > 0 && T > 0) {
    k_track_count<<<(Z + 255) / 256, 256, 0, s>>>(pr->kp_track, Z, pr->track_off);   // integer counts
    e = track_table(pr->kp_track, Z, T, pr->track_off, pr->track_idx, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_max);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

void launch_triangulate(const fm_problem* pr, const float* params, float max_err_px, float min_angle_rad,
                        float* pts, int* valid, int* ncam, cudaStream_t s) {
  const int T = pr->n_tracks;
  if (T <= 0) return;
  k_triangulate<<<(T + 127) / 128, 128, 0, s>>>(pr->kp, pr->kp_seg, pr->pair_i, pr->pair_j, pr->focal, params,
                                                pr->track_off, pr->track_idx, T, max_err_px,
                                                cosf(min_angle_rad), pts, valid, ncam);
}

}  // namespace fm
