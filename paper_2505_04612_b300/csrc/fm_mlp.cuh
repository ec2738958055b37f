// The features of a keypoint pair for the learned inlier network, shared by
// the feature-only kernel and the tcgen05 network kernel.  Definitions (readings) are those of
// the learned-weights section of include/fastmap.h: the epipolar residual
// over the image pair's mean residual, the log of the residual over its
// Sampson scale, the log of the track length, the angle between the two
// viewing rays, the mean distance of the keypoints from the principal point,
// the solve's progress, the log of the image pair's keypoint count and the
// current weight on a log scale.
#pragma once

#include "fm_device.cuh"

namespace fm {

constexpr int kMlpTab = 32;   // floats per image-pair row of the feature tables

struct InferArgs {
  const float4* kp;
  const int* kp_seg;
  const float* tab;
  const int* kp_track;     // or null
  const int* track_off;    // or null
  const float* w;          // current per-pair weights, or null (1)
  float iter_frac;
  float inv_log_delta;     // 1 / log1p(1/delta)
  const float* theta;      // or null: features only
  const float* x;          // feature rows [Z][8] in place of pair features, or null
  int64_t Z;
  float* prob;             // [Z] or null
  float* logit;            // [Z] or null
  float* feat;             // [Z][8] or null
  float* resid;            // [Z] or null
};

__device__ __forceinline__ void pair_features(const InferArgs& a, int64_t m, float* f, float& r) {
  const int n = a.kp_seg[m];
  const float* T = a.tab + (size_t)kMlpTab * n;
  const float4 x = __ldg(a.kp + m);
  const float a0 = fmaf(T[0], x.x, fmaf(T[1], x.y, T[2]));
  const float a1 = fmaf(T[3], x.x, fmaf(T[4], x.y, T[5]));
  const float a2 = fmaf(T[6], x.x, fmaf(T[7], x.y, T[8]));
  r = fmaf(x.z, a0, fmaf(x.w, a1, a2));
  const float b0 = fmaf(T[0], x.z, fmaf(T[3], x.w, T[6]));
  const float b1 = fmaf(T[1], x.z, fmaf(T[4], x.w, T[7]));
  const float ar = fabsf(r);
  f[0] = ar / (T[27] + 1e-12f);
  f[1] = log1pf(T[29] * ar / sqrtf(a0 * a0 + a1 * a1 + b0 * b0 + b1 * b1));
  f[2] = 0.f;
  if (a.kp_track) {
    const int tr = a.kp_track[m];
    const float c = (float)(a.track_off[tr + 1] - a.track_off[tr]);
    f[2] = logf(0.5f * (1.f + sqrtf(1.f + 8.f * c)));
  }
  // viewing rays R^T x~ of both keypoints; their angle via atan2 (accurate
  // for small angles)
  const float* Ri = T + 9;
  const float* Rj = T + 18;
  float d1[3], d2[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d1[k] = fmaf(Ri[k], x.x, fmaf(Ri[3 + k], x.y, Ri[6 + k]));
    d2[k] = fmaf(Rj[k], x.z, fmaf(Rj[3 + k], x.w, Rj[6 + k]));
  }
  float cr[3];
  cross3(d1, d2, cr);
  f[3] = atan2f(sqrtf(dot3(cr, cr)), dot3(d1, d2));
  f[4] = 0.5f * (sqrtf(x.x * x.x + x.y * x.y) + sqrtf(x.z * x.z + x.w * x.w));
  f[5] = a.iter_frac;
  f[6] = T[28];
  f[7] = log1pf(a.w ? a.w[m] : 1.f) * a.inv_log_delta;
}

}  // namespace fm
