// Focal lengths inside epipolar adjustment (Sec. 3.3, last paragraph of
// "Epipolar Adjustment"): camera c carries a log focal ratio phi_c
// (f_c = f0_c e^phi_c, keypoints calibrated once at f0); recalibrating scales
// the first two calibrated coordinates by s_c = e^-phi_c, so the objective is
// the direct one at E'_n = S_j E_n S_i, S = diag(s, s, 1).
//
//   k_ea_tables     (fm_ea.cu) writes E'_n into the image-pair tables when
//                   given phi, so the direct kernel runs unchanged and its
//                   per-pair sums are dL/dE';
//   k_focal_dlde    E_n from the poses, G' = dL/dE'_n -> dL/dE_n = S_j G' S_i (for the pose
//                   chain rule) and the pair's focal terms
//                   dL/dphi_i = -s_i <G', S_j E D>, dL/dphi_j = -s_j <G', D E S_i>
//                   with D = diag(1, 1, 0);
//   k_focal_cam     per camera (one warp), the focal terms of its image pairs
//                   in a fixed order (deterministic).
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

__device__ __forceinline__ float row_scale(int a, float s) { return a < 2 ? s : 1.f; }

__global__ void k_focal_dlde(const float* __restrict__ params, const float* __restrict__ Gp,
                             const int* __restrict__ pi, const int* __restrict__ pj, const float* __restrict__ phi,
                             const float* __restrict__ grad_loss, const int* __restrict__ pair_scene, int P,
                             float* __restrict__ G_out, float* __restrict__ dphi) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= P) return;
  const int ci = pi[n], cj = pj[n];
  const float si = __expf(-phi[ci]), sj = __expf(-phi[cj]);
  float qi[9], qj[9];
  load_plain(params + 9 * ci, qi, 9);
  load_plain(params + 9 * cj, qj, 9);
  PairGeo g;
  pair_geometry(qi, qj, g);
  float E[9];
  essential(g, E);
  const float gl = grad_loss ? grad_loss[pair_scene ? pair_scene[n] : 0] : 1.f;
  float di = 0.f, dj = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float g = Gp[9 * (size_t)n + 3 * a + b];
      const float ra = row_scale(a, sj), cb = row_scale(b, si);
      G_out[9 * (size_t)n + 3 * a + b] = g * ra * cb;
      if (b < 2) di = fmaf(g * ra, E[3 * a + b], di);   // <G', S_j E D>
      if (a < 2) dj = fmaf(g * cb, E[3 * a + b], dj);   // <G', D E S_i>
    }
  dphi[2 * n] = -si * di * gl;
  dphi[2 * n + 1] = -sj * dj * gl;
}

// one warp per camera: lane l takes the camera's incident pairs l, l + 32,
// ... in order, then a fixed xor tree (deterministic)
__global__ void k_focal_cam(const int* __restrict__ cam_seg_off, const int* __restrict__ cam_seg,
                            const float* __restrict__ dphi, int N, float* __restrict__ gphi) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= N) return;   // warp-uniform
  float s = 0.f;
  for (int k = cam_seg_off[c] + lane; k < cam_seg_off[c + 1]; k += 32) {
    const unsigned e = (unsigned)cam_seg[k];
    const int n = (int)(e & 0x7fffffffu), role = (int)(e >> 31);   // role 1: camera is j
    s += dphi[2 * n + role];
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if (lane == 0) gphi[c] = s;
}

}  // namespace

void launch_focal_dlde(const fm_problem* pr, const float* params, const float* Gp, const float* phi,
                       const float* grad_loss, float* G_out, float* dphi, cudaStream_t s) {
  if (pr->P == 0) return;
  k_focal_dlde<<<(pr->P + 127) / 128, 128, 0, s>>>(params, Gp, pr->pair_i, pr->pair_j, phi, grad_loss,
                                                    pr->pair_scene, pr->P, G_out, dphi);
}

void launch_focal_cam(const fm_problem* pr, const float* dphi, float* gphi, cudaStream_t s) {
  k_focal_cam<<<(pr->N + 3) / 4, 128, 0, s>>>(pr->cam_seg_off, pr->cam_seg, dphi, pr->N, gphi);
}

}  // namespace fm
