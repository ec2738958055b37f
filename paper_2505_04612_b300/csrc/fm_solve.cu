// Setup steps and the end-to-end solve (host orchestration of the kernels).
//
// fm_solve runs the paper's pipeline after matching and intrinsics (Sec. 3;
// Appendix "Global Rotation", "Global Translation", "Epipolar Adjustment",
// "Sparse Reconstruction"): rotation initialisation, Adam on the rotation
// loss, relative translations re-estimated by grid search, m translation runs
// from random starts merged per camera plus a final run, IRLS/filtering rounds
// of epipolar adjustment on the compact form, and triangulation.  Every step
// runs in this library's kernels; the host only sequences them.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

// epipolar-stage parameters from the rotation stage (6D) and the centres o:
// t = -R o
__global__ void k_ea_from_stages(const float* __restrict__ rot6, const float* __restrict__ o, int N,
                                 float* __restrict__ ea) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  Rot6 s;
  rot6_forward(rot6 + 6 * c, s);
  float R[9];
  rot6_matrix(s, R);
  for (int k = 0; k < 6; ++k) ea[9 * c + k] = rot6[6 * c + k];
  for (int r = 0; r < 3; ++r)
    ea[9 * c + 6 + r] = -(R[3 * r] * o[3 * c] + R[3 * r + 1] * o[3 * c + 1] + R[3 * r + 2] * o[3 * c + 2]);
}

// world-to-camera R (row-major) and t of the epipolar-stage parameters
__global__ void k_ea_to_Rt(const float* __restrict__ ea, int N, float* __restrict__ R, float* __restrict__ t) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  Rot6 s;
  rot6_forward(ea + 9 * c, s);
  rot6_matrix(s, R + 9 * c);
  for (int k = 0; k < 3; ++k) t[3 * c + k] = ea[9 * c + 6 + k];
}

}  // namespace

void launch_ea_from_stages(const float* rot6, const float* o, int N, float* ea, cudaStream_t s) {
  k_ea_from_stages<<<(N + 127) / 128, 128, 0, s>>>(rot6, o, N, ea);
}
void launch_ea_to_Rt(const float* ea, int N, float* R, float* t, cudaStream_t s) {
  k_ea_to_Rt<<<(N + 127) / 128, 128, 0, s>>>(ea, N, R, t);
}

}  // namespace fm
