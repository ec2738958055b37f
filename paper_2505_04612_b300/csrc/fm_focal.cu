// Focal length interval search (Sec. 3.1 "Focal Length Estimation", Eq.
// focal-vote; Appendix "Focal Length Estimation") and recalibration of the
// keypoints at new focal lengths.
//
// The candidate essential matrix of an image pair at focal ratios rho_i,
// rho_j (f = rho f0, principal point fixed) is D_j E0 D_i with
// D = diag(rho, rho, 1) and E0 the eight-point estimate in coordinates
// calibrated at f0.  k_focal_vote: one CTA per candidate rho_k; its threads
// stride over the listed image pairs, each forming M = D_j E0 D_i, the
// eigenvalues of M^T M (3 x 3 Jacobi) and the term exp((1 - lambda1/lambda2)
// / tau) with lambda the singular values; a fixed-order tree over the threads
// gives the candidate's score.  A listed pair may fix one side's rho (the
// other image's group is already estimated).
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

constexpr int kVoteThreads = 256;

__global__ void __launch_bounds__(kVoteThreads) k_focal_vote(const float* __restrict__ e0, const int* __restrict__ idx,
                                                            const float* __restrict__ fix_i,
                                                            const float* __restrict__ fix_j, int M,
                                                            const float* __restrict__ rhos, float tau,
                                                            float* __restrict__ votes) {
  __shared__ float part[kVoteThreads];
  const int k = blockIdx.x;
  const float rho = rhos[k];
  float s = 0.f;
  for (int q = threadIdx.x; q < M; q += kVoteThreads) {
    const int n = idx[q];
    const float ri = fix_i[q] >= 0.f ? fix_i[q] : rho;
    const float rj = fix_j[q] >= 0.f ? fix_j[q] : rho;
    const float* E = e0 + 9 * (size_t)n;
    // M = D_j E D_i: rows 0, 1 scaled by rj, columns 0, 1 by ri
    float Mx[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Mx[a * 3 + b] = E[a * 3 + b] * (a < 2 ? rj : 1.f) * (b < 2 ? ri : 1.f);
    float S[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        S[a * 3 + b] = Mx[0 * 3 + a] * Mx[0 * 3 + b] + Mx[1 * 3 + a] * Mx[1 * 3 + b] + Mx[2 * 3 + a] * Mx[2 * 3 + b];
    float Q[9];
    jacobi3(S, Q);
    float l0 = S[0], l1 = S[4], l2 = S[8];
    // the two largest eigenvalues of M^T M
    const float hi = fmaxf(l0, fmaxf(l1, l2));
    const float lo = fminf(l0, fminf(l1, l2));
    const float mid = l0 + l1 + l2 - hi - lo;
    const float ratio = sqrtf(fmaxf(hi, 0.f) / fmaxf(mid, 1e-30f));
    s += expf((1.f - ratio) / tau);
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int d = kVoteThreads / 2; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) part[threadIdx.x] += part[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) votes[k] = part[0];
}

__global__ void k_recalibrate(float4* __restrict__ kp, const int* __restrict__ kp_seg, const int* __restrict__ pi,
                              const int* __restrict__ pj, const float* __restrict__ f_old,
                              const float* __restrict__ f_new, int64_t Z) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < Z; m += (int64_t)gridDim.x * blockDim.x) {
    const int n = kp_seg[m];
    const int i = pi[n], j = pj[n];
    const float si = f_old[i] / f_new[i], sj = f_old[j] / f_new[j];
    float4 x = kp[m];
    x.x *= si;
    x.y *= si;
    x.z *= sj;
    x.w *= sj;
    kp[m] = x;
  }
}

}  // namespace

void launch_focal_vote(const float* e0, const int* idx, const float* fix_i, const float* fix_j, int M,
                       const float* rhos, int K, float tau, float* votes, cudaStream_t s) {
  if (K == 0) return;
  k_focal_vote<<<K, kVoteThreads, 0, s>>>(e0, idx, fix_i, fix_j, M, rhos, tau, votes);
}

void launch_recalibrate(const fm_problem* pr, const float* f_old, const float* f_new, cudaStream_t s) {
  if (pr->Z == 0) return;
  int64_t g = (pr->Z + 255) / 256;
  if (g > 148 * 32) g = 148 * 32;
  k_recalibrate<<<(unsigned)g, 256, 0, s>>>(pr->kp, pr->kp_seg, pr->pair_i, pr->pair_j, f_old, f_new, pr->Z);
}

}  // namespace fm
