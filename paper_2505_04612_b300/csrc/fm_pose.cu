// Global rotation (Sec. 3.3, Eqs. 3-4) and global translation (Sec. 3.3,
// Eqs. 5-6): loss and per-image-pair gradient, one thread per image pair
// (and per initialisation run for the translation stage).
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

// L_R term of image pair n: d(R_j, R_ij R_i) with M = R_j^T R_ij R_i.
// The angle is taken as atan2(|w|, (tr M - 1)/2), w = vee(M - M^T)/2, which
// equals the paper's arccos((tr M - 1)/2) for a rotation M and stays accurate
// in float32 near 0, where arccos of a value next to 1 does not.
// dtheta/dM = (c [w]_x / (2|w|) - |w| I / 2) / (|w|^2 + c^2); 0 at |w| = 0.
// A CTA's 128 image pairs read their relative rotations as one contiguous
// block and write their gradients (two 48-byte slots, 9 floats each) as one
// (through shared memory, odd strides: no bank conflicts), instead of
// strided accesses per thread.
constexpr int kPairThreads = 128;

// cnt rows of W floats between contiguous global memory and shared-memory
// rows of STRIDE floats (STRIDE odd: a thread's row reads are free of bank
// conflicts)
template <int W, int STRIDE>
__device__ __forceinline__ void load_rows(const float* __restrict__ src, int cnt, float* rows) {
  for (int i = threadIdx.x; i < cnt * W; i += kPairThreads) rows[(i / W) * STRIDE + i % W] = src[i];
}
template <int W, int STRIDE>
__device__ __forceinline__ void store_rows(const float* rows, int cnt, float* __restrict__ dst) {
  for (int i = threadIdx.x; i < cnt * W; i += kPairThreads) dst[i] = rows[(i / W) * STRIDE + i % W];
}

__global__ void __launch_bounds__(kPairThreads) k_rot_pairs(const float* __restrict__ params,
                                                            const int* __restrict__ pi,
                                                            const int* __restrict__ pj,
                                                            const float* __restrict__ relR, int P,
                                                            const float* __restrict__ pair_inv_p,
                                                            float* __restrict__ seg_grad,
                                                            float* __restrict__ seg_loss, int* step_counter) {
  constexpr int kOut = kSegGradRot, kOutStride = kSegGradRot + 1;
  __shared__ float rel_s[kPairThreads * 9];
  __shared__ float out_s[kPairThreads * kOutStride];
  const int n0 = blockIdx.x * kPairThreads;
  const int n = n0 + threadIdx.x;
  const int cnt = min(kPairThreads, P - n0);
  if (step_counter && n == 0) *step_counter += 1;
  load_rows<9, 9>(relR + 9 * (size_t)n0, cnt, rel_s);
  __syncthreads();
  if (n < P) {
    const float inv_p = pair_inv_p[n];   // 1/|P| of the image pair's scene
    Rot6 si, sj;
    rot6_forward(params + 6 * pi[n], si);
    rot6_forward(params + 6 * pj[n], sj);
    float Ri[9], Rj[9], Rij[9];
    rot6_matrix(si, Ri);
    rot6_matrix(sj, Rj);
    for (int k = 0; k < 9; ++k) Rij[k] = rel_s[9 * threadIdx.x + k];
    float K[9], M[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        K[r * 3 + c] = fmaf(Rij[r * 3 + 0], Ri[0 * 3 + c],
                       fmaf(Rij[r * 3 + 1], Ri[1 * 3 + c], Rij[r * 3 + 2] * Ri[2 * 3 + c]));
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        M[r * 3 + c] = fmaf(Rj[0 * 3 + r], K[0 * 3 + c],
                       fmaf(Rj[1 * 3 + r], K[1 * 3 + c], Rj[2 * 3 + r] * K[2 * 3 + c]));
    const float w0 = 0.5f * (M[7] - M[5]);
    const float w1 = 0.5f * (M[2] - M[6]);
    const float w2 = 0.5f * (M[3] - M[1]);
    const float c = 0.5f * (M[0] + M[4] + M[8] - 1.f);
    const float s = sqrtf(w0 * w0 + w1 * w1 + w2 * w2);
    seg_loss[n] = atan2f(s, c) * inv_p;
    float D[9];
    if (s > 0.f) {
      const float den = inv_p / (s * s + c * c);
      const float a = 0.5f * c / s * den;
      const float b = -0.5f * s * den;
      // a [w]_x + b I
      D[0] = b;       D[1] = -a * w2; D[2] = a * w1;
      D[3] = a * w2;  D[4] = b;       D[5] = -a * w0;
      D[6] = -a * w1; D[7] = a * w0;  D[8] = b;
    } else {
      for (int k = 0; k < 9; ++k) D[k] = 0.f;
    }
    // dL/dR_i = R_ij^T R_j D ;  dL/dR_j = K D^T
    float T[9];
    for (int r = 0; r < 3; ++r)
      for (int cc = 0; cc < 3; ++cc)
        T[r * 3 + cc] = fmaf(Rij[0 * 3 + r], Rj[0 * 3 + cc],
                        fmaf(Rij[1 * 3 + r], Rj[1 * 3 + cc], Rij[2 * 3 + r] * Rj[2 * 3 + cc]));
    float* out = out_s + kOutStride * threadIdx.x;   // dR_i in [0, 9), dR_j in [12, 21), zeros between
    for (int r = 0; r < 3; ++r)
      for (int cc = 0; cc < 3; ++cc) {
        out[r * 3 + cc] = fmaf(T[r * 3 + 0], D[0 * 3 + cc],
                          fmaf(T[r * 3 + 1], D[1 * 3 + cc], T[r * 3 + 2] * D[2 * 3 + cc]));
        out[12 + r * 3 + cc] = fmaf(K[r * 3 + 0], D[cc * 3 + 0],
                               fmaf(K[r * 3 + 1], D[cc * 3 + 1], K[r * 3 + 2] * D[cc * 3 + 2]));
      }
    for (int k = 9; k < 12; ++k) out[k] = out[12 + k] = 0.f;
  }
  __syncthreads();
  if (cnt > 0) store_rows<kOut, kOutStride>(out_s, cnt, seg_grad + (size_t)kOut * n0);
}

// o^{i->j} = -R_j^T t^{i->j} (Eq. 5), R_j from the rotation-stage parameters
__global__ void k_trn_targets(const float* __restrict__ rot, const int* __restrict__ pj,
                              const float* __restrict__ relt, int P, float* __restrict__ tgt) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= P) return;
  Rot6 sj;
  rot6_forward(rot + 6 * pj[n], sj);
  float R[9];
  rot6_matrix(sj, R);
  const float t0 = relt[3 * n], t1 = relt[3 * n + 1], t2 = relt[3 * n + 2];
  for (int c = 0; c < 3; ++c) tgt[3 * n + c] = -fmaf(R[0 * 3 + c], t0, fmaf(R[1 * 3 + c], t1, R[2 * 3 + c] * t2));
}

// L_t term (Eq. 6): || u - o^{i->j} ||_1 with u = (o_j - o_i)/|o_j - o_i|;
// sign(0) = 0; |o_j - o_i| <= 1e-12 gives a zero gradient.
// (image pair, run) items idx = run * P + n; a CTA's 128 items write their
// gradients (two 16-byte slots, 3 floats each) as one contiguous block
// (through shared memory)
__global__ void __launch_bounds__(kPairThreads) k_trn_pairs(const float* __restrict__ o, const int* __restrict__ pi,
                                                            const int* __restrict__ pj,
                                                            const float* __restrict__ tgt, int N, int P, int runs,
                                                            const float* __restrict__ pair_inv_p,
                                                            float* __restrict__ seg_grad,
                                                            float* __restrict__ seg_loss, int* step_counter) {
  constexpr int kOut = kSegGradTrn, kOutStride = kSegGradTrn + 1;
  __shared__ float out_s[kPairThreads * kOutStride];
  const int i0 = blockIdx.x * kPairThreads;
  const int idx = i0 + threadIdx.x;
  const int cnt = min(kPairThreads, P * runs - i0);
  if (step_counter && idx == 0) *step_counter += 1;
  float* out = out_s + kOutStride * threadIdx.x;
  if (idx < P * runs) {
    const int run = idx / P, n = idx - run * P;
    const float inv_p = pair_inv_p[n];
    const float* orun = o + (size_t)3 * N * run;
    const int i = pi[n], j = pj[n];
    float d[3], u[3], gu[3];
    for (int k = 0; k < 3; ++k) d[k] = orun[3 * j + k] - orun[3 * i + k];
    const float nrm = sqrtf(dot3(d, d));
    if (!(nrm > 1e-12f)) {
      float l = 0.f;
      for (int k = 0; k < 3; ++k) l += fabsf(tgt[3 * n + k]);
      seg_loss[idx] = l * inv_p;
      for (int k = 0; k < 8; ++k) out[k] = 0.f;
    } else {
      const float inv = 1.f / nrm;
      float l = 0.f;
      for (int k = 0; k < 3; ++k) {
        u[k] = d[k] * inv;
        const float e = u[k] - tgt[3 * n + k];
        l += fabsf(e);
        gu[k] = ((e > 0.f) ? inv_p : ((e < 0.f) ? -inv_p : 0.f));
      }
      seg_loss[idx] = l * inv_p;
      const float q = dot3(u, gu);
      for (int k = 0; k < 3; ++k) {   // do_i in [0, 3), do_j in [4, 7), zeros between
        const float gd = (gu[k] - u[k] * q) * inv;
        out[k] = -gd;
        out[4 + k] = gd;
      }
      out[3] = out[7] = 0.f;
    }
  }
  __syncthreads();
  if (cnt > 0) store_rows<kOut, kOutStride>(out_s, cnt, seg_grad + (size_t)kOut * i0);
}

}  // namespace

void launch_rot_pairs(const float* params, const int* pi, const int* pj, const float* rel_R,
                      int P, const float* pair_inv_p, float* seg_grad, float* seg_loss, int* step_counter,
                      cudaStream_t s) {
  if (P <= 0) return;
  k_rot_pairs<<<(P + kPairThreads - 1) / kPairThreads, kPairThreads, 0, s>>>(params, pi, pj, rel_R, P, pair_inv_p,
                                                                              seg_grad, seg_loss, step_counter);
}

void launch_trn_targets(const float* rot_params, const int* pj, const float* rel_t, int P,
                        float* target, cudaStream_t s) {
  k_trn_targets<<<(P + 127) / 128, 128, 0, s>>>(rot_params, pj, rel_t, P, target);
}

void launch_trn_pairs(const float* o, const int* pi, const int* pj, const float* target, int N,
                      int P, int runs, const float* pair_inv_p, float* seg_grad, float* seg_loss,
                      int* step_counter, cudaStream_t s) {
  const int n = P * runs;
  if (n <= 0) return;
  k_trn_pairs<<<(n + kPairThreads - 1) / kPairThreads, kPairThreads, 0, s>>>(o, pi, pj, target, N, P, runs,
                                                                              pair_inv_p, seg_grad, seg_loss,
                                                                              step_counter);
}

}  // namespace fm
