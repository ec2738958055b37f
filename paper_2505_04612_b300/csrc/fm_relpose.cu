// Relative pose of every image pair from its keypoint pairs (the setup step
// that stands in for the upstream geometric verification; Sec. 3.3 "Global
// Rotation" takes R^{i->j}, t^{i->j} from decomposing the two-view matrix,
// Appendix "Limitations": the cheirality check keeps one decomposition, the
// lowest index on ties).
//
// One warp per image pair:
//   1. W_n = sum_m w_m v_m v_m^T with v_m = vec(x~2 x~1^T) (row-major; Eq. 17),
//      45 unique entries, lane-strided partial sums and a butterfly;
//   2. the eigenvector of W_n's smallest eigenvalue (the linear eight-point
//      estimate of E in calibrated coordinates) by cyclic Jacobi sweeps on the
//      9 x 9 matrix in shared memory, the nine lanes of a row updating it in
//      parallel; rotation angles by the symmetric 2 x 2 Schur decomposition
//      (Golub and Van Loan, Matrix Computations, Sec. 8.5);
//   3. optional IRLS rounds: weights 1/max(|x~2^T E x~1|, delta), step 1 and 2
//      again;
//   4. the projection of E onto the essential matrices (singular values
//      (1, 1, 0), Sec. 3.1) through the eigen-decomposition of E^T E (3 x 3
//      Jacobi), E = U diag(s) V^T with det U = det V = 1;
//   5. the four decompositions (R1, t), (R1, -t), (R2, t), (R2, -t) with
//      R1 = U W V^T, R2 = U W^T V^T, t = u3, and for each the number of
//      keypoint pairs with both depths positive (least-squares depths of
//      l2 x~2 = l1 R x~1 + t); the first maximum wins.
// Image pairs with fewer than 8 keypoint pairs get R = I, t = 0, valid = 0.
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kRelposeWarps = 4;
constexpr int kJacobiSweeps = 12;

// upper-triangle index of (a, b), a <= b, in a 9 x 9 symmetric matrix
__host__ __device__ constexpr int tri9(int a, int b) { return a * 9 - a * (a - 1) / 2 + (b - a); }

__device__ __forceinline__ void vec9(float4 x, float* v) {
  // v = vec(x~2 x~1^T), x~1 = (x.x, x.y, 1), x~2 = (x.z, x.w, 1)
  v[0] = x.z * x.x; v[1] = x.z * x.y; v[2] = x.z;
  v[3] = x.w * x.x; v[4] = x.w * x.y; v[5] = x.w;
  v[6] = x.x;       v[7] = x.y;       v[8] = 1.f;
}

// smallest-eigenvalue eigenvector of sum_m w_m v_m v_m^T over pairs [b, e);
// A, V: this warp's 81-float shared-memory scratch matrices
__device__ void eight_point(const float4* __restrict__ kp, const float* E_w, float delta, int b, int e, int lane,
                            float* A, float* V, float* out) {
  float acc[45];
#pragma unroll
  for (int k = 0; k < 45; ++k) acc[k] = 0.f;
  for (int m = b + lane; m < e; m += 32) {
    const float4 x = kp[m];
    float v[9];
    vec9(x, v);
    float w = 1.f;
    if (E_w) {   // IRLS weight from the previous estimate
      const float r = x.z * (E_w[0] * x.x + E_w[1] * x.y + E_w[2]) + x.w * (E_w[3] * x.x + E_w[4] * x.y + E_w[5]) +
                      (E_w[6] * x.x + E_w[7] * x.y + E_w[8]);
      w = 1.f / fmaxf(fabsf(r), delta);
    }
#pragma unroll
    for (int a = 0; a < 9; ++a)
#pragma unroll
      for (int c = a; c < 9; ++c) acc[tri9(a, c)] = fmaf(w * v[a], v[c], acc[tri9(a, c)]);
  }
#pragma unroll
  for (int k = 0; k < 45; ++k) acc[k] = warp_sum(acc[k]);
  // full matrix into shared memory (every lane holds the sums; lanes < 9 write rows)
  if (lane < 9) {
#pragma unroll
    for (int a = 0; a < 9; ++a)
#pragma unroll
      for (int c = 0; c < 9; ++c)
        if (lane == a) {
          A[a * 9 + c] = acc[a <= c ? tri9(a, c) : tri9(c, a)];
          V[a * 9 + c] = (a == c) ? 1.f : 0.f;
        }
  }
  __syncwarp();
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    for (int p = 0; p < 8; ++p)
      for (int q = p + 1; q < 9; ++q) {
        const float apq = A[p * 9 + q];
        if (apq == 0.f) continue;   // uniform: every lane reads the same value
        const float tau = (A[q * 9 + q] - A[p * 9 + p]) / (2.f * apq);
        const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
        const float c = rsqrtf(fmaf(t, t, 1.f)), s = t * c;
        __syncwarp();
        if (lane < 9) {   // A <- A J (columns p, q of row `lane`), V <- V J
          const float akp = A[lane * 9 + p], akq = A[lane * 9 + q];
          A[lane * 9 + p] = c * akp - s * akq;
          A[lane * 9 + q] = s * akp + c * akq;
          const float vkp = V[lane * 9 + p], vkq = V[lane * 9 + q];
          V[lane * 9 + p] = c * vkp - s * vkq;
          V[lane * 9 + q] = s * vkp + c * vkq;
        }
        __syncwarp();
        if (lane < 9) {   // A <- J^T A (rows p, q of column `lane`)
          const float apk = A[p * 9 + lane], aqk = A[q * 9 + lane];
          A[p * 9 + lane] = c * apk - s * aqk;
          A[q * 9 + lane] = s * apk + c * aqk;
        }
        __syncwarp();
      }
  }
  int best = 0;
  float lo = A[0];
  for (int k = 1; k < 9; ++k)
    if (A[k * 9 + k] < lo) {
      lo = A[k * 9 + k];
      best = k;
    }
#pragma unroll
  for (int a = 0; a < 9; ++a) out[a] = V[a * 9 + best];
  __syncwarp();   // the scratch is reused by the next call
}

// U, V (columns u_k, v_k; det +1) of the projection of E onto the essential
// matrices: E = U diag(s1, s2, s3) V^T with s1 >= s2 >= s3
__device__ void essential_frames(const float* E, float* U, float* V) {
  float S[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) S[a * 3 + b] = E[0 * 3 + a] * E[0 * 3 + b] + E[1 * 3 + a] * E[1 * 3 + b] +
                                                E[2 * 3 + a] * E[2 * 3 + b];   // E^T E
  float Q[9];
  jacobi3(S, Q);
  // order the eigenvectors by decreasing eigenvalue
  int o[3] = {0, 1, 2};
  float l[3] = {S[0], S[4], S[8]};
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2 - i; ++j)
      if (l[o[j]] < l[o[j + 1]]) {
        const int tmp = o[j];
        o[j] = o[j + 1];
        o[j + 1] = tmp;
      }
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int a = 0; a < 3; ++a) V[a * 3 + k] = Q[a * 3 + o[k]];
  float v1[3] = {V[0], V[3], V[6]}, v2[3] = {V[1], V[4], V[7]}, v3[3] = {V[2], V[5], V[8]};
  float c3[3];
  cross3(v1, v2, c3);
  if (dot3(c3, v3) < 0.f) {   // det V = +1 (v3 spans the null direction: its sign is free)
    V[2] = -V[2];
    V[5] = -V[5];
    V[8] = -V[8];
  }
  float u1[3], u2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u1[a] = E[a * 3 + 0] * v1[0] + E[a * 3 + 1] * v1[1] + E[a * 3 + 2] * v1[2];
    u2[a] = E[a * 3 + 0] * v2[0] + E[a * 3 + 1] * v2[1] + E[a * 3 + 2] * v2[2];
  }
  const float n1 = rsqrtf(fmaxf(dot3(u1, u1), 1e-30f));
#pragma unroll
  for (int a = 0; a < 3; ++a) u1[a] *= n1;
  const float d = dot3(u1, u2);
#pragma unroll
  for (int a = 0; a < 3; ++a) u2[a] -= d * u1[a];
  const float n2 = rsqrtf(fmaxf(dot3(u2, u2), 1e-30f));
#pragma unroll
  for (int a = 0; a < 3; ++a) u2[a] *= n2;
  float u3[3];
  cross3(u1, u2, u3);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    U[a * 3 + 0] = u1[a];
    U[a * 3 + 1] = u2[a];
    U[a * 3 + 2] = u3[a];
  }
}

// 1 when both least-squares depths of the pair are positive under (R, t)
__device__ __forceinline__ int in_front(const float* R, const float* t, float4 x) {
  const float a0 = R[0] * x.x + R[1] * x.y + R[2];
  const float a1 = R[3] * x.x + R[4] * x.y + R[5];
  const float a2 = R[6] * x.x + R[7] * x.y + R[8];
  const float A11 = a0 * a0 + a1 * a1 + a2 * a2;
  const float A12 = -(a0 * x.z + a1 * x.w + a2);
  const float A22 = x.z * x.z + x.w * x.w + 1.f;
  const float b1 = -(a0 * t[0] + a1 * t[1] + a2 * t[2]);
  const float b2 = x.z * t[0] + x.w * t[1] + t[2];
  const float det = A11 * A22 - A12 * A12;
  if (!(fabsf(det) > 1e-12f)) return 0;
  const float l1 = (A22 * b1 - A12 * b2) / det;
  const float l2 = (A11 * b2 - A12 * b1) / det;
  return (l1 > 0.f && l2 > 0.f) ? 1 : 0;
}

// rel_R == nullptr: only the (IRLS) eight-point estimates E0 [P*9] and valid
__global__ void __launch_bounds__(kRelposeWarps * 32) k_relpose(const float4* __restrict__ kp,
                                                                const int* __restrict__ seg_off, int P,
                                                                int irls_iters, float delta, float* __restrict__ rel_R,
                                                                float* __restrict__ rel_t, int* __restrict__ valid,
                                                                float* __restrict__ e0_out) {
  __shared__ float scratch[kRelposeWarps][2][81];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int n = blockIdx.x * kRelposeWarps + wib;
  if (n >= P) return;   // uniform per warp
  const int b = seg_off[n], e = seg_off[n + 1];
  float* A = scratch[wib][0];
  float* V = scratch[wib][1];
  if (e - b < 8) {
    if (rel_R) {
      if (lane < 9) rel_R[9 * (size_t)n + lane] = (lane % 4 == 0) ? 1.f : 0.f;
      if (lane < 3) rel_t[3 * (size_t)n + lane] = 0.f;
    }
    if (e0_out && lane < 9) e0_out[9 * (size_t)n + lane] = 0.f;
    if (lane == 0) valid[n] = 0;
    return;
  }
  float E[9];
  eight_point(kp, nullptr, delta, b, e, lane, A, V, E);
  for (int it = 0; it < irls_iters; ++it) {
    float En[9];
    eight_point(kp, E, delta, b, e, lane, A, V, En);
#pragma unroll
    for (int k = 0; k < 9; ++k) E[k] = En[k];
  }
  if (e0_out && lane < 9) {
    float v = E[0];
#pragma unroll
    for (int k = 1; k < 9; ++k)
      if (lane == k) v = E[k];
    e0_out[9 * (size_t)n + lane] = v;
  }
  if (!rel_R) {
    if (lane == 0) valid[n] = 1;
    return;
  }
  float U[9], Vf[9];
  essential_frames(E, U, Vf);
  // R1 = U Wm V^T, R2 = U Wm^T V^T with Wm = [[0,-1,0],[1,0,0],[0,0,1]]
  float R[2][9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // (U Wm)[a][:] = (u_a1, -u_a0, u_a2);  (U Wm^T)[a][:] = (-u_a1, u_a0, u_a2)
      const float w0 = U[a * 3 + 1], w1 = -U[a * 3 + 0], w2 = U[a * 3 + 2];
      R[0][a * 3 + c] = w0 * Vf[c * 3 + 0] + w1 * Vf[c * 3 + 1] + w2 * Vf[c * 3 + 2];
      R[1][a * 3 + c] = -w0 * Vf[c * 3 + 0] - w1 * Vf[c * 3 + 1] + w2 * Vf[c * 3 + 2];
    }
  const float tp[3] = {U[2], U[5], U[8]}, tn[3] = {-U[2], -U[5], -U[8]};
  int cnt[4] = {0, 0, 0, 0};
  for (int m = b + lane; m < e; m += 32) {
    const float4 x = kp[m];
    cnt[0] += in_front(R[0], tp, x);
    cnt[1] += in_front(R[0], tn, x);
    cnt[2] += in_front(R[1], tp, x);
    cnt[3] += in_front(R[1], tn, x);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt[k] += __shfl_xor_sync(FULL, cnt[k], d);
  int best = 0;
#pragma unroll
  for (int k = 1; k < 4; ++k)
    if (cnt[k] > cnt[best]) best = k;
  const float* Rb = R[best >> 1];
  const float* tb = (best & 1) ? tn : tp;
  if (lane < 9) {
    float v = Rb[0];
#pragma unroll
    for (int k = 1; k < 9; ++k)
      if (lane == k) v = Rb[k];
    rel_R[9 * (size_t)n + lane] = v;
  }
  if (lane < 3) rel_t[3 * (size_t)n + lane] = lane == 0 ? tb[0] : (lane == 1 ? tb[1] : tb[2]);
  if (lane == 0) valid[n] = 1;
}

}  // namespace

void launch_relpose(const fm_problem* pr, int irls_iters, float delta, float* rel_R, float* rel_t, int* valid,
                    cudaStream_t s, float* e0_out) {
  if (pr->P == 0) return;
  k_relpose<<<(pr->P + kRelposeWarps - 1) / kRelposeWarps, kRelposeWarps * 32, 0, s>>>(
      pr->kp, pr->seg_off, pr->P, irls_iters, delta, rel_R, rel_t, valid, e0_out);
}

}  // namespace fm
