// Device-side geometry shared by the kernels of the library (float32).
//
// Rotations are row-major 3x3 arrays R[r*3 + c].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fm {

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialisation attribute may start while its predecessor in the stream
// still runs.  pdl_wait() blocks until the predecessor grid has completed and
// its writes are visible (a no-op without the attribute); pdl_trigger() lets
// the successor start launching early -- it still waits in its own pdl_wait().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// A kernel launched this way is resident while its predecessor still writes,
// so nothing the predecessor (or an earlier kernel of the chain) produces may
// be read through the non-coherent read-only path (__ldg, or const
// __restrict__ pointers the compiler may turn into it): that path assumes the
// data is constant for the kernel's lifetime, and its lines were seen stale.
// Such data is read with ordinary loads after pdl_wait(), which makes the
// predecessors' writes visible to them.  Inputs that no kernel writes may
// still use __ldg.
__device__ __forceinline__ void load_plain(const float* p, float* out, int n) {
  for (int k = 0; k < n; ++k) out[k] = p[k];
}

__device__ __forceinline__ float dot3(const float* a, const float* b) {
  return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

__device__ __forceinline__ void cross3(const float* a, const float* b, float* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// 6D representation (Sec. 3.3): a = (a1, a2); b1 = a1/|a1|,
// b2 = normalise(a2 - (b1.a2) b1), b3 = b1 x b2; R = [b1 b2 b3] (columns).
struct Rot6 {
  float b1[3], b2[3], b3[3];
  float n1, n2, d12;   // |a1|, |u2|, b1.a2 (kept for the adjoint)
};

__device__ __forceinline__ void rot6_forward(const float* a, Rot6& s) {
  const float* a1 = a;
  const float* a2 = a + 3;
  s.n1 = sqrtf(dot3(a1, a1));
  float inv1 = 1.0f / s.n1;
  for (int k = 0; k < 3; ++k) s.b1[k] = a1[k] * inv1;
  s.d12 = dot3(s.b1, a2);
  float u2[3];
  for (int k = 0; k < 3; ++k) u2[k] = a2[k] - s.d12 * s.b1[k];
  s.n2 = sqrtf(dot3(u2, u2));
  float inv2 = 1.0f / s.n2;
  for (int k = 0; k < 3; ++k) s.b2[k] = u2[k] * inv2;
  cross3(s.b1, s.b2, s.b3);
}

__device__ __forceinline__ void rot6_matrix(const Rot6& s, float* R) {
  for (int r = 0; r < 3; ++r) {
    R[r * 3 + 0] = s.b1[r];
    R[r * 3 + 1] = s.b2[r];
    R[r * 3 + 2] = s.b3[r];
  }
}

// Gradient with respect to (a1, a2) of <gR, R(a)>; gR row-major.  The
// Gram-Schmidt steps above are differentiated in reverse order.
__device__ __forceinline__ void rot6_adjoint(const float* a, const Rot6& s, const float* gR,
                                             float* ga) {
  const float* a2 = a + 3;
  float gb1[3], gb2[3], gb3[3];
  for (int r = 0; r < 3; ++r) {
    gb1[r] = gR[r * 3 + 0];
    gb2[r] = gR[r * 3 + 1];
    gb3[r] = gR[r * 3 + 2];
  }
  float c[3];
  cross3(s.b2, gb3, c);            // b3 = b1 x b2
  for (int k = 0; k < 3; ++k) gb1[k] += c[k];
  cross3(gb3, s.b1, c);
  for (int k = 0; k < 3; ++k) gb2[k] += c[k];
  float q = dot3(s.b2, gb2);       // b2 = u2/|u2|
  float gu2[3];
  float inv2 = 1.0f / s.n2;
  for (int k = 0; k < 3; ++k) gu2[k] = (gb2[k] - s.b2[k] * q) * inv2;
  float p = dot3(s.b1, gu2);       // u2 = a2 - (b1.a2) b1
  for (int k = 0; k < 3; ++k) {
    ga[3 + k] = gu2[k] - s.b1[k] * p;
    gb1[k] += -s.d12 * gu2[k] - a2[k] * p;
  }
  float q1 = dot3(s.b1, gb1);      // b1 = a1/|a1|
  float inv1 = 1.0f / s.n1;
  for (int k = 0; k < 3; ++k) ga[k] = (gb1[k] - s.b1[k] * q1) * inv1;
}

// Epipolar geometry of an image pair (Sec. 3.3, epipolar adjustment):
// R_ij = R_j R_i^T, t_ij = t_j - R_ij t_i, t^ = t_ij/|t_ij|, E = [t^]_x R_ij.
struct PairGeo {
  float Ri[9], Rj[9], Rij[9];
  float ti[3], that[3];
  float inv_norm;      // 1/|t_ij|
};

__device__ __forceinline__ void pair_geometry(const float* pi, const float* pj, PairGeo& g) {
  Rot6 si, sj;
  rot6_forward(pi, si);
  rot6_forward(pj, sj);
  rot6_matrix(si, g.Ri);
  rot6_matrix(sj, g.Rj);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      // (R_j R_i^T)[r][c] = sum_k Rj[r][k] Ri[c][k]
      g.Rij[r * 3 + c] = fmaf(g.Rj[r * 3 + 0], g.Ri[c * 3 + 0],
                         fmaf(g.Rj[r * 3 + 1], g.Ri[c * 3 + 1], g.Rj[r * 3 + 2] * g.Ri[c * 3 + 2]));
    }
  float tij[3];
  for (int k = 0; k < 3; ++k) g.ti[k] = pi[6 + k];
  for (int r = 0; r < 3; ++r)
    tij[r] = pj[6 + r] - fmaf(g.Rij[r * 3 + 0], g.ti[0],
                          fmaf(g.Rij[r * 3 + 1], g.ti[1], g.Rij[r * 3 + 2] * g.ti[2]));
  float n = sqrtf(dot3(tij, tij));
  g.inv_norm = 1.0f / n;
  for (int k = 0; k < 3; ++k) g.that[k] = tij[k] * g.inv_norm;
}

__device__ __forceinline__ void essential(const PairGeo& g, float* E) {
  // [t]_x R: row r of [t]_x is (0,-t2,t1), (t2,0,-t0), (-t1,t0,0)
  const float* t = g.that;
  const float* R = g.Rij;
  for (int c = 0; c < 3; ++c) {
    E[0 * 3 + c] = -t[2] * R[1 * 3 + c] + t[1] * R[2 * 3 + c];
    E[1 * 3 + c] = t[2] * R[0 * 3 + c] - t[0] * R[2 * 3 + c];
    E[2 * 3 + c] = -t[1] * R[0 * 3 + c] + t[0] * R[1 * 3 + c];
  }
}

// Chain rule from G = dL/dE (row-major) to dL/dR_i, dL/dt_i, dL/dR_j, dL/dt_j.
// out[0..8] dR_i, out[9..11] dt_i, out[12..20] dR_j, out[21..23] dt_j.
__device__ __forceinline__ void pair_backward(const PairGeo& g, const float* G, float* out) {
  const float* t = g.that;
  const float* R = g.Rij;
  // through E = [t^]_x R with t^ fixed: dR = [t^]_x^T G = -[t^]_x G
  float dR[9];
  for (int c = 0; c < 3; ++c) {
    float g0 = G[0 * 3 + c], g1 = G[1 * 3 + c], g2 = G[2 * 3 + c];
    dR[0 * 3 + c] = t[2] * g1 - t[1] * g2;
    dR[1 * 3 + c] = -t[2] * g0 + t[0] * g2;
    dR[2 * 3 + c] = t[1] * g0 - t[0] * g1;
  }
  // dL/dt^ = (A23 - A32, A31 - A13, A12 - A21) (1-based) with A = R G^T
  float A[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      A[r * 3 + c] = fmaf(R[r * 3 + 0], G[c * 3 + 0], fmaf(R[r * 3 + 1], G[c * 3 + 1], R[r * 3 + 2] * G[c * 3 + 2]));
  float gt[3] = {A[1 * 3 + 2] - A[2 * 3 + 1], A[2 * 3 + 0] - A[0 * 3 + 2], A[0 * 3 + 1] - A[1 * 3 + 0]};
  // t^ = t_ij/|t_ij|
  float q = dot3(t, gt);
  float gtij[3];
  for (int k = 0; k < 3; ++k) gtij[k] = (gt[k] - t[k] * q) * g.inv_norm;
  // t_ij = t_j - R_ij t_i
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) dR[r * 3 + c] -= gtij[r] * g.ti[c];
  for (int k = 0; k < 3; ++k) out[21 + k] = gtij[k];
  for (int c = 0; c < 3; ++c)
    out[9 + c] = -fmaf(R[0 * 3 + c], gtij[0], fmaf(R[1 * 3 + c], gtij[1], R[2 * 3 + c] * gtij[2]));
  // R_ij = R_j R_i^T: dR_j = dR R_i, dR_i = dR^T R_j
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      out[12 + r * 3 + c] = fmaf(dR[r * 3 + 0], g.Ri[0 * 3 + c],
                            fmaf(dR[r * 3 + 1], g.Ri[1 * 3 + c], dR[r * 3 + 2] * g.Ri[2 * 3 + c]));
      out[r * 3 + c] = fmaf(dR[0 * 3 + r], g.Rj[0 * 3 + c],
                       fmaf(dR[1 * 3 + r], g.Rj[1 * 3 + c], dR[2 * 3 + r] * g.Rj[2 * 3 + c]));
    }
}

// eigen-decomposition of a symmetric 3 x 3 matrix S (row-major), cyclic
// Jacobi; on return S's diagonal holds the eigenvalues, Q's columns the
// eigenvectors
__device__ __forceinline__ void jacobi3(float* S, float* Q) {
#pragma unroll
  for (int k = 0; k < 9; ++k) Q[k] = (k % 4 == 0) ? 1.f : 0.f;
#pragma unroll 1
  for (int sweep = 0; sweep < 10; ++sweep) {
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const float apq = S[p * 3 + q];
      if (apq == 0.f) continue;
      const float tau = (S[q * 3 + q] - S[p * 3 + p]) / (2.f * apq);
      const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
      const float c = rsqrtf(fmaf(t, t, 1.f)), s = t * c;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float akp = S[k * 3 + p], akq = S[k * 3 + q];
        S[k * 3 + p] = c * akp - s * akq;
        S[k * 3 + q] = s * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float apk = S[p * 3 + k], aqk = S[q * 3 + k];
        S[p * 3 + k] = c * apk - s * aqk;
        S[q * 3 + k] = s * apk + c * aqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float vkp = Q[k * 3 + p], vkq = Q[k * 3 + q];
        Q[k * 3 + p] = c * vkp - s * vkq;
        Q[k * 3 + q] = s * vkp + c * vkq;
      }
    }
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

}  // namespace fm
