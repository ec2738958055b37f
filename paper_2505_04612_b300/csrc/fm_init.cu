// Rotation initialisation (Appendix "Global Rotation / Initialization",
// Eqs. 10-14) and the multi-run translation merge (Appendix "Multiple
// Initializations").
//
// Martinec-Pajdla column problems.  With x stacking one 3-vector per camera,
// sum_{(i,j)} ||x_j - R_ij x_i||^2 = x^T A x where, per image pair,
// A_ii += I, A_jj += I, A_ji -= R_ij, A_ij -= R_ij^T (R_ij orthogonal).  The
// first columns are the eigenvector of A's smallest eigenvalue (Eq. 12); the
// second columns that of B = A/|P| + (1/|I|) blockdiag(c1_i c1_i^T) (Eq. 13).
// Both are found by power iteration on I - A/sigma with sigma = 1.05 d_max
// (B: 1.05 (d_max/|P| + 1/|I|)): x^T A x <= 2 sum_i d_i |x_i|^2 bounds
// lambda_max by 2 d_max, so the spectrum of I - A/sigma lies in [-0.905, 1]
// with the wanted eigenvector at the top.  A problem holding several scenes is block
// diagonal: every scene gets its own sigma, |P|, |I| and normalisation, so
// each one converges as it would alone.  Any vector of
// the (near-)null space is a valid answer (x_i = R_i v for some v), so only
// the gap to the fourth eigenvalue matters for convergence.
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

// y = x - (B x)/sigma with B = A/scaleP + (1/N) diag(c1 c1^T) (c1 may be
// null); coef[3 s + {0,1,2}] = (1/sigma, 1/scaleP, 1/N) of scene s.  One
// CTA of 128 threads per camera: thread t adds the incident image pairs
// t, t + 128, ... of the camera CSR, the warps reduce by butterflies and are
// added in warp order (a fixed order), and thread 0 writes the camera's row.
constexpr int kMartThreads = 128;

__global__ void __launch_bounds__(kMartThreads) k_mart_iter(const int* __restrict__ cam_seg_off,
                                                            const int* __restrict__ cam_seg,
                                                            const int* __restrict__ pi, const int* __restrict__ pj,
                                                            const float* __restrict__ relR,
                                                            const float* __restrict__ x,
                                                            const float* __restrict__ c1, float* __restrict__ y,
                                                            int N, const int* __restrict__ cam_scene,
                                                            const float* __restrict__ coef) {
  __shared__ float part[kMartThreads / 32][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  const int b = cam_seg_off[c], e = cam_seg_off[c + 1];
  for (int idx = b + threadIdx.x; idx < e; idx += kMartThreads) {
    const unsigned v = (unsigned)cam_seg[idx];
    const int n = (int)(v & 0x7fffffffu);
    const float* R = relR + 9 * n;
    if ((v >> 31) == 0) {
      // camera is i: row block i has -R^T x_j
      const float* xj = x + 3 * pj[n];
      a0 -= R[0] * xj[0] + R[3] * xj[1] + R[6] * xj[2];
      a1 -= R[1] * xj[0] + R[4] * xj[1] + R[7] * xj[2];
      a2 -= R[2] * xj[0] + R[5] * xj[1] + R[8] * xj[2];
    } else {
      // camera is j: row block j has -R x_i
      const float* xi = x + 3 * pi[n];
      a0 -= R[0] * xi[0] + R[1] * xi[1] + R[2] * xi[2];
      a1 -= R[3] * xi[0] + R[4] * xi[1] + R[5] * xi[2];
      a2 -= R[6] * xi[0] + R[7] * xi[1] + R[8] * xi[2];
    }
  }
  a0 = warp_sum(a0);
  a1 = warp_sum(a1);
  a2 = warp_sum(a2);
  if (lane == 0) {
    part[warp][0] = a0;
    part[warp][1] = a1;
    part[warp][2] = a2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a0 = a1 = a2 = 0.f;
    for (int w = 0; w < kMartThreads / 32; ++w) {
      a0 += part[w][0];
      a1 += part[w][1];
      a2 += part[w][2];
    }
    const int sc = cam_scene[c];
    const float inv_sigma = coef[3 * sc], inv_scale_p = coef[3 * sc + 1], inv_n = coef[3 * sc + 2];
    const float xc0 = x[3 * c], xc1 = x[3 * c + 1], xc2 = x[3 * c + 2];
    const float deg = (float)(e - b);
    float b0 = (a0 + deg * xc0) * inv_scale_p;
    float b1 = (a1 + deg * xc1) * inv_scale_p;
    float b2 = (a2 + deg * xc2) * inv_scale_p;
    if (c1) {
      const float* u = c1 + 3 * c;
      const float d = (u[0] * xc0 + u[1] * xc1 + u[2] * xc2) * inv_n;
      b0 += d * u[0];
      b1 += d * u[1];
      b2 += d * u[2];
    }
    y[3 * c] = xc0 - b0 * inv_sigma;
    y[3 * c + 1] = xc1 - b1 * inv_sigma;
    y[3 * c + 2] = xc2 - b2 * inv_sigma;
  }
}

// per-camera normalisation of the first columns
__global__ void k_normalise3(float* __restrict__ x, int N) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float v[3] = {x[3 * c], x[3 * c + 1], x[3 * c + 2]};
  const float n = sqrtf(dot3(v, v));
  const float s = n > 0.f ? 1.f / n : 0.f;
  for (int k = 0; k < 3; ++k) x[3 * c + k] = v[k] * s;
}

// second columns: normalise, Gram-Schmidt against c1 (Eq. 14 takes c3 = c1 x c2
// implicitly through the 6D map); write the 6D parameters (c1, c2)
__global__ void k_mart_finish(const float* __restrict__ c1, const float* __restrict__ c2, int N,
                              float* __restrict__ params6) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float u[3] = {c1[3 * c], c1[3 * c + 1], c1[3 * c + 2]};
  float v[3] = {c2[3 * c], c2[3 * c + 1], c2[3 * c + 2]};
  const float d = dot3(u, v);
  for (int k = 0; k < 3; ++k) v[k] -= d * u[k];
  const float n = sqrtf(dot3(v, v));
  const float s = n > 0.f ? 1.f / n : 0.f;
  for (int k = 0; k < 3; ++k) {
    params6[6 * c + k] = u[k];
    params6[6 * c + 3 + k] = v[k] * s;
  }
}

// deterministic start vector: the index mixed by a Weyl increment and the
// MurmurHash3 32-bit finaliser (fmix32), mapped to [-1, 1).  x is
// [runs][N][3]; the index of an entry is the one it has within its camera's
// scene, (r N_s + c - c0_s) 3 + a, so that a scene draws the same values
// whether it is solved alone or with others.
__global__ void k_hash_fill(float* __restrict__ x, int runs, int N, const int* __restrict__ cam_scene,
                            const int* __restrict__ sc_cam_off, unsigned salt) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long long)runs * N * 3) return;
  const int r = (int)(k / (3LL * N));
  const int rem = (int)(k - (long long)r * 3 * N);
  const int c = rem / 3, a = rem - 3 * c;
  const int sc = cam_scene[c];
  const int c0 = sc_cam_off[sc], ns = sc_cam_off[sc + 1] - c0;
  const unsigned idx = (unsigned)(((long long)r * ns + (c - c0)) * 3 + a);
  unsigned z = idx * 0x9E3779B9u + salt;
  z = (z ^ (z >> 16)) * 0x85EBCA6Bu;
  z = (z ^ (z >> 13)) * 0xC2B2AE35u;
  z ^= z >> 16;
  x[k] = (float)(z >> 8) * (1.0f / 8388608.0f) - 1.0f;
}

// x <- x / |x| over each scene's cameras (one CTA per scene, fixed-order
// sum), so that the power iteration neither underflows nor overflows
__global__ void k_scale_to_unit(float* __restrict__ x_all, const int* __restrict__ sc_cam_off) {
  __shared__ float part[256];
  float* x = x_all + 3 * (size_t)sc_cam_off[blockIdx.x];
  const int n = 3 * (sc_cam_off[blockIdx.x + 1] - sc_cam_off[blockIdx.x]);
  float s = 0.f;
  for (int k = threadIdx.x; k < n; k += 256) s += x[k] * x[k];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) part[threadIdx.x] += part[threadIdx.x + d];
    __syncthreads();
  }
  const float tot = part[0];
  const float inv = tot > 0.f ? rsqrtf(tot) : 0.f;
  for (int k = threadIdx.x; k < n; k += 256) x[k] *= inv;
}

// ---------------------------------------------------------------- merge
// Per (scene, run): centroid and mean norm of the scene's centres (fixed
// order, one CTA each); stats[4 (run S + scene) + {0..3}].
__global__ void k_run_stats(const float* __restrict__ o, int N_all, const int* __restrict__ sc_cam_off,
                            float* __restrict__ stats) {
  __shared__ float s[4][256];
  const int sc = blockIdx.x, run = blockIdx.y;
  const int c0 = sc_cam_off[sc], N = sc_cam_off[sc + 1] - c0;
  const float* orun = o + (size_t)3 * N_all * run + 3 * (size_t)c0;
  const int out = run * gridDim.x + sc;
  float a[3] = {0.f, 0.f, 0.f};
  for (int c = threadIdx.x; c < N; c += 256)
    for (int k = 0; k < 3; ++k) a[k] += orun[3 * c + k];
  for (int k = 0; k < 3; ++k) s[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d)
      for (int k = 0; k < 3; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + d];
    __syncthreads();
  }
  const float cx = s[0][0] / N, cy = s[1][0] / N, cz = s[2][0] / N;
  __syncthreads();
  float m = 0.f;
  for (int c = threadIdx.x; c < N; c += 256) {
    const float dx = orun[3 * c] - cx, dy = orun[3 * c + 1] - cy, dz = orun[3 * c + 2] - cz;
    m += sqrtf(dx * dx + dy * dy + dz * dz);
  }
  s[3][threadIdx.x] = m;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) s[3][threadIdx.x] += s[3][threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[4 * out + 0] = cx;
    stats[4 * out + 1] = cy;
    stats[4 * out + 2] = cz;
    stats[4 * out + 3] = s[3][0] / N;
  }
}

// Per camera (one warp): mean loss term over its image pairs in every run at
// the normalised centres; keep the run with the lowest mean (lowest index on
// ties) and write its normalised centre.
__global__ void __launch_bounds__(128) k_merge(const float* __restrict__ o, const float* __restrict__ stats,
                                               const int* __restrict__ cam_seg_off,
                                               const int* __restrict__ cam_seg, const int* __restrict__ pi,
                                               const int* __restrict__ pj, const float* __restrict__ tgt,
                                               int N, int runs, const int* __restrict__ cam_scene, int S,
                                               float* __restrict__ out, int* __restrict__ best_run) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (c >= N) return;
  const int sc = cam_scene[c];
  const int b = cam_seg_off[c], e = cam_seg_off[c + 1];
  float best = 3.4e38f;
  int best_r = 0;
  for (int r = 0; r < runs; ++r) {
    const float* orun = o + (size_t)3 * N * r;
    const float* st = stats + 4 * (r * S + sc);
    const float inv = st[3] > 0.f ? 1.f / st[3] : 0.f;
    float acc = 0.f;
    for (int idx = b + lane; idx < e; idx += 32) {
      const int n = (int)((unsigned)cam_seg[idx] & 0x7fffffffu);
      const int i = pi[n], j = pj[n];
      float d[3];
      for (int k = 0; k < 3; ++k) d[k] = ((orun[3 * j + k] - st[k]) - (orun[3 * i + k] - st[k])) * inv;
      const float nn = sqrtf(dot3(d, d));
      float l = 0.f;
      if (nn > 1e-12f) {
        for (int k = 0; k < 3; ++k) l += fabsf(d[k] / nn - tgt[3 * n + k]);
      } else {
        for (int k = 0; k < 3; ++k) l += fabsf(d[k] - tgt[3 * n + k]);
      }
      acc += l;
    }
    acc = warp_sum(acc);
    const float mean = (e > b) ? acc / (float)(e - b) : 0.f;
    if (mean < best) {
      best = mean;
      best_r = r;
    }
  }
  if (lane < 3) {
    const float* st = stats + 4 * (best_r * S + sc);
    const float inv = st[3] > 0.f ? 1.f / st[3] : 0.f;
    out[3 * c + lane] = (o[(size_t)3 * N * best_r + 3 * c + lane] - st[lane]) * inv;
  }
  if (lane == 0 && best_run) best_run[c] = best_r;
}

}  // namespace

void launch_mart_iter(const fm_problem* pr, const float* x, const float* c1, float* y, cudaStream_t s) {
  if (pr->N <= 0) return;
  k_mart_iter<<<pr->N, kMartThreads, 0, s>>>(pr->cam_seg_off, pr->cam_seg, pr->pair_i, pr->pair_j,
                                              pr->rel_R, x, c1, y, pr->N, pr->cam_scene, pr->mart_coef);
}
void launch_scale_to_unit(const fm_problem* pr, float* x, cudaStream_t s) {
  k_scale_to_unit<<<pr->S, 256, 0, s>>>(x, pr->sc_cam_off);
}
void launch_normalise3(float* x, int N, cudaStream_t s) {
  k_normalise3<<<(N + 127) / 128, 128, 0, s>>>(x, N);
}
void launch_mart_finish(const float* c1, const float* c2, int N, float* params6, cudaStream_t s) {
  k_mart_finish<<<(N + 127) / 128, 128, 0, s>>>(c1, c2, N, params6);
}
void launch_hash_fill(const fm_problem* pr, float* x, int runs, unsigned salt, cudaStream_t s) {
  const long long n = (long long)runs * pr->N * 3;
  k_hash_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, runs, pr->N, pr->cam_scene, pr->sc_cam_off, salt);
}
void launch_merge(const fm_problem* pr, const float* o, int runs, float* stats, float* out,
                  int* best_run, cudaStream_t s) {
  k_run_stats<<<dim3(pr->S, runs), 256, 0, s>>>(o, pr->N, pr->sc_cam_off, stats);
  k_merge<<<(pr->N + 3) / 4, 128, 0, s>>>(o, stats, pr->cam_seg_off, pr->cam_seg, pr->pair_i, pr->pair_j,
                                         pr->trn_target, pr->N, runs, pr->cam_scene, pr->S, out, best_run);
}

}  // namespace fm
