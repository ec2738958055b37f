// Relative translation re-estimation (Appendix "Relative Translation"): with
// R_ij = R_j R_i^T from the global rotations, unit candidates t are scored by
// the mean absolute epipolar error  mean_m |x~2^T [t]_x R_ij x~1|
// = mean_m |t . a_m|,  a_m = (R_ij x~1) x x~2, and the lowest is kept.
//
// Candidates (the paper gives none; a reading): a Fibonacci lattice of 4096
// points on the hemisphere, then two Fibonacci lattices of 1024 points on
// spherical caps of radius twice the previous spacing around the best point.
// The error is even in t, so the sign is chosen by cheirality (more pairs
// with both depths positive; +t on ties).  Keypoint pairs whose weight is 0
// (filtered) are left out of both, unless the image pair has no other.
//
// One CTA per image pair.  The a_m of a tile of keypoint pairs are formed in
// shared memory; each thread scores its own candidates over the tile.  An ALU
// kernel: 4 FP32 operations per (pair, candidate), issued as packed f32x2
// instructions for pairs of candidates (the multiply and the two fmas) and
// two scalar adds of the absolute values; no tensor-core shape (inner
// dimension 3).  The hemisphere's 4096 points are the same for every
// image pair: k_lattice0 writes them once per problem (the same function and
// arguments as the per-CTA evaluation, so the same values), and an image pair
// whose keypoint pairs fit in one tile forms its a_m once for all three
// levels.
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

constexpr int kThreads = 256;
constexpr int kTile = 512;
// each a_m entry twice, (a, a): one 64-bit shared-memory load gives the
// operand that a packed f32x2 instruction applies to two candidates
using TileT = float2;
__device__ __forceinline__ TileT tile_val(float v) { return make_float2(v, v); }
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
constexpr int kK0 = 4096, kK1 = 1024;
constexpr unsigned kGolden32 = 0x61C88647u;   // round(2^32 (3 - sqrt 5)/2)

// k-th of K Fibonacci points on the cap of height H = 1 - cos(radius) around
// (0, 0, 1), rotated by Q (row-major) to the cap's centre
__device__ __forceinline__ void lattice_point(int k, int K, float H, const float* Q, float* t) {
  const float h = H * ((float)k + 0.5f) / (float)K;
  const float z = 1.f - h;
  const float r = sqrtf(fmaxf(h * (2.f - h), 0.f));
  const float frac = (float)((unsigned)k * kGolden32) * 2.3283064365386963e-10f;   // / 2^32
  float s, c;
  sincospif(2.f * frac, &s, &c);
  const float p[3] = {r * c, r * s, z};
  for (int a = 0; a < 3; ++a) t[a] = Q[3 * a] * p[0] + Q[3 * a + 1] * p[1] + Q[3 * a + 2] * p[2];
}

// rotation taking (0,0,1) to the unit vector c (Rodrigues)
__device__ void rotation_to(const float* c, float* Q) {
  const float v[3] = {-c[1], c[0], 0.f};   // (0,0,1) x c
  const float s = sqrtf(v[0] * v[0] + v[1] * v[1]);
  const float ct = c[2];
  if (s < 1e-12f) {
    for (int k = 0; k < 9; ++k) Q[k] = 0.f;
    Q[0] = 1.f;
    Q[4] = ct > 0.f ? 1.f : -1.f;
    Q[8] = ct > 0.f ? 1.f : -1.f;
    return;
  }
  const float u[3] = {v[0] / s, v[1] / s, 0.f};
  const float K[9] = {0.f, -u[2], u[1], u[2], 0.f, -u[0], -u[1], u[0], 0.f};
  const float ang = atan2f(s, ct);
  float sn, cs;
  sincosf(ang, &sn, &cs);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      float kk = 0.f;
      for (int m = 0; m < 3; ++m) kk += K[3 * a + m] * K[3 * m + b];
      Q[3 * a + b] = (a == b ? 1.f : 0.f) + sn * K[3 * a + b] + (1.f - cs) * kk;
    }
}

struct Best {
  float e;
  int k;
};

__device__ __forceinline__ Best better(Best a, Best b) {
  return (b.e < a.e || (b.e == a.e && b.k < a.k)) ? b : a;
}

// a_m of keypoint pairs [base, base + n) into the tile
__device__ __forceinline__ void fill_tile(const float4* __restrict__ kp, const float* __restrict__ w, int base,
                                          int n, const float* Rij, TileT (*a_s)[kTile]) {
  for (int m = threadIdx.x; m < n; m += kThreads) {
    const float4 x = kp[base + m];
    const float r0 = Rij[0] * x.x + Rij[1] * x.y + Rij[2];
    const float r1 = Rij[3] * x.x + Rij[4] * x.y + Rij[5];
    const float r2 = Rij[6] * x.x + Rij[7] * x.y + Rij[8];
    // (R x1) x x2 with x2 = (x.z, x.w, 1); a left-out pair adds |t . 0| = 0
    const float keep = (w == nullptr || w[base + m] > 0.f) ? 1.f : 0.f;
    a_s[0][m] = tile_val(keep * (r1 * 1.f - r2 * x.w));
    a_s[1][m] = tile_val(keep * (r2 * x.z - r0 * 1.f));
    a_s[2][m] = tile_val(keep * (r0 * x.w - r1 * x.z));
  }
}

// candidates k = threadIdx.x + kThreads i from `table` (level 0) or the cap
// lattice (K, H, Q); resident: the image pair's a_m already fill the tile
template <int PER>
__device__ Best score_level(const float4* __restrict__ kp, const float* __restrict__ w, int b, int e,
                            const float* Rij, int K, float H, const float* Q, const float4* __restrict__ table,
                            bool resident, TileT (*a_s)[kTile]) {
  float t[PER][3];
  float acc[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    if (table) {
      const float4 p = table[threadIdx.x + kThreads * i];
      t[i][0] = p.x;
      t[i][1] = p.y;
      t[i][2] = p.z;
    } else {
      lattice_point(threadIdx.x + kThreads * i, K, H, Q, t[i]);
    }
    acc[i] = 0.f;
  }
  // |t . a| = |t0 a0 + (t1 a1 + t2 a2)| (a multiply and two fmas) for
  // candidates 2i and 2i + 1 side by side, two per f32x2 instruction; the
  // absolute values are added one by one
  unsigned long long tp[PER / 2][3];
#pragma unroll
  for (int i = 0; i < PER / 2; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) tp[i][c] = pk2(t[2 * i][c], t[2 * i + 1][c]);
  for (int base = b; base < e; base += kTile) {
    const int n = min(kTile, e - base);
    if (!resident) {
      __syncthreads();
      fill_tile(kp, w, base, n, Rij, a_s);
      __syncthreads();
    }
    for (int m = 0; m < n; ++m) {
      const unsigned long long a0 = *reinterpret_cast<const unsigned long long*>(&a_s[0][m]);
      const unsigned long long a1 = *reinterpret_cast<const unsigned long long*>(&a_s[1][m]);
      const unsigned long long a2 = *reinterpret_cast<const unsigned long long*>(&a_s[2][m]);
#pragma unroll
      for (int i = 0; i < PER / 2; ++i) {
        const unsigned long long d = fma2(tp[i][0], a0, fma2(tp[i][1], a1, mul2(tp[i][2], a2)));
        float lo, hi;
        upk2(d, lo, hi);
        acc[2 * i] += fabsf(lo);
        acc[2 * i + 1] += fabsf(hi);
      }
    }
  }
  Best best{3.4e38f, 0x7fffffff};
#pragma unroll
  for (int i = 0; i < PER; ++i) best = better(best, Best{acc[i], (int)threadIdx.x + kThreads * i});
  return best;
}

__device__ Best block_best(Best v, Best* red) {
  for (int d = 16; d > 0; d >>= 1) {
    Best o;
    o.e = __shfl_xor_sync(0xffffffffu, v.e, d);
    o.k = __shfl_xor_sync(0xffffffffu, v.k, d);
    v = better(v, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  Best r = red[0];
  for (int w = 1; w < kThreads / 32; ++w) r = better(r, red[w]);
  return r;
}

// positive-depth count for (R, t): l2 x2 = l1 R x1 + t, least squares
__device__ __forceinline__ int positive_depths(const float4 x, const float* R, const float* t) {
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

__global__ void __launch_bounds__(kThreads) k_reltrans(const float4* __restrict__ kp, const int* __restrict__ seg_off,
                                                      const int* __restrict__ pi, const int* __restrict__ pj,
                                                      const float* __restrict__ rot6, const float* __restrict__ w_in,
                                                      const float4* __restrict__ lat0,
                                                      float* __restrict__ rel_t, float* __restrict__ err_out) {
  __shared__ TileT a_s[3][kTile];
  __shared__ Best red[kThreads / 32];
  __shared__ float Rij_s[9];
  __shared__ int cnt_s[2][kThreads / 32];
  __shared__ int kept_s;
  const int n = blockIdx.x;
  const int b = seg_off[n], e = seg_off[n + 1];
  // pairs that count: those with a positive weight, or all of them when the
  // image pair has none (or no weights are set)
  int kc = 0;
  if (w_in)
    for (int m = b + threadIdx.x; m < e; m += kThreads) kc += (w_in[m] > 0.f);
  for (int d = 16; d > 0; d >>= 1) kc += __shfl_xor_sync(0xffffffffu, kc, d);
  if (threadIdx.x == 0) kept_s = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0 && kc) atomicAdd(&kept_s, kc);   // integer: order-free
  if (threadIdx.x == 0) {
    Rot6 si, sj;
    rot6_forward(rot6 + 6 * pi[n], si);
    rot6_forward(rot6 + 6 * pj[n], sj);
    float Ri[9], Rj[9];
    rot6_matrix(si, Ri);
    rot6_matrix(sj, Rj);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        Rij_s[3 * r + c] = Rj[3 * r] * Ri[3 * c] + Rj[3 * r + 1] * Ri[3 * c + 1] + Rj[3 * r + 2] * Ri[3 * c + 2];
  }
  __syncthreads();
  const int kept = kept_s;
  const float* w = (w_in && kept > 0) ? w_in : nullptr;
  const int count = w ? kept : e - b;
  float Rij[9];
  for (int k = 0; k < 9; ++k) Rij[k] = Rij_s[k];
  if (e == b) {
    if (threadIdx.x < 3) rel_t[3 * n + threadIdx.x] = (threadIdx.x == 2) ? 1.f : 0.f;
    if (threadIdx.x == 0 && err_out) err_out[n] = 0.f;
    return;
  }
  const float I3[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
  const bool resident = e - b <= kTile;
  if (resident) {
    fill_tile(kp, w, b, e - b, Rij, a_s);
    __syncthreads();
  }
  // level 0: hemisphere
  Best bst = block_best(score_level<kK0 / kThreads>(kp, w, b, e, Rij, kK0, 1.f, I3, lat0, resident, a_s), red);
  float t[3] = {lat0[bst.k].x, lat0[bst.k].y, lat0[bst.k].z};
  float best_e = bst.e;
  float spacing = sqrtf(2.f * 3.14159265358979f * 1.f / kK0);
  for (int level = 0; level < 2; ++level) {
    const float radius = 2.f * spacing;
    const float sh = sinf(0.5f * radius);
    const float H = 2.f * sh * sh;   // 1 - cos(radius)
    float Q[9];
    rotation_to(t, Q);
    Best c = block_best(score_level<kK1 / kThreads>(kp, w, b, e, Rij, kK1, H, Q, nullptr, resident, a_s), red);
    if (c.e < best_e) {
      best_e = c.e;
      lattice_point(c.k, kK1, H, Q, t);
    }
    spacing = sqrtf(2.f * 3.14159265358979f * H / kK1);
  }
  // sign by cheirality
  int cp = 0, cm = 0;
  const float tm[3] = {-t[0], -t[1], -t[2]};
  for (int m = b + threadIdx.x; m < e; m += kThreads) {
    if (w && !(w[m] > 0.f)) continue;
    const float4 x = kp[m];
    cp += positive_depths(x, Rij, t);
    cm += positive_depths(x, Rij, tm);
  }
  for (int d = 16; d > 0; d >>= 1) {
    cp += __shfl_xor_sync(0xffffffffu, cp, d);
    cm += __shfl_xor_sync(0xffffffffu, cm, d);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    cnt_s[0][threadIdx.x >> 5] = cp;
    cnt_s[1][threadIdx.x >> 5] = cm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int P = 0, M = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
      P += cnt_s[0][w];
      M += cnt_s[1][w];
    }
    const float sg = (M > P) ? -1.f : 1.f;
    const float nn = sqrtf(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    for (int k = 0; k < 3; ++k) rel_t[3 * n + k] = sg * t[k] / nn;
    if (err_out) err_out[n] = best_e / (float)count;
  }
}

// the hemisphere's kK0 points, as score_level forms them on the fly
__global__ void k_lattice0(float4* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kK0) return;
  const float I3[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
  float t[3];
  lattice_point(k, kK0, 1.f, I3, t);
  out[k] = make_float4(t[0], t[1], t[2], 0.f);
}

}  // namespace

int reltrans_lattice_points() { return kK0; }

void launch_reltrans_lattice(float4* lat0, cudaStream_t s) { k_lattice0<<<kK0 / 256, 256, 0, s>>>(lat0); }

void launch_reltrans(const fm_problem* pr, const float* rot6, float* rel_t, float* err_out, cudaStream_t s) {
  if (pr->P <= 0) return;
  k_reltrans<<<pr->P, kThreads, 0, s>>>(pr->kp, pr->seg_off, pr->pair_i, pr->pair_j, rot6, pr->ea_w, pr->lattice0,
                                        rel_t, err_out);
}

}  // namespace fm
