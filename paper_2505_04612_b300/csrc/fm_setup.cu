// Problem build (run once by fm_problem_create): keypoint calibration,
// image-pair offsets and the tables of the direct epipolar kernel.
#include "fm_internal.h"

namespace fm {
namespace {

__device__ __forceinline__ bool finitef(float x) { return isfinite(x); }

// x~ = K^-1 [u, v, 1]^T with the principal point (cx, cy) (Sec. 3.1, camera
// assumptions; Sec. 3.3, normalised homogeneous coordinates with z = 1).
__global__ void k_calibrate(const float* __restrict__ kp1, const float* __restrict__ kp2,
                            const int* __restrict__ kp_pair, const int* __restrict__ pi,
                            const int* __restrict__ pj, const float* __restrict__ f,
                            const float* __restrict__ cx, const float* __restrict__ cy,
                            int64_t Z, int P, float4* __restrict__ out, int* err) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < Z;
       m += (int64_t)gridDim.x * blockDim.x) {
    int n = kp_pair[m];
    if (n < 0 || n >= P) {
      atomicOr(err, kErrKpRange);
      out[m] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    int i = pi[n], j = pj[n];
    float u1 = kp1[2 * m], v1 = kp1[2 * m + 1];
    float u2 = kp2[2 * m], v2 = kp2[2 * m + 1];
    if (!(finitef(u1) && finitef(v1) && finitef(u2) && finitef(v2))) atomicOr(err, kErrKpNonFinite);
    out[m] = make_float4((u1 - cx[i]) / f[i], (v1 - cy[i]) / f[i], (u2 - cx[j]) / f[j],
                         (v2 - cy[j]) / f[j]);
  }
}

// The order of the caller's keypoint pairs: flags[0] gets 1 when an image
// pair index lies outside [0, P), 2 when the pairs are not in (image pair,
// track) order (track compared only when given), 4 when a track is negative;
// flags[1] the largest track.
__global__ void k_kp_order_check(const int* __restrict__ kpp, const int* __restrict__ track, int64_t Z, int P,
                                 int* flags) {
  int bits = 0, tmax = 0;
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < Z; m += (int64_t)gridDim.x * blockDim.x) {
    const int n = kpp[m];
    if (n < 0 || n >= P) bits |= 1;
    const int t = track ? track[m] : 0;
    if (t < 0) bits |= 4;
    tmax = max(tmax, t);
    if (m > 0) {
      const int n0 = kpp[m - 1];
      if (n < n0 || (track && n == n0 && t < track[m - 1])) bits |= 2;
    }
  }
  bits = __reduce_or_sync(0xffffffffu, bits);
  tmax = __reduce_max_sync(0xffffffffu, tmax);
  if ((threadIdx.x & 31) == 0) {
    if (bits) atomicOr(flags, bits);
    if (track) atomicMax(flags + 1, tmax);
  }
}

// the caller's keypoint-pair inputs in the order perm (position k takes input
// perm[k]); track may be null
__global__ void k_kp_gather(const uint32_t* __restrict__ perm, int64_t Z, const float2* __restrict__ kp1,
                            const float2* __restrict__ kp2, const int* __restrict__ kpp, const int* __restrict__ track,
                            float2* __restrict__ o1, float2* __restrict__ o2, int* __restrict__ okpp,
                            int* __restrict__ otrack) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Z; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t m = perm[k];
    o1[k] = kp1[m];
    o2[k] = kp2[m];
    okpp[k] = kpp[m];
    if (track) otrack[k] = track[m];
  }
}

// per-pair values between the caller's order and the internal one:
// to_internal: out[k] = in[perm[k]]; else out[perm[k]] = in[k]
__global__ void k_permute(const float* __restrict__ in, const uint32_t* __restrict__ perm, int64_t Z, int to_internal,
                          float* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Z; k += (int64_t)gridDim.x * blockDim.x) {
    if (to_internal) out[k] = in[perm[k]];
    else out[perm[k]] = in[k];
  }
}

// seg_off[n] = index of the first keypoint pair of image pair n (CSR); the
// keypoint pairs are grouped by image pair in index order (sorted at
// creation when the caller's are not).
__global__ void k_seg_offsets(const int* __restrict__ kp_pair, int64_t Z, int P,
                              int* __restrict__ seg_off, int* err) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < Z;
       m += (int64_t)gridDim.x * blockDim.x) {
    int n = min(max(kp_pair[m], 0), P - 1);
    int prev = (m == 0) ? -1 : min(max(kp_pair[m - 1], 0), P - 1);
    if (m > 0 && kp_pair[m] < kp_pair[m - 1]) atomicOr(err, kErrKpOrder);
    for (int s = prev + 1; s <= n; ++s) seg_off[s] = (int)m;
    if (m == Z - 1)
      for (int s = n + 1; s <= P; ++s) seg_off[s] = (int)Z;
  }
}

// ---- lane tables of the direct kernel
// Image pair n (m_n keypoint pairs) gets L_n = max(1, ceil(m_n / U)) lanes;
// lane j of n holds pairs [seg_off[n] + j U, min(seg_off[n] + (j + 1) U,
// seg_off[n + 1])).  G = exclusive scan of L orders all lanes; warp run w is
// lanes [32 w, 32 w + 32).  A lane never crosses an image-pair end, so the
// direct kernel needs no per-pair selection of E; an empty image pair keeps
// one lane (with no pairs) so that a warp run spans at most 32 image pairs.

__device__ __forceinline__ int lanes_of(const int* __restrict__ seg_off, int n, int U) {
  const int m = seg_off[n + 1] - seg_off[n];
  return m > 0 ? (m + U - 1) / U : 1;
}

// G[n] = sum_{n' < n} L_n' for n in [0, P]; *T = G[P].  One CTA, fixed order.
// With err != null the offsets are validated first; a bad table gives no
// lanes at all (G = 0, T = 0) and the error bit kErrSegOff.
__global__ void __launch_bounds__(1024) k_scan_lanes(const int* __restrict__ seg_off, int P, int U,
                                                     int* __restrict__ G, int* __restrict__ T, long long Z,
                                                     int* err) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (P + 1023) / 1024;
  const int b = min(t * per, P), e = min(b + per, P);
  if (err) {
    bool bad = (t == 0) && (seg_off[0] != 0 || (long long)seg_off[P] != Z);
    for (int n = b; n < e; ++n) bad |= seg_off[n + 1] < seg_off[n];
    if (__syncthreads_or(bad)) {
      for (int n = t; n <= P; n += 1024) G[n] = 0;
      if (t == 0) {
        *T = 0;
        atomicOr(err, kErrSegOff);
      }
      return;
    }
  }
  int s = 0;
  for (int n = b; n < e; ++n) s += lanes_of(seg_off, n, U);
  part[t] = s;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    const int v = (t >= d) ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = (t == 0) ? 0 : part[t - 1];
  for (int n = b; n < e; ++n) {
    G[n] = run;
    run += lanes_of(seg_off, n, U);
  }
  if (t == 1023) {
    G[P] = part[1023];
    *T = part[1023];
  }
}

// one thread per lane slot g of n_slots = 32 n_runs (a warp is a warp run):
// desc[g] = offset | count << 10 | key << 15 with offset the lane's first
// pair relative to the run's first pair, count <= U its pairs, key its image
// pair relative to the run's first one; info[w] = {first image pair,
// n_img | len << 8, record base (filled by k_scan_info), first pair}.  Slots
// at or past T (the lanes in use) copy the last lane in use with count 0;
// a run with no lane in use gets n_img = 0.
__global__ void k_lane_desc(const int* __restrict__ seg_off, const int* __restrict__ G,
                            const int* __restrict__ T_dev, int P, int U, int n_slots, int* __restrict__ desc,
                            int4* __restrict__ info) {
  const unsigned FULL = 0xffffffffu;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;   // blockDim and n_slots are multiples of 32
  const int lane = threadIdx.x & 31;
  if (g - lane >= n_slots) return;                     // whole warp out of range
  const int T = *T_dev;
  const bool used = g < T;
  const int gg = used ? g : T - 1;
  int lo = 0, hi = P - 1;                                // largest n with G[n] <= gg
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (G[mid] <= gg) lo = mid; else hi = mid - 1;
  }
  const int n = lo;
  const int start = seg_off[n] + (gg - G[n]) * U;
  const int cnt = used ? min(U, seg_off[n + 1] - start) : 0;
  const int base = __shfl_sync(FULL, start, 0);
  const int s0 = __shfl_sync(FULL, n, 0);
  const int key = n - s0;
  desc[g] = (start - base) | (cnt << kDescCntShift) | (key << kDescKeyShift);
  int end = used ? start + cnt - base : 0;
  for (int d = 16; d > 0; d >>= 1) end = max(end, __shfl_xor_sync(FULL, end, d));
  const int n_img = __any_sync(FULL, used) ? __shfl_sync(FULL, key, 31) + 1 : 0;
  if (lane == 0) info[g >> 5] = make_int4(s0, n_img | (end << 8), 0, base);
}

// exclusive scan of the runs' image-pair counts (info[].y & 0xff) into
// info[].z, one CTA, fixed order; *total = the number of records
__global__ void k_scan_info(int4* info, int n, long long* total) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int b = min(t * per, n), e = min(b + per, n);
  long long s = 0;
  for (int k = b; k < e; ++k) s += info[k].y & 0xff;
  part[t] = s;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    long long v = (t >= d) ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  long long run = (t == 0) ? 0 : part[t - 1];
  for (int k = b; k < e; ++k) {
    int4 v = info[k];
    v.z = (int)run;
    run += v.y & 0xff;
    info[k] = v;
  }
  if (t == 1023) *total = part[1023];
}

// seg_rec[n] = {first record of image pair n, number of records}: one per
// warp run its lanes fall in, consecutive in record order
__global__ void k_seg_records(const int* __restrict__ seg_off, const int* __restrict__ G,
                              const int4* __restrict__ info, int P, int* __restrict__ seg_rec) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= P) return;
  if (seg_off[n] == seg_off[n + 1] || G[n + 1] <= G[n]) {   // no pairs, or no lanes (rejected table)
    seg_rec[2 * n] = 0;
    seg_rec[2 * n + 1] = 0;
    return;
  }
  const int w0 = G[n] >> 5, w1 = (G[n + 1] - 1) >> 5;
  const int4 i0 = info[w0];
  seg_rec[2 * n] = i0.z + (n - i0.x);
  seg_rec[2 * n + 1] = w1 - w0 + 1;
}

// reads n16 16-byte words (an L2 sweep after a memset, so that the cache
// holds clean lines); the store never happens for a buffer set by memset
__global__ void k_l2_sweep(const uint4* __restrict__ p, int64_t n16, unsigned marker) {
  unsigned acc = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n16; k += (int64_t)gridDim.x * blockDim.x) {
    const uint4 v = p[k];
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == marker) const_cast<uint4*>(p)[0].x = acc;
}

__global__ void k_check_finite(const float* __restrict__ x, int64_t n, int* err, int bit) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[k])) atomicOr(err, bit);
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 148 * 64) g = 148 * 64;
  return (int)g;
}

}  // namespace

void launch_calibrate(const float* kp1, const float* kp2, const int* kp_pair, const int* pi,
                      const int* pj, const float* f, const float* cx, const float* cy,
                      int64_t Z, int P, float4* out, int* err, cudaStream_t s) {
  if (Z == 0) return;
  k_calibrate<<<grid_for(Z, 256), 256, 0, s>>>(kp1, kp2, kp_pair, pi, pj, f, cx, cy, Z, P,
                                                out, err);
}

void launch_seg_offsets(const int* kp_pair, int64_t Z, int P, int* seg_off, int* err,
                        cudaStream_t s) {
  if (Z == 0) {
    cudaMemsetAsync(seg_off, 0, sizeof(int) * (P + 1), s);
    return;
  }
  k_seg_offsets<<<grid_for(Z, 256), 256, 0, s>>>(kp_pair, Z, P, seg_off, err);
}

void launch_kp_order_check(const int* kpp, const int* track, int64_t Z, int P, int* flags, cudaStream_t s) {
  if (Z == 0) return;
  k_kp_order_check<<<grid_for(Z, 256), 256, 0, s>>>(kpp, track, Z, P, flags);
}

void launch_kp_gather(const uint32_t* perm, int64_t Z, const float* kp1, const float* kp2, const int* kpp,
                      const int* track, float* o1, float* o2, int* okpp, int* otrack, cudaStream_t s) {
  if (Z == 0) return;
  k_kp_gather<<<grid_for(Z, 256), 256, 0, s>>>(perm, Z, reinterpret_cast<const float2*>(kp1),
                                               reinterpret_cast<const float2*>(kp2), kpp, track,
                                               reinterpret_cast<float2*>(o1), reinterpret_cast<float2*>(o2), okpp,
                                               otrack);
}

void launch_permute(const float* in, const uint32_t* perm, int64_t Z, bool to_internal, float* out, cudaStream_t s) {
  if (Z == 0) return;
  k_permute<<<grid_for(Z, 256), 256, 0, s>>>(in, perm, Z, to_internal ? 1 : 0, out);
}

void launch_lane_scan(const int* seg_off, int P, int U, int* G, int* T, cudaStream_t s, int64_t Z, int* err) {
  k_scan_lanes<<<1, 1024, 0, s>>>(seg_off, P, U, G, T, (long long)Z, err);
}

void launch_lane_desc(const int* seg_off, const int* G, const int* T, int P, int U, int n_runs, int* desc,
                      int4* wrun_info, cudaStream_t s) {
  if (n_runs == 0) return;
  const int n = 32 * n_runs;
  k_lane_desc<<<(n + 255) / 256, 256, 0, s>>>(seg_off, G, T, P, U, n, desc, wrun_info);
}

void launch_exclusive_scan_info(int4* wrun_info, int n, int64_t* total_out_dev, cudaStream_t s) {
  k_scan_info<<<1, 1024, 0, s>>>(wrun_info, n, (long long*)total_out_dev);
}

void launch_seg_records(const int* seg_off, const int* G, const int4* wrun_info, int P, int* seg_rec,
                        cudaStream_t s) {
  if (P == 0) return;
  k_seg_records<<<(P + 255) / 256, 256, 0, s>>>(seg_off, G, wrun_info, P, seg_rec);
}

// one thread idles for about ns nanoseconds (bounded: __nanosleep steps of
// at most 1 us, ns / 1000 + 1 of them)
__global__ void k_idle(unsigned ns) {
  for (unsigned k = 0; k <= ns / 1000u; ++k) __nanosleep(1000u);
}

void launch_idle(unsigned ns, cudaStream_t s) { k_idle<<<1, 1, 0, s>>>(ns); }

void launch_l2_flush(void* buf, size_t bytes, int fill, cudaStream_t s) {
  cudaMemsetAsync(buf, fill, bytes, s);
  // every byte equals fill: an even number of equal words xors to 0, never to 1
  k_l2_sweep<<<148 * 8, 256, 0, s>>>(static_cast<const uint4*>(buf), (int64_t)(bytes / 16) & ~int64_t(1), 1u);
}

void launch_check_finite(const float* x, int64_t n, int* err, int bit, cudaStream_t s) {
  if (n == 0) return;
  k_check_finite<<<grid_for(n, 256), 256, 0, s>>>(x, n, err, bit);
}

}  // namespace fm
