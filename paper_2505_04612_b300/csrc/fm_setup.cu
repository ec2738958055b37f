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

// seg_off[n] = index of the first keypoint pair of image pair n (CSR); the
// keypoint pairs must be grouped by image pair in index order.
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

// largest s in [0, P) with seg_off[s] <= p (the image pair holding pair p)
__device__ __forceinline__ int segment_of(const int* __restrict__ seg_off, int P, int p) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (seg_off[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_run_tables(const int* __restrict__ seg_off, int P, int Z, int n_wruns, int U,
                             int* __restrict__ run_seg, int4* __restrict__ info) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_wruns * 32) return;
  int p0 = min(q * U, Z - 1);
  int s = segment_of(seg_off, P, p0);
  run_seg[q] = s;
  if ((q & 31) == 0) {
    int w = q >> 5;
    int last = min((w + 1) * 32 * U, Z) - 1;
    int sl = segment_of(seg_off, P, last);
    info[w] = make_int4(s, sl - s + 1, 0, 0);
  }
}

// exclusive scan of info[].y into info[].z, one CTA, fixed order
__global__ void k_scan_info(int4* info, int n, long long* total) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int b = t * per, e = min(b + per, n);
  long long s = 0;
  for (int k = b; k < e; ++k) s += info[k].y;
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
    run += v.y;
    info[k] = v;
  }
  if (t == 1023) *total = part[1023];
}

__global__ void k_seg_records(const int* __restrict__ seg_off, const int* __restrict__ run_seg,
                              const int4* __restrict__ info, int P, int WP, int* __restrict__ seg_rec) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= P) return;
  int b = seg_off[n], e = seg_off[n + 1];
  if (b == e) {
    seg_rec[2 * n] = 0;
    seg_rec[2 * n + 1] = 0;
    return;
  }
  int w0 = b / WP, w1 = (e - 1) / WP;
  int4 i0 = info[w0];
  seg_rec[2 * n] = i0.z + (n - i0.x);
  seg_rec[2 * n + 1] = w1 - w0 + 1;
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

void launch_run_tables(const int* seg_off, int P, int64_t Z, int n_wruns, int U, int* run_seg,
                       int4* wrun_info, cudaStream_t s) {
  if (n_wruns == 0) return;
  int n = n_wruns * 32;
  k_run_tables<<<(n + 255) / 256, 256, 0, s>>>(seg_off, P, (int)Z, n_wruns, U, run_seg, wrun_info);
}

void launch_exclusive_scan_info(int4* wrun_info, int n, int64_t* total_out_dev, cudaStream_t s) {
  k_scan_info<<<1, 1024, 0, s>>>(wrun_info, n, (long long*)total_out_dev);
}

void launch_seg_records(const int* seg_off, const int* run_seg, const int4* wrun_info, int P, int U,
                        int* seg_rec, cudaStream_t s) {
  k_seg_records<<<(P + 255) / 256, 256, 0, s>>>(seg_off, run_seg, wrun_info, P, 32 * U, seg_rec);
}

void launch_check_finite(const float* x, int64_t n, int* err, int bit, cudaStream_t s) {
  if (n == 0) return;
  k_check_finite<<<grid_for(n, 256), 256, 0, s>>>(x, n, err, bit);
}

}  // namespace fm
