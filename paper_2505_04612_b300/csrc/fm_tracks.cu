// Track completion (Appendix "Tracks"): keypoints are the nodes of a graph
// whose edges are raw matches; a track is a connected component; every
// consistent track (at most one keypoint per image) becomes all pairwise
// combinations of its keypoints, an inconsistent one keeps its raw matches.
//
// Steps, all on the device:
//   1. union-find over the matches: lock-free, every link puts the larger
//      root under the smaller (atomicCAS on the root), finds halve paths with
//      atomicMin; each component's final root is its smallest keypoint id,
//      whatever the order of the links, so the labels are deterministic;
//   2. component sizes (atomics: counts are order-free), keypoints sorted by
//      label (stable LSD radix sort: within a component by keypoint id, hence
//      by image), consistency from adjacent members, track numbers by label;
//   3. emission in a canonical order: the consistent tracks' pairs by track
//      and member positions, then the inconsistent tracks' raw matches in
//      input order, each with its image-pair key i * N + j;
//   4. a stable radix sort by key groups the pairs by image pair without
//      disturbing the canonical order inside one; image pairs from the key
//      changes, optional removal of image pairs with too few pairs.
// Scans and sorts are multi-CTA and fixed-order (deterministic).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "fm_internal.h"

struct fm_tracks {
  int64_t n_tracks = 0, n_inconsistent = 0, P = 0, Z = 0;
  int* pair_i = nullptr;
  int* pair_j = nullptr;
  int* kp_img_pair = nullptr;
  int* node1 = nullptr;
  int* node2 = nullptr;
  int* track = nullptr;
  float2* px1 = nullptr;
  float2* px2 = nullptr;
  cudaStream_t stream = nullptr;   // the results' stream (allocation, copies, release)
};

namespace fm {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;   // 2048 elements per CTA in scans and sorts
// steps of one find / retries of one union at most: parent pointers only
// decrease, so a find ends within K steps and a union's retries (each one a
// root linked by another thread) are bounded by K as well
__host__ __device__ constexpr int64_t uf_bound(int K) { return 2 * (int64_t)K + 64; }

enum : int { kTrkBadMatch = 1, kTrkUfBound = 2 };

// ------------------------------------------------------------------ scans

template <typename T>
__global__ void __launch_bounds__(kThreads) k_tile_sums(const T* __restrict__ in, int64_t n, T* __restrict__ sums) {
  __shared__ T part[kThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  T s = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int64_t k = base + i * kThreads + threadIdx.x;
    if (k < n) s += in[k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = 0;
    for (int w = 0; w < kThreads / 32; ++w) t += part[w];
    sums[blockIdx.x] = t;
  }
}

// exclusive scan of nb block sums in place (one CTA, chunks in order), total
// -> *total
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_sums(T* __restrict__ a, int nb, T* __restrict__ total) {
  __shared__ T part[1024];
  const int t = threadIdx.x;
  const int per = (nb + 1023) / 1024;
  const int b = min(t * per, nb), e = min(b + per, nb);
  T s = 0;
  for (int k = b; k < e; ++k) s += a[k];
  part[t] = s;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    const T v = (t >= d) ? part[t - d] : (T)0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  T run = (t == 0) ? (T)0 : part[t - 1];
  for (int k = b; k < e; ++k) {
    const T v = a[k];
    a[k] = run;
    run += v;
  }
  if (t == 1023 && total) *total = part[1023];
}

// out = exclusive scan of in, tile by tile from the scanned tile sums (in may
// alias out)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_tile_scan(const T* in, T* out, int64_t n, const T* __restrict__ sums) {
  __shared__ T tile[kTile];
  __shared__ T wsum[kThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int64_t k = base + i * kThreads + threadIdx.x;
    tile[i * kThreads + threadIdx.x] = k < n ? in[k] : (T)0;
  }
  __syncthreads();
  T v[kItems];
  T s = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    v[i] = tile[threadIdx.x * kItems + i];
    s += v[i];
  }
  // inclusive scan of the thread totals: warp shuffles, then the warps in order
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  T woff = 0;
  for (int k = 0; k < w; ++k) woff += wsum[k];
  T run = sums[blockIdx.x] + woff + inc - s;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    tile[threadIdx.x * kItems + i] = run;
    run += v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int64_t k = base + i * kThreads + threadIdx.x;
    if (k < n) out[k] = tile[i * kThreads + threadIdx.x];
  }
}

// ------------------------------------------------------------- radix sort

__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                         int nblk, int* __restrict__ hist) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int64_t k = base + i * kThreads + threadIdx.x;
    if (k < n) atomicAdd(&cnt[(keys[k] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one 8-bit digit.  Warp w of the CTA owns elements
// [tile + 256 w, tile + 256 (w + 1)) in 8 rounds of 32; ranks among equal
// digits come from __match_any_sync in lane order, so the output keeps the
// input order of equal digits.  The tile is first ordered by digit in shared
// memory, then written with consecutive threads on consecutive elements, so
// that equal digits go out as contiguous runs (coalesced stores).
__global__ void __launch_bounds__(kThreads) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                            const uint32_t* __restrict__ vin,
                                                            uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                            int64_t n, int shift, int nblk,
                                                            const int* __restrict__ hist) {
  __shared__ int woff[kThreads / 32][256];
  __shared__ int tile_off[256];   // first position of each digit inside the ordered tile
  __shared__ int gbase[256];      // first global position of each digit of this tile
  __shared__ int wsum[kThreads / 32];
  __shared__ uint32_t sk[kTile], sv[kTile];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = lane; d < 256; d += 32) woff[w][d] = 0;
  __syncwarp();
  const int64_t tile = (int64_t)blockIdx.x * kTile;
  const int64_t base = tile + (int64_t)w * 256;
  const unsigned lt = (1u << lane) - 1u;
  // per-warp digit counts
  for (int r = 0; r < 8; ++r) {
    const int64_t k = base + r * 32 + lane;
    const bool ok = k < n;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const unsigned d = (kin[k] >> shift) & 255u;
      const unsigned peers = __match_any_sync(act, d);
      if ((peers & lt) == 0) woff[w][d] += __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  // per digit (one thread each): the warps' exclusive offsets inside the
  // digit, the digit's count, and an exclusive scan of the counts over the
  // digits (warp shuffles, then the warps in order)
  {
    const int d = threadIdx.x;   // kThreads == 256 digits
    gbase[d] = hist[(size_t)d * nblk + blockIdx.x];
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < kThreads / 32; ++k) {
      const int c = woff[k][d];
      woff[k][d] = cnt;
      cnt += c;
    }
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int off = inc - cnt;
    for (int k = 0; k < w; ++k) off += wsum[k];
    tile_off[d] = off;
#pragma unroll
    for (int k = 0; k < kThreads / 32; ++k) woff[k][d] += off;
  }
  __syncthreads();
  // ordered tile in shared memory
  for (int r = 0; r < 8; ++r) {
    const int64_t k = base + r * 32 + lane;
    const bool ok = k < n;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const uint32_t key = kin[k];
      const unsigned d = (key >> shift) & 255u;
      const unsigned peers = __match_any_sync(act, d);
      const int pos = woff[w][d] + __popc(peers & lt);
      sk[pos] = key;
      sv[pos] = vin[k];
      __syncwarp(act);
      if ((peers & lt) == 0) woff[w][d] += __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  // coalesced write: element j of the ordered tile goes to its digit's global
  // start plus its position inside the digit's run
  const int valid = (n - tile < kTile) ? (int)(n - tile) : kTile;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int j = i * kThreads + threadIdx.x;
    if (j < valid) {
      const uint32_t key = sk[j];
      const unsigned d = (key >> shift) & 255u;
      const int pos = gbase[d] + (j - tile_off[d]);
      kout[pos] = key;
      vout[pos] = sv[j];
    }
  }
}

// ------------------------------------------------------------- union-find

__device__ __forceinline__ int ld_parent(const int* p, int x) { return *((volatile const int*)(p + x)); }

__device__ __forceinline__ int find_root(int* parent, int x, int K, int* err) {
  const int64_t bound = uf_bound(K);
  for (int64_t it = 0; it < bound; ++it) {
    const int p = ld_parent(parent, x);
    if (p == x) return x;
    const int gp = ld_parent(parent, p);
    if (gp != p) atomicMin(parent + x, gp);   // pointers only move to ancestors (smaller ids)
    x = gp;
  }
  atomicOr(err, kTrkUfBound);
  return x;
}

__global__ void k_node_image(const int* __restrict__ kp_off, int N, int K, int* __restrict__ img,
                             int* __restrict__ parent) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < K; v += gridDim.x * blockDim.x) {
    int lo = 0, hi = N;   // the image c with kp_off[c] <= v < kp_off[c + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (kp_off[mid] <= v) lo = mid;
      else hi = mid;
    }
    img[v] = lo;
    parent[v] = v;
  }
}

__global__ void k_union(const int2* __restrict__ matches, int64_t M, int K, const int* __restrict__ img,
                        int* parent, int* err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < M; e += (int64_t)gridDim.x * blockDim.x) {
    const int2 m = matches[e];
    if (m.x < 0 || m.x >= K || m.y < 0 || m.y >= K || img[m.x] == img[m.y]) {
      atomicOr(err, kTrkBadMatch);
      continue;
    }
    const int64_t bound = uf_bound(K);
    int64_t it = 0;
    for (; it < bound; ++it) {
      const int ru = find_root(parent, m.x, K, err), rv = find_root(parent, m.y, K, err);
      if (ru == rv) break;
      const int hi = max(ru, rv), lo = min(ru, rv);
      if (atomicCAS(parent + hi, hi, lo) == hi) break;   // else hi was linked meanwhile: retry
    }
    if (it == bound) atomicOr(err, kTrkUfBound);
  }
}

__global__ void k_label(int* parent, int K, int* __restrict__ label, int* __restrict__ size, int* err) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < K; v += gridDim.x * blockDim.x) {
    const int r = find_root(parent, v, K, err);
    label[v] = r;
    atomicAdd(size + r, 1);
  }
}

// --------------------------------------------------------------- tracks

// after the sort by label: members of a component are contiguous, in
// increasing keypoint id (hence image); start of every component and the
// consistency flag (two members in one image)
__global__ void k_members(const uint32_t* __restrict__ slabel, const uint32_t* __restrict__ snode, int K,
                          const int* __restrict__ img, int* __restrict__ start, int* __restrict__ bad) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < K; s += gridDim.x * blockDim.x) {
    const int r = (int)slabel[s];
    if (s == 0 || (int)slabel[s - 1] != r) {
      start[r] = s;
    } else if (img[snode[s]] == img[snode[s - 1]]) {
      bad[r] = 1;
    }
  }
}

// per keypoint v: is_track (a root of a component of >= 2), emitted pairs of
// its track when consistent (64-bit)
__global__ void k_track_flags(const int* __restrict__ label, const int* __restrict__ size, const int* __restrict__ bad,
                              int K, int* __restrict__ is_track, long long* __restrict__ n_emit) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < K; v += gridDim.x * blockDim.x) {
    const bool root = label[v] == v && size[v] >= 2;
    is_track[v] = root ? 1 : 0;
    const long long k = size[v];
    n_emit[v] = (root && !bad[v]) ? k * (k - 1) / 2 : 0;
  }
}

// pairs of the consistent tracks: member p of a track of k emits (p, q) for
// q > p at the track's offset + p k - p (p + 1) / 2 + (q - p - 1)
__global__ void k_emit_tracks(const uint32_t* __restrict__ slabel, const uint32_t* __restrict__ snode, int K,
                              const int* __restrict__ start, const int* __restrict__ size,
                              const int* __restrict__ bad, const int* __restrict__ tid,
                              const long long* __restrict__ off, const int* __restrict__ img, int N,
                              uint32_t* __restrict__ key, int* __restrict__ n1, int* __restrict__ n2,
                              int* __restrict__ trk) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < K; s += gridDim.x * blockDim.x) {
    const int r = (int)slabel[s];
    const int k = size[r];
    if (k < 2 || bad[r]) continue;
    const int st = start[r], p = s - st;
    const int v = (int)snode[s];
    const long long b = off[r] + (long long)p * k - (long long)p * (p + 1) / 2;
    const uint32_t ki = (uint32_t)img[v] * (uint32_t)N;
    const int t = tid[r];
    for (int q = p + 1; q < k; ++q) {
      const long long e = b + (q - p - 1);
      const int u = (int)snode[st + q];
      key[e] = ki + (uint32_t)img[u];
      n1[e] = v;
      n2[e] = u;
      trk[e] = t;
    }
  }
}

// a match k_union accepted (both keypoints in [0, K), two images); the others
// are flagged there and must not be dereferenced here either
__device__ __forceinline__ bool valid_match(int2 m, int K, const int* __restrict__ img) {
  return m.x >= 0 && m.x < K && m.y >= 0 && m.y < K && img[m.x] != img[m.y];
}

__global__ void k_raw_flags(const int2* __restrict__ matches, int64_t M, int K, const int* __restrict__ img,
                            const int* __restrict__ label, const int* __restrict__ bad,
                            long long* __restrict__ flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < M; e += (int64_t)gridDim.x * blockDim.x) {
    const int2 m = matches[e];
    flag[e] = (valid_match(m, K, img) && bad[label[m.x]]) ? 1 : 0;
  }
}

// raw matches of inconsistent tracks, in input order, after the Z1 pairs of
// the consistent tracks, oriented from the lower image
__global__ void k_emit_raw(const int2* __restrict__ matches, int64_t M, int K, const int* __restrict__ label,
                           const int* __restrict__ bad, const long long* __restrict__ pos, long long Z1,
                           const int* __restrict__ tid, const int* __restrict__ img, int N,
                           uint32_t* __restrict__ key, int* __restrict__ n1, int* __restrict__ n2,
                           int* __restrict__ trk) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < M; e += (int64_t)gridDim.x * blockDim.x) {
    const int2 m = matches[e];
    if (!valid_match(m, K, img)) continue;
    const int r = label[m.x];
    if (!bad[r]) continue;
    const long long z = Z1 + pos[e];
    const bool sw = img[m.x] > img[m.y];
    const int a = sw ? m.y : m.x, b = sw ? m.x : m.y;
    key[z] = (uint32_t)img[a] * (uint32_t)N + (uint32_t)img[b];
    n1[z] = a;
    n2[z] = b;
    trk[z] = tid[r];
  }
}

__global__ void k_iota(uint32_t* __restrict__ a, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    a[k] = (uint32_t)k;
}

// heads of the image-pair runs of the sorted keys
__global__ void k_heads(const uint32_t* __restrict__ key, int64_t Z, int* __restrict__ head) {
  for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < Z; z += (int64_t)gridDim.x * blockDim.x)
    head[z] = (z == 0 || key[z] != key[z - 1]) ? 1 : 0;
}

// image pair of every sorted pair (inclusive count of heads - 1), the image
// pairs' keys and starts
__global__ void k_pairs(const uint32_t* __restrict__ key, const int* __restrict__ head, const int* __restrict__ hscan,
                        int64_t Z, int N, int* __restrict__ ipair, int* __restrict__ pi, int* __restrict__ pj,
                        int* __restrict__ pstart) {
  for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < Z; z += (int64_t)gridDim.x * blockDim.x) {
    const int p = hscan[z] + head[z] - 1;
    ipair[z] = p;
    if (head[z]) {
      pi[p] = (int)(key[z] / (uint32_t)N);
      pj[p] = (int)(key[z] % (uint32_t)N);
      pstart[p] = (int)z;
    }
  }
}

// keep[p] for p < Pmax: 1 for image pairs with >= min_pairs keypoint pairs;
// 0 past the image-pair count *P_dev (read on the device: no host round trip)
__global__ void k_pair_keep(const int* __restrict__ pstart, const int* __restrict__ P_dev, int Pmax, int64_t Z,
                            int min_pairs, int* __restrict__ keep) {
  const int P = *P_dev;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < Pmax; p += gridDim.x * blockDim.x) {
    if (p >= P) {
      keep[p] = 0;
      continue;
    }
    const int64_t e = p + 1 < P ? pstart[p + 1] : Z;
    keep[p] = (e - pstart[p] >= min_pairs) ? 1 : 0;
  }
}

// final outputs: sorted pair z goes to zpos[z] (its image pair kept) as image
// pair ppos[ipair[z]]
__global__ void k_gather(const uint32_t* __restrict__ perm, const int* __restrict__ ipair, int64_t Z,
                         const int* __restrict__ pkeep, const int* __restrict__ ppos, const long long* __restrict__ zpos,
                         const int* __restrict__ n1, const int* __restrict__ n2, const int* __restrict__ trk,
                         const float2* __restrict__ px, int* __restrict__ o_ip, int* __restrict__ o_n1,
                         int* __restrict__ o_n2, int* __restrict__ o_t, float2* __restrict__ o_px1,
                         float2* __restrict__ o_px2) {
  for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < Z; z += (int64_t)gridDim.x * blockDim.x) {
    const int p = ipair[z];
    if (pkeep && !pkeep[p]) continue;
    const int64_t o = zpos ? zpos[z] : z;
    const uint32_t e = perm[z];
    const int a = n1[e], b = n2[e];
    o_ip[o] = ppos ? ppos[p] : p;
    o_n1[o] = a;
    o_n2[o] = b;
    o_t[o] = trk[e];
    if (px) {
      o_px1[o] = px[a];
      o_px2[o] = px[b];
    }
  }
}

// the kept image pairs (all of them when keep is null) of the *P_dev found
__global__ void k_pair_compact(const int* __restrict__ pi, const int* __restrict__ pj, const int* __restrict__ keep,
                               const int* __restrict__ pos, const int* __restrict__ P_dev, int* __restrict__ o_pi,
                               int* __restrict__ o_pj) {
  const int P = *P_dev;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
    if (!keep || keep[p]) {
      const int q = keep ? pos[p] : p;
      o_pi[q] = pi[p];
      o_pj[q] = pj[p];
    }
}

__global__ void k_keep_flags(const int* __restrict__ ipair, const int* __restrict__ pkeep, int64_t Z,
                             long long* __restrict__ f) {
  for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < Z; z += (int64_t)gridDim.x * blockDim.x)
    f[z] = pkeep[ipair[z]];
}

// ------------------------------------------------------------------ host

int grid_for(int64_t n, int threads = 256) {
  const int64_t g = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 148 * 64));
}

// Stream-ordered memory pools of the track completion and the device sorts,
// one per device, owned by the library and kept for the process (their
// memory is reused from call to call instead of being mapped and unmapped
// with cudaMalloc / cudaFree, whose frees synchronise the device).
cudaMemPool_t tracks_pool() {
  constexpr int kDevices = 64;
  static std::mutex mu;
  static cudaMemPool_t pools[kDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPool_t p = nullptr;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

// scratch of one call: pool allocations on the call's stream, returned to
// the pool (stream-ordered) when the call ends
struct Buffers {
  cudaStream_t s;
  std::vector<void*> ptrs;
  cudaError_t ce = cudaSuccess;
  explicit Buffers(cudaStream_t st) : s(st) {
    if (!tracks_pool()) ce = cudaErrorMemoryAllocation;
  }
  template <typename T>
  T* get(size_t n) {
    void* q = nullptr;
    if (ce == cudaSuccess) ce = cudaMallocFromPoolAsync(&q, std::max<size_t>(n * sizeof(T), 16), tracks_pool(), s);
    if (ce == cudaSuccess) ptrs.push_back(q);
    return (T*)q;
  }
  ~Buffers() {
    for (void* q : ptrs) cudaFreeAsync(q, s);
  }
};

// exclusive scan of n values (in may equal out); *total_dev receives the sum
template <typename T>
void scan(Buffers& B, const T* in, T* out, int64_t n, T* total_dev, cudaStream_t s) {
  const int nb = (int)std::max<int64_t>(1, (n + kTile - 1) / kTile);
  T* sums = B.get<T>(nb);
  if (B.ce != cudaSuccess) return;
  if (n > 0) k_tile_sums<T><<<nb, kThreads, 0, s>>>(in, n, sums);
  else cudaMemsetAsync(sums, 0, sizeof(T), s);
  k_scan_sums<T><<<1, 1024, 0, s>>>(sums, nb, total_dev);
  if (n > 0) k_tile_scan<T><<<nb, kThreads, 0, s>>>(in, out, n, sums);
}

// stable sort of (key, value) by the low `bits` bits of key; the result ends
// in (k, v) (the buffers are swapped as needed)
void radix_sort(Buffers& B, uint32_t*& k, uint32_t*& v, int64_t n, int bits, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return;
  const int nb = (int)((n + kTile - 1) / kTile);
  uint32_t* k2 = B.get<uint32_t>(n);
  uint32_t* v2 = B.get<uint32_t>(n);
  int* hist = B.get<int>((size_t)256 * nb);
  if (B.ce != cudaSuccess) return;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<<<nb, kThreads, 0, s>>>(k, n, shift, nb, hist);
    scan<int>(B, hist, hist, (int64_t)256 * nb, nullptr, s);
    k_radix_scatter<<<nb, kThreads, 0, s>>>(k, v, k2, v2, n, shift, nb, hist);
    std::swap(k, k2);
    std::swap(v, v2);
  }
}

int bits_for(uint64_t max_value) {
  int b = 0;
  while (b < 32 && (max_value >> b) != 0) ++b;
  return b;
}

// out[k] = (uint32) key[idx[k]] (idx null: key[k])
__global__ void k_gather_key(const int* __restrict__ key, const uint32_t* __restrict__ idx, int64_t n,
                             uint32_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (uint32_t)key[idx ? idx[k] : k];
}

}  // namespace

// The order of the keypoint pairs by (image pair, track, input index): two
// stable radix sorts of the indices, by track, then by image pair.  perm [Z]
// receives, for each position of that order, the input index.
cudaError_t sort_kp_pairs(const int* kp_img_pair, const int* kp_track, int64_t Z, int P, int max_track,
                          uint32_t* perm, cudaStream_t s) {
  if (Z <= 0) return cudaSuccess;
  Buffers B(s);
  uint32_t* key = B.get<uint32_t>((size_t)Z);
  uint32_t* val = B.get<uint32_t>((size_t)Z);
  if (B.ce != cudaSuccess) return B.ce;
  k_iota<<<grid_for(Z), 256, 0, s>>>(val, Z);
  if (kp_track) {
    k_gather_key<<<grid_for(Z), 256, 0, s>>>(kp_track, nullptr, Z, key);
    radix_sort(B, key, val, Z, bits_for((uint64_t)(max_track > 0 ? max_track : 0)), s);
  }
  k_gather_key<<<grid_for(Z), 256, 0, s>>>(kp_img_pair, val, Z, key);
  radix_sort(B, key, val, Z, bits_for((uint64_t)(P > 1 ? P - 1 : 0)), s);
  if (B.ce != cudaSuccess) return B.ce;
  cudaMemcpyAsync(perm, val, sizeof(uint32_t) * (size_t)Z, cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

// The track table of a problem: off [T+1] the exclusive scan of the
// keypoint pairs per track (counted into off by the caller), idx [Z] the
// keypoint-pair indices ordered by track, ascending inside a track (one
// stable radix sort of the indices by track).
cudaError_t track_table(const int* kp_track, int64_t Z, int T, int* off, int* idx, cudaStream_t s) {
  if (Z <= 0 || T <= 0) return cudaSuccess;
  Buffers B(s);
  uint32_t* key = B.get<uint32_t>((size_t)Z);
  uint32_t* val = B.get<uint32_t>((size_t)Z);
  if (B.ce != cudaSuccess) return B.ce;
  scan<int>(B, off, off, (int64_t)T + 1, nullptr, s);
  k_iota<<<grid_for(Z), 256, 0, s>>>(val, Z);
  k_gather_key<<<grid_for(Z), 256, 0, s>>>(kp_track, nullptr, Z, key);
  radix_sort(B, key, val, Z, bits_for((uint64_t)(T - 1)), s);
  if (B.ce != cudaSuccess) return B.ce;
  cudaMemcpyAsync(idx, val, sizeof(uint32_t) * (size_t)Z, cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

}  // namespace fm

namespace {

void tracks_free(fm_tracks* t) {
  if (!t) return;
  for (void* q : {(void*)t->pair_i, (void*)t->pair_j, (void*)t->kp_img_pair, (void*)t->node1, (void*)t->node2,
                  (void*)t->track, (void*)t->px1, (void*)t->px2})
    if (q) cudaFreeAsync(q, t->stream);
  if (t->stream) {
    cudaStreamSynchronize(t->stream);
    cudaStreamDestroy(t->stream);
  }
  delete t;
}

fm_status tracks_fail(fm_status st, const std::string& msg) {
  fm::set_thread_error(msg);
  return st;
}

template <typename T>
cudaError_t to_device(fm::Buffers& B, const T* src, size_t n, bool on_device, const T*& out, cudaStream_t s) {
  if (on_device) {
    out = src;
    return cudaSuccess;
  }
  T* d = B.get<T>(n);
  if (B.ce != cudaSuccess) return B.ce;
  out = d;
  return n ? cudaMemcpyAsync(d, src, sizeof(T) * n, cudaMemcpyHostToDevice, s) : cudaSuccess;
}

}  // namespace

extern "C" {

fm_status fm_tracks_complete(int32_t n_images, const int32_t* kp_off, int64_t n_matches, const int32_t* matches,
                             const float* kp_px, int32_t min_pairs, int32_t on_device, fm_tracks** out) {
  using namespace fm;
  if (!out) return tracks_fail(FM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_images < 2 || n_images > 65535) return tracks_fail(FM_ERR_INVALID_ARG, "n_images must be in [2, 65535]");
  if (!kp_off) return tracks_fail(FM_ERR_INVALID_ARG, "kp_off is NULL");
  if (n_matches < 0 || (n_matches > 0 && !matches)) return tracks_fail(FM_ERR_INVALID_ARG, "matches");
  if (min_pairs < 1) return tracks_fail(FM_ERR_INVALID_ARG, "min_pairs must be >= 1");
  const int N = n_images;
  std::vector<int> off(N + 1);
  if (on_device) {
    if (cudaMemcpy(off.data(), kp_off, sizeof(int) * (N + 1), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return tracks_fail(FM_ERR_CUDA, "reading kp_off");
    }
  } else {
    std::copy(kp_off, kp_off + N + 1, off.begin());
  }
  if (off[0] != 0) return tracks_fail(FM_ERR_INVALID_ARG, "kp_off[0] must be 0");
  for (int c = 0; c < N; ++c)
    if (off[c + 1] < off[c]) return tracks_fail(FM_ERR_INVALID_ARG, "kp_off must be non-decreasing");
  const int K = off[N];
  if (n_matches > (int64_t)INT32_MAX) return tracks_fail(FM_ERR_INVALID_ARG, "too many matches");
  if (K == 0 && n_matches > 0) return tracks_fail(FM_ERR_INVALID_ARG, "matches without keypoints");
  const int64_t M = n_matches;

  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return tracks_fail(FM_ERR_CUDA, "stream");
  }
  fm_tracks* res = new fm_tracks();
  res->stream = s;
  fm_status st = FM_OK;
  std::string msg;
  {
    Buffers B(s);
    const int* d_off = nullptr;
    const int2* d_match = nullptr;
    const float2* d_px = nullptr;
    cudaError_t ce = to_device(B, kp_off, N + 1, on_device != 0, d_off, s);
    const int* mraw = nullptr;
    if (ce == cudaSuccess) ce = to_device(B, matches, (size_t)2 * M, on_device != 0, mraw, s);
    d_match = (const int2*)mraw;
    if (ce == cudaSuccess && kp_px) {
      const float* p = nullptr;
      ce = to_device(B, kp_px, (size_t)2 * K, on_device != 0, p, s);
      d_px = (const float2*)p;
    }
    int* img = B.get<int>(K);
    int* parent = B.get<int>(K);
    int* label = B.get<int>(K);
    int* size = B.get<int>(K);
    int* bad = B.get<int>(K);
    int* start = B.get<int>(K);
    int* tid = B.get<int>(K);
    long long* nemit = B.get<long long>(K);
    uint32_t* skey = B.get<uint32_t>(K);
    uint32_t* sval = B.get<uint32_t>(K);
    int* err = B.get<int>(1);
    long long* tot = B.get<long long>(2);
    int* itot = B.get<int>(3);
    if (ce == cudaSuccess) ce = B.ce;
    if (ce == cudaSuccess) ce = cudaMemsetAsync(size, 0, sizeof(int) * std::max(K, 1), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(bad, 0, sizeof(int) * std::max(K, 1), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (ce == cudaSuccess && K > 0) {
      k_node_image<<<grid_for(K), 256, 0, s>>>(d_off, N, K, img, parent);
      if (M > 0) k_union<<<grid_for(M), 256, 0, s>>>(d_match, M, K, img, parent, err);
      k_label<<<grid_for(K), 256, 0, s>>>(parent, K, label, size, err);
      // keypoints sorted by label (stable: by keypoint id inside a component)
      cudaMemcpyAsync(skey, label, sizeof(int) * K, cudaMemcpyDeviceToDevice, s);
      k_iota<<<grid_for(K), 256, 0, s>>>(sval, K);
      radix_sort(B, skey, sval, K, bits_for((uint64_t)K - 1), s);
      k_members<<<grid_for(K), 256, 0, s>>>(skey, sval, K, img, start, bad);
      // track numbers (by label) and emitted pairs of consistent tracks
      k_track_flags<<<grid_for(K), 256, 0, s>>>(label, size, bad, K, tid, nemit);
      ce = cudaGetLastError();
    }
    // tid holds is_track flags: numbers by an exclusive scan
    int h_err = 0;
    int h_counts[2] = {0, 0};
    long long h_tot[2] = {0, 0};
    if (ce == cudaSuccess && K > 0) {
      scan<int>(B, tid, tid, K, itot, s);
      scan<long long>(B, nemit, nemit, K, tot, s);
      ce = B.ce == cudaSuccess ? cudaGetLastError() : B.ce;
    }
    long long* rflag = nullptr;
    if (ce == cudaSuccess && M > 0) {
      rflag = B.get<long long>(M);
      ce = B.ce;
      if (ce == cudaSuccess) {
        k_raw_flags<<<grid_for(M), 256, 0, s>>>(d_match, M, K, img, label, bad, rflag);
        scan<long long>(B, rflag, rflag, M, tot + 1, s);
        ce = B.ce == cudaSuccess ? cudaGetLastError() : B.ce;
      }
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess && K > 0) ce = cudaMemcpyAsync(h_counts, itot, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess && K > 0) ce = cudaMemcpyAsync(h_tot, tot, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess && M > 0)
      ce = cudaMemcpyAsync(h_tot + 1, tot + 1, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
      st = ce == cudaErrorMemoryAllocation ? FM_ERR_OOM : FM_ERR_CUDA;
      msg = std::string("track completion: ") + cudaGetErrorString(ce);
    } else if (h_err & kTrkBadMatch) {
      st = FM_ERR_INVALID_ARG;
      msg = "a match joins a keypoint outside [0, K) or two keypoints of one image";
    } else if (h_err & kTrkUfBound) {
      st = FM_ERR_TIMEOUT;
      msg = "union-find step bound reached";
    } else if (h_tot[0] + h_tot[1] > (long long)INT32_MAX) {
      st = FM_ERR_INVALID_ARG;
      msg = "more than 2^31 - 1 completed keypoint pairs";
    }
    const int64_t Z1 = h_tot[0], Z = h_tot[0] + h_tot[1];
    res->n_tracks = h_counts[0];
    if (st == FM_OK) {
      uint32_t* key = B.get<uint32_t>(Z);
      uint32_t* perm = B.get<uint32_t>(Z);
      int* n1 = B.get<int>(Z);
      int* n2 = B.get<int>(Z);
      int* trk = B.get<int>(Z);
      int* head = B.get<int>(Z);
      int* hscan = B.get<int>(Z);
      int* ipair = B.get<int>(Z);
      ce = B.ce;
      if (ce == cudaSuccess && Z > 0) {
        k_emit_tracks<<<grid_for(K), 256, 0, s>>>(skey, sval, K, start, size, bad, tid, nemit, img, N, key, n1, n2,
                                                   trk);
        if (M > 0 && Z > Z1)
          k_emit_raw<<<grid_for(M), 256, 0, s>>>(d_match, M, K, label, bad, rflag, Z1, tid, img, N, key, n1, n2,
                                                  trk);
        k_iota<<<grid_for(Z), 256, 0, s>>>(perm, Z);
        radix_sort(B, key, perm, Z, bits_for((uint64_t)N * N - 1), s);
        k_heads<<<grid_for(Z), 256, 0, s>>>(key, Z, head);
        scan<int>(B, head, hscan, Z, itot + 1, s);
        ce = B.ce == cudaSuccess ? cudaGetLastError() : B.ce;
      }
      // the image-pair count P stays on the device (itot[1]): buffers indexed
      // by image pair are sized by the bound Pmax, and every count is read
      // back once, at the end
      const int64_t Pmax = std::max<int64_t>(1, std::min<int64_t>(Z, (int64_t)N * (N - 1) / 2));
      int* pi = nullptr;
      int* pj = nullptr;
      int* pstart = nullptr;
      if (ce == cudaSuccess && Z > 0) {
        pi = B.get<int>(Pmax);
        pj = B.get<int>(Pmax);
        pstart = B.get<int>(Pmax);
        ce = B.ce;
        if (ce == cudaSuccess) k_pairs<<<grid_for(Z), 256, 0, s>>>(key, head, hscan, Z, N, ipair, pi, pj, pstart);
      }
      // image pairs with fewer than min_pairs pairs dropped: kept counts in
      // itot[0] (image pairs) and tot[0] (keypoint pairs)
      int* pkeep = nullptr;
      int* ppos = nullptr;
      long long* zpos = nullptr;
      const bool filter = Z > 0 && min_pairs > 1;
      if (ce == cudaSuccess && filter) {
        pkeep = B.get<int>(Pmax);
        ppos = B.get<int>(Pmax);
        zpos = B.get<long long>(Z);
        ce = B.ce;
        if (ce == cudaSuccess) {
          k_pair_keep<<<grid_for(Pmax), 256, 0, s>>>(pstart, itot + 1, (int)Pmax, Z, min_pairs, pkeep);
          scan<int>(B, pkeep, ppos, Pmax, itot, s);
          k_keep_flags<<<grid_for(Z), 256, 0, s>>>(ipair, pkeep, Z, zpos);
          scan<long long>(B, zpos, zpos, Z, tot, s);
          ce = B.ce == cudaSuccess ? cudaGetLastError() : B.ce;
        }
      }
      if (ce == cudaSuccess) {
        // outputs sized by the counts before filtering (bounds of the kept ones)
        const int64_t Pcap = Z > 0 ? Pmax : 0;
        auto alloc = [&](auto*& p, size_t n) {
          if (ce == cudaSuccess)
            ce = cudaMallocFromPoolAsync((void**)&p, std::max<size_t>(n * sizeof(*p), 16), tracks_pool(), s);
        };
        alloc(res->pair_i, Pcap);
        alloc(res->pair_j, Pcap);
        alloc(res->kp_img_pair, Z);
        alloc(res->node1, Z);
        alloc(res->node2, Z);
        alloc(res->track, Z);
        if (d_px) {
          alloc(res->px1, Z);
          alloc(res->px2, Z);
        }
      }
      if (ce == cudaSuccess && Z > 0) {
        k_gather<<<grid_for(Z), 256, 0, s>>>(perm, ipair, Z, pkeep, ppos, zpos, n1, n2, trk, d_px,
                                              res->kp_img_pair, res->node1, res->node2, res->track, res->px1,
                                              res->px2);
        k_pair_compact<<<grid_for(Pmax), 256, 0, s>>>(pi, pj, pkeep, ppos, itot + 1, res->pair_i, res->pair_j);
        ce = cudaGetLastError();
      }
      // inconsistent tracks: the number of flags (a scan of bad into start,
      // which is no longer needed), into itot[2]
      if (ce == cudaSuccess && K > 0) {
        scan<int>(B, bad, start, K, itot + 2, s);
        ce = B.ce == cudaSuccess ? cudaGetLastError() : B.ce;
      }
      int h_cnt[3] = {0, 0, 0};
      long long Z_out = Z;
      if (ce == cudaSuccess && (Z > 0 || K > 0))
        ce = cudaMemcpyAsync(h_cnt, itot, sizeof(int) * 3, cudaMemcpyDeviceToHost, s);
      if (ce == cudaSuccess && filter) ce = cudaMemcpyAsync(&Z_out, tot, sizeof(long long), cudaMemcpyDeviceToHost, s);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
      res->P = Z > 0 ? (filter ? h_cnt[0] : h_cnt[1]) : 0;
      res->Z = Z > 0 ? Z_out : 0;
      res->n_inconsistent = K > 0 ? h_cnt[2] : 0;
      if (ce != cudaSuccess) {
        st = ce == cudaErrorMemoryAllocation ? FM_ERR_OOM : FM_ERR_CUDA;
        msg = std::string("track completion: ") + cudaGetErrorString(ce);
      }
    }
  }
  if (st != FM_OK) {
    cudaGetLastError();
    tracks_free(res);
    return tracks_fail(st, msg);
  }
  *out = res;
  return FM_OK;
}

fm_status fm_tracks_info(const fm_tracks* t, int64_t* n_tracks, int64_t* n_img_pairs, int64_t* n_kp_pairs,
                         int64_t* n_inconsistent) {
  if (!t) return tracks_fail(FM_ERR_INVALID_ARG, "tracks is NULL");
  if (n_tracks) *n_tracks = t->n_tracks;
  if (n_img_pairs) *n_img_pairs = t->P;
  if (n_kp_pairs) *n_kp_pairs = t->Z;
  if (n_inconsistent) *n_inconsistent = t->n_inconsistent;
  return FM_OK;
}

fm_status fm_tracks_copy(const fm_tracks* t, int32_t* pair_i, int32_t* pair_j, int32_t* kp_img_pair, int32_t* node1,
                         int32_t* node2, int32_t* kp_track, float* kp1_px, float* kp2_px, int32_t on_device) {
  if (!t) return tracks_fail(FM_ERR_INVALID_ARG, "tracks is NULL");
  if ((kp1_px || kp2_px) && !t->px1) return tracks_fail(FM_ERR_INVALID_ARG, "no keypoint pixels were given");
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t ce = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (dst && bytes && ce == cudaSuccess) ce = cudaMemcpyAsync(dst, src, bytes, kind, t->stream);
  };
  cp(pair_i, t->pair_i, sizeof(int) * t->P);
  cp(pair_j, t->pair_j, sizeof(int) * t->P);
  cp(kp_img_pair, t->kp_img_pair, sizeof(int) * t->Z);
  cp(node1, t->node1, sizeof(int) * t->Z);
  cp(node2, t->node2, sizeof(int) * t->Z);
  cp(kp_track, t->track, sizeof(int) * t->Z);
  cp(kp1_px, t->px1, sizeof(float2) * t->Z);
  cp(kp2_px, t->px2, sizeof(float2) * t->Z);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(t->stream);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return tracks_fail(FM_ERR_CUDA, std::string("tracks copy: ") + cudaGetErrorString(ce));
  }
  return FM_OK;
}

void fm_tracks_destroy(fm_tracks* t) { tracks_free(t); }

fm_status fm_filter_image_pairs(int32_t n_images, int32_t n_pairs, const int32_t* pair_i, const int32_t* pair_j,
                                const int32_t* counts, double t_start, double t_min, int32_t* keep,
                                int32_t* image_valid, double* t_used) {
  if (n_images < 1 || n_pairs < 0) return tracks_fail(FM_ERR_INVALID_ARG, "n_images >= 1, n_pairs >= 0");
  if (n_pairs > 0 && (!pair_i || !pair_j || !counts)) return tracks_fail(FM_ERR_INVALID_ARG, "inputs are NULL");
  if (!keep && n_pairs > 0) return tracks_fail(FM_ERR_INVALID_ARG, "keep is NULL");
  if (!(t_min >= 0.0) || !(t_start >= t_min) || !std::isfinite(t_start))
    return tracks_fail(FM_ERR_INVALID_ARG, "0 <= t_min <= t_start, finite");
  for (int n = 0; n < n_pairs; ++n)
    if (pair_i[n] < 0 || pair_i[n] >= n_images || pair_j[n] < 0 || pair_j[n] >= n_images || pair_i[n] == pair_j[n])
      return tracks_fail(FM_ERR_INVALID_ARG, "image pair " + std::to_string(n) + " out of range");
  std::vector<int> parent(n_images);
  auto find = [&](int x) {
    while (parent[x] != x) x = parent[x] = parent[parent[x]];
    return x;
  };
  // components of the image pairs above t; the smallest image id labels each
  auto label_at = [&](double t) {
    for (int c = 0; c < n_images; ++c) parent[c] = c;
    for (int n = 0; n < n_pairs; ++n)
      if ((double)counts[n] > t) {
        const int a = find(pair_i[n]), b = find(pair_j[n]);
        if (a != b) parent[std::max(a, b)] = std::min(a, b);
      }
    int n_comp = 0;
    for (int c = 0; c < n_images; ++c) n_comp += find(c) == c;
    return n_comp;
  };
  double t = t_start;
  for (int it = 0; it < 2100; ++it) {   // halvings from 1e308 reach any t_min >= 0 or underflow to 0
    if (label_at(t) == 1 || t <= t_min) break;
    t = std::max(t / 2.0, t_min);
  }
  std::vector<int> size(n_images, 0);
  for (int c = 0; c < n_images; ++c) size[find(c)]++;
  int best = 0;
  for (int c = 1; c < n_images; ++c)
    if (size[c] > size[best]) best = c;   // the first (smallest label) on ties
  for (int c = 0; c < n_images; ++c)
    if (image_valid) image_valid[c] = find(c) == best;
  for (int n = 0; n < n_pairs; ++n)
    keep[n] = (double)counts[n] > t && find(pair_i[n]) == best && find(pair_j[n]) == best;
  if (t_used) *t_used = t;
  return FM_OK;
}

}  // extern "C"
