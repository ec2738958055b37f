// Epipolar adjustment: loss and gradient over every keypoint pair (Sec. 3.3,
// Eq. 7 (L1) and Eqs. 8-9 (L2 / IRLS-weighted L2)).
//
// One evaluation is three launches:
//   k_ea_tables    per image pair n: E_n = [t^]_x R_ij from the two cameras'
//                  parameters, packed with the end offset of n's keypoint
//                  pairs (48 B per image pair);
//   k_ea_direct    streams the calibrated keypoint pairs (16 B each, plus 4 B
//                  when weighted) once and emits, per (warp run, image pair),
//                  the partial sums  sum rho'(r) x~2 x~1^T  (9 floats) and
//                  sum rho(r)  -- the residual r = x~2^T E_n x~1 is never
//                  written to memory;
//   k_ea_segments  per image pair: adds its partial sums in order, scales by
//                  1/Z, and applies the chain rule through E = [t^]_x R_ij to
//                  the two cameras (24 floats).
// The per-camera sums, the 6D adjoint and Adam follow in fm_cam.cu.
//
// k_ea_direct layout and schedule
//   * keypoint pairs are sorted by image pair (CSR seg_off);
//   * a warp run is 32 * U consecutive keypoint pairs; lane l owns the U
//     consecutive pairs [base + l*U, base + (l+1)*U);
//   * each warp is persistent over warp runs (grid-stride) and double-buffers
//     its next warp run in shared memory with cp.async (coalesced 512 B per
//     warp instruction); the image-pair table entries of the warp run
//     (up to kEaSegCap) are staged the same way;
//   * U is odd, so lanes reading their own contiguous pairs (stride U*16 B)
//     hit distinct 16-B bank groups in each quarter warp: no bank conflicts;
//   * each lane accumulates in registers along its run; a run spans at most
//     a few image pairs, so the lane keeps a "head" part (its first image
//     pair, which may continue from the previous lane), writes complete image
//     pairs inside its run directly, and keeps a "tail" part; a warp-level
//     segmented scan keyed by image pair combines heads and tails in fixed
//     lane order.  No atomics: the result is deterministic.
#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

constexpr int U = kEaPairsPerLane;
constexpr int WP = kEaWarpPairs;
constexpr int SEGCAP = kEaSegCap;
constexpr int WARPS = kEaWarpsPerCta;
constexpr unsigned FULL = 0xffffffffu;

__global__ void k_ea_tables(const float* __restrict__ params, const int* __restrict__ pi,
                            const int* __restrict__ pj, const int* __restrict__ seg_off, int P,
                            float4* __restrict__ tab, int* step_counter) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (step_counter && n == 0) *step_counter += 1;
  if (n >= P) return;
  PairGeo g;
  pair_geometry(params + 9 * pi[n], params + 9 * pj[n], g);
  float E[9];
  essential(g, E);
  int end = seg_off[n + 1];
  tab[3 * n + 0] = make_float4(E[0], E[1], E[2], E[3]);
  tab[3 * n + 1] = make_float4(E[4], E[5], E[6], E[7]);
  tab[3 * n + 2] = make_float4(E[8], __int_as_float(end), 0.f, 0.f);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async16_partial(void* smem, const void* gmem, int bytes) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

struct DirectArgs {
  const float4* kp;
  const float* wts;
  const int* run_seg;
  const int4* info;
  const float4* seg_tab;
  float4* rec;
  int Z;
  int n_wruns;
};

// shared memory per warp: [2][WP] float4 keypoints, [2][3*SEGCAP] float4
// image-pair entries, and (weighted) [2][WP] float weights
constexpr int kKpBuf = WP;
constexpr int kSegBuf = 3 * SEGCAP;
constexpr size_t kSmemPerWarp = 2 * (kKpBuf + kSegBuf) * sizeof(float4);
constexpr size_t kSmemPerWarpW = kSmemPerWarp + 2 * WP * sizeof(float);

template <bool WEIGHTED>
__device__ __forceinline__ void issue(const DirectArgs& a, int w, int4 info, float4* kb, float4* sb,
                                      float* wb, int lane) {
  const int base = w * WP;
#pragma unroll
  for (int k = 0; k < U; ++k) {
    int idx = lane + 32 * k;
    if (base + idx < a.Z) cp_async16(kb + idx, a.kp + base + idx);
  }
  const int ne = 3 * min(info.y, SEGCAP);
  for (int e = lane; e < ne; e += 32) cp_async16(sb + e, a.seg_tab + 3 * info.x + e);
  if (WEIGHTED) {
    for (int c = lane; c < WP / 4; c += 32) {
      int p4 = base + 4 * c;
      int bytes = 4 * min(4, a.Z - p4);
      if (bytes > 0) cp_async16_partial(wb + 4 * c, a.wts + p4, bytes);
    }
  }
  cp_async_commit();
}

__device__ __forceinline__ void load_entry(const float4* sb, const float4* seg_tab, int sl, int s,
                                           float* E, int& end) {
  float4 e0, e1, e2;
  if (sl < SEGCAP) {
    e0 = sb[3 * sl];
    e1 = sb[3 * sl + 1];
    e2 = sb[3 * sl + 2];
  } else {
    e0 = __ldg(seg_tab + 3 * s);
    e1 = __ldg(seg_tab + 3 * s + 1);
    e2 = __ldg(seg_tab + 3 * s + 2);
  }
  E[0] = e0.x; E[1] = e0.y; E[2] = e0.z; E[3] = e0.w;
  E[4] = e1.x; E[5] = e1.y; E[6] = e1.z; E[7] = e1.w;
  E[8] = e2.x;
  end = __float_as_int(e2.y);
}

__device__ __forceinline__ void store_record(float4* rec, int r, const float* v) {
  rec[3 * r + 0] = make_float4(v[0], v[1], v[2], v[3]);
  rec[3 * r + 1] = make_float4(v[4], v[5], v[6], v[7]);
  rec[3 * r + 2] = make_float4(v[8], v[9], 0.f, 0.f);
}

// LOSS 0: rho = w |r|, rho' = w sign(r) (sign(0) = 0)
// LOSS 1: rho = w r^2, rho'/2 = w r     (the factor 2 is applied per image pair)
template <int LOSS, bool WEIGHTED>
__device__ __forceinline__ void process(const DirectArgs& a, int w, int4 info, int s,
                                        const float4* kb, const float4* sb, const float* wb,
                                        int lane) {
  const int base = w * WP;
  const int p0 = base + lane * U;
  const int pend = min(p0 + U, a.Z);
  int sl = s - info.x;
  float E[9];
  int end;
  load_entry(sb, a.seg_tab, sl, s, E, end);
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.f;
  float head[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) head[k] = 0.f;
  bool has_head = false;
  const int head_key = s;

#pragma unroll
  for (int k = 0; k < U; ++k) {
    const int p = p0 + k;
    if (p < pend) {
      if (p >= end) {
        do {
          if (!has_head) {
#pragma unroll
            for (int c = 0; c < 10; ++c) head[c] = acc[c];
            has_head = true;
          } else {
            store_record(a.rec, info.z + sl, acc);
          }
#pragma unroll
          for (int c = 0; c < 10; ++c) acc[c] = 0.f;
          ++s;
          ++sl;
          load_entry(sb, a.seg_tab, sl, s, E, end);
        } while (p >= end);
      }
      const float4 x = kb[lane * U + k];
      const float ex = fmaf(E[0], x.x, fmaf(E[1], x.y, E[2]));
      const float ey = fmaf(E[3], x.x, fmaf(E[4], x.y, E[5]));
      const float ez = fmaf(E[6], x.x, fmaf(E[7], x.y, E[8]));
      const float r = fmaf(x.z, ex, fmaf(x.w, ey, ez));
      float c, l;
      if (LOSS == 0) {
        c = (r > 0.f) ? 1.f : ((r < 0.f) ? -1.f : 0.f);
        l = fabsf(r);
      } else {
        c = r;
        l = r * r;
      }
      if (WEIGHTED) {
        const float wt = wb[lane * U + k];
        c *= wt;
        l *= wt;
      }
      const float ca = c * x.x, cb = c * x.y;
      acc[0] = fmaf(ca, x.z, acc[0]);
      acc[1] = fmaf(cb, x.z, acc[1]);
      acc[2] = fmaf(c, x.z, acc[2]);
      acc[3] = fmaf(ca, x.w, acc[3]);
      acc[4] = fmaf(cb, x.w, acc[4]);
      acc[5] = fmaf(c, x.w, acc[5]);
      acc[6] += ca;
      acc[7] += cb;
      acc[8] += c;
      acc[9] += l;
    }
  }

  // warp combine: segmented inclusive scan of the tails keyed by image pair
  int key = s;
  float sc[10];
#pragma unroll
  for (int c = 0; c < 10; ++c) sc[c] = acc[c];
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int ku = __shfl_up_sync(FULL, key, d);
    const bool take = (lane >= d) && (ku == key);
#pragma unroll
    for (int c = 0; c < 10; ++c) {
      const float v = __shfl_up_sync(FULL, sc[c], d);
      if (take) sc[c] += v;
    }
  }
  const int key_next = __shfl_down_sync(FULL, key, 1);
  const int hk_next = __shfl_down_sync(FULL, has_head ? head_key : -1, 1);
  const int key_prev = __shfl_up_sync(FULL, key, 1);
  const bool last_of_key = (lane == 31) || (key_next != key);
  const bool absorb = (lane < 31) && (hk_next == key);
#pragma unroll
  for (int c = 0; c < 10; ++c) {
    const float hv = __shfl_down_sync(FULL, head[c], 1);
    if (absorb) sc[c] += hv;
  }
  if (last_of_key) store_record(a.rec, info.z + (key - info.x), sc);
  if (has_head && (lane == 0 || key_prev != head_key))
    store_record(a.rec, info.z + (head_key - info.x), head);
}

template <int LOSS, bool WEIGHTED>
__global__ void __launch_bounds__(WARPS * 32) k_ea_direct(DirectArgs a) {
  extern __shared__ float4 smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  constexpr size_t per_warp = (WEIGHTED ? kSmemPerWarpW : kSmemPerWarp) / sizeof(float4);
  float4* my = smem + wib * per_warp;
  // slot b: keypoints my + b*kKpBuf, image-pair entries my + 2*kKpBuf + b*kSegBuf,
  // weights (float) wbase + b*WP
  float* wbase = reinterpret_cast<float*>(my + 2 * (kKpBuf + kSegBuf));
  const int stride = gridDim.x * WARPS;
  int w = blockIdx.x * WARPS + wib;
  if (w >= a.n_wruns) return;   // uniform per warp

  int4 info_cur = a.info[w];
  int seg_cur = a.run_seg[w * 32 + lane];
  int4 info_nxt = make_int4(0, 0, 0, 0);
  if (w + stride < a.n_wruns) info_nxt = a.info[w + stride];
  issue<WEIGHTED>(a, w, info_cur, my, my + 2 * kKpBuf, wbase, lane);

  for (int it = 0; w < a.n_wruns; ++it, w += stride) {
    const int cur = it & 1;
    const int wn = w + stride;
    int seg_nxt = 0;
    int4 info_nn = make_int4(0, 0, 0, 0);
    if (wn < a.n_wruns) {
      seg_nxt = a.run_seg[wn * 32 + lane];
      if (wn + stride < a.n_wruns) info_nn = a.info[wn + stride];
      const int nb = cur ^ 1;
      issue<WEIGHTED>(a, wn, info_nxt, my + nb * kKpBuf, my + 2 * kKpBuf + nb * kSegBuf,
                      wbase + nb * WP, lane);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    process<LOSS, WEIGHTED>(a, w, info_cur, seg_cur, my + cur * kKpBuf,
                            my + 2 * kKpBuf + cur * kSegBuf, wbase + cur * WP, lane);
    __syncwarp();
    info_cur = info_nxt;
    info_nxt = info_nn;
    seg_cur = seg_nxt;
  }
}

// per image pair: sum its records (fixed order), scale, chain rule
template <int LOSS>
__global__ void k_ea_segments(const float4* __restrict__ rec, const int* __restrict__ seg_rec,
                              const float* __restrict__ params, const int* __restrict__ pi,
                              const int* __restrict__ pj, int P, float inv_z,
                              float* __restrict__ seg_grad, float* __restrict__ seg_loss) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= P) return;
  const int r0 = seg_rec[2 * n], cnt = seg_rec[2 * n + 1];
  float* out = seg_grad + (size_t)kSegGradEa * n;
  if (cnt == 0) {
    for (int k = 0; k < kSegGradEa; ++k) out[k] = 0.f;
    seg_loss[n] = 0.f;
    return;
  }
  float G[10];
  for (int k = 0; k < 10; ++k) G[k] = 0.f;
  for (int r = r0; r < r0 + cnt; ++r) {
    float4 v0 = rec[3 * r], v1 = rec[3 * r + 1], v2 = rec[3 * r + 2];
    G[0] += v0.x; G[1] += v0.y; G[2] += v0.z; G[3] += v0.w;
    G[4] += v1.x; G[5] += v1.y; G[6] += v1.z; G[7] += v1.w;
    G[8] += v2.x; G[9] += v2.y;
  }
  const float gs = (LOSS == 1) ? 2.f * inv_z : inv_z;
  for (int k = 0; k < 9; ++k) G[k] *= gs;
  seg_loss[n] = G[9] * inv_z;
  PairGeo g;
  pair_geometry(params + 9 * pi[n], params + 9 * pj[n], g);
  float o[kSegGradEa];
  pair_backward(g, G, o);
  for (int k = 0; k < kSegGradEa; ++k) out[k] = o[k];
}

}  // namespace

void launch_ea_tables(const float* params, const int* pi, const int* pj, const int* seg_off,
                      int P, float4* seg_tab, int* step_counter, cudaStream_t s) {
  k_ea_tables<<<(P + 127) / 128, 128, 0, s>>>(params, pi, pj, seg_off, P, seg_tab, step_counter);
}

template <int LOSS, bool WEIGHTED>
static void launch_direct_t(const fm_problem* pr, const float* weights, cudaStream_t s) {
  DirectArgs a;
  a.kp = pr->kp;
  a.wts = weights;
  a.run_seg = pr->run_seg;
  a.info = pr->wrun_info;
  a.seg_tab = pr->seg_tab;
  a.rec = pr->rec;
  a.Z = (int)pr->Z;
  a.n_wruns = pr->n_wruns;
  const size_t smem = WARPS * (WEIGHTED ? kSmemPerWarpW : kSmemPerWarp);
  static int per_sm = 0;   // resident CTAs per SM (one device per process)
  if (per_sm == 0) {
    cudaFuncSetAttribute(k_ea_direct<LOSS, WEIGHTED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ea_direct<LOSS, WEIGHTED>,
                                                  WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
  }
  int ctas = (pr->n_wruns + WARPS - 1) / WARPS;
  int cap = per_sm * pr->sm_count;
  if (ctas > cap) ctas = cap;
  k_ea_direct<LOSS, WEIGHTED><<<ctas, WARPS * 32, smem, s>>>(a);
}

void launch_ea_direct(const fm_problem* pr, const float* weights, int loss, cudaStream_t s) {
  if (pr->n_wruns == 0) return;
  if (loss == FM_EA_L1) {
    if (weights) launch_direct_t<0, true>(pr, weights, s);
    else launch_direct_t<0, false>(pr, nullptr, s);
  } else {
    if (weights) launch_direct_t<1, true>(pr, weights, s);
    else launch_direct_t<1, false>(pr, nullptr, s);
  }
}

void launch_ea_segments(const fm_problem* pr, const float* params, int loss, float inv_z,
                        cudaStream_t s) {
  const int P = pr->P;
  if (loss == FM_EA_L1)
    k_ea_segments<0><<<(P + 127) / 128, 128, 0, s>>>(pr->rec, pr->seg_rec, params, pr->pair_i,
                                                      pr->pair_j, P, inv_z, pr->seg_grad,
                                                      pr->seg_loss);
  else
    k_ea_segments<1><<<(P + 127) / 128, 128, 0, s>>>(pr->rec, pr->seg_rec, params, pr->pair_i,
                                                      pr->pair_j, P, inv_z, pr->seg_grad,
                                                      pr->seg_loss);
}

}  // namespace fm
