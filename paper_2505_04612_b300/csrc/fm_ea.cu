// Epipolar adjustment: loss and gradient over every keypoint pair (Sec. 3.3,
// Eq. 7 (L1) and Eqs. 8-9 (L2 / IRLS-weighted L2)).
//
// One evaluation is three launches:
//   k_ea_tables    per image pair n: E_n = [t^]_x R_ij from the two cameras'
//                  parameters (with free focal lengths, S_j E_n S_i), packed
//                  with the end offset of n's keypoint pairs (48 B per image
//                  pair);
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
//   * lanes: image pair n gets max(1, ceil(m_n / U)) lanes of at most U
//     consecutive pairs, so a lane never crosses an image-pair end; a warp
//     run is 32 consecutive lanes (at most 32 U pairs, at most 32 image
//     pairs), described by per-lane descriptors built once per problem;
//   * persistent warps: each warp stages its next warp run into shared memory
//     with one bulk copy (TMA) while it processes the current one (double
//     buffer, mbarrier completion);
//   * the E entries of the run's image pairs sit one per lane in registers;
//     a lane takes its own once per run and accumulates its pairs with no
//     per-pair selection;
//   * a segmented scan over the lanes (a butterfly when the run lies inside
//     one image pair) gives one record per (warp run, image pair), summed in
//     a fixed order: no atomics, deterministic.
//
// Modes of k_ea_direct (the split of one evaluation into a forward and a
// backward pass, for the autograd adjoint):
//   kFull      loss and dL/dE together (one pass, 16 B per pair);
//   kLossOnly  the loss alone; optionally writes each pair's coefficient
//              c = w drho/dr (4 B per pair) for a later kFromCoef pass;
//   kFromCoef  dL/dE from stored coefficients: no residual is recomputed, but
//              the pair's x~2 x~1^T still needs the keypoints (16 + 4 B).
#include <algorithm>
#include <atomic>

#include "fm_step.cuh"

namespace fm {
namespace {

constexpr int WARPS = kEaWarpsPerCta;
constexpr unsigned FULL = 0xffffffffu;

// snap (when not null): a copy of the n_snap parameters, which the camera
// pass of an Adam step reads for the image pairs' chain rule while it updates
// params in place
__global__ void k_ea_tables(const float* params, const int* __restrict__ pi,
                            const int* __restrict__ pj, const int* __restrict__ seg_off, int P,
                            float4* __restrict__ tab, int* step_counter, const float* __restrict__ phi,
                            float* __restrict__ snap, int n_snap) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_trigger();
  int end = 0, ci = 0, cj = 0;
  if (n < P) {
    end = seg_off[n + 1];   // static tables: read before waiting
    ci = pi[n];
    cj = pj[n];
  }
  pdl_wait();               // params come from the previous step's update
  if (step_counter && n == 0) atomicAdd(step_counter, 1);
  if (snap)
    for (int k = n; k < n_snap; k += gridDim.x * blockDim.x) snap[k] = params[k];
  if (n >= P) return;
  float qi[9], qj[9];
  load_plain(params + 9 * ci, qi, 9);
  load_plain(params + 9 * cj, qj, 9);
  PairGeo g;
  pair_geometry(qi, qj, g);
  float E[9];
  essential(g, E);
  if (phi) {   // focal lengths folded in: E' = S_j E S_i, S = diag(e^-phi, e^-phi, 1)
    const float si = __expf(-phi[ci]), sj = __expf(-phi[cj]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) E[3 * a + b] *= (a < 2 ? sj : 1.f) * (b < 2 ? si : 1.f);
  }
  tab[3 * n + 0] = make_float4(E[0], E[1], E[2], E[3]);
  tab[3 * n + 1] = make_float4(E[4], E[5], E[6], E[7]);
  tab[3 * n + 2] = make_float4(E[8], __int_as_float(end), 0.f, 0.f);
}

enum DirectMode { kFull = 0, kLossOnly = 1, kFromCoef = 2 };

struct DirectArgs {
  const float4* kp;
  const float* wts;      // per-pair weights; the stored coefficients in kFromCoef
  const int* lane_desc;  // [32 n_wruns] offset | count << 10 | key << 15 per lane
  const int4* info;      // [n_wruns] {first image pair, n_img | len << 8, record base, first pair}
  const float4* seg_tab;
  float4* rec;
  float* coef_out;       // kLossOnly: per-pair coefficients when not null
  int* err;              // error bits (kErrEaTimeout)
  int n_wruns;
};

__device__ __forceinline__ void store_record(float4* rec, int r, const float* v) {
  rec[3 * r + 0] = make_float4(v[0], v[1], v[2], v[3]);
  rec[3 * r + 1] = make_float4(v[4], v[5], v[6], v[7]);
  rec[3 * r + 2] = make_float4(v[8], v[9], 0.f, 0.f);
}

// c = w drho/dr and l = w rho of one pair.
// LOSS 0: rho = |r|, rho' = sign(r) (sign(0) = 0)
// LOSS 1: rho = r^2; c = w r in kFull (the factor 2 is applied per image pair)
//         and the full 2 w r when stored (kLossOnly), so that stored
//         coefficients need no per-loss factor.
// kFromCoef: c is the stored coefficient (passed in wt), l is not computed.
// MASKED: wt multiplies the pair even when unweighted (0 for lanes past Z).
template <int LOSS, bool WEIGHTED, int MODE, bool MASKED = false>
__device__ __forceinline__ void pair_terms(const float* E, float4 x, float wt, float& c, float& l) {
  if (MODE == kFromCoef) {
    c = wt;
    l = 0.f;
    return;
  }
  const float ex = fmaf(E[0], x.x, fmaf(E[1], x.y, E[2]));
  const float ey = fmaf(E[3], x.x, fmaf(E[4], x.y, E[5]));
  const float ez = fmaf(E[6], x.x, fmaf(E[7], x.y, E[8]));
  const float r = fmaf(x.z, ex, fmaf(x.w, ey, ez));
  if (LOSS == 0) {
    c = (r > 0.f) ? 1.f : ((r < 0.f) ? -1.f : 0.f);
    l = fabsf(r);
  } else {
    c = (MODE == kLossOnly) ? 2.f * r : r;
    l = r * r;
  }
  if (WEIGHTED || MASKED) {
    c *= wt;
    l *= wt;
  }
}

// v += the pair's record terms: c x~2 x~1^T (9, unless kLossOnly) and l
// (unless kFromCoef)
template <int MODE>
__device__ __forceinline__ void add_terms(float c, float l, float4 x, float* v) {
  if (MODE != kLossOnly) {
    const float ca = c * x.x, cb = c * x.y;
    v[0] = fmaf(ca, x.z, v[0]);
    v[1] = fmaf(cb, x.z, v[1]);
    v[2] = fmaf(c, x.z, v[2]);
    v[3] = fmaf(ca, x.w, v[3]);
    v[4] = fmaf(cb, x.w, v[4]);
    v[5] = fmaf(c, x.w, v[5]);
    v[6] += ca;
    v[7] += cb;
    v[8] += c;
  }
  if (MODE != kFromCoef) v[9] += l;
}

// accumulate one pair; returns its coefficient (for kLossOnly's store)
template <int LOSS, bool WEIGHTED, int MODE, bool MASKED = false>
__device__ __forceinline__ float accumulate(const float* E, float4 x, float wt, float* acc) {
  float c, l;
  pair_terms<LOSS, WEIGHTED, MODE, MASKED>(E, x, wt, c, l);
  add_terms<MODE>(c, l, x, acc);
  return c;
}

__device__ __forceinline__ void warp_store(float4* rec, int r, const float* v, int lane) {
  float s[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) s[k] = warp_sum(v[k]);
  if (lane == 0) store_record(rec, r, s);
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}

// shared memory per warp: kStages warp runs of keypoint pairs (each filled by
// one bulk copy), their weights (slot i filled by lane i % 32) and one
// mbarrier per stage
template <int U>
constexpr size_t smem_per_warp(bool weighted) {
  return kEaStages * 32 * U * (sizeof(float4) + (weighted ? sizeof(float) : 0)) + kEaStages * sizeof(uint64_t);
}

// state of a warp run, loaded before its pairs are processed
struct RunHead {
  int4 info;       // {first image pair, n_img | len << 8, record base, first pair}
  int desc;        // this lane's descriptor
  float Ereg[9];   // E of local image pair `lane` (lanes < n_img)
};

__device__ __forceinline__ void load_static_head(const DirectArgs& a, int w, int lane, RunHead& h) {
  h.info = __ldg(a.info + w);
  h.desc = __ldg(a.lane_desc + 32 * w + lane);
}

// the table entries are written by the preceding k_ea_tables launch: plain
// loads after the dependency wait
__device__ __forceinline__ void load_table_head(const DirectArgs& a, int lane, RunHead& h) {
  if (lane < (h.info.y & 0xff)) {
    const float4* e = a.seg_tab + 3 * (h.info.x + lane);
    const float4 e0 = e[0], e1 = e[1], e2 = e[2];
    h.Ereg[0] = e0.x; h.Ereg[1] = e0.y; h.Ereg[2] = e0.z; h.Ereg[3] = e0.w;
    h.Ereg[4] = e1.x; h.Ereg[5] = e1.y; h.Ereg[6] = e1.z; h.Ereg[7] = e1.w;
    h.Ereg[8] = e2.x;
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) h.Ereg[k] = 0.f;
  }
}

// the buffers start at zero, so that a lane reading past its own pairs
// (masked by a zero weight) only ever sees finite values: afterwards those
// slots hold earlier keypoints (finite, checked at creation) or stashed
// coefficients.  A weight slot is zeroed by the lane that later fills it; the
// keypoint slots are ordered before the bulk copies by a proxy fence.
template <int ROWS, bool WEIGHTED>
__device__ __forceinline__ void zero_buffers(int lane, float4* kb, float* wb) {
#pragma unroll
  for (int r = 0; r < ROWS; ++r) kb[32 * r + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (WEIGHTED)
#pragma unroll
    for (int r = 0; r < ROWS; ++r) wb[32 * r + lane] = 0.f;
}

// The coefficient of pair base + i goes into the x component of its own
// shared-memory slot (written only by the lane that owns the pair); the warp
// copies them out with coalesced stores after the warp run.
__device__ __forceinline__ void stash_coef(float4* kb, int i, float c) {
  reinterpret_cast<float*>(kb + i)[0] = c;
}

// Lane l owns pairs [off, off + cnt) of the warp run (cnt <= U), all of one
// image pair (local key): it takes E once, runs a branch-free U-step loop with
// a zero weight past cnt (stride-U float4 reads: conflict-free for odd U) and
// one accumulator.  A warp run inside one image pair ends with a butterfly
// sum; otherwise a segmented inclusive scan keyed by image pair (keys do not
// decrease with the lane) leaves each image pair's sum in its last lane.  Every
// (warp run, image pair) gets one record, summed in a fixed order.
template <int U, int LOSS, bool WEIGHTED, int MODE>
__device__ __forceinline__ void process(const DirectArgs& a, int lane, const RunHead& h, float4* kb,
                                        const float* wb) {
  const bool store = (MODE == kLossOnly) && a.coef_out != nullptr;
  const int n_img = h.info.y & 0xff;
  const int off = h.desc & ((1 << kDescCntShift) - 1);
  const int cnt = (h.desc >> kDescCntShift) & 31, key = h.desc >> kDescKeyShift;
  float E[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) E[q] = __shfl_sync(FULL, h.Ereg[q], key);
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.f;
#pragma unroll
  for (int k = 0; k < U; ++k) {
    const float4 x = kb[off + k];
    const float m = (k < cnt) ? 1.f : 0.f;
    const float wt = WEIGHTED ? wb[off + k] * m : m;
    float c, l;
    pair_terms<LOSS, WEIGHTED, MODE, true>(E, x, wt, c, l);
    if (MODE == kLossOnly && store && k < cnt) stash_coef(kb, off + k, c);
    add_terms<MODE>(c, l, x, acc);
  }
  if (n_img == 1) {
    warp_store(a.rec, h.info.z, acc, lane);
  } else {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int ku = __shfl_up_sync(FULL, key, d);
      const bool take = (lane >= d) && (ku == key);
#pragma unroll
      for (int c = 0; c < 10; ++c) {
        const float v = __shfl_up_sync(FULL, acc[c], d);
        if (take) acc[c] += v;
      }
    }
    const int key_next = __shfl_down_sync(FULL, key, 1);
    if (lane == 31 || key_next != key) store_record(a.rec, h.info.z + key, acc);
  }
  if (store) {
    // coalesced copy-out of the stashed coefficients
    __syncwarp();
    const int len = h.info.y >> 8;
#pragma unroll
    for (int r = 0; r < U; ++r) {
      const int i = 32 * r + lane;
      if (i < len) a.coef_out[h.info.w + i] = reinterpret_cast<const float*>(kb + i)[0];
    }
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t d;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(d) : "r"(bar), "r"(parity) : "memory");
  return d != 0;
}
constexpr int kBarPolls = 1 << 20;
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kBarPolls; ++i)
    if (bar_try(bar, parity)) return true;
  return false;
}

// lane 0 stages run `info`'s keypoint pairs with one bulk copy completing on bar
__device__ __forceinline__ void issue_bulk(const DirectArgs& a, int4 info, int lane, float4* kb, uint32_t bar) {
  if (lane == 0) {
    const int base = info.w, len = info.y >> 8;
    bar_expect_tx(bar, 16u * (uint32_t)len);   // len == 0: the arrive alone completes the phase
    if (len > 0)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                   ::"r"(smem_u32(kb)), "l"(a.kp + base), "r"(16u * (uint32_t)len), "r"(bar) : "memory");
  }
}

template <int U>
__device__ __forceinline__ void issue_weights(const DirectArgs& a, int4 info, int lane, float* wb) {
  const int base = info.w, len = info.y >> 8;
#pragma unroll
  for (int r = 0; r < U; ++r) {
    const int i = 32 * r + lane;
    if (i < len) cp_async4(wb + i, a.wts + base + i);
  }
}

// Schedule of a warp (persistent, runs w, w + stride, ...): kStages shared-
// memory buffers, each with an mbarrier.  One lane stages a run with a single
// bulk copy (TMA, cp.async.bulk) that completes on the buffer's mbarrier;
// while run k is processed, runs k + 1 .. k + kStages - 1 are in flight and
// the E entries of run k + 1 and the header of run k + kStages are being
// loaded, so that staging never waits on a header.  Weights (4 B per pair,
// not 16-B aligned per run) come with per-lane cp.async.  Every mbarrier wait
// is bounded: past the bound the warp sets kErrEaTimeout, waits (bounded) for
// its copies in flight and leaves.
template <int U, int LOSS, bool WEIGHTED, int MODE>
__global__ void __launch_bounds__(WARPS * 32, kEaMinCtas) k_ea_direct(DirectArgs a) {
  constexpr int WP = 32 * U;
  constexpr int S = kEaStages;
  extern __shared__ float4 smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float4* kb = smem + wib * S * WP;
  float* wb = WEIGHTED ? reinterpret_cast<float*>(smem + WARPS * S * WP) + wib * S * WP : nullptr;
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<float*>(smem + WARPS * S * WP) +
                                               (WEIGHTED ? WARPS * S * WP : 0)) + wib * S;
  const int stride = gridDim.x * WARPS;
  int w = blockIdx.x * WARPS + wib;
  if (w >= a.n_wruns) return;              // uniform per warp
  pdl_trigger();
  if (lane == 0) {
#pragma unroll
    for (int b = 0; b < S; ++b) bar_init(smem_u32(bars + b));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  zero_buffers<U * S, WEIGHTED>(lane, kb, wb);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  __syncwarp();
  // static heads (descriptor and run info) are loaded two runs before the
  // run's copy is issued: q[0 .. S-1] and far (run w + S stride)
  RunHead q[S];
  RunHead far;
#pragma unroll
  for (int k = 0; k < S; ++k)
    if (w + k * stride < a.n_wruns) load_static_head(a, w + k * stride, lane, q[k]);
  if (w + S * stride < a.n_wruns) load_static_head(a, w + S * stride, lane, far);
  unsigned pending = 0;                    // buffers with a bulk copy not yet waited for
#pragma unroll
  for (int k = 0; k < S - 1; ++k) {
    if (w + k * stride < a.n_wruns) {
      issue_bulk(a, q[k].info, lane, kb + k * WP, smem_u32(bars + k));
      pending |= 1u << k;
      if (WEIGHTED) issue_weights<U>(a, q[k].info, lane, wb + k * WP);
    }
    if (WEIGHTED) asm volatile("cp.async.commit_group;\n" ::);
  }
  pdl_wait();
  load_table_head(a, lane, q[0]);
  int buf = 0;
  unsigned phase = 0;                      // parity bit per buffer
  bool ok = true;
  for (; w < a.n_wruns; w += stride) {
    const int wl = w + (S - 1) * stride;
    int bl = buf + (S - 1);
    if (bl >= S) bl -= S;
    if (wl < a.n_wruns) {
      issue_bulk(a, q[S - 1].info, lane, kb + bl * WP, smem_u32(bars + bl));
      pending |= 1u << bl;
      if (WEIGHTED) issue_weights<U>(a, q[S - 1].info, lane, wb + bl * WP);
    }
    if (WEIGHTED) asm volatile("cp.async.commit_group;\n" ::);
    RunHead fresh;
    if (w + (S + 1) * stride < a.n_wruns) load_static_head(a, w + (S + 1) * stride, lane, fresh);
    if (w + stride < a.n_wruns) load_table_head(a, lane, q[1]);
    ok = bar_wait(smem_u32(bars + buf), (phase >> buf) & 1u);
    if (!__all_sync(FULL, ok)) { ok = false; break; }
    phase ^= 1u << buf;
    pending &= ~(1u << buf);
    if (WEIGHTED) asm volatile("cp.async.wait_group %0;\n" ::"n"(S - 1));
    __syncwarp();
    if ((q[0].info.y & 0xff) != 0)         // runs past the lanes in use are empty
      process<U, LOSS, WEIGHTED, MODE>(a, lane, q[0], kb + buf * WP, WEIGHTED ? wb + buf * WP : nullptr);
    // the buffer's generic reads and stash writes come before the next bulk
    // copy into it (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncwarp();
#pragma unroll
    for (int k = 0; k < S - 1; ++k) q[k] = q[k + 1];
    q[S - 1].info = far.info;
    q[S - 1].desc = far.desc;
    far.info = fresh.info;
    far.desc = fresh.desc;
    if (++buf == S) buf = 0;
  }
  if (!ok) {
    // a wait ran out: record it, then give every copy still in flight one
    // more bounded wait before the warp leaves its shared memory
    if (lane == 0) atomicOr(a.err, kErrEaTimeout);
#pragma unroll
    for (int b = 0; b < S; ++b)
      if (pending & (1u << b)) bar_wait(smem_u32(bars + b), (phase >> b) & 1u);
  }
  if (WEIGHTED) asm volatile("cp.async.wait_group 0;\n" ::);
}

// per image pair: sum its records -- or take dL/dE_n from a saved copy --
// scale, and apply the chain rule (step::segment_pair); kSegLanes lanes per
// image pair.
__global__ void k_ea_segments(SegArgs a) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = gid / step::kSegLanes;
  const int sub = gid % step::kSegLanes;
  pdl_trigger();
  const step::SegStatic st = step::seg_static(a, n);   // static tables: before the wait
  pdl_wait();               // records come from k_ea_direct
  step::segment_pair(a, n, sub, st);
}

}  // namespace

void launch_ea_tables(const float* params, const int* pi, const int* pj, const int* seg_off,
                      int P, float4* seg_tab, int* step_counter, cudaStream_t s, const float* phi, float* snap,
                      int n_snap) {
  launch_pdl(k_ea_tables, dim3((std::max(P, 1) + 127) / 128), dim3(128), 0, s, params, pi, pj, seg_off, P, seg_tab,
             step_counter, phi, snap, n_snap);
}

template <int U, int LOSS, bool WEIGHTED, int MODE>
static void launch_direct_u(const fm_problem* pr, const float* weights, float* coef_out, cudaStream_t s) {
  DirectArgs a;
  a.kp = pr->kp;
  a.wts = weights;
  a.lane_desc = pr->lane_desc;
  a.info = pr->wrun_info;
  a.seg_tab = pr->seg_tab;
  a.rec = pr->rec;
  a.coef_out = coef_out;
  a.err = pr->d_err;
  a.n_wruns = pr->n_wruns;
  const size_t smem = WARPS * smem_per_warp<U>(WEIGHTED);
  // resident CTAs per SM of this instantiation, per device: the shared-memory
  // limit is a per-device function attribute, set once on each device
  constexpr int kDevices = 64;
  static std::atomic<int> per_sm_dev[kDevices];
  const int dev = (pr->device >= 0 && pr->device < kDevices) ? pr->device : 0;
  int per_sm = per_sm_dev[dev].load(std::memory_order_relaxed);
  if (per_sm == 0) {
    cudaFuncSetAttribute(k_ea_direct<U, LOSS, WEIGHTED, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ea_direct<U, LOSS, WEIGHTED, MODE>, WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
    per_sm_dev[dev].store(per_sm, std::memory_order_relaxed);
  }
  const int want = pr->ea_ctas_per_sm > 0 ? std::min(pr->ea_ctas_per_sm, per_sm) : per_sm;
  int ctas = (pr->n_wruns + WARPS - 1) / WARPS;
  int cap = want * pr->sm_count;
  if (ctas > cap) ctas = cap;
  launch_pdl(k_ea_direct<U, LOSS, WEIGHTED, MODE>, dim3(ctas), dim3(WARPS * 32), smem, s, a);
}

// the tiles built into the library (pairs per lane, odd)
template <int LOSS, bool WEIGHTED, int MODE>
static void launch_direct_t(const fm_problem* pr, const float* weights, float* coef_out, cudaStream_t s) {
  switch (pr->ea_U) {
    case 11: launch_direct_u<11, LOSS, WEIGHTED, MODE>(pr, weights, coef_out, s); break;
    case 21: launch_direct_u<21, LOSS, WEIGHTED, MODE>(pr, weights, coef_out, s); break;
    default: launch_direct_u<15, LOSS, WEIGHTED, MODE>(pr, weights, coef_out, s); break;
  }
}

template <int U>
static int max_ctas_u() {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ea_direct<U, 0, false, kFull>, WARPS * 32,
                                                WARPS * smem_per_warp<U>(false));
  return per_sm > 0 ? per_sm : 1;
}

int direct_max_ctas_per_sm(const fm_problem* pr) {
  switch (pr->ea_U) {
    case 11: return max_ctas_u<11>();
    case 21: return max_ctas_u<21>();
    default: return max_ctas_u<15>();
  }
}

template <int MODE>
static void launch_direct_m(const fm_problem* pr, const float* weights, int loss, float* coef_out,
                            cudaStream_t s) {
  if (loss == FM_EA_L1) {
    if (weights) launch_direct_t<0, true, MODE>(pr, weights, coef_out, s);
    else launch_direct_t<0, false, MODE>(pr, nullptr, coef_out, s);
  } else {
    if (weights) launch_direct_t<1, true, MODE>(pr, weights, coef_out, s);
    else launch_direct_t<1, false, MODE>(pr, nullptr, coef_out, s);
  }
}

void launch_ea_direct(const fm_problem* pr, const float* weights, int loss, cudaStream_t s) {
  if (pr->n_wruns == 0) return;
  launch_direct_m<kFull>(pr, weights, loss, nullptr, s);
}

void launch_ea_direct_loss(const fm_problem* pr, const float* weights, int loss, float* coef_out,
                           cudaStream_t s) {
  if (pr->n_wruns == 0) return;
  launch_direct_m<kLossOnly>(pr, weights, loss, coef_out, s);
}

void launch_ea_direct_from_coef(const fm_problem* pr, const float* coef, cudaStream_t s) {
  if (pr->n_wruns == 0) return;
  launch_direct_t<0, true, kFromCoef>(pr, coef, nullptr, s);
}

SegArgs seg_args(const fm_problem* pr, const float* params) {
  SegArgs a;
  a.rec = pr->rec;
  a.seg_rec = pr->seg_rec;
  a.dlde_in = nullptr;
  a.params = params;
  a.pi = pr->pair_i;
  a.pj = pr->pair_j;
  a.P = pr->P;
  a.g_scale = 0.f;
  a.l_scale = 1.f;
  a.pair_scale = pr->pair_inv_z;
  a.grad_loss = nullptr;
  a.pair_scene = pr->pair_scene;
  a.seg_grad = pr->seg_grad;
  a.seg_loss = pr->seg_loss;
  a.dlde_out = nullptr;
  return a;
}

void launch_ea_segments(const SegArgs& a, cudaStream_t s) {
  const long long threads = (long long)a.P * step::kSegLanes;
  launch_pdl(k_ea_segments, dim3((unsigned)((threads + 127) / 128)), dim3(128), 0, s, a);
}

void launch_ea_segments(const fm_problem* pr, const float* params, int loss, cudaStream_t s) {
  SegArgs a = seg_args(pr, params);
  a.g_scale = (loss == FM_EA_L1) ? 1.f : 2.f;
  launch_ea_segments(a, s);
}

}  // namespace fm
