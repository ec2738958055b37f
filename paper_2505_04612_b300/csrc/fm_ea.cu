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
//   * a warp run is 15 rows of 32 consecutive pairs; lane l takes pair
//     base + 32 r + l of row r, so every row is one coalesced 512-B load
//     (LDG.128) and the warp issues all 15 rows before using them: 7.5 KB in
//     flight per warp, no shared memory, occupancy bounded by registers;
//   * the table entries (E and end offset) of the warp run's first 32 image
//     pairs sit one per lane in registers and are broadcast with shuffles;
//     entries beyond the first 32 come from global memory;
//   * a row that lies inside the current image pair is accumulated per lane
//     with no branches; a row that crosses one or more image-pair ends is
//     handled warp-uniformly: each lane finds its own image pair, the current
//     image pair is closed by a butterfly warp sum, image pairs that start and
//     end inside the row get their own warp sums, and the last one opens.
//     Every (warp run, image pair) gets exactly one record, summed in a fixed
//     order: no atomics, deterministic.
//
// Modes of k_ea_direct (the split of one evaluation into a forward and a
// backward pass, for the autograd adjoint):
//   kFull      loss and dL/dE together (one pass, 16 B per pair);
//   kLossOnly  the loss alone; optionally writes each pair's coefficient
//              c = w drho/dr (4 B per pair) for a later kFromCoef pass;
//   kFromCoef  dL/dE from stored coefficients: no residual is recomputed, but
//              the pair's x~2 x~1^T still needs the keypoints (16 + 4 B).
#include <algorithm>

#include "fm_device.cuh"
#include "fm_internal.h"

namespace fm {
namespace {

constexpr int WARPS = kEaWarpsPerCta;
constexpr unsigned FULL = 0xffffffffu;

__global__ void k_ea_tables(const float* params, const int* __restrict__ pi,
                            const int* __restrict__ pj, const int* __restrict__ seg_off, int P,
                            float4* __restrict__ tab, int* step_counter) {
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
  if (n >= P) return;
  float qi[9], qj[9];
  load_plain(params + 9 * ci, qi, 9);
  load_plain(params + 9 * cj, qj, 9);
  PairGeo g;
  pair_geometry(qi, qj, g);
  float E[9];
  essential(g, E);
  tab[3 * n + 0] = make_float4(E[0], E[1], E[2], E[3]);
  tab[3 * n + 1] = make_float4(E[4], E[5], E[6], E[7]);
  tab[3 * n + 2] = make_float4(E[8], __int_as_float(end), 0.f, 0.f);
}

enum DirectMode { kFull = 0, kLossOnly = 1, kFromCoef = 2 };

struct DirectArgs {
  const float4* kp;
  const float* wts;      // per-pair weights; the stored coefficients in kFromCoef
  int rows_max;          // warp runs touching at most this many image pairs go row by row
  const int* run_seg;
  const int4* info;
  const float4* seg_tab;
  float4* rec;
  float* coef_out;       // kLossOnly: per-pair coefficients when not null
  int Z;
  int n_wruns;
};


__device__ __forceinline__ void store_record(float4* rec, int r, const float* v) {
  rec[3 * r + 0] = make_float4(v[0], v[1], v[2], v[3]);
  rec[3 * r + 1] = make_float4(v[4], v[5], v[6], v[7]);
  rec[3 * r + 2] = make_float4(v[8], v[9], 0.f, 0.f);
}

// table entry t (local image-pair index of the warp run): lanes hold entries
// 0..31 in registers; later entries are read from global memory
struct Entry {
  float E[9];
  int end;
};

__device__ __forceinline__ void entry_uniform(const float* Ereg, int endreg, const float4* seg_tab,
                                              int s_first, int t, Entry& o) {
  if (t < 32) {
#pragma unroll
    for (int k = 0; k < 9; ++k) o.E[k] = __shfl_sync(FULL, Ereg[k], t);
    o.end = __shfl_sync(FULL, endreg, t);
  } else {
    const float4* e = seg_tab + 3 * (s_first + t);
    const float4 e0 = e[0], e1 = e[1], e2 = e[2];
    o.E[0] = e0.x; o.E[1] = e0.y; o.E[2] = e0.z; o.E[3] = e0.w;
    o.E[4] = e1.x; o.E[5] = e1.y; o.E[6] = e1.z; o.E[7] = e1.w;
    o.E[8] = e2.x;
    o.end = __float_as_int(e2.y);
  }
}

__device__ __forceinline__ int end_uniform(int endreg, const float4* seg_tab, int s_first, int t) {
  if (t < 32) return __shfl_sync(FULL, endreg, t);
  return __float_as_int(seg_tab[3 * (s_first + t) + 2].y);
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

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async16_partial(void* smem, const void* gmem, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes));
}

// shared memory per warp: two warp runs of keypoint pairs (double buffer),
// row-major (row r, lane l at 32 r + l: conflict-free 512-B row reads), and
// their weights
template <int U>
constexpr size_t smem_per_warp(bool weighted) {
  return 2 * 32 * U * (sizeof(float4) + (weighted ? sizeof(float) : 0));
}

// state of a warp run prefetched before its rows are processed
struct RunHead {
  int4 info;       // {first image pair, #image pairs, record base}
  float Ereg[9];   // table entry of local image pair `lane`
  int endreg;
  int rs;          // image pair of this lane's first pair in the lane-contiguous split
};

template <int U, bool WEIGHTED>
__device__ __forceinline__ void issue_rows(const DirectArgs& a, int w, int lane, float4* kb, float* wb) {
  constexpr int WP = 32 * U, ROWS = U;
  const int base = w * WP;
  // slots past Z are zero-filled (src-size 0), so that no lane ever reads
  // stale shared memory
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int p = base + 32 * r + lane;
    if (p < a.Z) cp_async16(kb + 32 * r + lane, a.kp + p);
    else cp_async16_partial(kb + 32 * r + lane, a.kp, 0);
  }
  if (WEIGHTED) {
#pragma unroll
    for (int k = 0; k < (WP / 4 + 31) / 32; ++k) {
      const int c = lane + 32 * k;
      if (c < WP / 4) {
        const int p4 = base + 4 * c;
        const int bytes = 4 * max(0, min(4, a.Z - p4));
        cp_async16_partial(wb + 4 * c, bytes > 0 ? a.wts + p4 : a.wts, bytes);
      }
    }
  }
  asm volatile("cp.async.commit_group;\n" ::);
}

__device__ __forceinline__ void load_static_head(const DirectArgs& a, int w, int lane, RunHead& h) {
  h.info = __ldg(a.info + w);
  h.rs = __ldg(a.run_seg + 32 * w + lane);
}

// the table entries are written by the preceding k_ea_tables launch
__device__ __forceinline__ void load_table_head(const DirectArgs& a, int lane, RunHead& h) {
  h.endreg = 0x7fffffff;
  if (lane < h.info.y) {
    const float4* e = a.seg_tab + 3 * (h.info.x + lane);
    const float4 e0 = e[0], e1 = e[1], e2 = e[2];
    h.Ereg[0] = e0.x; h.Ereg[1] = e0.y; h.Ereg[2] = e0.z; h.Ereg[3] = e0.w;
    h.Ereg[4] = e1.x; h.Ereg[5] = e1.y; h.Ereg[6] = e1.z; h.Ereg[7] = e1.w;
    h.Ereg[8] = e2.x;
    h.endreg = __float_as_int(e2.y);
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) h.Ereg[k] = 0.f;
  }
}

// The coefficient of pair base + i goes into the x component of its own
// shared-memory slot (read only by the lane that stores it); the warp copies
// them out with coalesced stores after the warp run (coef_store).
__device__ __forceinline__ void stash_coef(float4* kb, int i, float c) {
  reinterpret_cast<float*>(kb + i)[0] = c;
}

// Row-major processing: right for warp runs that touch one or two image pairs
// (at most one image-pair end to cross with a warp reduction).
template <int U, int LOSS, bool WEIGHTED, int MODE>
__device__ __forceinline__ void process_rows(const DirectArgs& a, int w, int lane, const RunHead& h,
                                             float4* kb, const float* wb, bool store) {
  constexpr int WP = 32 * U;
  const int base = w * WP;
  const int4 info = h.info;
  const int wend = min(base + WP, a.Z);    // one past the warp run's last pair
  const int full_rows = (wend - base) >> 5; // rows with 32 valid pairs
  int j = 0;                               // current local image pair (uniform)
  Entry cur;
  entry_uniform(h.Ereg, h.endreg, a.seg_tab, info.x, 0, cur);
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.f;

  int r = 0;
  const int n_rows = (wend - base + 31) >> 5;
  while (r < n_rows) {
    // rows [r, r_in) lie inside the current image pair and are full: no checks
    const int r_in = min(full_rows, max(r, (cur.end - base) >> 5));
    if (r < r_in) {
      int q = r;
#pragma unroll 1
      for (; q + 4 <= r_in; q += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 32 * (q + u) + lane;
          const float c = accumulate<LOSS, WEIGHTED, MODE>(cur.E, kb[i], WEIGHTED ? wb[i] : 1.f, acc);
          if (MODE == kLossOnly && store) stash_coef(kb, i, c);
        }
      }
#pragma unroll 1
      for (; q < r_in; ++q) {
        const int i = 32 * q + lane;
        const float c = accumulate<LOSS, WEIGHTED, MODE>(cur.E, kb[i], WEIGHTED ? wb[i] : 1.f, acc);
        if (MODE == kLossOnly && store) stash_coef(kb, i, c);
      }
      r = r_in;
      continue;
    }
    // row r crosses an image-pair end, or is the partial last row
    const int row_lo = base + 32 * r;
    const int row_hi = min(row_lo + 32, wend);
    const bool valid = row_lo + lane < wend;
    const float4 x = valid ? kb[32 * r + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float wt = valid ? (WEIGHTED ? wb[32 * r + lane] : 1.f) : 0.f;
    if (row_hi <= cur.end) {
      const float c = accumulate<LOSS, WEIGHTED, MODE, true>(cur.E, x, wt, acc);
      if (MODE == kLossOnly && store && valid) stash_coef(kb, 32 * r + lane, c);
      ++r;
      continue;
    }
    int jl_last = j;
    while (end_uniform(h.endreg, a.seg_tab, info.x, jl_last) < row_hi) ++jl_last;
    const int p = min(row_lo + lane, wend - 1);
    int jl = j;
    for (int t = j; t < jl_last; ++t) jl += (p >= end_uniform(h.endreg, a.seg_tab, info.x, t)) ? 1 : 0;
    float El[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) El[k] = __shfl_sync(FULL, h.Ereg[k], jl & 31);   // all lanes take part
    if (jl >= 32) {
      const float4* e = a.seg_tab + 3 * (info.x + jl);
      const float4 e0 = e[0], e1 = e[1], e2 = e[2];
      El[0] = e0.x; El[1] = e0.y; El[2] = e0.z; El[3] = e0.w;
      El[4] = e1.x; El[5] = e1.y; El[6] = e1.z; El[7] = e1.w;
      El[8] = e2.x;
    }
    float v[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) v[k] = 0.f;
    if (valid) {
      const float c = accumulate<LOSS, WEIGHTED, MODE, true>(El, x, wt, v);
      if (MODE == kLossOnly && store) stash_coef(kb, 32 * r + lane, c);
    }
    // close the current image pair
    float t10[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) t10[k] = acc[k] + ((jl == j) ? v[k] : 0.f);
    warp_store(a.rec, info.z + j, t10, lane);
    // image pairs that start and end inside this row
    for (int t = j + 1; t < jl_last; ++t) {
#pragma unroll
      for (int k = 0; k < 10; ++k) t10[k] = (jl == t) ? v[k] : 0.f;
      warp_store(a.rec, info.z + t, t10, lane);
    }
    // open the last one
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = (jl == jl_last) ? v[k] : 0.f;
    j = jl_last;
    entry_uniform(h.Ereg, h.endreg, a.seg_tab, info.x, j, cur);
    ++r;
  }
  warp_store(a.rec, info.z + j, acc, lane);
}

// Lane-contiguous processing for warp runs that touch three or more image
// pairs: lane l owns pairs [base + 15 l, base + 15 l + 15) (stride 15 float4 in
// shared memory: conflict-free since 15 is odd).  A lane whose run crosses at
// most one image-pair end splits it into a head part (its first image pair)
// and a tail part with a branch-free two-accumulator loop; a lane crossing two
// or more ends walks its pairs one by one and writes the image pairs that lie
// wholly inside its run.  A segmented scan keyed by image pair then combines
// the tails of consecutive lanes and absorbs heads, in fixed lane order.
template <int U, int LOSS, bool WEIGHTED, int MODE>
__device__ __forceinline__ void process_lanes(const DirectArgs& a, int w, int lane, const RunHead& h,
                                              float4* kb, const float* wb, bool store) {
  constexpr int WP = 32 * U;
  const int base = w * WP;
  const int4 info = h.info;
  const int wend = min(base + WP, a.Z);
  const int p0 = base + lane * U;
  const int pend = min(p0 + U, wend);
  const int j0 = h.rs - info.x;             // local image pair of the lane's first pair
  float E0[9], E1[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    E0[k] = __shfl_sync(FULL, h.Ereg[k], j0 & 31);
    E1[k] = __shfl_sync(FULL, h.Ereg[k], (j0 + 1) & 31);
  }
  const int end0 = __shfl_sync(FULL, h.endreg, j0 & 31);
  const int end1 = __shfl_sync(FULL, h.endreg, (j0 + 1) & 31);
  // split: pairs [p0, min(end0, pend)) are the head, the rest (if any) the tail
  const bool one_part = pend <= end0;
  const bool two_parts = !one_part && (j0 + 1 < 32) && (pend <= end1) && (end1 > end0);
  const bool fast = (j0 < 32) && (one_part || two_parts);
  float acc_h[10], acc_t[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    acc_h[k] = 0.f;
    acc_t[k] = 0.f;
  }
  int head_key = j0, key = j0;
  bool has_head = false;
  if (fast) {
    const int b = min(end0, pend) - p0;    // head pairs (>= 1)
    const int n = pend - p0;               // valid pairs of this lane (may be < U at the end)
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const float4 x = kb[lane * U + k];
      const bool in_head = k < b;
      float E[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) E[q] = in_head ? E0[q] : E1[q];
      const float wt = (k < n) ? (WEIGHTED ? wb[lane * U + k] : 1.f) : 0.f;
      float c, l;
      pair_terms<LOSS, WEIGHTED, MODE, true>(E, x, wt, c, l);
      if (MODE == kLossOnly && store && k < n) stash_coef(kb, lane * U + k, c);
      const float ch = in_head ? c : 0.f, ct = c - ch;
      const float lh = in_head ? l : 0.f, lt = l - lh;
      add_terms<MODE>(ch, lh, x, acc_h);
      add_terms<MODE>(ct, lt, x, acc_t);
    }
    if (two_parts) {
      has_head = true;
      key = j0 + 1;
    } else {
#pragma unroll
      for (int k = 0; k < 10; ++k) acc_t[k] = acc_h[k];
    }
  } else if (p0 < wend) {
    // two or more image-pair ends inside the lane's run: one pair at a time
    int s = info.x + j0, sl = j0;
    const float4* e = a.seg_tab + 3 * s;
    float4 e0 = e[0], e1 = e[1], e2 = e[2];
    int end = __float_as_int(e2.y);
    for (int p = p0; p < pend; ++p) {
      while (p >= end) {
        if (!has_head) {
#pragma unroll
          for (int k = 0; k < 10; ++k) acc_h[k] = acc_t[k];
          has_head = true;
        } else {
          store_record(a.rec, info.z + sl, acc_t);
        }
#pragma unroll
        for (int k = 0; k < 10; ++k) acc_t[k] = 0.f;
        ++s;
        ++sl;
        e = a.seg_tab + 3 * s;
        e0 = e[0];
        e1 = e[1];
        e2 = e[2];
        end = __float_as_int(e2.y);
      }
      const float Es[9] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w, e2.x};
      const int i = lane * U + (p - p0);
      const float c = accumulate<LOSS, WEIGHTED, MODE>(Es, kb[i], WEIGHTED ? wb[i] : 1.f, acc_t);
      if (MODE == kLossOnly && store) stash_coef(kb, i, c);
    }
    key = sl;
  }
  // lanes past the end of the data keep key = j0 (the last image pair) and zeros

  // segmented inclusive scan of the tails keyed by local image pair
  float sc[10];
#pragma unroll
  for (int c = 0; c < 10; ++c) sc[c] = acc_t[c];
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
    const float hv = __shfl_down_sync(FULL, acc_h[c], 1);
    if (absorb) sc[c] += hv;
  }
  if (last_of_key) store_record(a.rec, info.z + key, sc);
  if (has_head && (lane == 0 || key_prev != head_key)) store_record(a.rec, info.z + head_key, acc_h);
}

template <int U, int LOSS, bool WEIGHTED, int MODE>
__device__ __forceinline__ void process(const DirectArgs& a, int w, int lane, const RunHead& h,
                                        float4* kb, const float* wb) {
  constexpr int WP = 32 * U, ROWS = U;
  const bool store = (MODE == kLossOnly) && a.coef_out != nullptr;
  if (h.info.y <= a.rows_max) process_rows<U, LOSS, WEIGHTED, MODE>(a, w, lane, h, kb, wb, store);
  else process_lanes<U, LOSS, WEIGHTED, MODE>(a, w, lane, h, kb, wb, store);
  if (store) {
    // coalesced copy-out of the stashed coefficients
    __syncwarp();
    const int base = w * WP;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int i = 32 * r + lane;
      if (base + i < a.Z) a.coef_out[base + i] = reinterpret_cast<const float*>(kb + i)[0];
    }
  }
}

template <int U, int LOSS, bool WEIGHTED, int MODE>
__global__ void __launch_bounds__(WARPS * 32, kEaMinCtas) k_ea_direct(DirectArgs a) {
  constexpr int WP = 32 * U;
  extern __shared__ float4 smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float4* kb = smem + wib * 2 * WP;
  float* wb = WEIGHTED ? reinterpret_cast<float*>(smem + WARPS * 2 * WP) + wib * 2 * WP : nullptr;
  const int stride = gridDim.x * WARPS;
  int w = blockIdx.x * WARPS + wib;
  if (w >= a.n_wruns) return;              // uniform per warp
  pdl_trigger();
  RunHead head;
  load_static_head(a, w, lane, head);
  issue_rows<U, WEIGHTED>(a, w, lane, kb, wb);   // the keypoints do not depend on the predecessor
  pdl_wait();
  load_table_head(a, lane, head);
  for (int it = 0; w < a.n_wruns; ++it, w += stride) {
    const int cur = it & 1;
    const int wn = w + stride;
    RunHead next;
    if (wn < a.n_wruns) {
      load_static_head(a, wn, lane, next);
      load_table_head(a, lane, next);
      issue_rows<U, WEIGHTED>(a, wn, lane, kb + (cur ^ 1) * WP, WEIGHTED ? wb + (cur ^ 1) * WP : nullptr);
      asm volatile("cp.async.wait_group 1;\n" ::);
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::);
    }
    __syncwarp();
    process<U, LOSS, WEIGHTED, MODE>(a, w, lane, head, kb + cur * WP, WEIGHTED ? wb + cur * WP : nullptr);
    __syncwarp();   // this buffer is refilled two warp runs later
    head = next;
  }
}

// per image pair: sum its records -- or take dL/dE_n from a saved copy --
// scale, and apply the chain rule.  kSegLanes lanes share an image pair: they
// sum its records with a stride of kSegLanes and combine them with a
// butterfly inside the group (a fixed order), so that image pairs spanning
// many warp runs are not summed by one thread; the group's first lane then
// applies the chain rule.
constexpr int kSegLanes = 8;

__global__ void k_ea_segments(SegArgs a) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = gid / kSegLanes;
  const int sub = gid % kSegLanes;
  pdl_trigger();
  const bool valid = n < a.P;
  int r0 = 0, cnt = 0, ci = 0, cj = 0;
  if (valid) {
    r0 = a.seg_rec[2 * n];
    cnt = a.seg_rec[2 * n + 1];
    ci = a.pi[n];
    cj = a.pj[n];
  }
  pdl_wait();               // records come from k_ea_direct
  float G[10];
  for (int k = 0; k < 10; ++k) G[k] = 0.f;
  if (valid && !a.dlde_in) {
    for (int r = r0 + sub; r < r0 + cnt; r += kSegLanes) {
      const float4 v0 = a.rec[3 * r], v1 = a.rec[3 * r + 1], v2 = a.rec[3 * r + 2];
      G[0] += v0.x; G[1] += v0.y; G[2] += v0.z; G[3] += v0.w;
      G[4] += v1.x; G[5] += v1.y; G[6] += v1.z; G[7] += v1.w;
      G[8] += v2.x; G[9] += v2.y;
    }
  }
#pragma unroll
  for (int d = kSegLanes / 2; d > 0; d >>= 1)
#pragma unroll
    for (int k = 0; k < 10; ++k) G[k] += __shfl_xor_sync(0xffffffffu, G[k], d);
  if (!valid || sub != 0) return;
  const float ps = a.pair_scale ? a.pair_scale[n] : 1.f;
  if (a.dlde_in) {
    for (int k = 0; k < 9; ++k) G[k] = a.dlde_in[9 * (size_t)n + k];
  } else {
    const float gs = a.g_scale * ps;
    for (int k = 0; k < 9; ++k) G[k] *= gs;
  }
  if (a.seg_loss) a.seg_loss[n] = G[9] * (a.l_scale * ps);
  if (a.dlde_out)
    for (int k = 0; k < 9; ++k) a.dlde_out[9 * (size_t)n + k] = G[k];
  if (!a.seg_grad) return;
  float* out = a.seg_grad + (size_t)kSegGradEa * n;
  if (cnt == 0) {   // an image pair without keypoint pairs (its geometry may be degenerate)
    for (int k = 0; k < kSegGradEa; ++k) out[k] = 0.f;
    return;
  }
  if (a.grad_loss) {
    const float gl = a.grad_loss[a.pair_scene ? a.pair_scene[n] : 0];
    for (int k = 0; k < 9; ++k) G[k] *= gl;
  }
  float qi[9], qj[9];
  load_plain(a.params + 9 * ci, qi, 9);
  load_plain(a.params + 9 * cj, qj, 9);
  PairGeo g;
  pair_geometry(qi, qj, g);
  float o[kSegGradEa];
  pair_backward(g, G, o);
  if ((reinterpret_cast<uintptr_t>(out) & 15u) == 0) {   // library buffers: 96-B rows, 16-B aligned
    float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll
    for (int k = 0; k < kSegGradEa / 4; ++k) o4[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
  } else {
    for (int k = 0; k < kSegGradEa; ++k) out[k] = o[k];
  }
}

}  // namespace

void launch_ea_tables(const float* params, const int* pi, const int* pj, const int* seg_off,
                      int P, float4* seg_tab, int* step_counter, cudaStream_t s) {
  launch_pdl(k_ea_tables, dim3((P + 127) / 128), dim3(128), 0, s, params, pi, pj, seg_off, P, seg_tab,
             step_counter);
}

template <int U, int LOSS, bool WEIGHTED, int MODE>
static void launch_direct_u(const fm_problem* pr, const float* weights, float* coef_out, cudaStream_t s) {
  DirectArgs a;
  a.kp = pr->kp;
  a.wts = weights;
  a.rows_max = pr->ea_rows_max;
  a.run_seg = pr->run_seg;
  a.info = pr->wrun_info;
  a.seg_tab = pr->seg_tab;
  a.rec = pr->rec;
  a.coef_out = coef_out;
  a.Z = (int)pr->Z;
  a.n_wruns = pr->n_wruns;
  const size_t smem = WARPS * smem_per_warp<U>(WEIGHTED);
  static int per_sm = 0;   // resident CTAs per SM (one device per process)
  if (per_sm == 0) {
    cudaFuncSetAttribute(k_ea_direct<U, LOSS, WEIGHTED, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ea_direct<U, LOSS, WEIGHTED, MODE>, WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
  }
  const int want = pr->ea_ctas_per_sm > 0 ? std::min(pr->ea_ctas_per_sm, per_sm) : per_sm;
  int ctas = (pr->n_wruns + WARPS - 1) / WARPS;
  int cap = want * pr->sm_count;
  if (ctas > cap) ctas = cap;
  launch_pdl(k_ea_direct<U, LOSS, WEIGHTED, MODE>, dim3(ctas), dim3(WARPS * 32), smem, s, a);
}

// the tile sizes the library is built with (pairs per lane, odd)
template <int LOSS, bool WEIGHTED, int MODE>
static void launch_direct_t(const fm_problem* pr, const float* weights, float* coef_out, cudaStream_t s) {
  if (pr->ea_U == 11) launch_direct_u<11, LOSS, WEIGHTED, MODE>(pr, weights, coef_out, s);
  else launch_direct_u<15, LOSS, WEIGHTED, MODE>(pr, weights, coef_out, s);
}

int direct_max_ctas_per_sm(const fm_problem* pr) {
  const size_t smem = WARPS * (pr->ea_U == 11 ? smem_per_warp<11>(false) : smem_per_warp<15>(false));
  int per_sm = 0;
  if (pr->ea_U == 11)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ea_direct<11, 0, false, kFull>, WARPS * 32, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ea_direct<15, 0, false, kFull>, WARPS * 32, smem);
  return per_sm > 0 ? per_sm : 1;
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
  const long long threads = (long long)a.P * kSegLanes;
  launch_pdl(k_ea_segments, dim3((unsigned)((threads + 127) / 128)), dim3(128), 0, s, a);
}

void launch_ea_segments(const fm_problem* pr, const float* params, int loss, cudaStream_t s) {
  SegArgs a = seg_args(pr, params);
  a.g_scale = (loss == FM_EA_L1) ? 1.f : 2.f;
  launch_ea_segments(a, s);
}

}  // namespace fm
