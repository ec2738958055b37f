// Per-camera assembly and optimiser step: a camera's gradient is the sum,
// over the image pairs it belongs to (camera CSR, fixed order), of the
// per-image-pair gradients; rotations then go through the adjoint of the 6D
// map (Sec. 3.3), and Adam updates the camera's parameters in place.
//
// k_cam          one CTA per camera: thread t adds the incident image pairs
//                t, t + 128, ... (the first two read from the CSR before the
//                dependency wait), warps combine by butterflies and in warp
//                order, warp 0 applies the adjoint and Adam; its parameters
//                and moments are loaded while the parts are gathered.  When a
//                loss is wanted, more CTAs of the same launch sum it, one per
//                slice of 256 image pairs, while the cameras are updated.
// k_sum_fixed    the same loss slices alone.
// k_cam_ea       the epipolar step after k_ea_direct in one launch: one CTA
//                per camera whose threads each take an incident image pair,
//                add its records, apply the normalisers and the chain rule
//                themselves (the per-image-pair pass folded in: every image
//                pair's chain rule is evaluated by both of its cameras), then
//                the camera's sum and Adam as in k_cam; the loss CTAs form
//                each image pair's loss term from its records.  Same sums in
//                the same order as k_ea_segments followed by k_cam, so the
//                results are bit-identical; one launch and one dependency
//                wait instead of three (measured on the 5M-pair scene: each
//                wait after a predecessor's end costs ~1.1 us).
#include "fm_step.cuh"

namespace fm {
namespace {

using step::kThreads;
using step::Layout;

template <int STAGE, bool ADAM>
__global__ void __launch_bounds__(kThreads) k_cam(CamUpdate u) {
  using L = Layout<STAGE>;
  __shared__ float red[kThreads / 32][L::PART];
  const int run = blockIdx.y;
  pdl_trigger();
  if ((int)blockIdx.x >= u.N) {   // loss slices
    const int g = blockIdx.x - u.N;
    const int sc = step::slice_scene(u.loss.sc_slice_off, u.loss.S, g);
    const float* x = u.seg_loss + (size_t)run * u.P + u.loss.sc_pair_off[sc];
    pdl_wait();
    step::loss_slice(u.loss, sc, g, run, [&](int j, int k, float* v) { step::fill_stored(x, j, k, v); });
    return;
  }
  const int c = blockIdx.x, t = threadIdx.x, lane = t & 31;
  // static: before the wait
  const int b = u.cam_seg_off[c], e = u.cam_seg_off[c + 1];
  // this thread's first two camera-CSR entries, before the wait
  const int pre0 = (b + t < e && !u.csr_order) ? __ldg(u.cam_seg + b + t) : -1;
  const int pre1 = (b + t + kThreads < e && !u.csr_order) ? __ldg(u.cam_seg + b + t + kThreads) : -1;
  pdl_wait();
  // parameters and moments do not depend on the gather: loaded with it
  const size_t off = ((size_t)run * u.N + c) * L::PDIM;
  float p[L::PDIM];
  float m = 0.f, v = 0.f;
  step::CamPre cpre;
  if (t < 32) {
#pragma unroll
    for (int k = 0; k < L::PDIM; ++k) p[k] = u.params[off + k];
    if (ADAM && lane < L::PDIM) {
      m = u.m[off + lane];
      v = u.v[off + lane];
    }
    step::cam_pre<STAGE, ADAM>(u, p, cpre);
  }
  float acc[L::PART];
#pragma unroll
  for (int k = 0; k < L::PART; ++k) acc[k] = 0.f;
  const float* sg = u.seg_grad + (size_t)run * u.P * 2 * L::STRIDE;
  if (u.csr_order) {   // the parts already in camera-CSR order: contiguous, same order of additions
    for (int idx = b + t; idx < e; idx += kThreads)
      step::cam_add_part<L::PART, L::STRIDE>(sg + (size_t)idx * L::STRIDE, acc);
  } else {
    if (pre0 != -1) step::cam_add<L::PART, L::STRIDE>(sg, pre0, acc);
    if (pre1 != -1) step::cam_add<L::PART, L::STRIDE>(sg, pre1, acc);
    for (int idx = b + t + 2 * kThreads; idx < e; idx += kThreads)
      step::cam_add<L::PART, L::STRIDE>(sg, __ldg(u.cam_seg + idx), acc);
  }
  step::cam_reduce<L::PART>(acc, red);
  if (t < 32) step::cam_apply<STAGE, ADAM>(u, off, p, m, v, acc, lane, cpre);
}

// the loss slices alone: seg_loss summed per (scene, run)
__global__ void __launch_bounds__(kThreads) k_sum_fixed(const float* __restrict__ x, int P, LossArgs L) {
  const int g = blockIdx.x, run = blockIdx.y;
  pdl_trigger();
  const int sc = step::slice_scene(L.sc_slice_off, L.S, g);
  const float* xs = x + (size_t)run * P + L.sc_pair_off[sc];
  pdl_wait();
  step::loss_slice(L, sc, g, run, [&](int j, int k, float* v) { step::fill_stored(xs, j, k, v); });
}

// one incident image pair of a camera in k_cam_ea: camera-CSR entry, role,
// and its static inputs
struct CamEntry {
  int n = 0;
  bool role_j = false;
  bool ok = false;
  step::SegStatic st;
};

__device__ __forceinline__ CamEntry cam_entry(const SegArgs& s, const int* __restrict__ cam_seg, int idx, int e) {
  CamEntry c;
  c.ok = idx < e;
  const unsigned w = c.ok ? (unsigned)__ldg(cam_seg + idx) : 0u;
  c.n = (int)(w & 0x7fffffffu);
  c.role_j = (w >> 31) != 0;
  c.st = step::seg_static(s, c.ok ? c.n : s.P);
  return c;
}

// the part of camera entry c (dL/dR, dL/dt of its role) from records, with
// the cameras' parameters qi, qj loaded beforehand
__device__ __forceinline__ void cam_entry_part(const SegArgs& s, const CamEntry& c, const float* qi, const float* qj,
                                               float* acc) {
  float G[10];
  step::rec_sum_serial(s.rec, c.st.r0, c.st.cnt, G);
  const float gs = s.g_scale * (s.pair_scale ? s.pair_scale[c.n] : 1.f);
  for (int k = 0; k < 9; ++k) G[k] *= gs;
  float o[kSegGradEa];
  step::pair_grad(s, c.n, c.st.cnt, G, qi, qj, o);
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] += c.role_j ? o[12 + k] : o[k];
}

__device__ __forceinline__ void cam_entry_params(const SegArgs& s, const CamEntry& c, float* qi, float* qj) {
  if (c.ok && c.st.cnt > 0) {
    load_plain(s.params + 9 * c.st.ci, qi, 9);
    load_plain(s.params + 9 * c.st.cj, qj, 9);
  }
}

// 3 CTAs per SM: the 5M-pair scene's 300 camera CTAs and their loss CTAs run
// in one wave
template <bool ADAM>
__global__ void __launch_bounds__(kThreads, 3) k_cam_ea(EaCamArgs f) {
  __shared__ float red[kThreads / 32][12];
  const SegArgs& s = f.s;
  const CamUpdate& u = f.u;
  pdl_trigger();
  if ((int)blockIdx.x >= u.N) {   // loss slices: each image pair's loss term from its records
    const int g = blockIdx.x - u.N;
    const int sc = step::slice_scene(u.loss.sc_slice_off, u.loss.S, g);
    int j, k;
    step::slice_terms(u.loss, sc, g, j, k);
    step::RecRanges R;
    step::rec_ranges(s, u.loss.sc_pair_off[sc], j, k, R);   // static: before the wait
    pdl_wait();
    step::loss_slice(u.loss, sc, g, 0, [&](int, int kk, float* v) { step::fill_from_records(s, R, kk, v); });
    return;
  }
  const int c = blockIdx.x, t = threadIdx.x, lane = t & 31;
  // static: this thread's first two incident image pairs, before the wait
  const int b = u.cam_seg_off[c], e = u.cam_seg_off[c + 1];
  const CamEntry e0 = cam_entry(s, u.cam_seg, b + t, e);
  const CamEntry e1 = cam_entry(s, u.cam_seg, b + t + kThreads, e);
  pdl_wait();
  const size_t off = (size_t)c * 9;
  float p[9];
  float m = 0.f, v = 0.f;
  step::CamPre cpre;
  if (t < 32) {
#pragma unroll
    for (int k = 0; k < 9; ++k) p[k] = u.params[off + k];
    if (ADAM && lane < 9) {
      m = u.m[off + lane];
      v = u.v[off + lane];
    }
    step::cam_pre<2, ADAM>(u, p, cpre);
  }
  float acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = 0.f;
  // both entries' parameters first, then their records and chain rules, in
  // CSR order
  float qi0[9], qj0[9], qi1[9], qj1[9];
  cam_entry_params(s, e0, qi0, qj0);
  cam_entry_params(s, e1, qi1, qj1);
  if (e0.ok) cam_entry_part(s, e0, qi0, qj0, acc);
  if (e1.ok) cam_entry_part(s, e1, qi1, qj1, acc);
  for (int idx = b + t + 2 * kThreads; idx < e; idx += kThreads) {
    const CamEntry en = cam_entry(s, u.cam_seg, idx, e);
    float qi[9], qj[9];
    cam_entry_params(s, en, qi, qj);
    cam_entry_part(s, en, qi, qj, acc);
  }
  step::cam_reduce<12>(acc, red);
  if (t < 32) step::cam_apply<2, ADAM>(u, off, p, m, v, acc, lane, cpre);
}

template <int STAGE>
void launch_stage(const CamUpdate& u, cudaStream_t s) {
  dim3 grid(u.N + (u.loss.out ? u.loss.n_slices : 0), u.runs);
  if (u.params_out) launch_pdl(k_cam<STAGE, true>, grid, dim3(kThreads), 0, s, u);
  else launch_pdl(k_cam<STAGE, false>, grid, dim3(kThreads), 0, s, u);
}

}  // namespace

void launch_cam_update(int stage, const CamUpdate& u, cudaStream_t s) {
  if (stage == FM_STAGE_ROTATION) launch_stage<0>(u, s);
  else if (stage == FM_STAGE_TRANSLATION) launch_stage<1>(u, s);
  else launch_stage<2>(u, s);
}

void launch_sum_fixed(const float* x, int P, int runs, const LossArgs& L, cudaStream_t s) {
  launch_pdl(k_sum_fixed, dim3(L.n_slices, runs), dim3(kThreads), 0, s, x, P, L);
}

void launch_cam_ea(const EaCamArgs& f, cudaStream_t s) {
  dim3 grid(f.u.N + (f.u.loss.out ? f.u.loss.n_slices : 0));
  if (f.u.params_out) launch_pdl(k_cam_ea<true>, grid, dim3(kThreads), 0, s, f);
  else launch_pdl(k_cam_ea<false>, grid, dim3(kThreads), 0, s, f);
}

}  // namespace fm
