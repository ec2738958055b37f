// Per-camera assembly and optimiser step: a camera's gradient is the sum,
// over the image pairs it belongs to (camera CSR, fixed order), of the
// per-image-pair gradients; rotations then go through the adjoint of the 6D
// map (Sec. 3.3), and Adam updates the camera's parameters in place.
//
// k_cam          one warp per camera (four per CTA of 128 threads: small
//                CTAs find room beside the preceding kernel's, so that under
//                programmatic dependent launch they are resident before it
//                ends; 1024-thread CTAs were measured 9 us slower per step):
//                its first incident image pairs are read from the CSR before
//                the dependency wait, its parameters and Adam moments right
//                after it, together with the gathered parts; lanes stride
//                over the incident image pairs, a butterfly combines them,
//                lanes < 9 apply the adjoint and Adam.
// k_sum_fixed    the loss of each (scene, run): one CTA of 1024 threads (one
//                round of loads), a fixed order that depends on the number of
//                terms only.
#include "fm_step.cuh"

namespace fm {
namespace {

using step::Layout;

constexpr int kCamThreads = 128;    // one warp per camera
constexpr int kSumThreads = 1024;

template <int STAGE, bool ADAM>
__global__ void __launch_bounds__(kCamThreads) k_cam(CamUpdate u) {
  using L = Layout<STAGE>;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int run = blockIdx.y;
  pdl_trigger();
  const int c = blockIdx.x * (kCamThreads / 32) + warp;
  if (c >= u.N) return;
  // static: before the wait
  const int b = u.cam_seg_off[c], e = u.cam_seg_off[c + 1];
  int pre[step::kCamPre];
  step::cam_prefetch(u.cam_seg, b, e, lane, pre);
  pdl_wait();
  // parameters and moments do not depend on the gather: loaded with it
  const size_t off = ((size_t)run * u.N + c) * L::PDIM;
  float p[L::PDIM];
#pragma unroll
  for (int k = 0; k < L::PDIM; ++k) p[k] = u.params[off + k];
  float m = 0.f, v = 0.f;
  if (ADAM && lane < L::PDIM) {
    m = u.m[off + lane];
    v = u.v[off + lane];
  }
  float acc[L::PART];
  step::cam_gather<L::PART>(u.seg_grad + (size_t)run * u.P * 2 * L::PART, u.cam_seg, b, e, lane, pre, acc);
  step::cam_apply<STAGE, ADAM>(u, off, p, m, v, acc, lane);
}

// fixed-order sum of each scene's range of values per run (one CTA per
// (scene, run)) into out (and out2 when not null)
__global__ void __launch_bounds__(kSumThreads) k_sum_fixed(const float* __restrict__ x, int P,
                                                           const int* __restrict__ sc_pair_off,
                                                           float* __restrict__ out, float* __restrict__ out2) {
  __shared__ float part[kSumThreads];
  const int sc = blockIdx.x, run = blockIdx.y;
  pdl_trigger();
  const int b = sc_pair_off ? sc_pair_off[sc] : 0, e = sc_pair_off ? sc_pair_off[sc + 1] : P;
  pdl_wait();
  const float v = step::loss_sum_cta<kSumThreads>(x + (size_t)run * P + b, e - b, part);
  if (threadIdx.x == 0) {
    out[(size_t)run * gridDim.x + sc] = v;
    if (out2) out2[(size_t)run * gridDim.x + sc] = v;
  }
}

template <int STAGE>
void launch_stage(const CamUpdate& u, cudaStream_t s) {
  const int cam_blocks = (u.N + kCamThreads / 32 - 1) / (kCamThreads / 32);
  dim3 grid(cam_blocks, u.runs);
  if (u.params_out) launch_pdl(k_cam<STAGE, true>, grid, dim3(kCamThreads), 0, s, u);
  else launch_pdl(k_cam<STAGE, false>, grid, dim3(kCamThreads), 0, s, u);
}

}  // namespace

void launch_cam_update(int stage, const CamUpdate& u, cudaStream_t s) {
  if (stage == FM_STAGE_ROTATION) launch_stage<0>(u, s);
  else if (stage == FM_STAGE_TRANSLATION) launch_stage<1>(u, s);
  else launch_stage<2>(u, s);
}

void launch_sum_fixed(const float* x, int P, int runs, const int* sc_pair_off, int S, float* out,
                      cudaStream_t s, float* out2) {
  launch_pdl(k_sum_fixed, dim3(S, runs), dim3(kSumThreads), 0, s, x, P, sc_pair_off, out, out2);
}

}  // namespace fm
