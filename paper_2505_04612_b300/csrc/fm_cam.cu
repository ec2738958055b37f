// Per-camera assembly and optimiser step: a camera's gradient is the sum,
// over the image pairs it belongs to (camera CSR, fixed order), of the
// per-image-pair gradients; rotations then go through the adjoint of the 6D
// map (Sec. 3.3), and Adam updates the camera's parameters in place.
//
// k_cam          one warp per camera (four per CTA): lanes stride over the
//                incident image pairs, a butterfly combines them, lanes < 9
//                apply the adjoint and Adam.
// k_sum_fixed    the loss of each (scene, run): one CTA of 1024 threads, a
//                fixed order that depends on the number of terms only.
// k_ea_finish    the epipolar step's per-image-pair pass (k_ea_segments) and
//                per-camera pass (k_cam) in one launch (Sec. 3.4 fuses an
//                iteration's passes into one kernel): eight lanes per image
//                pair form its gradient block; every image pair then counts
//                itself done for its two cameras, and the warp that brings a
//                camera's count to its number of image pairs updates that
//                camera right away, with the same sums in the same order as
//                k_cam.  Camera updates thus overlap the image-pair pass
//                instead of waiting for all of it.  Each camera's counter
//                has a 128-byte line of its own: counters sharing a line
//                serialise each other's atomics (measured: 31k returning
//                atomics on 300 adjacent counters cost ~9 us, spread over
//                lines almost nothing).  Counters are reset by whoever
//                completes them, ready for the next launch.
#include "fm_step.cuh"

namespace fm {
namespace {

using step::kThreads;
using step::Layout;

template <int STAGE, bool ADAM>
__global__ void __launch_bounds__(kThreads) k_cam(CamUpdate u) {
  using L = Layout<STAGE>;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int run = blockIdx.y;
  pdl_trigger();
  const int c = blockIdx.x * (kThreads / 32) + warp;
  if (c >= u.N) return;
  const int b = u.cam_seg_off[c], e = u.cam_seg_off[c + 1];   // static: before the wait
  pdl_wait();
  float acc[L::PART];
  step::cam_gather<L::PART, false>(u.seg_grad + (size_t)run * u.P * 2 * L::PART, u.cam_seg, b, e, lane, acc);
  step::cam_apply<STAGE, ADAM>(u, c, run, acc, lane);
}

// fixed-order sum of each scene's range of values per run (one CTA per
// (scene, run)) into out (and out2 when not null)
constexpr int kSumThreads = 1024;
__global__ void __launch_bounds__(kSumThreads) k_sum_fixed(const float* __restrict__ x, int P,
                                                           const int* __restrict__ sc_pair_off,
                                                           float* __restrict__ out, float* __restrict__ out2) {
  __shared__ float part[kSumThreads];
  const int sc = blockIdx.x, run = blockIdx.y;
  pdl_trigger();
  const int b = sc_pair_off ? sc_pair_off[sc] : 0, e = sc_pair_off ? sc_pair_off[sc + 1] : P;
  pdl_wait();
  const float v = step::loss_sum_cta<kSumThreads, false>(x + (size_t)run * P + b, e - b, part);
  if (threadIdx.x == 0) {
    out[(size_t)run * gridDim.x + sc] = v;
    if (out2) out2[(size_t)run * gridDim.x + sc] = v;
  }
}

template <bool ADAM>
__global__ void __launch_bounds__(kThreads) k_ea_finish(FinishArgs f) {
  constexpr int kGroups = kThreads / step::kSegLanes;   // image pairs per CTA
  __shared__ int list[2 * kGroups];                      // cameras completed by this CTA
  __shared__ int n_list;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int gid = blockIdx.x * kThreads + t;
  const int n = gid / step::kSegLanes, sub = gid % step::kSegLanes;
  const CamUpdate& u = f.u;
  pdl_trigger();
  // static tables: before the wait
  const step::SegStatic st = step::seg_static(f.s, n);
  int deg_i = 0, deg_j = 0;
  if (n < f.s.P && sub == 0) {
    deg_i = u.cam_seg_off[st.ci + 1] - u.cam_seg_off[st.ci];
    deg_j = u.cam_seg_off[st.cj + 1] - u.cam_seg_off[st.cj];
  }
  if (t == 0) n_list = 0;
  pdl_wait();               // records come from k_ea_direct
  if (!ADAM && blockIdx.x == 0) {
    // cameras without image pairs are never completed: their gradient is 0
    for (int c = t; c < u.N; c += kThreads)
      if (u.cam_seg_off[c + 1] == u.cam_seg_off[c])
        for (int k = 0; k < 9; ++k) u.grad_out[9 * (size_t)c + k] = 0.f;
  }
  __syncthreads();
  if (step::segment_pair(f.s, n, sub, st)) {
    __threadfence();        // this image pair's block before its counts
    if (atomicAdd(f.cam_cnt + kCamCntStride * st.ci, 1) == deg_i - 1) {
      __threadfence();
      list[atomicAdd(&n_list, 1)] = st.ci;
    }
    if (atomicAdd(f.cam_cnt + kCamCntStride * st.cj, 1) == deg_j - 1) {
      __threadfence();
      list[atomicAdd(&n_list, 1)] = st.cj;
    }
  }
  __syncthreads();
  const int nl = n_list;
  for (int q = warp; q < nl; q += kThreads / 32) {
    const int c = list[q];
    __threadfence();
    float acc[12];
    step::cam_gather<12, true>(u.seg_grad, u.cam_seg, u.cam_seg_off[c], u.cam_seg_off[c + 1], lane, acc);
    step::cam_apply<2, ADAM>(u, c, 0, acc, lane);
    if (lane == 0) f.cam_cnt[kCamCntStride * c] = 0;   // ready for the next launch
  }
}

template <int STAGE>
void launch_stage(const CamUpdate& u, cudaStream_t s) {
  const int cam_blocks = (u.N + kThreads / 32 - 1) / (kThreads / 32);
  dim3 grid(cam_blocks, u.runs);
  if (u.params_out) launch_pdl(k_cam<STAGE, true>, grid, dim3(kThreads), 0, s, u);
  else launch_pdl(k_cam<STAGE, false>, grid, dim3(kThreads), 0, s, u);
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

void launch_ea_finish(const FinishArgs& f, cudaStream_t s) {
  const long long threads = (long long)f.s.P * step::kSegLanes;
  const dim3 grid((unsigned)((threads + kThreads - 1) / kThreads));
  if (f.u.params_out) launch_pdl(k_ea_finish<true>, grid, dim3(kThreads), 0, s, f);
  else launch_pdl(k_ea_finish<false>, grid, dim3(kThreads), 0, s, f);
}

}  // namespace fm
