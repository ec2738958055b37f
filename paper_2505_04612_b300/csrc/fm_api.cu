// Host runtime of the C ABI declared in include/fastmap.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fm_internal.h"

namespace {
thread_local std::string g_create_error = "no error";
}

namespace fm {
thread_local bool g_capturing = false;
thread_local bool g_plain_once = false;
void set_thread_error(const std::string& msg) { g_create_error = msg; }

const char* const kKernelNames[kKCount] = {
    "k_calibrate", "k_seg_offsets", "k_run_tables", "k_ea_tables", "k_ea_direct",
    "k_ea_segments", "k_rot_pairs", "k_trn_targets", "k_trn_pairs", "k_cam", "k_sum_fixed",
    "k_ea_reweight", "k_w_build", "k_ea_compact", "k_mart_iter", "k_reltrans", "k_merge",
    "k_triangulate", "k_ea_direct_loss", "k_ea_direct_coef", "k_mlp_pair_tables", "k_mlp_infer",
    "k_relpose", "k_focal_vote", "k_dist_errors", "k_dist_reduce", "k_cam_ea"};
}

namespace {

cudaEvent_t take_event(fm_problem* pr) {
  if (!pr->event_pool.empty()) {
    cudaEvent_t e = pr->event_pool.back();
    pr->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Counts every kernel launch; with timing on, brackets it with an event pair
// on the problem's stream.
struct Timed {
  fm_problem* pr;
  int kid;
  cudaEvent_t a = nullptr, b = nullptr;
  Timed(fm_problem* p, int k) : pr(p), kid(k) {
    if (pr->timing) {
      a = take_event(pr);
      b = take_event(pr);
      cudaEventRecord(a, pr->stream);
      // a timed kernel starts after the event, not overlapped with its
      // predecessor by programmatic dependent launch: the pair brackets
      // exactly this kernel
      fm::g_plain_once = true;
    }
  }
  ~Timed() {
    pr->k_launches[kid] += 1;
    if (pr->timing) {
      cudaEventRecord(b, pr->stream);
      pr->pending.push_back({kid, a, b});
    }
  }
};

void drain_timing(fm_problem* pr, bool accumulate) {
  if (pr->pending.empty()) return;
  cudaStreamSynchronize(pr->stream);
  for (auto& t : pr->pending) {
    float ms = 0.f;
    if (accumulate && cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) pr->k_ms[t.kid] += ms;
    pr->event_pool.push_back(t.start);
    pr->event_pool.push_back(t.stop);
  }
  cudaGetLastError();
  pr->pending.clear();
}

fm_status fail(fm_problem* pr, fm_status st, const std::string& msg) {
  if (pr) pr->last_error = msg;
  else g_create_error = msg;
  return st;
}

#define FM_CUDA(pr, expr)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail((pr), FM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define FM_LAUNCHED(pr)                                                                \
  do {                                                                                 \
    cudaError_t e_ = cudaGetLastError();                                               \
    if (e_ != cudaSuccess)                                                             \
      return fail((pr), FM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
fm_status dalloc(fm_problem* pr, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(pr, e == cudaErrorMemoryAllocation ? FM_ERR_OOM : FM_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  pr->device_bytes += (int64_t)(sizeof(T) * count);
  return FM_OK;
}

#define FM_ALLOC(pr, p, n)                 \
  do {                                     \
    fm_status s_ = dalloc((pr), &(p), (n)); \
    if (s_ != FM_OK) return s_;            \
  } while (0)

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

int stage_dim(fm_stage st) {
  return st == FM_STAGE_ROTATION ? 6 : (st == FM_STAGE_TRANSLATION ? 3 : 9);
}

// copy n elements from a host or device pointer into a host vector
template <typename T>
cudaError_t fetch(std::vector<T>& out, const T* src, size_t n, bool on_device) {
  out.resize(n);
  if (n == 0) return cudaSuccess;
  if (on_device) return cudaMemcpy(out.data(), src, sizeof(T) * n, cudaMemcpyDeviceToHost);
  std::memcpy(out.data(), src, sizeof(T) * n);
  return cudaSuccess;
}

fm_status check_err_bits(fm_problem* pr) {
  int bits = 0;
  FM_CUDA(pr, cudaMemcpyAsync(&bits, pr->d_err, sizeof(int), cudaMemcpyDeviceToHost, pr->stream));
  FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  if (bits == 0) return FM_OK;
  FM_CUDA(pr, cudaMemsetAsync(pr->d_err, 0, sizeof(int), pr->stream));
  // a launch cut short must not leave arrival counters behind
  if (pr->loss_cnt)
    FM_CUDA(pr, cudaMemsetAsync(pr->loss_cnt, 0, sizeof(int) * 64 * pr->S * fm::kLossCntStride, pr->stream));
  std::string msg;
  if (bits & fm::kErrKpRange) msg += "kp_img_pair outside [0, n_img_pairs); ";
  if (bits & fm::kErrKpOrder) msg += "kp_img_pair is not non-decreasing; ";
  if (bits & fm::kErrKpNonFinite) msg += "a keypoint coordinate is not finite; ";
  if (bits & fm::kErrParamNonFinite) msg += "a parameter is not finite; ";
  if (bits & (fm::kErrMlpTimeout | fm::kErrEaTimeout)) {
    if (bits & fm::kErrMlpTimeout) msg += "a bounded wait of the tensor-core network kernel ran out; ";
    if (bits & fm::kErrEaTimeout) msg += "a bounded wait of the direct epipolar kernel ran out; ";
    return fail(pr, FM_ERR_TIMEOUT, msg);
  }
  fm_status st = (bits & (fm::kErrKpNonFinite | fm::kErrParamNonFinite)) &&
                         !(bits & (fm::kErrKpRange | fm::kErrKpOrder))
                     ? FM_ERR_NAN
                     : FM_ERR_INVALID_ARG;
  return fail(pr, st, msg);
}

void release(fm_problem* pr) {
  if (!pr) return;
  cudaStreamSynchronize(pr->stream);
  dfree(pr->pair_i); dfree(pr->pair_j); dfree(pr->seg_off);
  dfree(pr->cam_seg_off); dfree(pr->cam_seg); dfree(pr->cam_pos);
  dfree(pr->kp); dfree(pr->kp_perm); dfree(pr->kp_track); dfree(pr->focal); dfree(pr->cx); dfree(pr->cy);
  dfree(pr->lane_desc); dfree(pr->wrun_info); dfree(pr->seg_rec); dfree(pr->rec);
  dfree(pr->seg_tab); dfree(pr->seg_grad); dfree(pr->seg_loss);
  dfree(pr->ea_w); dfree(pr->ea_params);
  dfree(pr->ea_adam.m); dfree(pr->ea_adam.v); dfree(pr->ea_adam.t);
  dfree(pr->rel_R); dfree(pr->rel_t); dfree(pr->rot_params);
  dfree(pr->rot_adam.m); dfree(pr->rot_adam.v); dfree(pr->rot_adam.t);
  dfree(pr->trn_target); dfree(pr->trn_params);
  dfree(pr->trn_adam.m); dfree(pr->trn_adam.v); dfree(pr->trn_adam.t);
  dfree(pr->scratch_params); dfree(pr->scratch_grad); dfree(pr->param_snap); dfree(pr->d_loss); dfree(pr->d_err); dfree(pr->sc_slice_off); dfree(pr->loss_part); dfree(pr->loss_cnt);
  dfree(pr->loss_hist);
  dfree(pr->W);
  dfree(pr->d_kept);
  dfree(pr->kp_seg); dfree(pr->track_off); dfree(pr->track_idx);
  dfree(pr->merge_buf); dfree(pr->best_run);
  dfree(pr->mlp_theta); dfree(pr->mlp_tab); dfree(pr->mlp_prob);
  dfree(pr->sc_cam_off); dfree(pr->sc_pair_off); dfree(pr->sc_kp_off); dfree(pr->cam_scene);
  dfree(pr->pair_scene); dfree(pr->pair_inv_p); dfree(pr->pair_inv_z); dfree(pr->mart_coef); dfree(pr->lattice0);
  for (auto& g : pr->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  pr->graphs.clear();
  if (pr->cap_stream) cudaStreamDestroy(pr->cap_stream);
  pr->cap_stream = nullptr;
  dfree(pr->focal_G);
  dfree(pr->focal_dphi);
  if (pr->aux_stream) cudaStreamDestroy(pr->aux_stream);
  if (pr->aux_fork) cudaEventDestroy(pr->aux_fork);
  if (pr->aux_join) cudaEventDestroy(pr->aux_join);
  pr->aux_stream = nullptr;
  pr->aux_fork = pr->aux_join = nullptr;
  if (pr->graph_in) cudaEventDestroy(pr->graph_in);
  if (pr->graph_out) cudaEventDestroy(pr->graph_out);
  pr->graph_in = pr->graph_out = nullptr;
  drain_timing(pr, false);
  for (cudaEvent_t e : pr->event_pool) cudaEventDestroy(e);
  pr->event_pool.clear();
  if (pr->h_loss) cudaFreeHost(pr->h_loss);
  pr->h_loss = nullptr;
  if (pr->h_err) cudaFreeHost(pr->h_err);
  pr->h_err = nullptr;
  if (pr->h_lg_in) cudaFreeHost(pr->h_lg_in);
  if (pr->h_lg_grad) cudaFreeHost(pr->h_lg_grad);
  pr->h_lg_in = pr->h_lg_grad = nullptr;
}

fm_status alloc_adam(fm_problem* pr, fm::AdamState& a, size_t n) {
  FM_ALLOC(pr, a.m, n);
  FM_ALLOC(pr, a.v, n);
  FM_ALLOC(pr, a.t, 1);
  return FM_OK;
}

fm_status reset_adam(fm_problem* pr, fm::AdamState& a, size_t n) {
  FM_CUDA(pr, cudaMemsetAsync(a.m, 0, sizeof(float) * n, pr->stream));
  FM_CUDA(pr, cudaMemsetAsync(a.v, 0, sizeof(float) * n, pr->stream));
  FM_CUDA(pr, cudaMemsetAsync(a.t, 0, sizeof(int), pr->stream));
  return FM_OK;
}

// Tables of the direct epipolar kernel for a tile of U keypoint pairs per
// lane: warp runs of 32 U pairs, each lane's first image pair, per warp run
// its image pairs and record base, per image pair its records.  Rebuilt when
// the tile changes (fm_autotune, fm_set_tuning).
fm_status build_direct_tables(fm_problem* pr, int U) {
  cudaStream_t s = pr->stream;
  const int P = pr->P;
  const int64_t Z = pr->Z;
  FM_CUDA(pr, cudaStreamSynchronize(s));
  if (pr->lane_desc) {   // tables of a previous tile
    pr->device_bytes -= (int64_t)sizeof(int) * 32 * std::max(pr->n_wruns, 1) +
                        (int64_t)sizeof(int4) * std::max(pr->n_wruns, 1) + (int64_t)sizeof(int) * 2 * P +
                        (int64_t)sizeof(float4) * 3 * std::max<int64_t>(pr->n_rec, 1);
  }
  dfree(pr->lane_desc);
  dfree(pr->wrun_info);
  dfree(pr->seg_rec);
  dfree(pr->rec);
  pr->ea_U = U;
  // lanes per image pair and their scan G (temporary)
  int* G = nullptr;
  int* d_T = nullptr;
  int64_t* d_total = nullptr;
  FM_ALLOC(pr, G, (size_t)P + 1);
  FM_ALLOC(pr, d_T, 1);
  FM_ALLOC(pr, d_total, 1);
  auto release_tmp = [&]() {
    cudaFree(G);
    cudaFree(d_T);
    cudaFree(d_total);
    pr->device_bytes -= (int64_t)sizeof(int) * (P + 2) + (int64_t)sizeof(int64_t);
  };
  int T = 0;
  if (Z > 0 && P > 0) {
    {
      Timed t(pr, fm::kKRunTables);
      fm::launch_lane_scan(pr->seg_off, P, U, G, d_T, s);
    }
    FM_LAUNCHED(pr);
    FM_CUDA(pr, cudaMemcpyAsync(&T, d_T, sizeof(int), cudaMemcpyDeviceToHost, s));
    FM_CUDA(pr, cudaStreamSynchronize(s));
  }
  pr->n_wruns = (T + 31) / 32;
  fm_status st = FM_OK;
  if ((st = dalloc(pr, &pr->lane_desc, (size_t)pr->n_wruns * 32)) != FM_OK ||
      (st = dalloc(pr, &pr->wrun_info, (size_t)pr->n_wruns)) != FM_OK ||
      (st = dalloc(pr, &pr->seg_rec, 2 * (size_t)P)) != FM_OK) {
    release_tmp();
    return st;
  }
  int64_t total = 0;
  if (pr->n_wruns > 0) {
    fm::launch_lane_desc(pr->seg_off, G, d_T, P, U, pr->n_wruns, pr->lane_desc, pr->wrun_info, s);
    FM_LAUNCHED(pr);
    fm::launch_exclusive_scan_info(pr->wrun_info, pr->n_wruns, d_total, s);
    FM_LAUNCHED(pr);
    FM_CUDA(pr, cudaMemcpyAsync(&total, d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FM_CUDA(pr, cudaStreamSynchronize(s));
  }
  pr->n_rec = total;
  if ((st = dalloc(pr, &pr->rec, 3 * (size_t)(pr->n_rec > 0 ? pr->n_rec : 1))) != FM_OK) {
    release_tmp();
    return st;
  }
  fm::launch_seg_records(pr->seg_off, G, pr->wrun_info, P, pr->seg_rec, s);
  FM_LAUNCHED(pr);
  FM_CUDA(pr, cudaStreamSynchronize(s));
  release_tmp();
  pr->graph_epoch += 1;   // captured launches hold the table pointers
  return FM_OK;
}

fm_status build(fm_problem* pr, const fm_problem_desc* d) {
  const int N = pr->N, P = pr->P;
  const int64_t Z = pr->Z;
  const bool dev = d->inputs_on_device != 0;
  cudaStream_t s = pr->stream;

  // ---- small arrays: validate on the host
  std::vector<int> hi, hj;
  std::vector<float> hf, hcx, hcy;
  FM_CUDA(pr, fetch(hi, d->pair_cam_i, P, dev));
  FM_CUDA(pr, fetch(hj, d->pair_cam_j, P, dev));
  FM_CUDA(pr, fetch(hf, d->focal, N, dev));
  FM_CUDA(pr, fetch(hcx, d->cx, N, dev));
  FM_CUDA(pr, fetch(hcy, d->cy, N, dev));
  for (int n = 0; n < P; ++n) {
    if (hi[n] < 0 || hi[n] >= N || hj[n] < 0 || hj[n] >= N)
      return fail(pr, FM_ERR_INVALID_ARG, "image pair " + std::to_string(n) + " has a camera index outside [0, n_cams)");
    if (hi[n] == hj[n])
      return fail(pr, FM_ERR_INVALID_ARG, "image pair " + std::to_string(n) + " joins a camera to itself");
  }
  for (int c = 0; c < N; ++c) {
    if (!(std::isfinite(hf[c]) && hf[c] > 0.f))
      return fail(pr, FM_ERR_INVALID_ARG, "focal[" + std::to_string(c) + "] must be finite and > 0");
    if (!(std::isfinite(hcx[c]) && std::isfinite(hcy[c])))
      return fail(pr, FM_ERR_INVALID_ARG, "principal point of camera " + std::to_string(c) + " is not finite");
  }
  // ---- scenes: camera ranges, image pairs grouped by scene
  const int S = d->n_scenes > 1 ? d->n_scenes : 1;
  pr->S = S;
  pr->h_sc_cam_off.assign(S + 1, 0);
  if (S > 1) {
    if (!d->scene_cam_off) return fail(pr, FM_ERR_INVALID_ARG, "scene_cam_off is required when n_scenes > 1");
    for (int q = 0; q <= S; ++q) pr->h_sc_cam_off[q] = d->scene_cam_off[q];
    if (pr->h_sc_cam_off[0] != 0 || pr->h_sc_cam_off[S] != N)
      return fail(pr, FM_ERR_INVALID_ARG, "scene_cam_off must start at 0 and end at n_cams");
    for (int q = 0; q < S; ++q)
      if (pr->h_sc_cam_off[q + 1] - pr->h_sc_cam_off[q] < 2)
        return fail(pr, FM_ERR_INVALID_ARG, "scene " + std::to_string(q) + " has fewer than 2 cameras");
  } else {
    pr->h_sc_cam_off[1] = N;
  }
  std::vector<int> cam_scene(N), pair_scene(P);
  for (int q = 0; q < S; ++q)
    for (int c = pr->h_sc_cam_off[q]; c < pr->h_sc_cam_off[q + 1]; ++c) cam_scene[c] = q;
  pr->h_sc_pair_off.assign(S + 1, 0);
  for (int n = 0; n < P; ++n) {
    const int q = cam_scene[hi[n]];
    if (cam_scene[hj[n]] != q)
      return fail(pr, FM_ERR_INVALID_ARG, "image pair " + std::to_string(n) + " joins cameras of two scenes");
    if (n > 0 && q < pair_scene[n - 1])
      return fail(pr, FM_ERR_INVALID_ARG, "image pairs are not grouped by scene in scene order");
    pair_scene[n] = q;
    pr->h_sc_pair_off[q + 1]++;
  }
  for (int q = 0; q < S; ++q) {
    if (pr->h_sc_pair_off[q + 1] == 0)
      return fail(pr, FM_ERR_INVALID_ARG, "scene " + std::to_string(q) + " has no image pair");
    pr->h_sc_pair_off[q + 1] += pr->h_sc_pair_off[q];
  }
  std::vector<float> inv_p(P);
  for (int n = 0; n < P; ++n) {
    const int q = pair_scene[n];
    inv_p[n] = 1.f / (float)(pr->h_sc_pair_off[q + 1] - pr->h_sc_pair_off[q]);
  }

  // connectivity filter: the largest connected component of each scene's view
  // graph (union-find; lowest camera index wins ties between components)
  {
    std::vector<int> parent(N);
    for (int c = 0; c < N; ++c) parent[c] = c;
    auto find = [&](int c) {
      while (parent[c] != c) c = parent[c] = parent[parent[c]];
      return c;
    };
    for (int n = 0; n < P; ++n) {
      const int a = find(hi[n]), b = find(hj[n]);
      if (a != b) parent[std::max(a, b)] = std::min(a, b);
    }
    std::vector<int> size(N, 0);
    for (int c = 0; c < N; ++c) size[find(c)]++;
    pr->h_cam_valid.assign(N, 0);
    for (int q = 0; q < S; ++q) {
      int best = -1;
      for (int c = pr->h_sc_cam_off[q]; c < pr->h_sc_cam_off[q + 1]; ++c)
        if (best < 0 || size[find(c)] > size[best]) best = find(c);
      for (int c = pr->h_sc_cam_off[q]; c < pr->h_sc_cam_off[q + 1]; ++c) pr->h_cam_valid[c] = find(c) == best;
    }
  }

  // camera -> incident image pairs, ordered by image pair (deterministic sums)
  std::vector<int> coff(N + 1, 0), cseg(2 * (size_t)P), cpos(2 * (size_t)P);
  for (int n = 0; n < P; ++n) { coff[hi[n] + 1]++; coff[hj[n] + 1]++; }
  for (int c = 0; c < N; ++c) pr->max_degree = std::max(pr->max_degree, coff[c + 1]);
  pr->h_sc_max_degree.assign(S, 0);
  for (int c = 0; c < N; ++c)
    pr->h_sc_max_degree[cam_scene[c]] = std::max(pr->h_sc_max_degree[cam_scene[c]], coff[c + 1]);
  for (int c = 0; c < N; ++c) coff[c + 1] += coff[c];
  {
    std::vector<int> fill(coff.begin(), coff.end() - 1);
    for (int n = 0; n < P; ++n) {
      cpos[2 * (size_t)n] = fill[hi[n]];
      cseg[fill[hi[n]]++] = n;
      cpos[2 * (size_t)n + 1] = fill[hj[n]];
      cseg[fill[hj[n]]++] = (int)((unsigned)n | 0x80000000u);
    }
  }

  FM_ALLOC(pr, pr->pair_i, P);
  FM_ALLOC(pr, pr->pair_j, P);
  FM_ALLOC(pr, pr->focal, N);
  FM_ALLOC(pr, pr->cx, N);
  FM_ALLOC(pr, pr->cy, N);
  FM_ALLOC(pr, pr->cam_seg_off, N + 1);
  FM_ALLOC(pr, pr->cam_seg, 2 * (size_t)P);
  FM_ALLOC(pr, pr->cam_pos, 2 * (size_t)P);
  FM_ALLOC(pr, pr->seg_off, P + 1);
  FM_ALLOC(pr, pr->d_err, 1);
  FM_CUDA(pr, cudaMemcpyAsync(pr->pair_i, hi.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaMemcpyAsync(pr->pair_j, hj.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaMemcpyAsync(pr->focal, hf.data(), sizeof(float) * N, cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaMemcpyAsync(pr->cx, hcx.data(), sizeof(float) * N, cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaMemcpyAsync(pr->cy, hcy.data(), sizeof(float) * N, cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaMemcpyAsync(pr->cam_seg_off, coff.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaMemcpyAsync(pr->cam_seg, cseg.data(), sizeof(int) * 2 * (size_t)P, cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaMemcpyAsync(pr->cam_pos, cpos.data(), sizeof(int) * 2 * (size_t)P, cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaMemsetAsync(pr->d_err, 0, sizeof(int), s));
  FM_ALLOC(pr, pr->sc_cam_off, S + 1);
  FM_ALLOC(pr, pr->sc_pair_off, S + 1);
  FM_ALLOC(pr, pr->sc_kp_off, S + 1);
  FM_ALLOC(pr, pr->cam_scene, N);
  FM_ALLOC(pr, pr->pair_scene, P);
  FM_ALLOC(pr, pr->pair_inv_p, P);
  FM_ALLOC(pr, pr->pair_inv_z, P);
  FM_ALLOC(pr, pr->mart_coef, 3 * (size_t)S);
  FM_CUDA(pr, cudaMemcpyAsync(pr->sc_cam_off, pr->h_sc_cam_off.data(), sizeof(int) * (S + 1), cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaMemcpyAsync(pr->sc_pair_off, pr->h_sc_pair_off.data(), sizeof(int) * (S + 1), cudaMemcpyHostToDevice, s));
  // loss slices: ceil(P_s / 1024) per scene, sums and arrival counters for up to 64 runs
  pr->h_sc_slice_off.assign(S + 1, 0);
  for (int q = 0; q < S; ++q)
    pr->h_sc_slice_off[q + 1] = pr->h_sc_slice_off[q] +
                                (pr->h_sc_pair_off[q + 1] - pr->h_sc_pair_off[q] + fm::kLossSlice - 1) / fm::kLossSlice;
  pr->n_slices = pr->h_sc_slice_off[S];
  FM_ALLOC(pr, pr->sc_slice_off, S + 1);
  FM_ALLOC(pr, pr->loss_part, (size_t)64 * pr->n_slices);
  FM_ALLOC(pr, pr->loss_cnt, (size_t)64 * S * fm::kLossCntStride);
  FM_CUDA(pr, cudaMemcpyAsync(pr->sc_slice_off, pr->h_sc_slice_off.data(), sizeof(int) * (S + 1),
                              cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaMemsetAsync(pr->loss_cnt, 0, sizeof(int) * 64 * S * fm::kLossCntStride, s));
  FM_CUDA(pr, cudaMemcpyAsync(pr->cam_scene, cam_scene.data(), sizeof(int) * N, cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaMemcpyAsync(pr->pair_scene, pair_scene.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaMemcpyAsync(pr->pair_inv_p, inv_p.data(), sizeof(float) * P, cudaMemcpyHostToDevice, s));
  FM_CUDA(pr, cudaStreamSynchronize(s));   // the host vectors above are locals

  // ---- keypoints: stage host inputs on the device, calibrate, offsets
  FM_ALLOC(pr, pr->kp, Z);
  const float* kp1 = d->kp1_px;
  const float* kp2 = d->kp2_px;
  const int* kpp = d->kp_img_pair;
  float* tmp1 = nullptr;
  float* tmp2 = nullptr;
  int* tmpp = nullptr;
  if (!dev && Z > 0) {
    FM_ALLOC(pr, tmp1, 2 * Z);
    FM_ALLOC(pr, tmp2, 2 * Z);
    FM_ALLOC(pr, tmpp, Z);
    FM_CUDA(pr, cudaMemcpyAsync(tmp1, kp1, sizeof(float) * 2 * Z, cudaMemcpyHostToDevice, s));
    FM_CUDA(pr, cudaMemcpyAsync(tmp2, kp2, sizeof(float) * 2 * Z, cudaMemcpyHostToDevice, s));
    FM_CUDA(pr, cudaMemcpyAsync(tmpp, kpp, sizeof(int) * Z, cudaMemcpyHostToDevice, s));
    kp1 = tmp1;
    kp2 = tmp2;
    kpp = tmpp;
  }
  if (d->kp_track && Z > 0) {
    FM_ALLOC(pr, pr->kp_track, Z);
    FM_CUDA(pr, cudaMemcpyAsync(pr->kp_track, d->kp_track, sizeof(int) * Z,
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  }
  // the keypoint pairs in (image pair, track) order: the caller's order when
  // it is one already, else sorted here (stable: equal keys keep the input
  // order) with the permutation kept for per-pair inputs and outputs
  float* srt1 = nullptr;
  float* srt2 = nullptr;
  int* srtp = nullptr;
  auto free_sorted = [&]() {
    if (srt1) { cudaFree(srt1); pr->device_bytes -= (int64_t)sizeof(float) * 2 * Z; srt1 = nullptr; }
    if (srt2) { cudaFree(srt2); pr->device_bytes -= (int64_t)sizeof(float) * 2 * Z; srt2 = nullptr; }
    if (srtp) { cudaFree(srtp); pr->device_bytes -= (int64_t)sizeof(int) * Z; srtp = nullptr; }
  };
  if (Z > 0) {
    int flags[2] = {0, 0};
    FM_CUDA(pr, cudaMemsetAsync(pr->d_err, 0, sizeof(int), s));
    int* d_flags = nullptr;
    FM_ALLOC(pr, d_flags, 2);
    FM_CUDA(pr, cudaMemsetAsync(d_flags, 0, sizeof(int) * 2, s));
    fm::launch_kp_order_check(kpp, pr->kp_track, Z, P, d_flags, s);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(flags, d_flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaFree(d_flags);
    pr->device_bytes -= (int64_t)sizeof(int) * 2;
    if (ce != cudaSuccess) return fail(pr, FM_ERR_CUDA, std::string("keypoint order: ") + cudaGetErrorString(ce));
    if (flags[0] & 1) {
      if (tmp1) { cudaFree(tmp1); cudaFree(tmp2); cudaFree(tmpp); }
      return fail(pr, FM_ERR_INVALID_ARG, "kp_img_pair outside [0, n_img_pairs)");
    }
    if (flags[0] & 2) {
      fm_status a = FM_OK;
      if ((a = dalloc(pr, &pr->kp_perm, (size_t)Z)) != FM_OK || (a = dalloc(pr, &srt1, 2 * (size_t)Z)) != FM_OK ||
          (a = dalloc(pr, &srt2, 2 * (size_t)Z)) != FM_OK || (a = dalloc(pr, &srtp, (size_t)Z)) != FM_OK) {
        free_sorted();
        return a;
      }
      int* srtt = nullptr;
      if (pr->kp_track && (a = dalloc(pr, &srtt, (size_t)Z)) != FM_OK) {
        free_sorted();
        return a;
      }
      ce = fm::sort_kp_pairs(kpp, pr->kp_track, Z, P, flags[1], pr->kp_perm, s);
      if (ce == cudaSuccess) {
        fm::launch_kp_gather(pr->kp_perm, Z, kp1, kp2, kpp, pr->kp_track, srt1, srt2, srtp, srtt, s);
        ce = cudaGetLastError();
      }
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) {
        free_sorted();
        if (srtt) cudaFree(srtt);
        return fail(pr, FM_ERR_CUDA, std::string("sorting the keypoint pairs: ") + cudaGetErrorString(ce));
      }
      kp1 = srt1;
      kp2 = srt2;
      kpp = srtp;
      if (srtt) {   // the sorted tracks replace the caller's order
        dfree(pr->kp_track);
        pr->device_bytes -= (int64_t)sizeof(int) * Z;
        pr->kp_track = srtt;
      }
    }
  }
  {
    Timed t(pr, fm::kKCalibrate);
    fm::launch_calibrate(kp1, kp2, kpp, pr->pair_i, pr->pair_j, pr->focal, pr->cx, pr->cy, Z, P,
                         pr->kp, pr->d_err, s);
  }
  FM_LAUNCHED(pr);
  {
    Timed t(pr, fm::kKSegOffsets);
    fm::launch_seg_offsets(kpp, Z, P, pr->seg_off, pr->d_err, s);
  }
  FM_LAUNCHED(pr);
  fm_status st = check_err_bits(pr);
  if (st == FM_OK && Z > 0) {
    // the image pair of every keypoint pair (triangulation, learned-weight features)
    FM_ALLOC(pr, pr->kp_seg, Z);
    FM_CUDA(pr, cudaMemcpyAsync(pr->kp_seg, kpp, sizeof(int) * Z, cudaMemcpyDeviceToDevice, s));
  }
  if (st == FM_OK && d->kp_track && Z > 0) {
    int T = 0;
    FM_CUDA(pr, fm::build_track_table(pr, &T));
    st = check_err_bits(pr);
  }
  if (tmp1) { cudaFree(tmp1); pr->device_bytes -= (int64_t)sizeof(float) * 2 * Z; }
  if (tmp2) { cudaFree(tmp2); pr->device_bytes -= (int64_t)sizeof(float) * 2 * Z; }
  if (tmpp) { cudaFree(tmpp); pr->device_bytes -= (int64_t)sizeof(int) * Z; }
  free_sorted();
  if (st != FM_OK) return st;

  {
    std::vector<int> so(P + 1);
    FM_CUDA(pr, cudaMemcpy(so.data(), pr->seg_off, sizeof(int) * (P + 1), cudaMemcpyDeviceToHost));
    int e = 0;
    for (int n = 0; n < P; ++n) e += (so[n] == so[n + 1]);
    pr->n_empty = e;
    // keypoint range of each scene, and the unit-weight normaliser 1/Z_s
    pr->h_sc_kp_off.assign(S + 1, 0);
    for (int q = 0; q <= S; ++q) pr->h_sc_kp_off[q] = so[pr->h_sc_pair_off[q]];
    std::vector<float> inv_z(P);
    for (int n = 0; n < P; ++n) {
      const int q = pair_scene[n];
      const int64_t zq = pr->h_sc_kp_off[q + 1] - pr->h_sc_kp_off[q];
      inv_z[n] = zq > 0 ? (float)(1.0 / (double)zq) : 0.f;
    }
    FM_CUDA(pr, cudaMemcpy(pr->sc_kp_off, pr->h_sc_kp_off.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice));
    FM_CUDA(pr, cudaMemcpy(pr->pair_inv_z, inv_z.data(), sizeof(float) * P, cudaMemcpyHostToDevice));
  }

  // ---- tables of the direct epipolar kernel
  {
    fm_status st2 = build_direct_tables(pr, pr->ea_U);
    if (st2 != FM_OK) return st2;
  }

  // ---- per-stage state
  FM_ALLOC(pr, pr->seg_tab, 3 * (size_t)P);
  FM_ALLOC(pr, pr->seg_grad, (size_t)fm::kSegGradEa * P);
  FM_ALLOC(pr, pr->seg_loss, (size_t)P);
  FM_ALLOC(pr, pr->ea_params, 9 * (size_t)N);
  FM_ALLOC(pr, pr->rot_params, 6 * (size_t)N);
  FM_ALLOC(pr, pr->trn_params, 3 * (size_t)N);
  FM_ALLOC(pr, pr->trn_target, 3 * (size_t)P);
  FM_ALLOC(pr, pr->rel_R, 9 * (size_t)P);
  FM_ALLOC(pr, pr->rel_t, 3 * (size_t)P);
  fm_status a;
  if ((a = alloc_adam(pr, pr->ea_adam, 9 * (size_t)N)) != FM_OK) return a;
  if ((a = alloc_adam(pr, pr->rot_adam, 6 * (size_t)N)) != FM_OK) return a;
  if ((a = alloc_adam(pr, pr->trn_adam, 3 * (size_t)N)) != FM_OK) return a;
  FM_ALLOC(pr, pr->scratch_params, 9 * (size_t)N);
  FM_ALLOC(pr, pr->scratch_grad, 9 * (size_t)N);
  FM_ALLOC(pr, pr->param_snap, 9 * (size_t)N);
  FM_ALLOC(pr, pr->d_loss, (size_t)S);
  FM_ALLOC(pr, pr->W, 64 * (((size_t)P + 31) & ~(size_t)31));   // tiles of 32 image pairs
  FM_ALLOC(pr, pr->d_kept, (size_t)S);
  FM_ALLOC(pr, pr->merge_buf, 3 * (size_t)N + 4 * 64 * (size_t)S);
  FM_ALLOC(pr, pr->best_run, (size_t)N);
  FM_CUDA(pr, cudaMallocHost((void**)&pr->h_loss, sizeof(float) * S));
  FM_CUDA(pr, cudaMallocHost((void**)&pr->h_err, sizeof(int)));
  {
    const int64_t z0 = pr->h_sc_kp_off[1] - pr->h_sc_kp_off[0];
    pr->ea_inv_z = z0 > 0 ? (float)(1.0 / (double)z0) : 0.f;
  }
  if (d->rel_R) {
    FM_CUDA(pr, cudaMemcpyAsync(pr->rel_R, d->rel_R, sizeof(float) * 9 * P,
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    pr->rel_R_set = true;
  }
  if (d->rel_t) {
    FM_CUDA(pr, cudaMemcpyAsync(pr->rel_t, d->rel_t, sizeof(float) * 3 * P,
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    pr->rel_t_set = true;
  }
  FM_CUDA(pr, cudaStreamSynchronize(s));
  return FM_OK;
}

// device pointer of a stage's parameters and Adam state
struct StageBuf {
  float* params;
  fm::AdamState* adam;
  size_t count;
  bool* set;
};

StageBuf stage_buf(fm_problem* pr, fm_stage st) {
  if (st == FM_STAGE_ROTATION) return {pr->rot_params, &pr->rot_adam, 6 * (size_t)pr->N, &pr->rot_params_set};
  if (st == FM_STAGE_TRANSLATION)
    return {pr->trn_params, &pr->trn_adam, 3 * (size_t)pr->N * pr->trn_runs, &pr->trn_params_set};
  return {pr->ea_params, &pr->ea_adam, 9 * (size_t)pr->N, &pr->ea_params_set};
}

bool valid_stage(int st) { return st >= FM_STAGE_ROTATION && st <= FM_STAGE_EPIPOLAR; }

fm_status ensure_targets(fm_problem* pr) {
  if (pr->trn_target_valid) return FM_OK;
  if (!pr->rot_params_set) return fail(pr, FM_ERR_STATE, "translation stage needs rotation-stage parameters (fm_set_params(FM_STAGE_ROTATION))");
  if (!pr->rel_t_set) return fail(pr, FM_ERR_STATE, "translation stage needs relative translations (rel_t)");
  {
    Timed t(pr, fm::kKTrnTargets);
    fm::launch_trn_targets(pr->rot_params, pr->pair_j, pr->rel_t, pr->P, pr->trn_target, pr->stream);
  }
  FM_LAUNCHED(pr);
  pr->trn_target_valid = true;
  return FM_OK;
}

// W_n together with its expansion around the essential matrices e0 of the
// parameters `centre` (see fm_irls.cu); built lazily after the weights change
fm_status rebuild_W(fm_problem* pr, const float* centre) {
  {
    Timed t(pr, fm::kKEaTables);
    fm::launch_ea_tables(centre, pr->pair_i, pr->pair_j, pr->seg_off, pr->P, pr->seg_tab, nullptr,
                         pr->stream);
  }
  FM_LAUNCHED(pr);
  {
    Timed t(pr, fm::kKWBuild);
    fm::launch_w_build(pr, pr->ea_w, pr->W, pr->stream);
  }
  FM_LAUNCHED(pr);
  pr->W_valid = true;
  return FM_OK;
}

// loss slices of the problem writing to out (and out2); out null: no loss
fm::LossArgs loss_args(const fm_problem* pr, float* out, float* out2) {
  fm::LossArgs L;
  L.sc_pair_off = pr->sc_pair_off;
  L.sc_slice_off = pr->sc_slice_off;
  L.S = pr->S;
  L.n_slices = pr->n_slices;
  L.partial = pr->loss_part;
  L.cnt = pr->loss_cnt;
  L.out = out;
  L.out2 = out ? out2 : nullptr;
  return L;
}

fm::CamUpdate cam_update(fm_problem* pr, const float* params, float* grad_dev, const fm_adam_opts* adam,
                         fm::AdamState* state, int* step, int runs) {
  fm::CamUpdate u{};
  u.cam_seg_off = pr->cam_seg_off;
  u.cam_seg = pr->cam_seg;
  u.seg_grad = pr->seg_grad;
  u.params = params;
  u.params_out = adam ? const_cast<float*>(params) : nullptr;
  u.grad_out = grad_dev;
  u.m = state ? state->m : nullptr;
  u.v = state ? state->v : nullptr;
  u.step = step;
  u.lr = adam ? adam->lr : 0.f;
  u.b1 = adam ? adam->beta1 : 0.f;
  u.b2 = adam ? adam->beta2 : 0.f;
  u.eps = adam ? adam->eps : 0.f;
  u.N = pr->N;
  u.P = pr->P;
  u.runs = runs;
  u.seg_loss = pr->seg_loss;
  u.loss = loss_args(pr, nullptr, nullptr);
  return u;
}

// One evaluation of a stage: per-image-pair pass, then the per-camera pass
// (Adam when adam != null, else the gradient into grad_dev); the loss of every
// run is reduced into loss_a and loss_b when they are not null.
fm_status evaluate(fm_problem* pr, fm_stage st, const float* params, float* grad_dev,
                   const fm_adam_opts* adam, fm::AdamState* state, float* loss_a,
                   float* loss_b = nullptr) {
  cudaStream_t s = pr->stream;
  const int P = pr->P, N = pr->N;
  int runs = 1;
  int* step = adam ? state->t : nullptr;

  if (st == FM_STAGE_EPIPOLAR && pr->ea_loss == FM_EA_COMPACT) {
    if (!pr->W_valid) {
      fm_status e = rebuild_W(pr, params);
      if (e != FM_OK) return e;
    }
    {
      Timed t(pr, fm::kKEaCompact);
      fm::launch_ea_compact(pr, params, step, s);
    }
    FM_LAUNCHED(pr);
  } else if (st == FM_STAGE_EPIPOLAR) {
    {
      // an Adam step updates params in place while the camera pass still
      // reads other cameras' parameters for the chain rule: that pass reads
      // the copy taken here instead
      Timed t(pr, fm::kKEaTables);
      fm::launch_ea_tables(params, pr->pair_i, pr->pair_j, pr->seg_off, P, pr->seg_tab, step, s, nullptr,
                           adam ? pr->param_snap : nullptr, 9 * N);
    }
    FM_LAUNCHED(pr);
    if (pr->n_wruns > 0) {
      Timed t(pr, fm::kKEaDirect);
      fm::launch_ea_direct(pr, pr->ea_w, pr->ea_loss, s);
    }
    FM_LAUNCHED(pr);
    if (adam || grad_dev) {
      // the per-image-pair chain rule, the cameras and the loss in one launch
      fm::EaCamArgs f;
      f.s = fm::seg_args(pr, adam ? pr->param_snap : params);
      f.s.g_scale = (pr->ea_loss == FM_EA_L1) ? 1.f : 2.f;
      f.u = cam_update(pr, params, grad_dev, adam, state, step, 1);
      f.u.loss = loss_args(pr, loss_a ? loss_a : loss_b, loss_a ? loss_b : nullptr);
      {
        Timed t(pr, fm::kKCamEa);
        fm::launch_cam_ea(f, s);
      }
      FM_LAUNCHED(pr);
      return FM_OK;
    }
    {
      Timed t(pr, fm::kKEaSegments);
      fm::launch_ea_segments(pr, params, pr->ea_loss, s);
    }
    FM_LAUNCHED(pr);
  } else if (st == FM_STAGE_ROTATION) {
    if (!pr->rel_R_set) return fail(pr, FM_ERR_STATE, "rotation stage needs relative rotations (rel_R)");
    {
      Timed t(pr, fm::kKRotPairs);
      fm::launch_rot_pairs(params, pr->pair_i, pr->pair_j, pr->rel_R, P, pr->pair_inv_p, pr->seg_grad,
                           pr->seg_loss, step, s);
    }
    FM_LAUNCHED(pr);
  } else {
    fm_status e = ensure_targets(pr);
    if (e != FM_OK) return e;
    runs = pr->trn_runs;
    {
      Timed t(pr, fm::kKTrnPairs);
      fm::launch_trn_pairs(params, pr->pair_i, pr->pair_j, pr->trn_target, N, P, runs, pr->pair_inv_p,
                           pr->seg_grad, pr->seg_loss, step, s);
    }
    FM_LAUNCHED(pr);
  }
  float* first = loss_a ? loss_a : loss_b;
  float* second = loss_a ? loss_b : nullptr;
  if (adam || grad_dev) {
    // the cameras, and the loss in slices of the same launch
    fm::CamUpdate u = cam_update(pr, params, grad_dev, adam, state, step, runs);
    u.loss = loss_args(pr, first, second);
    u.csr_order = (st == FM_STAGE_EPIPOLAR && pr->ea_loss == FM_EA_COMPACT);   // k_ea_compact's layout
    {
      Timed t(pr, fm::kKCamUpdate);
      fm::launch_cam_update((int)st, u, s);
    }
    FM_LAUNCHED(pr);
  } else if (first) {
    Timed t(pr, fm::kKLossSum);
    fm::launch_sum_fixed(pr->seg_loss, P, runs, loss_args(pr, first, second), s);
  }
  FM_LAUNCHED(pr);
  return FM_OK;
}

fm_status resize_runs(fm_problem* pr, int runs) {
  if (runs == pr->trn_runs) return FM_OK;
  pr->graph_epoch += 1;   // buffers are reallocated
  const size_t n = 3 * (size_t)pr->N * runs;
  dfree(pr->trn_params);
  dfree(pr->trn_adam.m);
  dfree(pr->trn_adam.v);
  dfree(pr->seg_grad);
  dfree(pr->seg_loss);
  dfree(pr->scratch_params);
  dfree(pr->scratch_grad);
  dfree(pr->d_loss);
  if (pr->h_loss) cudaFreeHost(pr->h_loss);
  pr->h_loss = nullptr;
  FM_ALLOC(pr, pr->trn_params, n);
  FM_ALLOC(pr, pr->trn_adam.m, n);
  FM_ALLOC(pr, pr->trn_adam.v, n);
  const size_t sg = std::max((size_t)fm::kSegGradEa * pr->P, (size_t)fm::kSegGradTrn * pr->P * runs);
  FM_ALLOC(pr, pr->seg_grad, sg);
  FM_ALLOC(pr, pr->seg_loss, (size_t)pr->P * runs);
  const size_t sp = std::max((size_t)9 * pr->N, n);
  FM_ALLOC(pr, pr->scratch_params, sp);
  FM_ALLOC(pr, pr->scratch_grad, sp);
  FM_ALLOC(pr, pr->d_loss, (size_t)runs * pr->S);
  FM_CUDA(pr, cudaMallocHost((void**)&pr->h_loss, sizeof(float) * runs * pr->S));
  pr->trn_runs = runs;
  pr->trn_params_set = false;
  return FM_OK;
}


// Greedy order of the cameras (groups of images sharing intrinsics) of the
// focal and distortion searches: an image pair is ready for a group when both
// images are in it, or one is and the other's group is done; the group with
// the most ready image pairs goes next (the lowest id on ties), never one
// with none.  Counts are kept incrementally.
struct ReadyOrder {
  const std::vector<int>& g;
  const std::vector<int>& hi;
  const std::vector<int>& hj;
  std::vector<std::vector<int>> inc;   // usable image pairs touching each group
  std::vector<int64_t> ready;
  std::vector<char> done;

  ReadyOrder(const std::vector<int>& g_, const std::vector<int>& hi_, const std::vector<int>& hj_,
             const std::vector<int>& usable, int n_groups)
      : g(g_), hi(hi_), hj(hj_), inc(n_groups), ready(n_groups, 0), done(n_groups, 0) {
    for (size_t n = 0; n < hi.size(); ++n) {
      if (!usable[n]) continue;
      const int a = g[hi[n]], b = g[hj[n]];
      inc[a].push_back((int)n);
      if (b != a) inc[b].push_back((int)n);
      else ready[a] += 1;
    }
  }
  int next() const {
    int best = -1;
    int64_t bn = 0;
    for (size_t q = 0; q < ready.size(); ++q)
      if (!done[q] && ready[q] > bn) {
        best = (int)q;
        bn = ready[q];
      }
    return best;
  }
  // ready pairs of `best` in increasing order, with the group of each side
  // (-1 where the side belongs to `best`)
  void list(int best, std::vector<int>& pairs, std::vector<int>& gi_fixed, std::vector<int>& gj_fixed) const {
    pairs.clear();
    gi_fixed.clear();
    gj_fixed.clear();
    for (int n : inc[best]) {
      const int a = g[hi[n]], b = g[hj[n]];
      if (!((a == best && b == best) || (a == best && done[b]) || (b == best && done[a]))) continue;
      pairs.push_back(n);
      gi_fixed.push_back(a == best ? -1 : a);
      gj_fixed.push_back(b == best ? -1 : b);
    }
  }
  void finish(int best) {
    done[best] = 1;
    for (int n : inc[best]) {
      const int a = g[hi[n]], b = g[hj[n]];
      if (a == b) continue;
      const int other = (a == best) ? b : a;
      if (!done[other]) ready[other] += 1;
    }
  }
};

fm_status check_groups(fm_problem* pr, const int32_t* group, int32_t n_groups, std::vector<int>& g) {
  if (n_groups < 1 || (!group && n_groups != 1)) return fail(pr, FM_ERR_INVALID_ARG, "n_groups >= 1 (1 without group)");
  g.assign(pr->N, 0);
  if (group)
    for (int c = 0; c < pr->N; ++c) {
      g[c] = group[c];
      if (g[c] < 0 || g[c] >= n_groups) return fail(pr, FM_ERR_INVALID_ARG, "group id outside [0, n_groups)");
    }
  return FM_OK;
}

// device scratch of one search call, freed on every return path
struct Scratch {
  std::vector<void*> ptrs;
  cudaError_t ce = cudaSuccess;
  template <typename T>
  T* get(size_t n) {
    void* q = nullptr;
    if (ce == cudaSuccess) ce = cudaMalloc(&q, std::max<size_t>(n * sizeof(T), 16));
    if (ce == cudaSuccess) ptrs.push_back(q);
    return (T*)q;
  }
  ~Scratch() {
    for (void* q : ptrs) cudaFree(q);
  }
};

// work items of k_dist_errors: image pairs and their output rows, those of at
// most kDistSplit keypoint pairs (one warp each) first, then the larger ones
// (one CTA each), each class largest first so that the longest items start
// first (the outputs do not depend on the order); returns the number of small
// ones
int split_by_size(const std::vector<int>& pairs, const std::vector<int>& off, std::vector<int>& idx,
                  std::vector<int>& row) {
  // key: class (small 0, large 1), then the size descending, then the row
  std::vector<uint64_t> key(pairs.size());
  int n_small = 0;
  for (size_t q = 0; q < pairs.size(); ++q) {
    const uint64_t m = (uint64_t)(off[pairs[q] + 1] - off[pairs[q]]);
    const uint64_t big = m > (uint64_t)fm::kDistSplit;
    n_small += big == 0;
    key[q] = (big << 62) | ((0x7fffffffull - m) << 31) | (uint64_t)q;
  }
  std::sort(key.begin(), key.end());
  idx.resize(pairs.size());
  row.resize(pairs.size());
  for (size_t k = 0; k < key.size(); ++k) {
    const int q = (int)(key[k] & 0x7fffffffull);
    idx[k] = pairs[q];
    row[k] = q;
  }
  return n_small;
}

// One level of distortion scores: the items of more than kDistSplit keypoint
// pairs (one CTA each) on the auxiliary stream, forked from and joined back
// to the problem's stream, the others (one warp each) on the problem's
// stream, so that the two launches overlap.  items/rows: n_small small items
// first, then M - n_small large ones.
cudaError_t dist_level(fm_problem* pr, const float* scale, const int* items, const int* rows, const float* fix_i,
                       const float* fix_j, int M, int n_small, const float* cand, int K, float* err) {
  cudaStream_t s = pr->stream;
  const int n_big = M - n_small;
  if (n_big > 0 && !pr->aux_stream) {
    cudaError_t ce = cudaStreamCreateWithFlags(&pr->aux_stream, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pr->aux_fork, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&pr->aux_join, cudaEventDisableTiming);
    if (ce != cudaSuccess) return ce;
  }
  Timed t(pr, fm::kKDistErrors);
  if (n_big > 0) {
    cudaError_t ce = cudaEventRecord(pr->aux_fork, s);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(pr->aux_stream, pr->aux_fork, 0);
    if (ce != cudaSuccess) return ce;
    fm::launch_dist_errors(pr, scale, items + n_small, rows + n_small, fix_i, fix_j, n_big, true, cand, K, err,
                           pr->aux_stream);
  }
  fm::launch_dist_errors(pr, scale, items, rows, fix_i, fix_j, n_small, false, cand, K, err, s);
  if (n_big > 0) {
    if (n_small > 0) pr->k_launches[fm::kKDistErrors] += 1;   // two launches in one bracket
    cudaError_t ce = cudaEventRecord(pr->aux_join, pr->aux_stream);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, pr->aux_join, 0);
    if (ce != cudaSuccess) return ce;
  }
  return cudaGetLastError();
}

// f0 / half diagonal of every image (x_d = s x_c for keypoints calibrated at f0)
cudaError_t image_scales(const fm_problem* pr, std::vector<float>& scale) {
  std::vector<float> f, cx, cy;
  cudaError_t ce = fetch(f, pr->focal, pr->N, true);
  if (ce == cudaSuccess) ce = fetch(cx, pr->cx, pr->N, true);
  if (ce == cudaSuccess) ce = fetch(cy, pr->cy, pr->N, true);
  if (ce != cudaSuccess) return ce;
  scale.resize(pr->N);
  for (int c = 0; c < pr->N; ++c)
    scale[c] = (float)((double)f[c] / std::sqrt((double)cx[c] * cx[c] + (double)cy[c] * cy[c]));
  return cudaSuccess;
}

}  // namespace

extern "C" {

fm_status fm_problem_create(const fm_problem_desc* d, fm_problem** out) {
  if (!out) return fail(nullptr, FM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!d) return fail(nullptr, FM_ERR_INVALID_ARG, "desc is NULL");
  if (d->n_cams < 2) return fail(nullptr, FM_ERR_INVALID_ARG, "n_cams must be >= 2");
  if (d->n_img_pairs < 1) return fail(nullptr, FM_ERR_INVALID_ARG, "n_img_pairs must be >= 1");
  if (d->n_kp_pairs < 0 || d->n_kp_pairs >= (int64_t(1) << 31) - (int64_t(1) << 20))
    return fail(nullptr, FM_ERR_INVALID_ARG, "n_kp_pairs must be in [0, 2^31 - 2^20)");
  if (!d->pair_cam_i || !d->pair_cam_j || !d->focal || !d->cx || !d->cy)
    return fail(nullptr, FM_ERR_INVALID_ARG, "pair_cam_i, pair_cam_j, focal, cx and cy are required");
  if (d->n_kp_pairs > 0 && (!d->kp1_px || !d->kp2_px || !d->kp_img_pair))
    return fail(nullptr, FM_ERR_INVALID_ARG, "kp1_px, kp2_px and kp_img_pair are required when n_kp_pairs > 0");
  fm_problem* pr = new (std::nothrow) fm_problem();
  if (!pr) return fail(nullptr, FM_ERR_OOM, "host allocation failed");
  pr->N = d->n_cams;
  pr->P = d->n_img_pairs;
  pr->Z = d->n_kp_pairs;
  pr->stream = (cudaStream_t)d->cuda_stream;
  cudaError_t e = cudaGetDevice(&pr->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&pr->sm_count, cudaDevAttrMultiProcessorCount, pr->device);
  if (e != cudaSuccess) {
    std::string msg = std::string("no usable CUDA device: ") + cudaGetErrorString(e);
    delete pr;
    return fail(nullptr, FM_ERR_CUDA, msg);
  }
  fm_status st = build(pr, d);
  if (st != FM_OK) {
    g_create_error = pr->last_error;
    release(pr);
    delete pr;
    return st;
  }
  *out = pr;
  return FM_OK;
}

void fm_problem_destroy(fm_problem* pr) {
  if (!pr) return;
  release(pr);
  delete pr;
}

const char* fm_last_error(const fm_problem* pr) {
  return pr ? pr->last_error.c_str() : g_create_error.c_str();
}

fm_status fm_problem_info_get(const fm_problem* pr, fm_problem_info* out) {
  if (!pr || !out) return FM_ERR_INVALID_ARG;
  out->n_cams = pr->N;
  out->n_img_pairs = pr->P;
  out->n_kp_pairs = pr->Z;
  out->n_empty_img_pairs = pr->n_empty;
  out->pairs_per_lane = pr->ea_U;
  out->n_records = pr->n_rec;
  out->device_bytes = pr->device_bytes;
  out->n_scenes = pr->S;
  int nv = 0;
  for (int v : pr->h_cam_valid) nv += v;
  out->n_cams_connected = nv;
  return FM_OK;
}

fm_status fm_set_params(fm_problem* pr, fm_stage st, const float* params, int32_t on_device) {
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!valid_stage(st)) return fail(pr, FM_ERR_INVALID_ARG, "unknown stage");
  if (!params) return fail(pr, FM_ERR_INVALID_ARG, "params is NULL");
  StageBuf b = stage_buf(pr, st);
  FM_CUDA(pr, cudaMemcpyAsync(b.params, params, sizeof(float) * b.count,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, pr->stream));
  fm::launch_check_finite(b.params, (int64_t)b.count, pr->d_err, fm::kErrParamNonFinite, pr->stream);
  FM_LAUNCHED(pr);
  fm_status e = check_err_bits(pr);
  if (e != FM_OK) return e;
  e = reset_adam(pr, *b.adam, b.count);
  if (e != FM_OK) return e;
  *b.set = true;
  if (st == FM_STAGE_ROTATION) pr->trn_target_valid = false;
  return FM_OK;
}

fm_status fm_get_params(const fm_problem* cpr, fm_stage st, float* out, int32_t on_device) {
  fm_problem* pr = const_cast<fm_problem*>(cpr);
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!valid_stage(st)) return fail(pr, FM_ERR_INVALID_ARG, "unknown stage");
  if (!out) return fail(pr, FM_ERR_INVALID_ARG, "params_out is NULL");
  StageBuf b = stage_buf(pr, st);
  if (!*b.set) return fail(pr, FM_ERR_STATE, "the stage's parameters have not been set");
  FM_CUDA(pr, cudaMemcpyAsync(out, b.params, sizeof(float) * b.count,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, pr->stream));
  if (!on_device) FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  return FM_OK;
}

fm_status fm_set_rel_poses(fm_problem* pr, const float* rel_R, const float* rel_t, int32_t on_device) {
  if (!pr) return FM_ERR_INVALID_ARG;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (rel_R) {
    FM_CUDA(pr, cudaMemcpyAsync(pr->rel_R, rel_R, sizeof(float) * 9 * pr->P, k, pr->stream));
    pr->rel_R_set = true;
  }
  if (rel_t) {
    FM_CUDA(pr, cudaMemcpyAsync(pr->rel_t, rel_t, sizeof(float) * 3 * pr->P, k, pr->stream));
    pr->rel_t_set = true;
    pr->trn_target_valid = false;
  }
  return FM_OK;
}

fm_status fm_relative_poses(fm_problem* pr, int32_t irls_iters, float delta, int32_t* n_valid) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  if (irls_iters < 0 || irls_iters > 16) return fail(pr, FM_ERR_INVALID_ARG, "irls_iters must be in [0, 16]");
  if (!(delta > 0.f) || !std::isfinite(delta)) return fail(pr, FM_ERR_INVALID_ARG, "delta must be finite and > 0");
  cudaStream_t s = pr->stream;
  int* d_valid = nullptr;
  FM_ALLOC(pr, d_valid, (size_t)pr->P);
  {
    Timed t(pr, fm::kKRelpose);
    fm::launch_relpose(pr, irls_iters, delta, pr->rel_R, pr->rel_t, d_valid, s);
  }
  cudaError_t le = cudaGetLastError();
  std::vector<int> h(pr->P);
  cudaError_t ce = le;
  if (ce == cudaSuccess && pr->P > 0)
    ce = cudaMemcpyAsync(h.data(), d_valid, sizeof(int) * pr->P, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  cudaFree(d_valid);
  pr->device_bytes -= (int64_t)sizeof(int) * std::max(pr->P, 1);
  if (ce != cudaSuccess) return fail(pr, FM_ERR_CUDA, std::string("relative poses: ") + cudaGetErrorString(ce));
  int cnt = 0;
  for (int v : h) cnt += v;
  if (n_valid) *n_valid = cnt;
  pr->rel_R_set = true;
  pr->rel_t_set = true;
  pr->trn_target_valid = false;
  return FM_OK;
}

fm_status fm_focal_search(fm_problem* pr, const int32_t* group, int32_t n_groups, float rho_min, float rho_max,
                          int32_t n_cand, float tau, int32_t irls_iters, float* focal_out, int32_t* n_estimated) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!focal_out) return fail(pr, FM_ERR_INVALID_ARG, "focal_out is NULL");
  if (!(rho_min > 0.f && rho_max > rho_min) || !std::isfinite(rho_max))
    return fail(pr, FM_ERR_INVALID_ARG, "0 < rho_min < rho_max required");
  if (n_cand < 2 || n_cand > 65536) return fail(pr, FM_ERR_INVALID_ARG, "n_cand must be in [2, 65536]");
  if (!(tau > 0.f) || !std::isfinite(tau)) return fail(pr, FM_ERR_INVALID_ARG, "tau must be finite and > 0");
  if (irls_iters < 0 || irls_iters > 16) return fail(pr, FM_ERR_INVALID_ARG, "irls_iters must be in [0, 16]");
  std::vector<int> g;
  {
    fm_status st = check_groups(pr, group, n_groups, g);
    if (st != FM_OK) return st;
  }
  const int N = pr->N, P = pr->P;
  cudaStream_t s = pr->stream;
  std::vector<int> hi, hj;
  std::vector<float> f0;
  FM_CUDA(pr, fetch(hi, pr->pair_i, P, true));
  FM_CUDA(pr, fetch(hj, pr->pair_j, P, true));
  FM_CUDA(pr, fetch(f0, pr->focal, N, true));
  // candidates rho_k = exp(log rho_min + k (log rho_max - log rho_min) / (n - 1))
  std::vector<float> rhos(n_cand);
  for (int k = 0; k < n_cand; ++k)
    rhos[k] = (float)std::exp(std::log((double)rho_min) +
                              k * (std::log((double)rho_max) - std::log((double)rho_min)) / (n_cand - 1));
  Scratch sc;
  float* e0 = sc.get<float>((size_t)9 * P);
  int* valid = sc.get<int>(P);
  float* d_rhos = sc.get<float>(n_cand);
  float* votes = sc.get<float>(n_cand);
  int* idx = sc.get<int>(P);
  float* fix = sc.get<float>((size_t)2 * P);
  cudaError_t ce = sc.ce;
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return fail(pr, ce == cudaErrorMemoryAllocation ? FM_ERR_OOM : FM_ERR_CUDA, "focal search: allocation");
  }
  {
    Timed t(pr, fm::kKRelpose);
    fm::launch_relpose(pr, irls_iters, 1e-5f, nullptr, nullptr, valid, s, e0);
  }
  ce = cudaGetLastError();
  std::vector<int> hv(P);
  if (ce == cudaSuccess && P > 0) ce = cudaMemcpyAsync(hv.data(), valid, sizeof(int) * P, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_rhos, rhos.data(), sizeof(float) * n_cand, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return fail(pr, FM_ERR_CUDA, std::string("focal search: ") + cudaGetErrorString(ce));
  ReadyOrder order(g, hi, hj, hv, n_groups);
  std::vector<float> rho_g(n_groups, 1.f);
  std::vector<int> list, fi, fj;
  std::vector<float> fixes(2 * (size_t)std::max(P, 1));
  std::vector<float> hvotes(n_cand);
  int n_done = 0;
  for (int best = order.next(); best >= 0 && ce == cudaSuccess; best = order.next()) {
    order.list(best, list, fi, fj);
    const int M = (int)list.size();
    for (int q = 0; q < M; ++q) {
      fixes[q] = fi[q] < 0 ? -1.f : rho_g[fi[q]];
      fixes[P + q] = fj[q] < 0 ? -1.f : rho_g[fj[q]];
    }
    ce = cudaMemcpyAsync(idx, list.data(), sizeof(int) * M, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(fix, fixes.data(), sizeof(float) * 2 * P, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) break;
    {
      Timed t(pr, fm::kKFocalVote);
      fm::launch_focal_vote(e0, idx, fix, fix + P, M, d_rhos, n_cand, tau, votes, s);
    }
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(hvotes.data(), votes, sizeof(float) * n_cand, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) break;
    int k = 0;
    for (int q = 1; q < n_cand; ++q)
      if (hvotes[q] > hvotes[k]) k = q;   // the first maximum
    rho_g[best] = rhos[k];
    order.finish(best);
    ++n_done;
  }
  if (ce != cudaSuccess) return fail(pr, FM_ERR_CUDA, std::string("focal search: ") + cudaGetErrorString(ce));
  for (int c = 0; c < N; ++c) focal_out[c] = order.done[g[c]] ? f0[c] * rho_g[g[c]] : f0[c];
  if (n_estimated) *n_estimated = n_done;
  return FM_OK;
}

fm_status fm_distortion_search(fm_problem* pr, const int32_t* group, int32_t n_groups, float alpha_min,
                               float alpha_max, int32_t n_cand, int32_t n_levels, float* alpha_out,
                               int32_t* n_estimated) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!alpha_out) return fail(pr, FM_ERR_INVALID_ARG, "alpha_out is NULL");
  if (!(alpha_max > alpha_min) || !std::isfinite(alpha_min) || !std::isfinite(alpha_max))
    return fail(pr, FM_ERR_INVALID_ARG, "finite alpha_min < alpha_max required");
  if (n_cand < 2 || n_cand > 32) return fail(pr, FM_ERR_INVALID_ARG, "n_cand must be in [2, 32]");
  if (n_levels < 1 || n_levels > 16) return fail(pr, FM_ERR_INVALID_ARG, "n_levels must be in [1, 16]");
  std::vector<int> g;
  {
    fm_status st = check_groups(pr, group, n_groups, g);
    if (st != FM_OK) return st;
  }
  const int N = pr->N, P = pr->P;
  cudaStream_t s = pr->stream;
  std::vector<int> hi, hj, off;
  std::vector<float> scale;
  FM_CUDA(pr, fetch(hi, pr->pair_i, P, true));
  FM_CUDA(pr, fetch(hj, pr->pair_j, P, true));
  FM_CUDA(pr, fetch(off, pr->seg_off, (size_t)P + 1, true));
  FM_CUDA(pr, image_scales(pr, scale));
  std::vector<int> usable(P);
  for (int n = 0; n < P; ++n) usable[n] = off[n + 1] - off[n] >= 8;
  Scratch sc;
  float* d_scale = sc.get<float>(N);
  int* idx = sc.get<int>((size_t)2 * P);   // pairs, then rows
  float* fix = sc.get<float>((size_t)2 * P);
  float* d_cand = sc.get<float>(32);
  float* err = sc.get<float>((size_t)32 * P);
  float* sums = sc.get<float>(32);
  cudaError_t ce = sc.ce;
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return fail(pr, ce == cudaErrorMemoryAllocation ? FM_ERR_OOM : FM_ERR_CUDA, "distortion search: allocation");
  }
  ce = cudaMemcpyAsync(d_scale, scale.data(), sizeof(float) * N, cudaMemcpyHostToDevice, s);
  ReadyOrder order(g, hi, hj, usable, n_groups);
  std::vector<float> alpha_g(n_groups, 0.f);
  std::vector<int> list, fi, fj, items, rows;
  std::vector<float> fixes(2 * (size_t)std::max(P, 1));
  std::vector<float> cand(n_cand), hs(n_cand);
  int n_done = 0;
  for (int best = ce == cudaSuccess ? order.next() : -1; best >= 0 && ce == cudaSuccess; best = order.next()) {
    order.list(best, list, fi, fj);
    const int M = (int)list.size();
    for (int q = 0; q < M; ++q) {
      fixes[q] = fi[q] < 0 ? NAN : alpha_g[fi[q]];
      fixes[P + q] = fj[q] < 0 ? NAN : alpha_g[fj[q]];
    }
    const int n_small = split_by_size(list, off, items, rows);
    ce = cudaMemcpyAsync(idx, items.data(), sizeof(int) * M, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(idx + P, rows.data(), sizeof(int) * M, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(fix, fixes.data(), sizeof(float) * 2 * P, cudaMemcpyHostToDevice, s);
    // hierarchical levels: candidates evenly over [lo, hi]; the winner's
    // neighbours (the end candidate at an end) bound the next level
    double lo = alpha_min, hi_a = alpha_max, est = alpha_min;
    for (int level = 0; level < n_levels && ce == cudaSuccess; ++level) {
      for (int k = 0; k < n_cand; ++k) cand[k] = (float)(lo + (hi_a - lo) * k / (n_cand - 1));
      ce = cudaMemcpyAsync(d_cand, cand.data(), sizeof(float) * n_cand, cudaMemcpyHostToDevice, s);
      if (ce != cudaSuccess) break;
      ce = dist_level(pr, d_scale, idx, idx + P, fix, fix + P, M, n_small, d_cand, n_cand, err);
      if (ce != cudaSuccess) break;
      {
        Timed t(pr, fm::kKDistReduce);
        fm::launch_dist_reduce(err, M, n_cand, sums, s);
      }
      ce = cudaGetLastError();
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(hs.data(), sums, sizeof(float) * n_cand, cudaMemcpyDeviceToHost, s);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) break;
      // every candidate's average divides by the same keypoint-pair count, so
      // the sums rank them alike
      int k = -1;
      for (int q = 0; q < n_cand; ++q)   // the first minimum; NaN never wins
        if (!std::isnan(hs[q]) && (k < 0 || hs[q] < hs[k])) k = q;
      if (k < 0) k = 0;
      est = cand[k];
      lo = cand[std::max(k - 1, 0)];
      hi_a = cand[std::min(k + 1, n_cand - 1)];
    }
    alpha_g[best] = (float)est;
    order.finish(best);
    ++n_done;
  }
  if (ce != cudaSuccess) return fail(pr, FM_ERR_CUDA, std::string("distortion search: ") + cudaGetErrorString(ce));
  for (int c = 0; c < N; ++c) alpha_out[c] = order.done[g[c]] ? alpha_g[g[c]] : 0.f;
  if (n_estimated) *n_estimated = n_done;
  return FM_OK;
}

fm_status fm_distortion_pair_errors(fm_problem* pr, const float* alpha_cand, int32_t n_cand, float* err_out,
                                    int32_t on_device) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!alpha_cand || !err_out) return fail(pr, FM_ERR_INVALID_ARG, "alpha_cand and err_out are required");
  if (n_cand < 1 || n_cand > 32) return fail(pr, FM_ERR_INVALID_ARG, "n_cand must be in [1, 32]");
  const int N = pr->N, P = pr->P;
  cudaStream_t s = pr->stream;
  std::vector<float> cand, scale;
  std::vector<int> off, all(P), items, rows;
  FM_CUDA(pr, fetch(cand, alpha_cand, n_cand, on_device != 0));
  FM_CUDA(pr, image_scales(pr, scale));
  FM_CUDA(pr, fetch(off, pr->seg_off, (size_t)P + 1, true));
  for (int n = 0; n < P; ++n) all[n] = n;
  const int n_small = split_by_size(all, off, items, rows);
  Scratch sc;
  float* d_scale = sc.get<float>(N);
  float* d_cand = sc.get<float>(32);
  int* d_idx = sc.get<int>((size_t)2 * P);
  float* err = on_device ? err_out : sc.get<float>((size_t)n_cand * P);
  cudaError_t ce = sc.ce;
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return fail(pr, ce == cudaErrorMemoryAllocation ? FM_ERR_OOM : FM_ERR_CUDA, "distortion errors: allocation");
  }
  ce = cudaMemcpyAsync(d_scale, scale.data(), sizeof(float) * N, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_cand, cand.data(), sizeof(float) * n_cand, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess && P > 0) ce = cudaMemcpyAsync(d_idx, items.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess && P > 0)
    ce = cudaMemcpyAsync(d_idx + P, rows.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = dist_level(pr, d_scale, d_idx, d_idx + P, nullptr, nullptr, P, n_small, d_cand, n_cand, err);
  if (ce == cudaSuccess && !on_device && P > 0)
    ce = cudaMemcpyAsync(err_out, err, sizeof(float) * n_cand * P, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return fail(pr, FM_ERR_CUDA, std::string("distortion errors: ") + cudaGetErrorString(ce));
  return FM_OK;
}

fm_status fm_set_distortion(fm_problem* pr, const float* alpha, int32_t on_device) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!alpha) return fail(pr, FM_ERR_INVALID_ARG, "alpha is NULL");
  std::vector<float> a, scale;
  FM_CUDA(pr, fetch(a, alpha, pr->N, on_device != 0));
  for (int c = 0; c < pr->N; ++c)
    if (!std::isfinite(a[c])) return fail(pr, FM_ERR_INVALID_ARG, "alpha[" + std::to_string(c) + "] must be finite");
  FM_CUDA(pr, image_scales(pr, scale));
  Scratch sc;
  float* d_scale = sc.get<float>(pr->N);
  float* d_alpha = sc.get<float>(pr->N);
  int* bad = sc.get<int>(1);
  cudaError_t ce = sc.ce;
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return fail(pr, ce == cudaErrorMemoryAllocation ? FM_ERR_OOM : FM_ERR_CUDA, "set distortion: allocation");
  }
  cudaStream_t s = pr->stream;
  int h_bad = 0;
  ce = cudaMemcpyAsync(d_scale, scale.data(), sizeof(float) * pr->N, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_alpha, a.data(), sizeof(float) * pr->N, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (ce == cudaSuccess) {
    fm::launch_undistort(pr, d_scale, d_alpha, bad, s);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return fail(pr, FM_ERR_CUDA, std::string("set distortion: ") + cudaGetErrorString(ce));
  pr->W_valid = false;
  pr->graph_epoch += 1;
  if (h_bad)
    return fail(pr, FM_ERR_INVALID_ARG,
                "1 + alpha r^2 <= 0 at some keypoint: those keypoint pairs were left as they were");
  return FM_OK;
}

fm_status fm_set_focal(fm_problem* pr, const float* focal, int32_t on_device) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!focal) return fail(pr, FM_ERR_INVALID_ARG, "focal is NULL");
  std::vector<float> f;
  FM_CUDA(pr, fetch(f, focal, pr->N, on_device != 0));
  for (int c = 0; c < pr->N; ++c)
    if (!(std::isfinite(f[c]) && f[c] > 0.f))
      return fail(pr, FM_ERR_INVALID_ARG, "focal[" + std::to_string(c) + "] must be finite and > 0");
  float* f_new = nullptr;
  FM_ALLOC(pr, f_new, (size_t)pr->N);
  cudaStream_t s = pr->stream;
  cudaError_t ce = cudaMemcpyAsync(f_new, f.data(), sizeof(float) * pr->N, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) {
    fm::launch_recalibrate(pr, pr->focal, f_new, s);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(pr->focal, f_new, sizeof(float) * pr->N, cudaMemcpyDeviceToDevice, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  cudaFree(f_new);
  pr->device_bytes -= (int64_t)sizeof(float) * std::max(pr->N, 1);
  if (ce != cudaSuccess) return fail(pr, FM_ERR_CUDA, std::string("set focal: ") + cudaGetErrorString(ce));
  pr->W_valid = false;
  pr->graph_epoch += 1;
  return FM_OK;
}

fm_status fm_translation_set_runs(fm_problem* pr, int32_t n_runs) {
  if (!pr) return FM_ERR_INVALID_ARG;
  if (n_runs < 1 || n_runs > 64) return fail(pr, FM_ERR_INVALID_ARG, "n_runs must be in [1, 64]");
  FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  return resize_runs(pr, n_runs);
}

fm_status fm_ea_set_loss(fm_problem* pr, fm_ea_loss loss) {
  if (!pr) return FM_ERR_INVALID_ARG;
  if (loss != FM_EA_L1 && loss != FM_EA_L2 && loss != FM_EA_COMPACT)
    return fail(pr, FM_ERR_INVALID_ARG, "unknown epipolar loss");
  pr->ea_loss = loss;
  pr->graph_epoch += 1;
  return FM_OK;
}

// pair_inv_z = 1/Z_s (unit weights) for every image pair of scene s
static fm_status set_unit_normalisers(fm_problem* pr) {
  std::vector<float> inv_z(pr->P);
  for (int q = 0; q < pr->S; ++q) {
    const int64_t zq = pr->h_sc_kp_off[q + 1] - pr->h_sc_kp_off[q];
    const float v = zq > 0 ? (float)(1.0 / (double)zq) : 0.f;
    for (int n = pr->h_sc_pair_off[q]; n < pr->h_sc_pair_off[q + 1]; ++n) inv_z[n] = v;
  }
  FM_CUDA(pr, cudaMemcpyAsync(pr->pair_inv_z, inv_z.data(), sizeof(float) * pr->P, cudaMemcpyHostToDevice,
                              pr->stream));
  FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  const int64_t z0 = pr->h_sc_kp_off[1] - pr->h_sc_kp_off[0];
  pr->ea_inv_z = z0 > 0 ? (float)(1.0 / (double)z0) : 0.f;
  return FM_OK;
}

// pair_inv_z from the per-scene counts in d_kept; returns the total on the host
static fm_status normalisers_from_counts(fm_problem* pr, int64_t* total) {
  fm::launch_pair_inv_from_counts(pr, pr->d_kept, pr->stream);
  FM_LAUNCHED(pr);
  std::vector<unsigned long long> kept(pr->S);
  FM_CUDA(pr, cudaMemcpyAsync(kept.data(), pr->d_kept, sizeof(unsigned long long) * pr->S,
                              cudaMemcpyDeviceToHost, pr->stream));
  FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  int64_t t = 0;
  for (int q = 0; q < pr->S; ++q) t += (int64_t)kept[q];
  if (total) *total = t;
  pr->ea_inv_z = kept[0] > 0 ? (float)(1.0 / (double)kept[0]) : 0.f;
  return FM_OK;
}

fm_status fm_ea_set_weights(fm_problem* pr, const float* w, int32_t on_device, float inv_z) {
  if (!pr) return FM_ERR_INVALID_ARG;
  pr->graph_epoch += 1;   // the weight pointer of the captured launches may change
  if (!w) {
    dfree(pr->ea_w);
    pr->W_valid = false;
    return set_unit_normalisers(pr);
  }
  if (!(std::isfinite(inv_z) && inv_z >= 0.f)) return fail(pr, FM_ERR_INVALID_ARG, "inv_z must be finite and >= 0");
  if (!pr->ea_w) FM_ALLOC(pr, pr->ea_w, (size_t)pr->Z);
  if (pr->Z > 0 && pr->kp_perm) {
    // the caller's order -> the internal (sorted) order
    const float* src = w;
    float* tmp = nullptr;
    if (!on_device) {
      FM_ALLOC(pr, tmp, (size_t)pr->Z);
      FM_CUDA(pr, cudaMemcpyAsync(tmp, w, sizeof(float) * pr->Z, cudaMemcpyHostToDevice, pr->stream));
      src = tmp;
    }
    fm::launch_permute(src, pr->kp_perm, pr->Z, true, pr->ea_w, pr->stream);
    cudaError_t ce = cudaGetLastError();
    if (tmp) {
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(pr->stream);
      cudaFree(tmp);
      pr->device_bytes -= (int64_t)sizeof(float) * pr->Z;
    }
    if (ce != cudaSuccess) return fail(pr, FM_ERR_CUDA, std::string("weights: ") + cudaGetErrorString(ce));
  } else if (pr->Z > 0) {
    FM_CUDA(pr, cudaMemcpyAsync(pr->ea_w, w, sizeof(float) * pr->Z,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, pr->stream));
  }
  if (pr->Z > 0) {
    fm::launch_check_finite(pr->ea_w, pr->Z, pr->d_err, fm::kErrParamNonFinite, pr->stream);
    FM_LAUNCHED(pr);
    fm_status e = check_err_bits(pr);
    if (e != FM_OK) return e;
  }
  pr->W_valid = false;
  if (inv_z > 0.f) {
    std::vector<float> v(pr->P, inv_z);
    FM_CUDA(pr, cudaMemcpyAsync(pr->pair_inv_z, v.data(), sizeof(float) * pr->P, cudaMemcpyHostToDevice,
                                pr->stream));
    FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
    pr->ea_inv_z = inv_z;
    return FM_OK;
  }
  // inv_z == 0: each scene's 1/(number of its pairs with a positive weight)
  FM_CUDA(pr, cudaMemsetAsync(pr->d_kept, 0, sizeof(unsigned long long) * pr->S, pr->stream));
  fm::launch_count_positive(pr, pr->ea_w, pr->d_kept, pr->stream);
  FM_LAUNCHED(pr);
  return normalisers_from_counts(pr, nullptr);
}

fm_status fm_ea_reweight(fm_problem* pr, float tau, float delta, int32_t irls, int64_t* n_kept) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!(tau > 0.f) || !(delta > 0.f) || !std::isfinite(delta))
    return fail(pr, FM_ERR_INVALID_ARG, "tau > 0 and finite delta > 0 required");
  if (!pr->ea_params_set) return fail(pr, FM_ERR_STATE, "the epipolar-stage parameters have not been set");
  cudaStream_t s = pr->stream;
  pr->graph_epoch += 1;
  if (!pr->ea_w) FM_ALLOC(pr, pr->ea_w, (size_t)pr->Z);
  {
    Timed t(pr, fm::kKEaTables);
    fm::launch_ea_tables(pr->ea_params, pr->pair_i, pr->pair_j, pr->seg_off, pr->P, pr->seg_tab, nullptr, s);
  }
  FM_LAUNCHED(pr);
  FM_CUDA(pr, cudaMemsetAsync(pr->d_kept, 0, sizeof(unsigned long long) * pr->S, s));
  {
    Timed t(pr, fm::kKEaReweight);
    fm::launch_ea_reweight(pr, tau, delta, irls, pr->ea_w, pr->d_kept, s);
  }
  FM_LAUNCHED(pr);
  {
    Timed t(pr, fm::kKWBuild);
    fm::launch_w_build(pr, pr->ea_w, pr->W, s);   // centred at the reweighting pose
  }
  FM_LAUNCHED(pr);
  pr->W_valid = true;
  int64_t total = 0;
  fm_status e = normalisers_from_counts(pr, &total);
  if (e != FM_OK) return e;
  if (n_kept) *n_kept = total;
  return FM_OK;
}

fm_status fm_ea_get_weights(fm_problem* pr, float* out, int32_t on_device, float* inv_z) {
  if (!pr || !out) return FM_ERR_INVALID_ARG;
  if (!pr->ea_w) return fail(pr, FM_ERR_STATE, "no per-pair weights are set");
  if (pr->Z > 0 && pr->kp_perm) {
    // the internal (sorted) order -> the caller's order
    float* dst = on_device ? out : nullptr;
    if (!on_device) FM_ALLOC(pr, dst, (size_t)pr->Z);
    fm::launch_permute(pr->ea_w, pr->kp_perm, pr->Z, false, dst, pr->stream);
    cudaError_t ce = cudaGetLastError();
    if (!on_device) {
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(out, dst, sizeof(float) * pr->Z, cudaMemcpyDeviceToHost, pr->stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(pr->stream);
      cudaFree(dst);
      pr->device_bytes -= (int64_t)sizeof(float) * pr->Z;
    }
    if (ce != cudaSuccess) return fail(pr, FM_ERR_CUDA, std::string("weights: ") + cudaGetErrorString(ce));
  } else if (pr->Z > 0) {
    FM_CUDA(pr, cudaMemcpyAsync(out, pr->ea_w, sizeof(float) * pr->Z,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, pr->stream));
  }
  FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  if (inv_z) *inv_z = pr->ea_inv_z;
  return FM_OK;
}

fm_status fm_kp_order(const fm_problem* cpr, int32_t* perm_out, int32_t on_device) {
  fm_problem* pr = const_cast<fm_problem*>(cpr);
  if (!pr || !perm_out) return FM_ERR_INVALID_ARG;
  if (pr->Z == 0) return FM_OK;
  if (pr->kp_perm) {
    FM_CUDA(pr, cudaMemcpyAsync(perm_out, pr->kp_perm, sizeof(int32_t) * pr->Z,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, pr->stream));
    FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
    return FM_OK;
  }
  if (!on_device) {
    for (int64_t k = 0; k < pr->Z; ++k) perm_out[k] = (int32_t)k;
    return FM_OK;
  }
  std::vector<int32_t> iota((size_t)pr->Z);
  for (int64_t k = 0; k < pr->Z; ++k) iota[(size_t)k] = (int32_t)k;
  FM_CUDA(pr, cudaMemcpyAsync(perm_out, iota.data(), sizeof(int32_t) * pr->Z, cudaMemcpyHostToDevice, pr->stream));
  FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  return FM_OK;
}

static fm_status replay(fm_problem* pr, cudaGraphExec_t exec);
static void evict_lru(fm_problem* pr);

// waits for the problem's stream: polls for up to 5 ms (a synchronous call
// that returns results to the host is latency-bound; a blocking wait adds the
// host's wake-up latency), then blocks
static fm_status wait_stream(fm_problem* pr) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t q = cudaStreamQuery(pr->stream);
    if (q == cudaSuccess) return FM_OK;
    if (q != cudaErrorNotReady) return fail(pr, FM_ERR_CUDA, std::string("cudaStreamQuery: ") + cudaGetErrorString(q));
    if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(5)) break;
  }
  FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  return FM_OK;
}
static fm_status capture_loss_grad(fm_problem* pr, fm_stage st, size_t count, bool want_loss,
                                   bool want_grad, fm_problem::GraphEntry* out);

// fm_loss_grad with host buffers through a captured graph (from the second
// call at an epoch on); *done = false leaves the call to the direct path
static fm_status loss_grad_graph(fm_problem* pr, fm_stage st, const float* params, float* loss, float* grad,
                                 size_t count, size_t nl, bool* done) {
  *done = false;
  // lazily built state is settled by a direct evaluation first
  if (st == FM_STAGE_TRANSLATION && !pr->trn_target_valid) return FM_OK;
  if (st == FM_STAGE_EPIPOLAR && pr->ea_loss == FM_EA_COMPACT && !pr->W_valid) return FM_OK;
  const int flags = (loss ? 1 : 0) | (grad ? 2 : 0);
  fm_problem::GraphEntry* g = nullptr;
  for (auto& e : pr->graphs)
    if (e.kind == 1 && e.stage == (int)st && e.flags == flags && e.epoch == pr->graph_epoch && e.exec) g = &e;
  if (!g) {
    // the first call at an epoch runs directly: it settles lazily built state
    // (the compact form's W, the translation targets) outside any graph
    if (pr->lg_seen[st] != pr->graph_epoch) {
      pr->lg_seen[st] = pr->graph_epoch;
      return FM_OK;
    }
    if (pr->h_lg_cap < count) {
      if (pr->h_lg_in) cudaFreeHost(pr->h_lg_in);
      if (pr->h_lg_grad) cudaFreeHost(pr->h_lg_grad);
      pr->h_lg_in = pr->h_lg_grad = nullptr;
      pr->h_lg_cap = 0;
      FM_CUDA(pr, cudaMallocHost((void**)&pr->h_lg_in, sizeof(float) * count));
      FM_CUDA(pr, cudaMallocHost((void**)&pr->h_lg_grad, sizeof(float) * count));
      pr->h_lg_cap = count;
      for (auto& e : pr->graphs)   // graphs of the old buffers
        if (e.kind == 1 && e.exec) {
          cudaGraphExecDestroy(e.exec);
          e.exec = nullptr;
        }
    }
    evict_lru(pr);
    fm_problem::GraphEntry e;
    e.stage = (int)st;
    e.kind = 1;
    e.flags = flags;
    e.epoch = pr->graph_epoch;
    fm_status r = capture_loss_grad(pr, st, count, loss != nullptr, grad != nullptr, &e);
    if (r != FM_OK) return r;
    pr->graphs.push_back(e);
    g = &pr->graphs.back();
  }
  g->last_use = ++pr->graph_clock;
  std::memcpy(pr->h_lg_in, params, sizeof(float) * count);
  // one launch on the problem's stream (stream order covers the copies in and
  // out); the wait spins first, which avoids the blocking wake-up latency
  FM_CUDA(pr, cudaGraphLaunch(g->exec, pr->stream));
  fm::g_plain_once = true;
  for (int k = 0; k < fm::kKCount; ++k) pr->k_launches[k] += g->counts[k];
  pr->graph_replays += 1;
  fm_status r = wait_stream(pr);
  if (r != FM_OK) return r;
  if (*pr->h_err) return check_err_bits(pr);
  if (grad) std::memcpy(grad, pr->h_lg_grad, sizeof(float) * count);
  if (loss) std::memcpy(loss, pr->h_loss, sizeof(float) * nl);
  *done = true;
  return FM_OK;
}

fm_status fm_loss_grad(fm_problem* pr, fm_stage st, const float* params, float* loss, float* grad,
                       int32_t mem_on_device) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!valid_stage(st)) return fail(pr, FM_ERR_INVALID_ARG, "unknown stage");
  if (!params) return fail(pr, FM_ERR_INVALID_ARG, "params is NULL");
  cudaStream_t s = pr->stream;
  const size_t count = (size_t)stage_dim(st) * pr->N * (st == FM_STAGE_TRANSLATION ? pr->trn_runs : 1);
  if (!mem_on_device && (loss || grad) && pr->use_graphs && !pr->timing) {
    bool done = false;
    const size_t nl = (size_t)((st == FM_STAGE_TRANSLATION) ? pr->trn_runs : 1) * pr->S;
    fm_status e = loss_grad_graph(pr, st, params, loss, grad, count, nl, &done);
    if (e != FM_OK || done) return e;
  }
  const float* p = params;
  if (!mem_on_device) {
    FM_CUDA(pr, cudaMemcpyAsync(pr->scratch_params, params, sizeof(float) * count, cudaMemcpyHostToDevice, s));
    p = pr->scratch_params;
  }
  float* g = nullptr;
  if (grad) g = mem_on_device ? grad : pr->scratch_grad;
  fm_status e = evaluate(pr, st, p, g, nullptr, nullptr, loss ? pr->d_loss : nullptr);
  if (e != FM_OK) return e;
  const int runs = (st == FM_STAGE_TRANSLATION) ? pr->trn_runs : 1;
  if (grad && !mem_on_device)
    FM_CUDA(pr, cudaMemcpyAsync(grad, g, sizeof(float) * count, cudaMemcpyDeviceToHost, s));
  const size_t nl = (size_t)runs * pr->S;
  if (loss) FM_CUDA(pr, cudaMemcpyAsync(pr->h_loss, pr->d_loss, sizeof(float) * nl, cudaMemcpyDeviceToHost, s));
  if (loss || (grad && !mem_on_device)) {
    // the error bits travel with the results (no extra synchronisation)
    FM_CUDA(pr, cudaMemcpyAsync(pr->h_err, pr->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    fm_status w = wait_stream(pr);
    if (w != FM_OK) return w;
    if (*pr->h_err) return check_err_bits(pr);
    if (loss) std::memcpy(loss, pr->h_loss, sizeof(float) * nl);
  }
  return FM_OK;
}

static fm_status ea_split_check(fm_problem* pr, const float* params, int32_t save, const void* saved) {
  if (!params) return fail(pr, FM_ERR_INVALID_ARG, "params_dev is NULL");
  if (save < FM_EA_SAVE_NONE || save > FM_EA_SAVE_DLDE) return fail(pr, FM_ERR_INVALID_ARG, "unknown save mode");
  if (save != FM_EA_SAVE_NONE && !saved) return fail(pr, FM_ERR_INVALID_ARG, "saved_dev is NULL");
  if (save != FM_EA_SAVE_NONE && (reinterpret_cast<uintptr_t>(saved) & 15u))
    return fail(pr, FM_ERR_INVALID_ARG, "saved_dev must be 16-byte aligned");
  if (pr->ea_loss == FM_EA_COMPACT)
    return fail(pr, FM_ERR_STATE,
                "the forward/backward split evaluates the direct forms (FM_EA_L1, FM_EA_L2); "
                "the compact form goes through fm_loss_grad");
  return FM_OK;
}

fm_status fm_ea_forward(fm_problem* pr, const float* params, float* loss_dev, int32_t save, float* saved) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  fm_status e = ea_split_check(pr, params, save, saved);
  if (e != FM_OK) return e;
  if (!loss_dev) return fail(pr, FM_ERR_INVALID_ARG, "loss_dev is NULL");
  cudaStream_t s = pr->stream;
  {
    Timed t(pr, fm::kKEaTables);
    fm::launch_ea_tables(params, pr->pair_i, pr->pair_j, pr->seg_off, pr->P, pr->seg_tab, nullptr, s);
  }
  FM_LAUNCHED(pr);
  fm::SegArgs a = fm::seg_args(pr, params);   // per-pair (per-scene) normalisers
  a.seg_grad = nullptr;
  if (save == FM_EA_SAVE_DLDE) {
    if (pr->n_wruns > 0) {
      Timed t(pr, fm::kKEaDirect);
      fm::launch_ea_direct(pr, pr->ea_w, pr->ea_loss, s);
    }
    a.g_scale = (pr->ea_loss == FM_EA_L1) ? 1.f : 2.f;
    a.dlde_out = saved;
  } else if (pr->n_wruns > 0) {
    Timed t(pr, fm::kKEaDirectLoss);
    fm::launch_ea_direct_loss(pr, pr->ea_w, pr->ea_loss, save == FM_EA_SAVE_COEF ? saved : nullptr, s);
  }
  FM_LAUNCHED(pr);
  {
    Timed t(pr, fm::kKEaSegments);
    fm::launch_ea_segments(a, s);
  }
  FM_LAUNCHED(pr);
  {
    Timed t(pr, fm::kKLossSum);
    fm::launch_sum_fixed(pr->seg_loss, pr->P, 1, loss_args(pr, loss_dev, nullptr), s);
  }
  FM_LAUNCHED(pr);
  return FM_OK;
}

fm_status fm_ea_focal_forward(fm_problem* pr, const float* params, const float* phi, float* loss_dev,
                              float* dlde_saved) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  fm_status e = ea_split_check(pr, params, FM_EA_SAVE_DLDE, dlde_saved);
  if (e != FM_OK) return e;
  if (!phi || !loss_dev) return fail(pr, FM_ERR_INVALID_ARG, "phi_dev and loss_dev are required");
  cudaStream_t s = pr->stream;
  {
    Timed t(pr, fm::kKEaTables);
    fm::launch_ea_tables(params, pr->pair_i, pr->pair_j, pr->seg_off, pr->P, pr->seg_tab, nullptr, s,
                         phi);   // E'_n = S_j E_n S_i
  }
  FM_LAUNCHED(pr);
  fm::SegArgs a = fm::seg_args(pr, params);
  a.seg_grad = nullptr;
  if (pr->n_wruns > 0) {
    Timed t(pr, fm::kKEaDirect);
    fm::launch_ea_direct(pr, pr->ea_w, pr->ea_loss, s);
  }
  a.g_scale = (pr->ea_loss == FM_EA_L1) ? 1.f : 2.f;
  a.dlde_out = dlde_saved;   // dL/dE'_n
  FM_LAUNCHED(pr);
  {
    Timed t(pr, fm::kKEaSegments);
    fm::launch_ea_segments(a, s);
  }
  {
    Timed t(pr, fm::kKLossSum);
    fm::launch_sum_fixed(pr->seg_loss, pr->P, 1, loss_args(pr, loss_dev, nullptr), s);
  }
  FM_LAUNCHED(pr);
  return FM_OK;
}

fm_status fm_ea_focal_backward(fm_problem* pr, const float* params, const float* phi, const float* dlde_saved,
                               const float* grad_loss, float* grad, float* grad_phi) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  fm_status e = ea_split_check(pr, params, FM_EA_SAVE_DLDE, dlde_saved);
  if (e != FM_OK) return e;
  if (!phi || !grad || !grad_phi) return fail(pr, FM_ERR_INVALID_ARG, "phi_dev, grad_dev and grad_phi_dev are required");
  cudaStream_t s = pr->stream;
  if (!pr->focal_G) FM_ALLOC(pr, pr->focal_G, 9 * (size_t)std::max(pr->P, 1));
  if (!pr->focal_dphi) FM_ALLOC(pr, pr->focal_dphi, 2 * (size_t)std::max(pr->P, 1));
  fm::launch_focal_dlde(pr, params, dlde_saved, phi, grad_loss, pr->focal_G, pr->focal_dphi, s);
  FM_LAUNCHED(pr);
  fm::SegArgs a = fm::seg_args(pr, params);
  a.seg_loss = nullptr;
  a.grad_loss = grad_loss;
  a.dlde_in = pr->focal_G;   // dL/dE_n = S_j G' S_i
  {
    Timed t(pr, fm::kKEaSegments);
    fm::launch_ea_segments(a, s);
  }
  FM_LAUNCHED(pr);
  fm::CamUpdate u = cam_update(pr, params, grad, nullptr, nullptr, nullptr, 1);
  {
    Timed t(pr, fm::kKCamUpdate);
    fm::launch_cam_update(FM_STAGE_EPIPOLAR, u, s);
  }
  fm::launch_focal_cam(pr, pr->focal_dphi, grad_phi, s);
  FM_LAUNCHED(pr);
  return FM_OK;
}

fm_status fm_ea_backward(fm_problem* pr, const float* params, int32_t save, const float* saved,
                         const float* grad_loss, float* grad) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  fm_status e = ea_split_check(pr, params, save, saved);
  if (e != FM_OK) return e;
  if (!grad) return fail(pr, FM_ERR_INVALID_ARG, "grad_dev is NULL");
  cudaStream_t s = pr->stream;
  fm::SegArgs a = fm::seg_args(pr, params);
  a.seg_loss = nullptr;
  a.grad_loss = grad_loss;
  if (save == FM_EA_SAVE_DLDE) {
    a.dlde_in = saved;
  } else {
    {
      Timed t(pr, fm::kKEaTables);
      fm::launch_ea_tables(params, pr->pair_i, pr->pair_j, pr->seg_off, pr->P, pr->seg_tab, nullptr, s);
    }
    FM_LAUNCHED(pr);
    if (save == FM_EA_SAVE_COEF) {
      if (pr->n_wruns > 0) {
        Timed t(pr, fm::kKEaDirectCoef);
        fm::launch_ea_direct_from_coef(pr, saved, s);
      }
      a.g_scale = 1.f;   // the stored coefficients carry rho' in full
    } else {
      if (pr->n_wruns > 0) {
        Timed t(pr, fm::kKEaDirect);
        fm::launch_ea_direct(pr, pr->ea_w, pr->ea_loss, s);
      }
      a.g_scale = (pr->ea_loss == FM_EA_L1) ? 1.f : 2.f;
    }
    FM_LAUNCHED(pr);
  }
  {
    Timed t(pr, fm::kKEaSegments);
    fm::launch_ea_segments(a, s);
  }
  FM_LAUNCHED(pr);
  fm::CamUpdate u = cam_update(pr, params, grad, nullptr, nullptr, nullptr, 1);
  {
    Timed t(pr, fm::kKCamUpdate);
    fm::launch_cam_update(FM_STAGE_EPIPOLAR, u, s);
  }
  FM_LAUNCHED(pr);
  return FM_OK;
}

// ---- captured iterations
// fm_step replays a CUDA graph of kGraphIters iterations (each one the
// stage's launches of `evaluate` with Adam) instead of launching every kernel
// from the host.  Captured arguments are device pointers and the Adam
// constants; the graphs are keyed by stage, constants and an epoch that every
// call able to change a captured pointer or branch bumps.  Capture runs on a
// private stream (the legacy default stream cannot be captured); replays go
// to the problem's stream.
//
// A replay is ordered by events on both sides: the kernels of this library
// signal their successors early (programmatic dependent launch), and a graph
// launched right behind such a kernel was seen to start before that kernel's
// writes were done.  An event records the completion of everything before
// it, so the graph runs on the private stream behind one event, and the
// problem's stream waits for a second one.
constexpr int kGraphIters = 16;

static fm_status replay(fm_problem* pr, cudaGraphExec_t exec) {
  if (!pr->graph_in) FM_CUDA(pr, cudaEventCreateWithFlags(&pr->graph_in, cudaEventDisableTiming));
  if (!pr->graph_out) FM_CUDA(pr, cudaEventCreateWithFlags(&pr->graph_out, cudaEventDisableTiming));
  FM_CUDA(pr, cudaEventRecord(pr->graph_in, pr->stream));
  FM_CUDA(pr, cudaStreamWaitEvent(pr->cap_stream, pr->graph_in, 0));
  FM_CUDA(pr, cudaGraphLaunch(exec, pr->cap_stream));
  FM_CUDA(pr, cudaEventRecord(pr->graph_out, pr->cap_stream));
  FM_CUDA(pr, cudaStreamWaitEvent(pr->stream, pr->graph_out, 0));
  fm::g_plain_once = true;
  return FM_OK;
}

static fm_status capture_graph(fm_problem* pr, fm_stage st, const fm_adam_opts* opts, float* params,
                               fm::AdamState* adam, fm_problem::GraphEntry* out) {
  if (!pr->cap_stream) FM_CUDA(pr, cudaStreamCreateWithFlags(&pr->cap_stream, cudaStreamNonBlocking));
  int64_t before[fm::kKCount];
  std::memcpy(before, pr->k_launches, sizeof(before));
  cudaStream_t orig = pr->stream;
  pr->stream = pr->cap_stream;
  cudaError_t ce = cudaStreamBeginCapture(pr->cap_stream, cudaStreamCaptureModeThreadLocal);
  fm_status e = FM_OK;
  const bool was = fm::g_capturing;
  fm::g_capturing = true;
  if (ce == cudaSuccess)
    for (int k = 0; k < kGraphIters && e == FM_OK; ++k) e = evaluate(pr, st, params, nullptr, opts, adam, nullptr);
  fm::g_capturing = was;
  cudaGraph_t graph = nullptr;
  cudaError_t ce2 = (ce == cudaSuccess) ? cudaStreamEndCapture(pr->cap_stream, &graph) : ce;
  pr->stream = orig;
  for (int k = 0; k < fm::kKCount; ++k) {
    out->counts[k] = pr->k_launches[k] - before[k];
    pr->k_launches[k] = before[k];
  }
  if (e != FM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return e;
  }
  if (ce != cudaSuccess || ce2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return fail(pr, FM_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
  }
  cudaError_t ci = cudaGraphInstantiate(&out->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ci != cudaSuccess) {
    out->exec = nullptr;
    return fail(pr, FM_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ci));
  }
  return FM_OK;
}

static void evict_lru(fm_problem* pr) {
  constexpr size_t kMaxGraphs = 16;
  if (pr->graphs.size() < kMaxGraphs) return;
  size_t lru = 0;
  for (size_t k = 1; k < pr->graphs.size(); ++k)
    if (pr->graphs[k].last_use < pr->graphs[lru].last_use) lru = k;
  if (pr->graphs[lru].exec) cudaGraphExecDestroy(pr->graphs[lru].exec);
  pr->graphs.erase(pr->graphs.begin() + lru);
}

// fm_loss_grad with host buffers as one graph: parameters in from the pinned
// staging buffer, the evaluation writing gradient and loss into pinned
// buffers, the error word out.  Replaying it costs one launch instead of one
// per copy and kernel.
static fm_status capture_loss_grad(fm_problem* pr, fm_stage st, size_t count, bool want_loss,
                                   bool want_grad, fm_problem::GraphEntry* out) {
  if (!pr->cap_stream) FM_CUDA(pr, cudaStreamCreateWithFlags(&pr->cap_stream, cudaStreamNonBlocking));
  int64_t before[fm::kKCount];
  std::memcpy(before, pr->k_launches, sizeof(before));
  cudaStream_t orig = pr->stream;
  pr->stream = pr->cap_stream;
  cudaStream_t s = pr->cap_stream;
  cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  fm_status e = FM_OK;
  const bool was = fm::g_capturing;
  fm::g_capturing = true;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(pr->scratch_params, pr->h_lg_in, sizeof(float) * count,
                                              cudaMemcpyHostToDevice, s);
  // the last kernel writes the gradient and the loss straight into the
  // pinned staging buffers (mapped into the device's address space), so no
  // copy node follows it for them; the 4-byte error word is copied
  if (ce == cudaSuccess)
    e = evaluate(pr, st, pr->scratch_params, want_grad ? pr->h_lg_grad : nullptr, nullptr, nullptr,
                 want_loss ? pr->h_loss : nullptr);
  if (ce == cudaSuccess && e == FM_OK)
    ce = cudaMemcpyAsync(pr->h_err, pr->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  fm::g_capturing = was;
  cudaGraph_t graph = nullptr;
  cudaError_t ce2 = cudaStreamEndCapture(s, &graph);
  pr->stream = orig;
  for (int k = 0; k < fm::kKCount; ++k) {
    out->counts[k] = pr->k_launches[k] - before[k];
    pr->k_launches[k] = before[k];
  }
  if (e != FM_OK || ce != cudaSuccess || ce2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (e != FM_OK) return e;
    return fail(pr, FM_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
  }
  cudaError_t ci = cudaGraphInstantiate(&out->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ci != cudaSuccess) {
    out->exec = nullptr;
    return fail(pr, FM_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ci));
  }
  return FM_OK;
}

static fm_status graph_for(fm_problem* pr, fm_stage st, const fm_adam_opts* opts, float* params,
                           fm::AdamState* adam, fm_problem::GraphEntry** g) {
  for (auto& e : pr->graphs)
    if (e.kind == 0 && e.stage == (int)st && e.lr == opts->lr && e.b1 == opts->beta1 && e.b2 == opts->beta2 &&
        e.eps == opts->eps && e.epoch == pr->graph_epoch && e.exec) {
      e.last_use = ++pr->graph_clock;
      *g = &e;
      return FM_OK;
    }
  evict_lru(pr);
  fm_problem::GraphEntry e;
  e.stage = (int)st;
  e.lr = opts->lr;
  e.b1 = opts->beta1;
  e.b2 = opts->beta2;
  e.eps = opts->eps;
  e.epoch = pr->graph_epoch;
  fm_status r = capture_graph(pr, st, opts, params, adam, &e);
  if (r != FM_OK) return r;
  e.last_use = ++pr->graph_clock;
  pr->graphs.push_back(e);
  *g = &pr->graphs.back();
  return FM_OK;
}

fm_status fm_step(fm_problem* pr, fm_stage st, const fm_adam_opts* opts, int32_t n_iters, float* loss) {
  fm::g_plain_once = true;
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!valid_stage(st)) return fail(pr, FM_ERR_INVALID_ARG, "unknown stage");
  if (!opts) return fail(pr, FM_ERR_INVALID_ARG, "opts is NULL");
  if (!(opts->lr > 0.f && opts->beta1 >= 0.f && opts->beta1 < 1.f && opts->beta2 >= 0.f &&
        opts->beta2 < 1.f && opts->eps >= 0.f))
    return fail(pr, FM_ERR_INVALID_ARG, "invalid Adam options");
  if (n_iters < 0) return fail(pr, FM_ERR_INVALID_ARG, "n_iters must be >= 0");
  StageBuf b = stage_buf(pr, st);
  if (!*b.set) return fail(pr, FM_ERR_STATE, "the stage's parameters have not been set");
  const int runs = (st == FM_STAGE_TRANSLATION) ? pr->trn_runs : 1;
  // graphs need no per-iteration host decisions: no per-kernel timing, no
  // loss trace; the first iteration runs directly (it settles the lazily
  // built state: W of the compact form, the translation targets)
  const bool graphs = pr->use_graphs && !pr->timing && pr->loss_every == 0;
  for (int it = 0; it < n_iters;) {
    const bool last = (it == n_iters - 1);
    const int left_for_graph = n_iters - it - (loss ? 1 : 0);
    if (graphs && it > 0 && left_for_graph >= kGraphIters) {
      fm_problem::GraphEntry* g = nullptr;
      fm_status e = graph_for(pr, st, opts, b.params, b.adam, &g);
      if (e != FM_OK) return e;
      e = replay(pr, g->exec);
      if (e != FM_OK) return e;
      for (int k = 0; k < fm::kKCount; ++k) pr->k_launches[k] += g->counts[k];
      pr->graph_replays += 1;
      it += kGraphIters;
      continue;
    }
    float* trace = nullptr;
    if (pr->loss_every > 0) {
      if (pr->iter_count % pr->loss_every == 0) {
        trace = pr->loss_hist + (size_t)(pr->loss_count % pr->loss_cap) * 64 * pr->S;
        pr->loss_count += 1;
      }
      pr->iter_count += 1;
    }
    fm_status e = evaluate(pr, st, b.params, nullptr, opts, b.adam, (last && loss) ? pr->d_loss : nullptr,
                           trace);
    if (e != FM_OK) return e;
    ++it;
  }
  if (st == FM_STAGE_ROTATION && n_iters > 0) pr->trn_target_valid = false;
  if (loss && n_iters > 0) {
    const size_t nl = (size_t)runs * pr->S;
    FM_CUDA(pr, cudaMemcpyAsync(pr->h_loss, pr->d_loss, sizeof(float) * nl, cudaMemcpyDeviceToHost, pr->stream));
    FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
    std::memcpy(loss, pr->h_loss, sizeof(float) * nl);
  }
  return FM_OK;
}

// ---- learned per-pair weights

fm_status fm_mlp_set_params(fm_problem* pr, const float* theta, int32_t on_device) {
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!theta) {
    dfree(pr->mlp_theta);
    return FM_OK;
  }
  if (!pr->mlp_theta) FM_ALLOC(pr, pr->mlp_theta, (size_t)fm::kMlpParams);
  FM_CUDA(pr, cudaMemcpyAsync(pr->mlp_theta, theta, sizeof(float) * fm::kMlpParams,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, pr->stream));
  fm::launch_check_finite(pr->mlp_theta, fm::kMlpParams, pr->d_err, fm::kErrParamNonFinite, pr->stream);
  FM_LAUNCHED(pr);
  return check_err_bits(pr);
}

// relative: E from the rotation stage and rel_t (params ignored)
static fm_status mlp_eval(fm_problem* pr, const float* params, float iter_frac, float delta, float* feat,
                          float* resid, float* prob, const float* w, bool relative = false) {
  if (relative) {
    if (!pr->rot_params_set) return fail(pr, FM_ERR_STATE, "the rotation-stage parameters have not been set");
    if (!pr->rel_t_set) return fail(pr, FM_ERR_STATE, "no relative translations (rel_t)");
    params = pr->rot_params;
  } else if (!params) {
    if (!pr->ea_params_set) return fail(pr, FM_ERR_STATE, "the epipolar-stage parameters have not been set");
    params = pr->ea_params;
  }
  if (prob && !pr->mlp_theta) return fail(pr, FM_ERR_STATE, "no network parameters (fm_mlp_set_params)");
  if (!(delta > 0.f) || !std::isfinite(delta)) return fail(pr, FM_ERR_INVALID_ARG, "delta must be finite and > 0");
  if (!(iter_frac >= 0.f && iter_frac <= 1.f)) return fail(pr, FM_ERR_INVALID_ARG, "iter_frac must lie in [0, 1]");
  if (!pr->mlp_tab) FM_ALLOC(pr, pr->mlp_tab, (size_t)32 * pr->P);
  cudaStream_t s = pr->stream;
  {
    Timed t(pr, fm::kKMlpTables);
    fm::launch_mlp_pair_tables(pr, params, relative ? pr->rel_t : nullptr, pr->mlp_tab, s);
  }
  FM_LAUNCHED(pr);
  {
    Timed t(pr, fm::kKMlpInfer);
    fm::launch_mlp_infer(pr, pr->mlp_tab, prob ? pr->mlp_theta : nullptr, w, iter_frac, delta, prob, nullptr,
                         feat, resid, s);
  }
  FM_LAUNCHED(pr);
  return prob ? check_err_bits(pr) : FM_OK;
}

fm_status fm_mlp_eval(fm_problem* pr, const float* params_dev, float iter_frac, float delta, float* feat_dev,
                      float* resid_dev, float* prob_dev) {
  if (!pr) return FM_ERR_INVALID_ARG;
  fm::g_plain_once = true;
  return mlp_eval(pr, params_dev, iter_frac, delta, feat_dev, resid_dev, prob_dev, pr->ea_w);
}

fm_status fm_mlp_eval_relative(fm_problem* pr, float iter_frac, float delta, float* feat_dev, float* resid_dev,
                               float* prob_dev) {
  if (!pr) return FM_ERR_INVALID_ARG;
  fm::g_plain_once = true;
  return mlp_eval(pr, nullptr, iter_frac, delta, feat_dev, resid_dev, prob_dev, pr->ea_w, true);
}

fm_status fm_mlp_prune(fm_problem* pr, float iter_frac, float delta, float p_min, int64_t* n_kept) {
  if (!pr) return FM_ERR_INVALID_ARG;
  fm::g_plain_once = true;
  if (!(p_min >= 0.f && p_min <= 1.f)) return fail(pr, FM_ERR_INVALID_ARG, "p_min must lie in [0, 1]");
  cudaStream_t s = pr->stream;
  pr->graph_epoch += 1;
  if (!pr->mlp_prob) FM_ALLOC(pr, pr->mlp_prob, (size_t)pr->Z);
  fm_status e = mlp_eval(pr, nullptr, iter_frac, delta, nullptr, nullptr, pr->mlp_prob, pr->ea_w, true);
  if (e != FM_OK) return e;
  if (!pr->ea_w) FM_ALLOC(pr, pr->ea_w, (size_t)pr->Z);
  fm::launch_mask_from_prob(pr->mlp_prob, pr->Z, p_min, pr->ea_w, s);
  FM_LAUNCHED(pr);
  pr->W_valid = false;
  FM_CUDA(pr, cudaMemsetAsync(pr->d_kept, 0, sizeof(unsigned long long) * pr->S, s));
  fm::launch_count_positive(pr, pr->ea_w, pr->d_kept, s);
  FM_LAUNCHED(pr);
  int64_t total = 0;
  e = normalisers_from_counts(pr, &total);
  if (e != FM_OK) return e;
  if (n_kept) *n_kept = total;
  return FM_OK;
}

fm_status fm_mlp_reweight(fm_problem* pr, float iter_frac, float delta, float p_min, int32_t irls,
                          int64_t* n_kept) {
  if (!pr) return FM_ERR_INVALID_ARG;
  fm::g_plain_once = true;
  if (!(p_min >= 0.f && p_min <= 1.f)) return fail(pr, FM_ERR_INVALID_ARG, "p_min must lie in [0, 1]");
  if (!pr->ea_params_set) return fail(pr, FM_ERR_STATE, "the epipolar-stage parameters have not been set");
  cudaStream_t s = pr->stream;
  pr->graph_epoch += 1;
  if (!pr->mlp_prob) FM_ALLOC(pr, pr->mlp_prob, (size_t)pr->Z);
  // probabilities from the features at the current poses and weights
  fm_status e = mlp_eval(pr, pr->ea_params, iter_frac, delta, nullptr, nullptr, pr->mlp_prob, pr->ea_w);
  if (e != FM_OK) return e;
  if (!pr->ea_w) FM_ALLOC(pr, pr->ea_w, (size_t)pr->Z);
  {
    Timed t(pr, fm::kKEaTables);
    fm::launch_ea_tables(pr->ea_params, pr->pair_i, pr->pair_j, pr->seg_off, pr->P, pr->seg_tab, nullptr, s);
  }
  FM_LAUNCHED(pr);
  FM_CUDA(pr, cudaMemsetAsync(pr->d_kept, 0, sizeof(unsigned long long) * pr->S, s));
  {
    Timed t(pr, fm::kKEaReweight);
    fm::launch_ea_reweight(pr, 0.f, delta, irls, pr->ea_w, pr->d_kept, s, pr->mlp_prob, p_min);
  }
  FM_LAUNCHED(pr);
  {
    Timed t(pr, fm::kKWBuild);
    fm::launch_w_build(pr, pr->ea_w, pr->W, s);
  }
  FM_LAUNCHED(pr);
  pr->W_valid = true;
  int64_t total = 0;
  e = normalisers_from_counts(pr, &total);
  if (e != FM_OK) return e;
  if (n_kept) *n_kept = total;
  return FM_OK;
}

fm_status fm_get_tuning(const fm_problem* pr, fm_tuning* out) {
  if (!pr || !out) return FM_ERR_INVALID_ARG;
  out->pairs_per_lane = pr->ea_U;
  out->ctas_per_sm = pr->ea_ctas_per_sm;
  out->us_per_eval = 0.f;
  return FM_OK;
}

fm_status fm_set_tuning(fm_problem* pr, const fm_tuning* t) {
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!t) return fail(pr, FM_ERR_INVALID_ARG, "tuning is NULL");
  if (!fm::ea_tile_built(t->pairs_per_lane))
    return fail(pr, FM_ERR_INVALID_ARG, "pairs_per_lane must be 11, 15 or 21 (the tiles built into the library)");
  if (t->ctas_per_sm < 0) return fail(pr, FM_ERR_INVALID_ARG, "ctas_per_sm >= 0 required");
  if (t->pairs_per_lane != pr->ea_U) {
    fm_status e = build_direct_tables(pr, t->pairs_per_lane);
    if (e != FM_OK) return e;
  }
  pr->ea_ctas_per_sm = t->ctas_per_sm;
  pr->graph_epoch += 1;
  return FM_OK;
}

// Times k_ea_direct (L1, the problem's weights) for every tile built into
// the library and every CTA count per SM, each launch after a flush of L2,
// and keeps the fastest (median of `repeats`).
fm_status fm_autotune(fm_problem* pr, int32_t repeats, fm_tuning* best_out) {
  if (!pr) return FM_ERR_INVALID_ARG;
  if (repeats < 1) return fail(pr, FM_ERR_INVALID_ARG, "repeats must be >= 1");
  cudaStream_t s = pr->stream;
  FM_CUDA(pr, cudaStreamSynchronize(s));
  // table entries E_n: the epipolar parameters if set, else generated ones
  const float* params = pr->ea_params;
  if (!pr->ea_params_set) {
    fm::launch_hash_fill(pr, pr->scratch_params, 3, 0x5EED5u, s);   // [N][9] values in [-1, 1)
    params = pr->scratch_params;
  }
  // each sample is one gradient evaluation of the direct L1 objective as
  // fm_step chains it (E tables, the streaming kernel, the per-camera pass
  // with the loss): the streaming kernel's configuration also decides how
  // the next launch overlaps its end (measured on the 5M-pair scene: equal
  // times of the streaming kernel alone, steps 29.5 to 37.3 us)
  const int old_loss = pr->ea_loss;
  const bool old_timing = pr->timing;
  pr->ea_loss = FM_EA_L1;
  pr->timing = false;
  // an L2-sized flush between timed launches (skipped if it cannot be allocated)
  void* flush = nullptr;
  const size_t flush_bytes = (size_t)256 << 20;
  if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
    cudaGetLastError();
    flush = nullptr;
  }
  const int old_u = pr->ea_U, old_c = pr->ea_ctas_per_sm;
  fm_tuning best{old_u, old_c, 3.4e38f};
  fm_status st = FM_OK;
  std::vector<cudaEvent_t> ev;
  for (int U : {15, 11, 21}) {
    if (pr->Z == 0) break;
    if (U != pr->ea_U && (st = build_direct_tables(pr, U)) != FM_OK) break;
    const int max_c = fm::direct_max_ctas_per_sm(pr);
    // round robin over the CTA counts, so that a slow drift of the device
    // (clocks, power) does not favour the first ones; every sample after an
    // L2 flush and a 0.2 ms device idle, no host synchronisation in between
    const size_t n_ev = 2 * (size_t)repeats * max_c;
    while (ev.size() < n_ev) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) break;
      ev.push_back(e);
    }
    if (ev.size() < n_ev) {
      cudaGetLastError();
      st = fail(pr, FM_ERR_CUDA, "autotune: events");
      break;
    }
    size_t q = 0;
    for (int k = 0; k < repeats; ++k)
      for (int c = 1; c <= max_c; ++c, q += 2) {
        pr->ea_ctas_per_sm = c;
        if (flush) fm::launch_l2_flush(flush, flush_bytes, k & 0xff, s);
        fm::launch_idle(200000u, s);
        cudaEventRecord(ev[q], s);
        fm::g_plain_once = true;
        if (st == FM_OK) st = evaluate(pr, FM_STAGE_EPIPOLAR, params, pr->scratch_grad, nullptr, nullptr, pr->d_loss);
        cudaEventRecord(ev[q + 1], s);
      }
    if (st != FM_OK) break;
    cudaError_t ce = cudaStreamSynchronize(s);
    // the mean over the samples of each CTA count: event timestamps come in
    // steps of about 2 us on this part, so minima tie; means resolve below that
    std::vector<float> fastest(max_c + 1, 0.f);
    q = 0;
    for (int k = 0; k < repeats && ce == cudaSuccess; ++k)
      for (int c = 1; c <= max_c && ce == cudaSuccess; ++c, q += 2) {
        float t = 0.f;
        ce = cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
        fastest[c] += 1000.f * t / (float)repeats;
      }
    if (ce != cudaSuccess) {
      st = fail(pr, FM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(ce));
      break;
    }
    for (int c = 1; c <= max_c; ++c)
      if (fastest[c] < best.us_per_eval) best = fm_tuning{U, c, fastest[c]};
  }
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
  if (flush) cudaFree(flush);
  pr->ea_loss = old_loss;
  pr->timing = old_timing;
  if (st == FM_OK) st = check_err_bits(pr);
  if (st == FM_OK && pr->Z > 0) st = fm_set_tuning(pr, &best);
  if (st != FM_OK) {   // leave the previous tile in place
    if (pr->ea_U != old_u) build_direct_tables(pr, old_u);
    pr->ea_ctas_per_sm = old_c;
    return st;
  }
  if (best_out) *best_out = best;
  return FM_OK;
}

fm_status fm_graphs_enable(fm_problem* pr, int32_t enable) {
  if (!pr) return FM_ERR_INVALID_ARG;
  pr->use_graphs = enable != 0;
  return FM_OK;
}

fm_status fm_rotation_init(fm_problem* pr, int32_t n_iters) {
  if (!pr) return FM_ERR_INVALID_ARG;
  if (n_iters < 1) return fail(pr, FM_ERR_INVALID_ARG, "n_iters must be >= 1");
  if (!pr->rel_R_set) return fail(pr, FM_ERR_STATE, "rotation initialisation needs relative rotations (rel_R)");
  cudaStream_t s = pr->stream;
  const int N = pr->N;
  float* x = pr->scratch_params;           // [3N]
  float* y = pr->scratch_params + 3 * N;   // [3N]
  float* c1 = pr->scratch_grad;            // [3N]
  // per scene: x^T A x = sum ||x_j - R_ij x_i||^2 <= 2 sum_i d_i ||x_i||^2, so
  // lambda_max(A) <= 2 d_max, and lambda_max(B) <= 2 (d_max/|P| + 1/|I|) for
  // B = A/|P| + diag(c1 c1^T)/|I|.  The shift sigma = 1.05 (d_max[/|P| + 1/|I|])
  // keeps every eigenvalue of I - A/sigma above 1 - 2/1.05 = -0.905, so the
  // top end decays too, while the wanted end converges twice as fast as with
  // sigma = 2 d_max (the gap to the first unwanted eigenvalue, divided by sigma)
  const int S = pr->S;
  std::vector<float> coef1(3 * (size_t)S), coef2(3 * (size_t)S);
  for (int q = 0; q < S; ++q) {
    const float Pq = (float)(pr->h_sc_pair_off[q + 1] - pr->h_sc_pair_off[q]);
    const float Nq = (float)(pr->h_sc_cam_off[q + 1] - pr->h_sc_cam_off[q]);
    const float dq = (float)std::max(pr->h_sc_max_degree[q], 1);
    const float sigma1 = 1.05f * dq;
    const float sigma2 = 1.05f * (dq / Pq + 1.f / Nq);
    coef1[3 * q] = 1.f / sigma1; coef1[3 * q + 1] = 1.f;      coef1[3 * q + 2] = 1.f / Nq;
    coef2[3 * q] = 1.f / sigma2; coef2[3 * q + 1] = 1.f / Pq; coef2[3 * q + 2] = 1.f / Nq;
  }
  for (int col = 0; col < 2; ++col) {
    FM_CUDA(pr, cudaMemcpyAsync(pr->mart_coef, (col == 0 ? coef1 : coef2).data(), sizeof(float) * 3 * S,
                                cudaMemcpyHostToDevice, s));
    FM_CUDA(pr, cudaStreamSynchronize(s));   // the host vector is reused
    fm::launch_hash_fill(pr, x, 1, col == 0 ? 0x1234567u : 0x89ABCDEu, s);
    fm::launch_scale_to_unit(pr, x, s);
    int it = 0;
    // blocks of 32 iterations (an even count: x and y swap back) followed by
    // the rescaling, replayed from one captured graph
    if (pr->use_graphs && !pr->timing && n_iters >= 64) {
      if (!pr->cap_stream) FM_CUDA(pr, cudaStreamCreateWithFlags(&pr->cap_stream, cudaStreamNonBlocking));
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      FM_CUDA(pr, cudaStreamBeginCapture(pr->cap_stream, cudaStreamCaptureModeThreadLocal));
      const bool was = fm::g_capturing;
      fm::g_capturing = true;   // (these launches are plain ones anyway)
      float* gx = x;
      float* gy = y;
      for (int k = 0; k < 32; ++k) {
        fm::launch_mart_iter(pr, gx, col == 0 ? nullptr : c1, gy, pr->cap_stream);
        std::swap(gx, gy);
      }
      fm::launch_scale_to_unit(pr, gx, pr->cap_stream);
      fm::g_capturing = was;
      cudaError_t ce = cudaStreamEndCapture(pr->cap_stream, &graph);
      if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        cudaGetLastError();
        return fail(pr, FM_ERR_CUDA, std::string("rotation-init graph: ") + cudaGetErrorString(ce));
      }
      for (; it + 32 <= n_iters; it += 32) {
        cudaError_t le = cudaGraphLaunch(exec, s);
        if (le != cudaSuccess) {
          cudaGraphExecDestroy(exec);
          return fail(pr, FM_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(le));
        }
        pr->k_launches[fm::kKMartIter] += 32;
      }
      FM_CUDA(pr, cudaStreamSynchronize(s));
      cudaGraphExecDestroy(exec);
    }
    for (; it < n_iters; ++it) {
      {
        Timed t(pr, fm::kKMartIter);
        fm::launch_mart_iter(pr, x, col == 0 ? nullptr : c1, y, s);
      }
      std::swap(x, y);
      if ((it & 31) == 31) fm::launch_scale_to_unit(pr, x, s);
    }
    FM_LAUNCHED(pr);
    if (col == 0) {
      fm::launch_normalise3(x, N, s);
      FM_CUDA(pr, cudaMemcpyAsync(c1, x, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, s));
    }
  }
  fm::launch_mart_finish(c1, x, N, pr->rot_params, s);
  FM_LAUNCHED(pr);
  fm_status e = reset_adam(pr, pr->rot_adam, 6 * (size_t)N);
  if (e != FM_OK) return e;
  pr->rot_params_set = true;
  pr->trn_target_valid = false;
  return FM_OK;
}

fm_status fm_relative_translations(fm_problem* pr, float* err_out, int32_t err_on_device) {
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!pr->rot_params_set) return fail(pr, FM_ERR_STATE, "the grid search needs rotation-stage parameters");
  float* err = nullptr;
  if (err_out) err = err_on_device ? err_out : pr->seg_loss;
  if (!pr->lattice0) {
    FM_ALLOC(pr, pr->lattice0, (size_t)fm::reltrans_lattice_points());
    fm::launch_reltrans_lattice(pr->lattice0, pr->stream);
    FM_LAUNCHED(pr);
  }
  {
    Timed t(pr, fm::kKRelTrans);
    fm::launch_reltrans(pr, pr->rot_params, pr->rel_t, err, pr->stream);
  }
  FM_LAUNCHED(pr);
  pr->rel_t_set = true;
  pr->trn_target_valid = false;
  if (err_out && !err_on_device) {
    FM_CUDA(pr, cudaMemcpyAsync(err_out, err, sizeof(float) * pr->P, cudaMemcpyDeviceToHost, pr->stream));
    FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  }
  return FM_OK;
}

fm_status fm_get_rel_poses(fm_problem* pr, float* rel_R, float* rel_t, int32_t out_on_device) {
  if (!pr) return FM_ERR_INVALID_ARG;
  const cudaMemcpyKind k = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (rel_R) {
    if (!pr->rel_R_set) return fail(pr, FM_ERR_STATE, "no relative rotations are set");
    FM_CUDA(pr, cudaMemcpyAsync(rel_R, pr->rel_R, sizeof(float) * 9 * pr->P, k, pr->stream));
  }
  if (rel_t) {
    if (!pr->rel_t_set) return fail(pr, FM_ERR_STATE, "no relative translations are set");
    FM_CUDA(pr, cudaMemcpyAsync(rel_t, pr->rel_t, sizeof(float) * 3 * pr->P, k, pr->stream));
  }
  if (!out_on_device) FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  return FM_OK;
}

fm_status fm_translation_random_init(fm_problem* pr, uint32_t seed) {
  if (!pr) return FM_ERR_INVALID_ARG;
  const size_t n = 3 * (size_t)pr->N * pr->trn_runs;
  fm::launch_hash_fill(pr, pr->trn_params, pr->trn_runs, seed, pr->stream);
  FM_LAUNCHED(pr);
  fm_status e = reset_adam(pr, pr->trn_adam, n);
  if (e != FM_OK) return e;
  pr->trn_params_set = true;
  return FM_OK;
}

fm_status fm_translation_merge(fm_problem* pr, int32_t* best_run_out) {
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!pr->trn_params_set) return fail(pr, FM_ERR_STATE, "the translation-stage parameters have not been set");
  fm_status e = ensure_targets(pr);
  if (e != FM_OK) return e;
  cudaStream_t s = pr->stream;
  const int N = pr->N, runs = pr->trn_runs;
  float* merged = pr->merge_buf;
  float* stats = pr->merge_buf + 3 * N;
  {
    Timed t(pr, fm::kKMerge);
    fm::launch_merge(pr, pr->trn_params, runs, stats, merged, pr->best_run, s);
  }
  FM_LAUNCHED(pr);
  if (best_run_out) {
    FM_CUDA(pr, cudaMemcpyAsync(best_run_out, pr->best_run, sizeof(int) * N, cudaMemcpyDeviceToHost, s));
  }
  FM_CUDA(pr, cudaStreamSynchronize(s));
  if (runs != 1) {
    e = resize_runs(pr, 1);
    if (e != FM_OK) return e;
  }
  FM_CUDA(pr, cudaMemcpyAsync(pr->trn_params, merged, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, s));
  e = reset_adam(pr, pr->trn_adam, 3 * (size_t)N);
  if (e != FM_OK) return e;
  pr->trn_params_set = true;
  FM_CUDA(pr, cudaStreamSynchronize(s));
  return FM_OK;
}

fm_status fm_epipolar_init_from_stages(fm_problem* pr) {
  if (!pr) return FM_ERR_INVALID_ARG;
  if (!pr->rot_params_set || !pr->trn_params_set)
    return fail(pr, FM_ERR_STATE, "needs rotation- and translation-stage parameters");
  if (pr->trn_runs != 1) return fail(pr, FM_ERR_STATE, "merge the translation runs first");
  fm::launch_ea_from_stages(pr->rot_params, pr->trn_params, pr->N, pr->ea_params, pr->stream);
  FM_LAUNCHED(pr);
  fm_status e = reset_adam(pr, pr->ea_adam, 9 * (size_t)pr->N);
  if (e != FM_OK) return e;
  pr->ea_params_set = true;
  pr->W_valid = false;
  return FM_OK;
}

fm_status fm_triangulate(fm_problem* pr, const fm_tri_opts* opts, float* points, int32_t* valid,
                         int32_t* n_inlier_cams, int32_t out_on_device, int32_t* n_tracks) {
  if (!pr || !opts) return FM_ERR_INVALID_ARG;
  if (!pr->track_idx) return fail(pr, FM_ERR_STATE, "triangulation needs kp_track at creation");
  if (!pr->ea_params_set) return fail(pr, FM_ERR_STATE, "the epipolar-stage parameters have not been set");
  const int T = pr->n_tracks;
  if (n_tracks) *n_tracks = T;
  if (T <= 0) return FM_OK;
  cudaStream_t s = pr->stream;
  float* d_pts = nullptr;
  int* d_valid = nullptr;
  int* d_ncam = nullptr;
  FM_ALLOC(pr, d_pts, 3 * (size_t)T);
  FM_ALLOC(pr, d_valid, (size_t)T);
  FM_ALLOC(pr, d_ncam, (size_t)T);
  {
    Timed t(pr, fm::kKTriangulate);
    fm::launch_triangulate(pr, pr->ea_params, opts->max_err_px, opts->min_angle_deg * 3.14159265358979f / 180.f,
                           d_pts, d_valid, d_ncam, s);
  }
  cudaError_t le = cudaGetLastError();
  const cudaMemcpyKind k = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (le == cudaSuccess && points) le = cudaMemcpyAsync(points, d_pts, sizeof(float) * 3 * T, k, s);
  if (le == cudaSuccess && valid) le = cudaMemcpyAsync(valid, d_valid, sizeof(int) * T, k, s);
  if (le == cudaSuccess && n_inlier_cams) le = cudaMemcpyAsync(n_inlier_cams, d_ncam, sizeof(int) * T, k, s);
  if (le == cudaSuccess) le = cudaStreamSynchronize(s);
  cudaFree(d_pts);
  cudaFree(d_valid);
  cudaFree(d_ncam);
  pr->device_bytes -= (int64_t)(sizeof(float) * 3 + 2 * sizeof(int)) * T;
  if (le != cudaSuccess) return fail(pr, FM_ERR_CUDA, std::string("triangulation: ") + cudaGetErrorString(le));
  return FM_OK;
}

void fm_solve_opts_default(fm_solve_opts* o) {
  if (!o) return;
  o->rot_given = 0;
  o->rot_init_iters = 2000;
  o->rot_iters = 2000;
  o->rot_lr = 1e-3f;
  o->reestimate_rel_t = 1;
  o->trn_runs = 4;
  o->trn_iters = 2000;
  o->trn_lr = 1e-2f;
  o->trn_final_iters = 1000;
  o->seed = 0;
  o->ea_rounds = 5;
  o->ea_iters = 500;
  o->ea_lr = 1e-4f;
  o->ea_tau0 = 0.05f;
  o->ea_tau_min = 0.005f;
  o->ea_delta = 1e-5f;
  o->tri_max_err_px = 4.f;
  o->tri_min_angle_deg = 2.f;
  o->beta1 = 0.9f;
  o->beta2 = 0.999f;
  o->eps = 1e-8f;
  o->learned = 0;
  o->learned_p_min = 0.5f;
  o->learned_prune_passes = 1;
}

// Adam steps in four equal phases with the learning rate scaled by
// 1, 0.3, 0.1, 0.03 (the moments carry over between phases)
static fm_status stepped(fm_problem* pr, fm_stage st, const fm_solve_opts* o, float lr, int iters, float* loss) {
  static const float kPhase[4] = {1.f, 0.3f, 0.1f, 0.03f};
  const int per = iters / 4;
  for (int ph = 0; ph < 4; ++ph) {
    const int n = (ph < 3) ? per : iters - 3 * per;
    fm_adam_opts a{lr * kPhase[ph], o->beta1, o->beta2, o->eps};
    fm_status e = fm_step(pr, st, &a, n, (ph == 3) ? loss : nullptr);
    if (e != FM_OK) return e;
  }
  return FM_OK;
}

namespace {

// The output gauge of fm_solve, per scene, applied to the epipolar-stage
// parameters themselves (so that the outputs and the triangulated points
// share it): the world frame is rotated so that the scene's first valid
// camera has R = I, then moved and scaled so that the valid cameras' centres
// have their centroid at the origin and unit mean norm.  With G = R_ref, mu
// and sigma the centroid and mean norm of G c_i: R_i' = R_i G^T and
// t_i' = (R_i' mu + t_i) / sigma, so that c_i' = (G c_i - mu) / sigma.
cudaError_t apply_output_gauge(fm_problem* pr) {
  const int N = pr->N;
  std::vector<float> P;
  cudaError_t ce = fetch(P, pr->ea_params, (size_t)9 * N, true);
  if (ce != cudaSuccess) return ce;
  auto rot = [&](int c, double R[9]) {   // 6D (two columns) -> R, Gram-Schmidt
    const float* a = &P[9 * (size_t)c];
    double b1[3] = {a[0], a[1], a[2]}, b2[3] = {a[3], a[4], a[5]};
    double n1 = std::sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2]);
    for (double& v : b1) v /= n1;
    const double d = b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2];
    for (int k = 0; k < 3; ++k) b2[k] -= d * b1[k];
    const double n2 = std::sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]);
    for (double& v : b2) v /= n2;
    const double b3[3] = {b1[1] * b2[2] - b1[2] * b2[1], b1[2] * b2[0] - b1[0] * b2[2], b1[0] * b2[1] - b1[1] * b2[0]};
    for (int r = 0; r < 3; ++r) {
      R[3 * r] = b1[r];
      R[3 * r + 1] = b2[r];
      R[3 * r + 2] = b3[r];
    }
  };
  for (int q = 0; q < pr->S; ++q) {
    const int b = pr->h_sc_cam_off[q], e = pr->h_sc_cam_off[q + 1];
    int ref = -1;
    for (int c = b; c < e && ref < 0; ++c)
      if (pr->h_cam_valid[c]) ref = c;
    if (ref < 0) continue;
    double G[9];
    rot(ref, G);
    // centres G c_i of the valid cameras, c_i = -R_i^T t_i
    std::vector<double> gc(3 * (size_t)(e - b), 0.0);
    double mu[3] = {0, 0, 0};
    int nv = 0;
    for (int c = b; c < e; ++c) {
      double R[9];
      rot(c, R);
      const float* t = &P[9 * (size_t)c + 6];
      double ci[3];
      for (int k = 0; k < 3; ++k) ci[k] = -(R[k] * t[0] + R[3 + k] * t[1] + R[6 + k] * t[2]);
      for (int r = 0; r < 3; ++r) gc[3 * (c - b) + r] = G[3 * r] * ci[0] + G[3 * r + 1] * ci[1] + G[3 * r + 2] * ci[2];
      if (pr->h_cam_valid[c]) {
        for (int r = 0; r < 3; ++r) mu[r] += gc[3 * (c - b) + r];
        ++nv;
      }
    }
    for (double& v : mu) v /= nv;
    double sigma = 0.0;
    for (int c = b; c < e; ++c)
      if (pr->h_cam_valid[c]) {
        const double* g = &gc[3 * (c - b)];
        sigma += std::sqrt((g[0] - mu[0]) * (g[0] - mu[0]) + (g[1] - mu[1]) * (g[1] - mu[1]) +
                           (g[2] - mu[2]) * (g[2] - mu[2]));
      }
    sigma /= nv;
    if (!(sigma > 1e-30)) sigma = 1.0;   // one valid camera: no scale to fix
    for (int c = b; c < e; ++c) {
      double R[9], Rn[9];
      rot(c, R);
      for (int r = 0; r < 3; ++r)   // R' = R G^T
        for (int k = 0; k < 3; ++k) Rn[3 * r + k] = R[3 * r] * G[3 * k] + R[3 * r + 1] * G[3 * k + 1] + R[3 * r + 2] * G[3 * k + 2];
      float* a = &P[9 * (size_t)c];
      double tn[3];
      for (int r = 0; r < 3; ++r) tn[r] = (Rn[3 * r] * mu[0] + Rn[3 * r + 1] * mu[1] + Rn[3 * r + 2] * mu[2] + a[6 + r]) / sigma;
      for (int r = 0; r < 3; ++r) {
        a[r] = (float)Rn[3 * r];
        a[3 + r] = (float)Rn[3 * r + 1];
        a[6 + r] = (float)tn[r];
      }
    }
  }
  ce = cudaMemcpyAsync(pr->ea_params, P.data(), sizeof(float) * 9 * N, cudaMemcpyHostToDevice, pr->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(pr->stream);
  return ce;
}

}  // namespace

fm_status fm_solve(fm_problem* pr, const fm_solve_opts* o, fm_result* res) {
  if (!pr || !o || !res) return FM_ERR_INVALID_ARG;
  if (!res->R || !res->t) return fail(pr, FM_ERR_INVALID_ARG, "result R and t buffers are required");
  if (o->trn_runs < 1 || o->trn_runs > 64 || o->ea_rounds < 0 || o->rot_init_iters < 1)
    return fail(pr, FM_ERR_INVALID_ARG, "invalid solve options");
  if (o->learned && !pr->mlp_theta)
    return fail(pr, FM_ERR_STATE, "learned filtering needs the network parameters (fm_mlp_set_params)");
  fm_status e;
  // every solve starts from unit weights (a previous solve leaves its own)
  if ((e = fm_ea_set_weights(pr, nullptr, 0, 0.f)) != FM_OK) return e;
  // per-scene losses; the result reports their sum
  std::vector<float> Lv(pr->S);
  auto total = [&]() {
    float t = 0.f;
    for (float v : Lv) t += v;
    return t;
  };
  // divergence: a stage whose final loss is not finite ends the solve
  auto finite = [&](const std::vector<float>& L, const char* stage) -> fm_status {
    for (size_t k = 0; k < L.size(); ++k)
      if (!std::isfinite(L[k]))
        return fail(pr, FM_ERR_NAN, std::string(stage) + " stage diverged: its final loss is not finite (scene " +
                                        std::to_string(k % pr->S) + ")");
    return FM_OK;
  };
  if (o->rot_given) {
    // rotations given (e.g. aligned on another problem's raw matches)
    if (!pr->rot_params_set)
      return fail(pr, FM_ERR_STATE, "rot_given needs the rotation-stage parameters (fm_set_params)");
    if (!o->reestimate_rel_t && !pr->rel_t_set)
      return fail(pr, FM_ERR_STATE, "rot_given needs reestimate_rel_t or rel_t");
    res->loss_rotation = NAN;
  } else {
    // 0. relative poses from the keypoints when none were given
    if (!pr->rel_R_set && (e = fm_relative_poses(pr, 0, o->ea_delta, nullptr)) != FM_OK) return e;
    // 1-2. rotations
    if ((e = fm_rotation_init(pr, o->rot_init_iters)) != FM_OK) return e;
    if ((e = stepped(pr, FM_STAGE_ROTATION, o, o->rot_lr, o->rot_iters, Lv.data())) != FM_OK) return e;
    if ((e = finite(Lv, "rotation")) != FM_OK) return e;
    res->loss_rotation = total();
  }
  // 3. relative translations
  if (o->reestimate_rel_t) {
    if ((e = fm_relative_translations(pr, nullptr, 0)) != FM_OK) return e;
  } else if (!pr->rel_t_set) {
    return fail(pr, FM_ERR_STATE, "rel_t is needed when reestimate_rel_t is 0");
  }
  if (o->learned) {   // early pruning, then the relative translations of the kept pairs
    for (int pass = 0; pass < std::max(o->learned_prune_passes, 1); ++pass) {
      if ((e = fm_mlp_prune(pr, 0.f, o->ea_delta, o->learned_p_min, nullptr)) != FM_OK) return e;
      if (o->reestimate_rel_t && (e = fm_relative_translations(pr, nullptr, 0)) != FM_OK) return e;
    }
  }
  // 4. translation runs, merge, final run
  if ((e = fm_translation_set_runs(pr, o->trn_runs)) != FM_OK) return e;
  if ((e = fm_translation_random_init(pr, o->seed)) != FM_OK) return e;
  std::vector<float> run_loss((size_t)o->trn_runs * pr->S);
  if ((e = stepped(pr, FM_STAGE_TRANSLATION, o, o->trn_lr, o->trn_iters, run_loss.data())) != FM_OK) return e;
  if ((e = fm_translation_merge(pr, nullptr)) != FM_OK) return e;
  if ((e = stepped(pr, FM_STAGE_TRANSLATION, o, o->trn_lr, o->trn_final_iters, Lv.data())) != FM_OK) return e;
  if ((e = finite(Lv, "translation")) != FM_OK) return e;
  res->loss_translation = total();
  // 5. epipolar adjustment: IRLS / filtering rounds on the compact form
  if ((e = fm_epipolar_init_from_stages(pr)) != FM_OK) return e;
  if ((e = fm_ea_set_loss(pr, FM_EA_COMPACT)) != FM_OK) return e;
  res->loss_epipolar = 0.f;
  res->n_kept = pr->Z;
  for (int k = 0; k < o->ea_rounds; ++k) {
    const float tau = std::max(o->ea_tau0 * std::pow(0.5f, (float)k), o->ea_tau_min);
    int64_t kept = 0;
    if (o->learned)
      e = fm_mlp_reweight(pr, (float)(k + 1) / (float)(o->ea_rounds + 1), o->ea_delta, o->learned_p_min, 1,
                          &kept);
    else
      e = fm_ea_reweight(pr, tau, o->ea_delta, 1, &kept);
    if (e != FM_OK) return e;
    res->n_kept = kept;
    if ((e = stepped(pr, FM_STAGE_EPIPOLAR, o, o->ea_lr, o->ea_iters, Lv.data())) != FM_OK) return e;
    if ((e = finite(Lv, "epipolar")) != FM_OK) return e;
    res->loss_epipolar = total();
  }
  // outputs, in the output gauge
  FM_CUDA(pr, apply_output_gauge(pr));
  float* dR = pr->scratch_params;     // [9N]
  float* dt = pr->scratch_grad;       // [3N]
  fm::launch_ea_to_Rt(pr->ea_params, pr->N, dR, dt, pr->stream);
  FM_LAUNCHED(pr);
  FM_CUDA(pr, cudaMemcpyAsync(res->R, dR, sizeof(float) * 9 * pr->N, cudaMemcpyDeviceToHost, pr->stream));
  FM_CUDA(pr, cudaMemcpyAsync(res->t, dt, sizeof(float) * 3 * pr->N, cudaMemcpyDeviceToHost, pr->stream));
  FM_CUDA(pr, cudaMemcpyAsync(pr->h_err, pr->d_err, sizeof(int), cudaMemcpyDeviceToHost, pr->stream));
  FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  if (*pr->h_err) return check_err_bits(pr);
  for (int64_t k = 0; k < 9 * (int64_t)pr->N; ++k)
    if (!std::isfinite(res->R[k]) || (k < 3 * (int64_t)pr->N && !std::isfinite(res->t[k])))
      return fail(pr, FM_ERR_NAN, "the solved poses are not finite (the last update diverged)");
  if (res->cam_valid)
    for (int c = 0; c < pr->N; ++c) res->cam_valid[c] = pr->h_cam_valid[c];
  res->n_tracks = 0;
  res->n_points_valid = 0;
  if (pr->track_idx && (res->points || res->point_valid)) {
    fm_tri_opts to{o->tri_max_err_px, o->tri_min_angle_deg};
    int32_t T = 0;
    if ((e = fm_triangulate(pr, &to, res->points, res->point_valid, nullptr, 0, &T)) != FM_OK) return e;
    res->n_tracks = T;
    if (res->point_valid)
      for (int k = 0; k < T; ++k) res->n_points_valid += res->point_valid[k] != 0;
  }
  return FM_OK;
}

fm_status fm_timing_enable(fm_problem* pr, int32_t enable) {
  if (!pr) return FM_ERR_INVALID_ARG;
  drain_timing(pr, false);
  for (int k = 0; k < fm::kKCount; ++k) {
    pr->k_ms[k] = 0.0;
    pr->k_launches[k] = 0;
  }
  pr->timing = enable != 0;
  return FM_OK;
}

fm_status fm_timing_read(fm_problem* pr, fm_kernel_time* out, int32_t capacity, int32_t* count) {
  if (!pr || !count || (capacity > 0 && !out)) return FM_ERR_INVALID_ARG;
  drain_timing(pr, true);
  FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  int n = 0;
  for (int k = 0; k < fm::kKCount; ++k) {
    if (pr->k_launches[k] == 0) continue;
    if (n < capacity) {
      std::memset(out[n].name, 0, sizeof(out[n].name));
      std::strncpy(out[n].name, fm::kKernelNames[k], sizeof(out[n].name) - 1);
      out[n].launches = pr->k_launches[k];
      out[n].total_ms = pr->timing ? pr->k_ms[k] : 0.0;
    }
    ++n;
  }
  *count = n;
  return FM_OK;
}

fm_status fm_track_loss(fm_problem* pr, int32_t every, int32_t capacity) {
  if (!pr) return FM_ERR_INVALID_ARG;
  if (every < 0 || (every > 0 && capacity < 1)) return fail(pr, FM_ERR_INVALID_ARG, "every >= 0 and capacity >= 1 required");
  FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  dfree(pr->loss_hist);
  pr->loss_every = 0;
  pr->loss_cap = 0;
  pr->loss_count = 0;
  pr->iter_count = 0;
  if (every == 0) return FM_OK;
  FM_ALLOC(pr, pr->loss_hist, (size_t)capacity * 64 * pr->S);
  pr->loss_every = every;
  pr->loss_cap = capacity;
  return FM_OK;
}

fm_status fm_loss_history(fm_problem* pr, float* out, int32_t capacity, int32_t* count) {
  if (!pr || !count || (capacity > 0 && !out)) return FM_ERR_INVALID_ARG;
  if (pr->loss_every == 0) {
    *count = 0;
    return FM_OK;
  }
  const int64_t have = std::min<int64_t>(pr->loss_count, pr->loss_cap);
  const int64_t n = std::min<int64_t>(have, capacity);
  std::vector<float> ring((size_t)pr->loss_cap * 64 * pr->S);
  FM_CUDA(pr, cudaMemcpyAsync(ring.data(), pr->loss_hist, sizeof(float) * ring.size(),
                              cudaMemcpyDeviceToHost, pr->stream));
  FM_CUDA(pr, cudaStreamSynchronize(pr->stream));
  for (int64_t k = 0; k < n; ++k) {
    const int64_t idx = pr->loss_count - n + k;
    out[k] = ring[(size_t)(idx % pr->loss_cap) * 64 * pr->S];   // scene 0 (run 0 of the translation stage)
  }
  *count = (int32_t)n;
  return FM_OK;
}


// ---- network trainer (no problem needed)

struct fm_mlp_trainer {
  cudaStream_t stream = nullptr;
  int64_t max_batch = 0;
  int step = 0;
  int sm_count = 0;
  int* err = nullptr;   // device error bits of the tensor-core kernels
  float* theta = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  float* loss = nullptr;
  float* partial = nullptr;
};

static fm_status trainer_fail(fm_status st, const std::string& msg) {
  fm::set_thread_error(msg);
  return st;
}

static void trainer_free(fm_mlp_trainer* t) {
  if (!t) return;
  for (float* p : {t->theta, t->m, t->v, t->grad, t->loss, t->partial})
    if (p) cudaFree(p);
  if (t->err) cudaFree(t->err);
}

fm_status fm_mlp_trainer_create(int64_t max_batch, void* cuda_stream, fm_mlp_trainer** out) {
  if (!out) return trainer_fail(FM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (max_batch < 1 || max_batch > (int64_t(1) << 31))
    return trainer_fail(FM_ERR_INVALID_ARG, "max_batch must be in [1, 2^31]");
  fm_mlp_trainer* t = new (std::nothrow) fm_mlp_trainer();
  if (!t) return trainer_fail(FM_ERR_OOM, "host allocation failed");
  t->stream = (cudaStream_t)cuda_stream;
  t->max_batch = max_batch;
  const size_t n = fm::kMlpParams;
  const size_t parts = (size_t)fm::mlp_grad_parts(max_batch) * fm::mlp_part_stride();
  cudaError_t e = cudaSuccess;
  for (auto pp : {&t->theta, &t->m, &t->v, &t->grad})
    if (e == cudaSuccess) e = cudaMalloc((void**)pp, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&t->loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&t->partial, sizeof(float) * parts);
  if (e == cudaSuccess) e = cudaMalloc((void**)&t->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(t->err, 0, sizeof(int), t->stream);
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->theta, 0, sizeof(float) * n, t->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->m, 0, sizeof(float) * n, t->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->v, 0, sizeof(float) * n, t->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    trainer_free(t);
    delete t;
    return trainer_fail(e == cudaErrorMemoryAllocation ? FM_ERR_OOM : FM_ERR_CUDA,
                        std::string("trainer: ") + cudaGetErrorString(e));
  }
  *out = t;
  return FM_OK;
}

void fm_mlp_trainer_destroy(fm_mlp_trainer* t) {
  if (!t) return;
  cudaStreamSynchronize(t->stream);
  trainer_free(t);
  delete t;
}

fm_status fm_mlp_trainer_set_params(fm_mlp_trainer* t, const float* theta, int32_t on_device) {
  if (!t || !theta) return trainer_fail(FM_ERR_INVALID_ARG, "trainer and theta are required");
  const size_t n = sizeof(float) * fm::kMlpParams;
  cudaError_t e = cudaMemcpyAsync(t->theta, theta, n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  t->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->m, 0, n, t->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->v, 0, n, t->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) return trainer_fail(FM_ERR_CUDA, std::string("trainer: ") + cudaGetErrorString(e));
  t->step = 0;
  return FM_OK;
}

fm_status fm_mlp_trainer_get_params(fm_mlp_trainer* t, float* theta, int32_t on_device) {
  if (!t || !theta) return trainer_fail(FM_ERR_INVALID_ARG, "trainer and theta are required");
  cudaError_t e = cudaMemcpyAsync(theta, t->theta, sizeof(float) * fm::kMlpParams,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, t->stream);
  if (on_device) {
    if (e != cudaSuccess) return trainer_fail(FM_ERR_CUDA, std::string("trainer: ") + cudaGetErrorString(e));
    return FM_OK;
  }
  int bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, t->err, sizeof(int), cudaMemcpyDeviceToHost, t->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) return trainer_fail(FM_ERR_CUDA, std::string("trainer: ") + cudaGetErrorString(e));
  if (bits & fm::kErrMlpTimeout) {
    cudaMemsetAsync(t->err, 0, sizeof(int), t->stream);
    return trainer_fail(FM_ERR_TIMEOUT, "a bounded wait of the tensor-core network kernel ran out");
  }
  return FM_OK;
}

static fm_status trainer_check_batch(fm_mlp_trainer* t, const float* x, int64_t B) {
  if (!t) return trainer_fail(FM_ERR_INVALID_ARG, "trainer is NULL");
  if (B < 0 || B > t->max_batch) return trainer_fail(FM_ERR_INVALID_ARG, "batch size outside [0, max_batch]");
  if (B > 0 && !x) return trainer_fail(FM_ERR_INVALID_ARG, "x_dev is NULL");
  return FM_OK;
}

fm_status fm_mlp_trainer_loss_grad(fm_mlp_trainer* t, const float* x, const float* y, int64_t B, float* loss_dev,
                                   float* grad_dev) {
  fm_status st = trainer_check_batch(t, x, B);
  if (st != FM_OK) return st;
  if (B > 0 && !y) return trainer_fail(FM_ERR_INVALID_ARG, "y_dev is NULL");
  fm::launch_mlp_grad(t->theta, x, y, B, t->partial, grad_dev, loss_dev, t->err, t->stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return trainer_fail(FM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return FM_OK;
}

fm_status fm_mlp_trainer_step(fm_mlp_trainer* t, const float* x, const float* y, int64_t B, const fm_adam_opts* o,
                              float* loss_dev) {
  fm_status st = trainer_check_batch(t, x, B);
  if (st != FM_OK) return st;
  if (B > 0 && !y) return trainer_fail(FM_ERR_INVALID_ARG, "y_dev is NULL");
  if (!o || !(o->lr > 0.f && o->beta1 >= 0.f && o->beta1 < 1.f && o->beta2 >= 0.f && o->beta2 < 1.f && o->eps >= 0.f))
    return trainer_fail(FM_ERR_INVALID_ARG, "invalid Adam options");
  fm::launch_mlp_grad(t->theta, x, y, B, t->partial, t->grad, loss_dev ? loss_dev : t->loss, t->err, t->stream);
  t->step += 1;
  fm::launch_mlp_adam(t->theta, t->grad, t->m, t->v, t->step, o->lr, o->beta1, o->beta2, o->eps, t->stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return trainer_fail(FM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return FM_OK;
}

fm_status fm_mlp_trainer_forward(fm_mlp_trainer* t, const float* x, int64_t B, float* logit_dev) {
  fm_status st = trainer_check_batch(t, x, B);
  if (st != FM_OK) return st;
  if (B > 0 && !logit_dev) return trainer_fail(FM_ERR_INVALID_ARG, "logit_dev is NULL");
  fm::launch_mlp_forward_tc(t->theta, x, B, logit_dev, t->err, t->sm_count, t->stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return trainer_fail(FM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  int bits = 0;
  e = cudaMemcpyAsync(&bits, t->err, sizeof(int), cudaMemcpyDeviceToHost, t->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) return trainer_fail(FM_ERR_CUDA, std::string("trainer: ") + cudaGetErrorString(e));
  if (bits & fm::kErrMlpTimeout) {
    cudaMemsetAsync(t->err, 0, sizeof(int), t->stream);
    return trainer_fail(FM_ERR_TIMEOUT, "a bounded wait of the tensor-core network kernel ran out");
  }
  return FM_OK;
}

}  // extern "C"
