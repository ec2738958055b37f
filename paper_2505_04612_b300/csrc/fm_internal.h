// Internal declarations shared by the host runtime and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/fastmap.h"

namespace fm {

// ---------------------------------------------------------------- constants
// tile of the direct epipolar kernel (overridable at build time for tuning)
#ifndef FM_EA_PAIRS_PER_LANE
#define FM_EA_PAIRS_PER_LANE 15
#endif
#ifndef FM_EA_WARPS_PER_CTA
#define FM_EA_WARPS_PER_CTA 4
#endif
constexpr int kEaPairsPerLane = FM_EA_PAIRS_PER_LANE;  // U: keypoint pairs per lane at most (odd)
// the tiles U built into k_ea_direct (odd: stride-U float4 reads from shared
// memory are free of bank conflicts)
inline bool ea_tile_built(int U) { return U == 11 || U == 15 || U == 21; }
// lane descriptor of k_ea_direct: offset | count << 10 | key << 15
constexpr int kDescCntShift = 10, kDescKeyShift = 15;
constexpr int kEaWarpsPerCta = FM_EA_WARPS_PER_CTA;
// shared-memory stages of k_ea_direct per warp (warp runs in flight + 1)
#ifndef FM_EA_STAGES
#define FM_EA_STAGES 2
#endif
constexpr int kEaStages = FM_EA_STAGES;
// register budget of k_ea_direct: at least this many CTAs per SM, i.e. 128
// registers a thread at four warps per CTA (room to interleave a lane's
// pairs); at 11 pairs per lane 4 CTAs are resident, 16 warps per SM, as many
// as 8 CTAs of two warps, in half as many CTAs to start
#ifndef FM_EA_MIN_CTAS
#define FM_EA_MIN_CTAS 4
#endif
constexpr int kEaMinCtas = FM_EA_MIN_CTAS;

// learned per-pair inlier weights (fm_mlp.cu)
constexpr int kMlpParams = 4801;   // W1 [8][64], b1, W2 [64][64], b2, w3, b3
constexpr int kMlpFeatures = 8;
static_assert(kEaPairsPerLane % 2 == 1, "lane-contiguous shared-memory reads need an odd stride");
constexpr int kSegGradEa = 24;                   // dR_i, dt_i, dR_j, dt_j
constexpr int kSegGradRot = 24;                  // dR_i, dR_j: 9 floats each in a 48-byte slot
constexpr int kSegGradTrn = 8;                   // do_i, do_j: 3 floats each in a 16-byte slot
// the per-image-pair gradient buffer holds max(kSegGradEa P, kSegGradTrn P runs) floats
static_assert(kSegGradRot <= kSegGradEa, "rotation parts must fit the epipolar stage's buffer");

// error bits raised by device-side validation
enum : int {
  kErrKpOrder = 1,       // kp_img_pair decreasing
  kErrKpRange = 2,       // kp_img_pair outside [0, P)
  kErrKpNonFinite = 4,   // keypoint not finite
  kErrParamNonFinite = 8,
  kErrMlpTimeout = 16,   // a bounded wait of the tensor-core network kernel ran out
  kErrEaTimeout = 32,    // a bounded wait of the direct epipolar kernel ran out
  kErrSegOff = 64,       // keypoint-pair offsets not a valid CSR table (allocation-free entry)
};

enum KernelId : int {
  kKCalibrate = 0, kKSegOffsets, kKRunTables, kKEaTables, kKEaDirect, kKEaSegments,
  kKRotPairs, kKTrnTargets, kKTrnPairs, kKCamUpdate, kKLossSum, kKEaReweight, kKWBuild,
  kKEaCompact, kKMartIter, kKRelTrans, kKMerge, kKTriangulate, kKEaDirectLoss, kKEaDirectCoef, kKMlpTables, kKMlpInfer,
  kKRelpose, kKFocalVote, kKDistErrors, kKDistReduce, kKCamEa, kKCount
};
extern const char* const kKernelNames[kKCount];

struct PendingTiming {
  int kid;
  cudaEvent_t start, stop;
};

struct AdamState {
  float* m = nullptr;
  float* v = nullptr;
  int* t = nullptr;      // device step counter (incremented on the device)
};

}  // namespace fm

struct fm_problem {
  int N = 0, P = 0;
  int64_t Z = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sm_count = 0;
  std::string last_error;
  int64_t device_bytes = 0;

  // scenes: a problem may hold S independent scenes, cameras and image pairs
  // grouped by scene; every loss is per scene (normalised within its scene)
  int S = 1;
  std::vector<int> h_sc_cam_off;   // [S+1]
  std::vector<int> h_sc_pair_off;  // [S+1]
  std::vector<int64_t> h_sc_kp_off;  // [S+1]
  std::vector<int> h_sc_max_degree;  // [S]
  std::vector<int> h_cam_valid;      // [N] 1: in the largest connected component of its scene
  int* sc_cam_off = nullptr;     // [S+1]
  int* sc_pair_off = nullptr;    // [S+1]
  int64_t* sc_kp_off = nullptr;  // [S+1] keypoint-pair range of each scene
  int* cam_scene = nullptr;      // [N]
  int* pair_scene = nullptr;     // [P]
  float* pair_inv_p = nullptr;   // [P] 1/P_s: normaliser of the rotation and translation losses
  float* pair_inv_z = nullptr;   // [P] normaliser of the epipolar loss of the pair's scene
  float* mart_coef = nullptr;    // [3S] per-scene constants of the rotation initialisation
  float4* lattice0 = nullptr;    // [4096] hemisphere candidates of the relative-translation search
  int* cam_pos = nullptr;        // [2P] camera-CSR index of (image pair n, role i / j)
  float* param_snap = nullptr;   // [9N] epipolar parameters at the start of a direct Adam step

  // image-pair graph
  int* pair_i = nullptr;         // [P]
  int* pair_j = nullptr;         // [P]
  int* seg_off = nullptr;        // [P+1] keypoint-pair offsets of each image pair
  int* cam_seg_off = nullptr;    // [N+1]
  int* cam_seg = nullptr;        // [2P] image pair | role << 31 (role 1: camera is j)
  int n_empty = 0;
  int max_degree = 0;            // largest number of image pairs of one camera
  float* merge_buf = nullptr;    // [3N + 4*64*S] merged centres and per-(run, scene) statistics
  int* best_run = nullptr;       // [N]

  // keypoints
  float4* kp = nullptr;          // [Z] calibrated (x1, y1, x2, y2)
  uint32_t* kp_perm = nullptr;   // [Z] input index of each internal position, or null (input order kept)
  int* kp_track = nullptr;       // [Z] or null
  int* kp_seg = nullptr;         // [Z] image pair of each keypoint pair (kept with tracks)
  int n_tracks = 0;
  int* track_off = nullptr;      // [T+1] keypoint pairs grouped by track
  int* track_idx = nullptr;      // [Z]
  float* focal = nullptr;
  float* cx = nullptr;
  float* cy = nullptr;

  // direct epipolar kernel: tile (chosen by fm_autotune or fm_set_tuning) and tables
  int ea_U = fm::kEaPairsPerLane;  // keypoint pairs per lane at most (a tile built into the library)
  int ea_ctas_per_sm = 0;        // persistent CTAs per SM (0: as many as fit)
  int n_wruns = 0;               // warp runs of 32 lanes
  int* lane_desc = nullptr;      // [n_wruns*32] offset | count << 10 | key << 15 of each lane
  int4* wrun_info = nullptr;     // [n_wruns] {first image pair, n_img | len << 8, record base, first pair}
  int* seg_rec = nullptr;        // [2P] {first record, #records} per image pair
  int64_t n_rec = 0;
  float4* rec = nullptr;         // [n_rec*3] per-(warp run, image pair) partial sums
  float4* seg_tab = nullptr;     // [P*3] E (9) + end offset per image pair

  // per image pair outputs of the segment pass
  float* seg_grad = nullptr;     // [max(m,1)*P*24]
  float* seg_loss = nullptr;     // [max(m,1)*P]

  // epipolar stage
  int ea_loss = FM_EA_L1;
  float* ea_w = nullptr;         // [Z] weights or null
  float ea_inv_z = 0.f;
  float* W = nullptr;            // [P*45] packed upper triangle of W_n (Eq. 17)
  bool W_valid = false;
  unsigned long long* d_kept = nullptr;  // [S] kept keypoint pairs per scene
  float* ea_params = nullptr;    // [N*9]
  fm::AdamState ea_adam;
  bool ea_params_set = false;

  // rotation stage
  float* rel_R = nullptr;        // [P*9]
  float* rel_t = nullptr;        // [P*3]
  bool rel_R_set = false;
  bool rel_t_set = false;
  float* rot_params = nullptr;   // [N*6]
  fm::AdamState rot_adam;
  bool rot_params_set = false;

  // translation stage
  int trn_runs = 1;
  float* trn_target = nullptr;   // [P*3] o^{i->j}
  bool trn_target_valid = false;
  float* trn_params = nullptr;   // [m*N*3]
  fm::AdamState trn_adam;
  bool trn_params_set = false;

  // learned weights
  float* mlp_theta = nullptr;    // [kMlpParams] network parameters, or null
  float* mlp_tab = nullptr;      // [P][32] per-image-pair feature table
  float* mlp_prob = nullptr;     // [Z] inlier probabilities of the last evaluation

  // observability
  bool timing = false;
  std::vector<fm::PendingTiming> pending;
  std::vector<cudaEvent_t> event_pool;
  int64_t k_launches[fm::kKCount] = {};
  double k_ms[fm::kKCount] = {};
  int loss_every = 0;
  int loss_cap = 0;
  int64_t loss_count = 0;     // traced values written so far
  int64_t iter_count = 0;     // fm_step iterations while tracing
  float* loss_hist = nullptr; // [loss_cap * 64 * S]: one row of [m][S] losses per traced iteration

  // captured iteration graphs of fm_step (see fm_api.cu)
  struct GraphEntry {
    int stage = 0;
    int kind = 0;                 // 0: 16 Adam iterations (fm_step); 1: fm_loss_grad with host buffers
    int flags = 0;                // kind 1: 1 loss, 2 gradient
    float lr = 0.f, b1 = 0.f, b2 = 0.f, eps = 0.f;
    uint64_t epoch = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t counts[fm::kKCount] = {};   // kernel launches of one replay
    uint64_t last_use = 0;
  };
  std::vector<GraphEntry> graphs;
  uint64_t graph_epoch = 1;      // bumped whenever captured launch arguments may change
  uint64_t graph_clock = 0;
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t aux_stream = nullptr;   // second stream of the distortion scoring (created on first use)
  cudaEvent_t aux_fork = nullptr, aux_join = nullptr;
  float* focal_G = nullptr;      // [P*9] dL/dE of the focal backward (allocated on first use)
  float* focal_dphi = nullptr;   // [P*2] per-pair focal terms
  cudaEvent_t graph_in = nullptr, graph_out = nullptr;   // orders replays by completion
  int64_t graph_replays = 0;
  // fm_loss_grad with host buffers: pinned staging of the parameters and the
  // gradient (captured by its graphs), and the epoch each stage was last
  // evaluated at without a graph (a graph is captured on the second call)
  float* h_lg_in = nullptr;
  float* h_lg_grad = nullptr;
  size_t h_lg_cap = 0;               // floats in each
  uint64_t lg_seen[3] = {0, 0, 0};

  // scratch
  float* scratch_params = nullptr;  // [max(m,1)*N*9] parameters of fm_loss_grad
  float* scratch_grad = nullptr;    // [max(m,1)*N*9]
  float* d_loss = nullptr;          // [max(m,1)*S]
  float* h_loss = nullptr;          // pinned [max(m,1)*S]
  int* h_err = nullptr;             // pinned copy of d_err
  int* d_err = nullptr;             // device error bits
  // loss slices (fm_step.cuh): per scene ceil(P_s / 1024) slices
  std::vector<int> h_sc_slice_off;  // [S+1]
  int n_slices = 0;
  int* sc_slice_off = nullptr;      // [S+1]
  float* loss_part = nullptr;       // [64][n_slices]
  int* loss_cnt = nullptr;          // [64][S][kLossCntStride]
};

namespace fm {

// Set while this thread captures a graph.  Captured programmatic edges do not
// order a kernel's reads after its predecessor's writes the way stream
// launches do (measured: replays were not even repeatable), so launches made
// during a capture are plain, fully ordered ones.
extern thread_local bool g_capturing;
// The next launch_pdl on this thread is a plain launch.  Every entry point of
// the library sets it, so that its first kernel is ordered after whatever the
// stream ran before (a caller's graph, copies, other libraries' kernels), and
// fm_step sets it after each graph replay; launches that follow one of this
// library's own kernels overlap with it.
extern thread_local bool g_plain_once;

// Launch with programmatic stream serialisation (see pdl_wait / pdl_trigger);
// a plain launch while capturing.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (g_capturing || g_plain_once) ? 0 : 1;
  g_plain_once = false;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// message returned by fm_last_error(NULL) on the calling thread
void set_thread_error(const std::string& msg);

// ---------------------------------------------------------------- launchers
// setup (fm_setup.cu)
void launch_calibrate(const float* kp1, const float* kp2, const int* kp_pair, const int* pi,
                      const int* pj, const float* f, const float* cx, const float* cy,
                      int64_t Z, int P, float4* out, int* err, cudaStream_t s);
void launch_seg_offsets(const int* kp_pair, int64_t Z, int P, int* seg_off, int* err,
                        cudaStream_t s);
// order of the caller's keypoint pairs (see k_kp_order_check): flags[0] bits
// 1 index out of range, 2 not in (image pair, track) order, 4 negative
// track; flags[1] the largest track (flags zeroed by the caller)
void launch_kp_order_check(const int* kpp, const int* track, int64_t Z, int P, int* flags, cudaStream_t s);
// perm [Z]: the input index of each position of the (image pair, track,
// input index) order (fm_tracks.cu; scratch from the library's pool)
cudaError_t sort_kp_pairs(const int* kp_img_pair, const int* kp_track, int64_t Z, int P, int max_track,
                          uint32_t* perm, cudaStream_t s);
// the inputs (kp1, kp2 [Z][2], kpp, track [Z] or null) in the order perm
void launch_kp_gather(const uint32_t* perm, int64_t Z, const float* kp1, const float* kp2, const int* kpp,
                      const int* track, float* o1, float* o2, int* okpp, int* otrack, cudaStream_t s);
// per-pair values: to_internal out[k] = in[perm[k]], else out[perm[k]] = in[k]
void launch_permute(const float* in, const uint32_t* perm, int64_t Z, bool to_internal, float* out, cudaStream_t s);
// lane tables of the direct kernel: G [P+1] = exclusive scan of the lanes per
// image pair, *T = lanes in use; then the lane descriptors and run headers of
// n_runs warp runs (n_runs >= ceil(T / 32); runs past the lanes in use are
// empty), the record bases, and seg_rec
// With err != null the offsets are checked first (seg_off[0] = 0,
// non-decreasing, seg_off[P] = Z): on a bad table err gets kErrSegOff and
// G = 0, *T = 0, so that no later kernel reads a keypoint pair.
void launch_lane_scan(const int* seg_off, int P, int U, int* G, int* T, cudaStream_t s, int64_t Z = -1,
                      int* err = nullptr);
void launch_lane_desc(const int* seg_off, const int* G, const int* T, int P, int U, int n_runs, int* desc,
                      int4* wrun_info, cudaStream_t s);
void launch_seg_records(const int* seg_off, const int* G, const int4* wrun_info, int P, int* seg_rec,
                        cudaStream_t s);
void launch_check_finite(const float* x, int64_t n, int* err, int bit, cudaStream_t s);
// fills buf and reads it back, leaving L2 full of clean lines of buf
// the stream idles on the device for about ns nanoseconds (one thread)
void launch_idle(unsigned ns, cudaStream_t s);
void launch_l2_flush(void* buf, size_t bytes, int fill, cudaStream_t s);
void launch_exclusive_scan_info(int4* wrun_info, int n, int64_t* total_out_dev, cudaStream_t s);

// epipolar (fm_ea.cu)
// snap (optional): receives a copy of the n_snap parameters (read by the
// camera pass of an Adam step, which updates params in place)
void launch_ea_tables(const float* params, const int* pi, const int* pj, const int* seg_off,
                      int P, float4* seg_tab, int* step_counter, cudaStream_t s, const float* phi = nullptr,
                      float* snap = nullptr, int n_snap = 0);
void launch_ea_direct(const fm_problem* pr, const float* weights, int loss, cudaStream_t s);
// the loss alone; coef_out (optional, Z floats) receives w drho/dr per pair
void launch_ea_direct_loss(const fm_problem* pr, const float* weights, int loss, float* coef_out,
                           cudaStream_t s);
// dL/dE records from stored per-pair coefficients (no residual recompute)
void launch_ea_direct_from_coef(const fm_problem* pr, const float* coef, cudaStream_t s);
// CTAs of k_ea_direct that fit on one SM at the problem's tile
int direct_max_ctas_per_sm(const fm_problem* pr);

// per-image-pair pass after k_ea_direct
struct SegArgs {
  const float4* rec;       // records of k_ea_direct
  const int* seg_rec;      // [P][2] first record, count
  const float* dlde_in;    // [P][9] saved dL/dE_n: used instead of the records when not null
  const float* params;     // [N][9]
  const int* pi;
  const int* pj;
  int P;
  float g_scale;           // factor on the summed coefficient terms
  float l_scale;           // factor on the summed loss terms
  const float* pair_scale; // [P] per-image-pair normaliser (null: 1), applied with g_scale / l_scale
  const float* grad_loss;  // [S] per-scene factor on the gradient (null: 1)
  const int* pair_scene;   // [P] scene of each image pair (null: scene 0)
  float* seg_grad;         // [P][24] chain rule (null: skipped)
  float* seg_loss;         // [P] (null: skipped)
  float* dlde_out;         // [P][9] scaled dL/dE_n (null: skipped)
};
SegArgs seg_args(const fm_problem* pr, const float* params);
void launch_ea_segments(const SegArgs& a, cudaStream_t s);
// the problem's own normalisers (per image pair, i.e. per scene)
void launch_ea_segments(const fm_problem* pr, const float* params, int loss, cudaStream_t s);

// IRLS / compact form (fm_irls.cu)
// prob (optional): keep a pair when prob >= p_min instead of |eps^| < tau
void launch_ea_reweight(const fm_problem* pr, float tau, float delta, int irls, float* w,
                        unsigned long long* kept, cudaStream_t s, const float* prob = nullptr,
                        float p_min = 0.5f);
void launch_w_build(const fm_problem* pr, const float* w, float* W, cudaStream_t s);
void launch_ea_compact(const fm_problem* pr, const float* params, int* step_counter, cudaStream_t s);
// pair_inv_z from per-scene counts: 1/count[scene] (0 when the count is 0)
void launch_pair_inv_from_counts(const fm_problem* pr, const unsigned long long* count, cudaStream_t s);
// count[s] = number of keypoint pairs of scene s with a weight > 0
void launch_count_positive(const fm_problem* pr, const float* w, unsigned long long* count, cudaStream_t s);

// relative poses from keypoints (fm_relpose.cu)
// rel_R == nullptr: only the eight-point estimates E0 into e0_out [P*9]
void launch_relpose(const fm_problem* pr, int irls_iters, float delta, float* rel_R, float* rel_t, int* valid,
                    cudaStream_t s, float* e0_out = nullptr);
// focal interval search (fm_focal.cu): votes[k] = sum over the listed image
// pairs of exp((1 - lambda1/lambda2)/tau) of D_j E0 D_i at candidate rho_k
// (fix_i / fix_j >= 0: that side's rho is fixed), fixed order
void launch_focal_vote(const float* e0, const int* idx, const float* fix_i, const float* fix_j, int M,
                       const float* rhos, int K, float tau, float* votes, cudaStream_t s);
// kp (x1, y1) *= f_old[i]/f_new[i], (x2, y2) *= f_old[j]/f_new[j] per keypoint pair
void launch_recalibrate(const fm_problem* pr, const float* f_old, const float* f_new, cudaStream_t s);

// distortion interval search (fm_distortion.cu): err[row[q]*K + k] = sum over
// the keypoint pairs of work item q's image pair idx[q] of |y_2^T F^ y_1| at
// candidate k (idx/row null: identity; fix_i/fix_j: known alpha per row or
// NaN, may be null).  big: the items have more than kDistSplit keypoint pairs
// (a CTA each), else at most kDistSplit (a warp each).
constexpr int kDistSplit = 1024;
void launch_dist_errors(const fm_problem* pr, const float* scale, const int* idx, const int* row,
                        const float* fix_i, const float* fix_j, int M, bool big, const float* cand, int K,
                        float* err, cudaStream_t s);
void launch_dist_reduce(const float* err, int M, int K, float* out, cudaStream_t s);
// kp <- undistorted at alpha [N] (scale [N] = f0 / half diagonal); *bad |= 1 where 1 + alpha r^2 <= 0
void launch_undistort(const fm_problem* pr, const float* scale, const float* alpha, int* bad, cudaStream_t s);

// focal lengths inside epipolar adjustment (fm_focal_ea.cu; E'_n in the
// tables through launch_ea_tables' phi): G' -> S_j G' S_i and per-pair focal
// terms [P][2]; per-camera sums
void launch_focal_dlde(const fm_problem* pr, const float* params, const float* Gp, const float* phi,
                       const float* grad_loss, float* G_out, float* dphi, cudaStream_t s);
void launch_focal_cam(const fm_problem* pr, const float* dphi, float* gphi, cudaStream_t s);

// learned weights (fm_mlp.cu)
void launch_mlp_pair_tables(const fm_problem* pr, const float* params, const float* rel_t, float* tab,
                            cudaStream_t s);
void launch_mask_from_prob(const float* prob, int64_t Z, float p_min, float* w, cudaStream_t s);
void launch_mlp_infer(const fm_problem* pr, const float* tab, const float* theta, const float* w, float iter_frac,
                      float delta, float* prob, float* logit, float* feat, float* resid, cudaStream_t s);
// tcgen05 forward pass (fm_mlp_tc.cu); err: device error bits
struct InferArgs;
// the network on the tcgen05 tensor cores over the pairs of a (features
// computed in the kernel); err gets kErrMlpTimeout if a bounded wait ran out
void launch_mlp_infer_tc(const InferArgs& a, int* err, int sm_count, cudaStream_t s);
void launch_mlp_forward_tc(const float* theta, const float* x, int64_t B, float* logit, int* err, int sm_count,
                           cudaStream_t s);
// training on tcgen05 (fm_mlp_tc.cu): per-CTA partials of the loss and
// gradient of a batch, [mlp_grad_parts(B)][mlp_part_stride()]
int mlp_grad_parts(int64_t B);
int mlp_part_stride();
void launch_mlp_grad_tc(const float* theta, const float* x, const float* y, int64_t B, float* partial, int* err,
                        cudaStream_t s);
// the partials and their fixed-order sum into grad [kMlpParams] and loss
void launch_mlp_grad(const float* theta, const float* x, const float* y, int64_t B, float* partial, float* grad,
                     float* loss, int* err, cudaStream_t s);
void launch_mlp_adam(float* theta, const float* grad, float* m, float* v, int step, float lr, float b1, float b2,
                     float eps, cudaStream_t s);

// setup steps (fm_init.cu, fm_reltrans.cu, fm_points.cu)
// y = x - (B x)/sigma_s per camera, with the constants of the camera's scene
// in pr->mart_coef (see fm_rotation_init); c1 null for the first column
void launch_mart_iter(const fm_problem* pr, const float* x, const float* c1, float* y, cudaStream_t s);
void launch_normalise3(float* x, int N, cudaStream_t s);
void launch_mart_finish(const float* c1, const float* c2, int N, float* params6, cudaStream_t s);
// x[r][c][a] (runs x N x 3) from the counter-based generator at the index the
// value would have in the camera's own scene: (r N_s + c - c0_s) 3 + a
void launch_hash_fill(const fm_problem* pr, float* x, int runs, unsigned salt, cudaStream_t s);
void launch_merge(const fm_problem* pr, const float* o, int runs, float* stats, float* out,
                  int* best_run, cudaStream_t s);
void launch_reltrans(const fm_problem* pr, const float* rot6, float* rel_t, float* err_out, cudaStream_t s);
int reltrans_lattice_points();
void launch_reltrans_lattice(float4* lat0, cudaStream_t s);   // fills pr->lattice0 (needed by launch_reltrans)
cudaError_t build_track_table(fm_problem* pr, int* T_out);
// (fm_tracks.cu) off: per-track counts in, exclusive scan out; idx: keypoint
// pairs ordered by track, ascending inside a track
cudaError_t track_table(const int* kp_track, int64_t Z, int T, int* off, int* idx, cudaStream_t s);
void launch_triangulate(const fm_problem* pr, const float* params, float max_err_px, float min_angle_rad,
                        float* pts, int* valid, int* ncam, cudaStream_t s);
// x <- x/|x| over each scene's cameras ([N][3])
void launch_scale_to_unit(const fm_problem* pr, float* x, cudaStream_t s);
void launch_ea_from_stages(const float* rot6, const float* o, int N, float* ea, cudaStream_t s);
void launch_ea_to_Rt(const float* ea, int N, float* R, float* t, cudaStream_t s);

// rotation / translation (fm_pose.cu)
void launch_rot_pairs(const float* params, const int* pi, const int* pj, const float* rel_R,
                      int P, const float* pair_inv_p, float* seg_grad, float* seg_loss, int* step_counter,
                      cudaStream_t s);
void launch_trn_targets(const float* rot_params, const int* pj, const float* rel_t, int P,
                        float* target, cudaStream_t s);
void launch_trn_pairs(const float* o, const int* pi, const int* pj, const float* target, int N,
                      int P, int runs, const float* pair_inv_p, float* seg_grad, float* seg_loss,
                      int* step_counter, cudaStream_t s);

// loss reductions in slices of image pairs (fm_step.cuh): the loss of scene
// s is summed by ceil(P_s / 1024) CTAs, the last of which adds their sums
constexpr int kLossCntStride = 32;   // ints between two arrival counters: a 128-B line each
constexpr int kLossSlice = 256;      // image pairs per slice (two per thread)
struct LossArgs {
  const int* sc_pair_off;  // [S+1] image-pair range of each scene
  const int* sc_slice_off; // [S+1] first slice of each scene
  int S;
  int n_slices;            // slices of all scenes (per run)
  float* partial;          // [runs][n_slices] slice sums
  int* cnt;                // [runs][S][kLossCntStride] arrival counters, zero between launches
  float* out;              // [runs][S] losses, or null (no loss wanted)
  float* out2;             // a second destination of the same losses, or null
};

// per-camera reduction, 6D adjoint and Adam (fm_cam.cu)
struct CamUpdate {
  const int* cam_seg_off;
  const int* cam_seg;
  const float* seg_grad;   // [runs][P][2*stride]: two 16-byte-aligned slots per image pair
  const float* params;     // [runs][N][pdim] parameters the gradient was taken at
  float* params_out;       // Adam: updated in place (== params); else null
  float* grad_out;         // gradient output or null
  float* m;
  float* v;
  const int* step;
  float lr, b1, b2, eps;
  int N, P, runs;
  const float* seg_loss;   // [runs][P] per-image-pair loss terms (k_cam's loss slices)
  LossArgs loss;           // loss.out null: no loss
  bool csr_order;          // seg_grad holds the parts in camera-CSR order ([2P][stride], one run)
};
void launch_cam_update(int stage, const CamUpdate& u, cudaStream_t s);
// the epipolar step after k_ea_direct: s as for k_ea_segments (its seg_grad,
// seg_loss, dlde_* unused), u as for k_cam of the epipolar stage (one run)
struct EaCamArgs {
  SegArgs s;
  CamUpdate u;
};
void launch_cam_ea(const EaCamArgs& f, cudaStream_t s);
// L.out[r*S + s] (and L.out2) = fixed-order sum of x[r*P + sc_pair_off[s] ..
// sc_pair_off[s+1]) in the slices of L
void launch_sum_fixed(const float* x, int P, int runs, const LossArgs& L, cudaStream_t s);

}  // namespace fm
