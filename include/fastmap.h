/*
 * fastmap.h -- C ABI of the B300 (sm_103a) first-order solver for FastMap
 * (arxiv 2505.04612, "FastMap: Revisiting Structure from Motion through
 * First-Order Optimization").
 *
 * The library evaluates, on one GPU, the loss and gradient of the paper's
 * first-order objectives and takes Adam steps on them:
 *   - global rotation      (Sec. 3.3, Eqs. 3-4)
 *   - global translation   (Sec. 3.3, Eqs. 5-6)
 *   - epipolar adjustment  (Sec. 3.3, Eqs. 7-9; Appendix "Epipolar
 *                           Adjustment", Eqs. 15-17)
 *
 * Conventions used by every entry point
 *   - Pose of camera c is world-to-camera: x_cam = R_c X + t_c.
 *   - Image pair n = (i_n, j_n), i_n != j_n; in a keypoint pair of image pair
 *     n the first keypoint lies in image i_n and the second in image j_n.
 *   - Keypoints are pixels (u, v); calibration uses a pinhole with focal f
 *     and principal point (cx, cy):  x~ = ((u - cx)/f, (v - cy)/f, 1)
 *     (Sec. 3.3, "normalized homogeneous coordinates"; Sec. 3.1, camera
 *     assumptions).
 *   - Parameters of a stage are one float32 row per camera:
 *       FM_STAGE_ROTATION     6 floats  (a1, a2): the 6D representation,
 *                             R = [b1 b2 b3], b1 = a1/|a1|,
 *                             b2 = normalise(a2 - (b1.a2) b1), b3 = b1 x b2
 *       FM_STAGE_TRANSLATION  3 floats  o: camera centre, one block of
 *                             n_cams rows per initialisation run
 *       FM_STAGE_EPIPOLAR     9 floats  (a1, a2, t): 6D rotation + translation
 *   - Matrices are row-major float32.
 *   - All floating point arithmetic on the GPU is float32.
 *
 * Memory and ownership
 *   - fm_problem_create copies everything it needs; the caller keeps
 *     ownership of its arrays and may free them after the call returns.
 *   - Pointers are host pointers unless the argument or flag says device.
 *   - Output buffers always belong to the caller.
 *   - Every entry point runs on the CUDA stream given at creation and
 *     returns after the work is enqueued, unless it writes a host buffer, in
 *     which case it synchronises that stream first.
 *
 * Scenes (batches)
 *   - One problem may hold S independent scenes (fm_problem_desc.n_scenes):
 *     their cameras, image pairs and keypoint pairs are concatenated, scene
 *     by scene.  Every kernel runs once over all of them; every loss is the
 *     scene's own (normalised by the scene's own |P| or Z), so that a scene
 *     gets the same losses, gradients and Adam steps as when solved alone.
 *   - Loss outputs hold one value per scene: [S] for the rotation and
 *     epipolar stages, [m][S] (run-major) for m translation runs.
 *
 * Errors
 *   - Every entry point returns an fm_status; no C++ exception crosses the
 *     ABI and the library never exits or aborts.
 *   - fm_last_error(problem) describes the last failure on that problem;
 *     fm_last_error(NULL) describes the last failure of fm_problem_create (or
 *     of fm_ea_loss_grad_static) on the calling thread.
 *   - Results are deterministic: no floating-point atomics are used, so the
 *     same inputs give bitwise identical outputs on the same GPU.
 */
#ifndef FASTMAP_H
#define FASTMAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fm_problem fm_problem;   /* opaque; owned by the library */

typedef enum {
  FM_OK = 0,
  FM_ERR_INVALID_ARG = 1,   /* a size, index, pointer or value is invalid */
  FM_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  FM_ERR_OOM = 3,           /* device memory could not be allocated */
  FM_ERR_NAN = 4,           /* a non-finite value was produced or given */
  FM_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
  FM_ERR_NOT_CONVERGED = 6,  /* reserved (kept for ABI stability): the method runs
                               fixed iteration counts and has no convergence test */
  FM_ERR_STATE = 7          /* the call needs state that has not been set */
} fm_status;

typedef enum {
  FM_STAGE_ROTATION = 0,
  FM_STAGE_TRANSLATION = 1,
  FM_STAGE_EPIPOLAR = 2
} fm_stage;

/* Robust loss of the epipolar stage.
 *   FM_EA_L1       direct, per keypoint pair:  (1/Z) sum w_m |r_m|      (Eq. 7)
 *   FM_EA_L2       direct, per keypoint pair:  (1/Z) sum w_m r_m^2      (Eqs. 8-9)
 *   FM_EA_COMPACT  per image pair:  (1/Z) sum_n e_n^T W_n e_n           (Eqs. 8-9,
 *                  right-hand side; W_n = sum_m w_m vec(x~2 x~1^T)vec(.)^T,
 *                  Eq. 17, rebuilt whenever the weights change) -- the same
 *                  objective as FM_EA_L2 at a per-step cost independent of Z
 * with r_m = x~2^T E_n x~1 and E_n = [t_ij/|t_ij|]_x R_ij,
 * R_ij = R_j R_i^T, t_ij = t_j - R_ij t_i.  w_m = 1 until fm_ea_set_weights
 * sets per-pair weights; Z is the number of keypoint pairs, or the value
 * given to fm_ea_set_weights. */
typedef enum {
  FM_EA_L1 = 0,
  FM_EA_L2 = 1,
  FM_EA_COMPACT = 2
} fm_ea_loss;

/* Problem description (Sec. 3.3: the inputs of the pose stages are the image
 * pairs, their inlier keypoint pairs and the calibrated intrinsics). */
typedef struct {
  int32_t n_cams;              /* N >= 2 */
  int32_t n_img_pairs;         /* P >= 1 */
  int64_t n_kp_pairs;          /* Z >= 0, Z < 2^31 - 2^20 */
  const int32_t* pair_cam_i;   /* [P] first image of each image pair */
  const int32_t* pair_cam_j;   /* [P] second image; != pair_cam_i */
  const int32_t* kp_img_pair;  /* [Z] image pair of each keypoint pair, in
                                  [0, P), in any order: the library keeps the
                                  keypoint pairs sorted by (image pair,
                                  track), see fm_kp_order */
  const float* kp1_px;         /* [Z*2] (u, v) of the keypoint in image i_n */
  const float* kp2_px;         /* [Z*2] (u, v) of the keypoint in image j_n */
  const int32_t* kp_track;     /* [Z] track id (>= 0), or NULL; needed by
                                  fm_triangulate only */
  const float* focal;          /* [N] > 0 */
  const float* cx;             /* [N] */
  const float* cy;             /* [N] */
  const float* rel_R;          /* [P*9] R^{i->j}, or NULL */
  const float* rel_t;          /* [P*3] unit t^{i->j}, or NULL */
  int32_t inputs_on_device;    /* 1: every pointer above is device memory */
  void* cuda_stream;           /* cudaStream_t to run on; NULL = default */
  int32_t n_scenes;            /* S: independent scenes held by the problem;
                                  0 or 1 = one scene (scene_cam_off unused) */
  const int32_t* scene_cam_off; /* [S+1] host memory: cameras of scene s are
                                  [off[s], off[s+1]), off[0] = 0, off[S] = N,
                                  >= 2 cameras each; every image pair joins two
                                  cameras of one scene, image pairs are grouped
                                  by scene in scene order, >= 1 per scene */
} fm_problem_desc;

typedef struct {
  int32_t n_cams;
  int32_t n_img_pairs;
  int64_t n_kp_pairs;
  int32_t n_empty_img_pairs;   /* image pairs with no keypoint pair */
  int32_t pairs_per_lane;      /* keypoint pairs per thread in the direct kernel */
  int64_t n_records;           /* per-(warp run, image pair) partial sums */
  int64_t device_bytes;        /* device memory held by the problem */
  int32_t n_scenes;            /* S */
  int32_t n_cams_connected;    /* cameras in the largest connected component of
                                  their scene's view graph */
} fm_problem_info;

/* Adam (the paper's cited adaptive first-order method, Sec. 1, Sec. 3.2; no
 * constants are given there).  Bias-corrected, as Kingma & Ba define it. */
typedef struct {
  float lr;
  float beta1;
  float beta2;
  float eps;
} fm_adam_opts;

/* Creates a problem on the current CUDA device.  Validates the description
 * (sizes, camera indices of the image pairs, intrinsics on the host side;
 * range of kp_img_pair and finiteness of the keypoints on the device) and
 * returns FM_ERR_INVALID_ARG / FM_ERR_NAN on bad input.  Copies the keypoint
 * pairs in (image pair, track) order -- the set of keypoint pairs Q_n of
 * image pair n (Sec. 3.3) contiguous, the data marshalled on the GPU (Sec. 4,
 * setup): when the caller's order is not that one already, they are sorted
 * on the device (stable: pairs with equal keys keep the caller's relative
 * order; without kp_track the key is the image pair alone) and the
 * permutation is kept.  Calibrates the keypoints (Sec. 3.3, x~ = K^-1 [u, v,
 * 1]^T) and builds the image-pair and camera tables.  Synchronises the
 * stream.  On success *out owns device memory until fm_problem_destroy. */
fm_status fm_problem_create(const fm_problem_desc* desc, fm_problem** out);

/* The library's order of the keypoint pairs: perm_out [Z] (host or device
 * as flagged) receives, for each internal position k, the index in the
 * caller's arrays of the keypoint pair held there (the identity when the
 * caller's order was kept).  fm_ea_set_weights and fm_ea_get_weights take
 * and give per-pair values in the caller's order; the per-pair device
 * outputs of fm_mlp_eval / fm_mlp_eval_relative and the coefficients saved
 * by fm_ea_forward are in the internal order (value k belongs to caller
 * pair perm_out[k]).  Synchronises. */
fm_status fm_kp_order(const fm_problem* problem, int32_t* perm_out, int32_t out_on_device);

/* Releases every resource of the problem (NULL is a no-op).  Synchronises. */
void fm_problem_destroy(fm_problem* problem);

/* Text of the last error (see the Errors paragraph above); never NULL. */
const char* fm_last_error(const fm_problem* problem);

/* Sizes and memory use of a problem. */
fm_status fm_problem_info_get(const fm_problem* problem, fm_problem_info* out);

/* Replaces the parameters of a stage (layout above) and resets the stage's
 * Adam moments and step counter.  params_on_device: 1 if params is a device
 * pointer.  FM_ERR_NAN if a value is not finite. */
fm_status fm_set_params(fm_problem* problem, fm_stage stage, const float* params,
                        int32_t params_on_device);

/* Copies the current parameters of a stage into params_out (host or device
 * as flagged).  Synchronises when params_out is a host pointer. */
fm_status fm_get_params(const fm_problem* problem, fm_stage stage, float* params_out,
                        int32_t out_on_device);

/* Relative rotations R^{i->j} [P*9] and unit relative translations t^{i->j}
 * [P*3] of the image pairs (the inputs of Eqs. 3 and 5); either may be NULL
 * to keep the current one.  Replacing rel_t invalidates the translation
 * targets, which are rebuilt from the rotation-stage parameters on the next
 * translation-stage call. */
fm_status fm_set_rel_poses(fm_problem* problem, const float* rel_R, const float* rel_t,
                           int32_t on_device);

/* Number m of independent translation runs solved together (Appendix
 * "Multiple Initializations"); 1 <= m <= 64.  The translation-stage
 * parameters become [m*N*3] (one block of N centres per run), losses [m];
 * the parameters must be set again afterwards. */
fm_status fm_translation_set_runs(fm_problem* problem, int32_t n_runs);

/* Selects the robust loss of the epipolar stage (default FM_EA_L1). */
fm_status fm_ea_set_loss(fm_problem* problem, fm_ea_loss loss);

/* Per-keypoint-pair weights w_m of the epipolar stage (Eq. 9: IRLS weights
 * 1/|eps^_m|; a weight of 0 removes a filtered pair), in the order of the
 * keypoint pairs given at creation, and the normaliser 1/Z of the loss:
 * inv_z > 0 is used for every scene; inv_z == 0 gives each scene
 * 1/(number of its pairs with a positive weight).  weights == NULL restores
 * unit weights and 1/(the scene's keypoint pairs).  The compact
 * matrices W_n (Eq. 17) are rebuilt by the next FM_EA_COMPACT evaluation,
 * stored as an expansion around the essential matrices of the parameters of
 * that evaluation. */
fm_status fm_ea_set_weights(fm_problem* problem, const float* weights,
                            int32_t weights_on_device, float inv_z);

/* IRLS reweighting and outlier filtering at the current epipolar-stage
 * parameters (Sec. 3.3: weights from the absolute epipolar error eps^ of the
 * previous round, Eq. 9; periodic filtering of pairs with a large error).
 * For every keypoint pair, eps^ = x~2^T E_n x~1; the pair is kept when
 * |eps^| < tau and then weighted 1/max(|eps^|, delta) when irls != 0, or 1
 * when irls == 0; filtered pairs get weight 0.  Sets each scene's inv_z to
 * 1/(its kept pairs), rebuilds W_n around the current poses, and writes the
 * total #kept over all scenes to *n_kept (may be NULL).  Synchronises. */
fm_status fm_ea_reweight(fm_problem* problem, float tau, float delta, int32_t irls,
                         int64_t* n_kept);

/* Copies the current per-pair weights (host or device as flagged) and the
 * loss normaliser (of scene 0).  FM_ERR_STATE when no weights are set.
 * Synchronises. */
fm_status fm_ea_get_weights(fm_problem* problem, float* weights_out, int32_t out_on_device,
                            float* inv_z);

/* Loss and gradient of a stage at the given parameters (Eqs. 3-4 for the
 * rotation stage; Eqs. 5-6 for the translation stage, with targets
 * o^{i->j} = -R_j^T t^{i->j} from the rotation-stage parameters; Eq. 7 or
 * Eqs. 8-9 for the epipolar stage, with the loss chosen by fm_ea_set_loss).
 * params: [N*dim] (layout above; [m*N*3] for m translation runs); grad: same
 * layout, or NULL; loss: host array of one value per scene ([m][S] for the
 * translation stage), or NULL.  mem_on_device: 1 if params and grad are device pointers.
 * The stage's own parameters and Adam state are not touched.  Synchronises
 * when loss or a host grad is requested. */
fm_status fm_loss_grad(fm_problem* problem, fm_stage stage, const float* params,
                       float* loss, float* grad, int32_t mem_on_device);

/* ------------------------------------------- epipolar forward / backward */

/* What fm_ea_forward keeps for fm_ea_backward.  The paper evaluates loss and
 * gradient together (Sec. 3.3); these calls split the direct epipolar
 * objective (Eq. 7, or Eqs. 8-9 with per-pair weights: losses FM_EA_L1 and
 * FM_EA_L2) into a forward pass and its adjoint, for reverse-mode use (e.g.
 * behind torch.autograd.Function).
 *   FM_EA_SAVE_NONE  nothing: the backward pass re-reads every keypoint pair
 *                    and recomputes its residual (16 B per pair);
 *   FM_EA_SAVE_COEF  per keypoint pair the coefficient c_m = w_m rho'(r_m)
 *                    (sign(r) for L1, 2r for L2), Z floats in the library's
 *                    internal pair order (sorted by image pair, stable);
 *                    the backward pass reads c_m and the pair's keypoints
 *                    (4 + 16 B per pair) and recomputes no residual;
 *   FM_EA_SAVE_DLDE  per image pair dL/dE_n = (1/Z) sum_m c_m x~2 x~1^T
 *                    (row-major 3x3), P*9 floats; the forward pass does all
 *                    the per-pair work and the backward pass only the chain
 *                    rule through E_n and the per-camera sums. */
typedef enum {
  FM_EA_SAVE_NONE = 0,
  FM_EA_SAVE_COEF = 1,
  FM_EA_SAVE_DLDE = 2
} fm_ea_save;

/* Forward pass: the epipolar loss (current loss and weights of the problem;
 * FM_ERR_STATE for FM_EA_COMPACT) at params_dev [N*9] into loss_dev (one
 * device float per scene), and the intermediates selected by `save` into saved_dev
 * (device, 16-byte aligned: Z floats for FM_EA_SAVE_COEF, P*9 for
 * FM_EA_SAVE_DLDE, ignored for FM_EA_SAVE_NONE).  All pointers are device
 * memory owned by the caller.  Asynchronous on the problem's stream. */
fm_status fm_ea_forward(fm_problem* problem, const float* params_dev, float* loss_dev,
                        int32_t save, float* saved_dev);

/* Backward pass: grad_dev [N*9] = sum_s g_s dL_s/dparams at params_dev, where
 * g_s is grad_loss_dev[s], one device float per scene (all 1 when
 * grad_loss_dev is NULL).  `save` and saved_dev must be those of the forward
 * call at the same params_dev, and the loss and weights must be unchanged
 * since.  Asynchronous. */
fm_status fm_ea_backward(fm_problem* problem, const float* params_dev, int32_t save,
                         const float* saved_dev, const float* grad_loss_dev, float* grad_dev);

/* n_iters Adam steps on the stage's parameters, each one a full evaluation of
 * the loss and gradient (over all keypoint pairs for the epipolar stage)
 * followed by the update (Sec. 3.2-3.4).  loss (host, or NULL; [S], or
 * [m][S] for the translation stage) receives the loss of the last evaluation, i.e. at the
 * parameters before the last update; passing NULL keeps the call
 * asynchronous. */
fm_status fm_step(fm_problem* problem, fm_stage stage, const fm_adam_opts* opts,
                  int32_t n_iters, float* loss);

/* ------------------------------------------------------------- setup steps */

/* Rotation initialisation (Appendix "Global Rotation / Initialization",
 * Eqs. 10-14): the first columns of all world-to-camera rotations minimise
 * sum ||c1_j - R^{i->j} c1_i||^2 (Eq. 12), the second columns the same plus
 * the orthogonality penalty (Eq. 13); each is the eigenvector of the smallest
 * eigenvalue of its sparse quadratic form, found here by n_iters steps of
 * power iteration on I - A/sigma; columns are normalised per camera,
 * Gram-Schmidt orthogonalised, and c3 = c1 x c2 (Eq. 14).  Writes the
 * rotation-stage parameters (6D = (c1, c2)) and resets their Adam state.
 * Needs rel_R.  The result is defined up to a global rotation (a gauge). */
fm_status fm_rotation_init(fm_problem* problem, int32_t n_iters);

/* Relative translation re-estimation (Appendix "Relative Translation"): with
 * R^{i->j} = R_j R_i^T from the rotation-stage parameters, the unit
 * translation of every image pair minimising the mean |x~2^T [t]_x R x~1|
 * over a Fibonacci lattice of 4096 points on the hemisphere refined by two
 * 1024-point lattices on spherical caps (radius twice the previous spacing),
 * sign by cheirality (+t on ties).  Replaces rel_t.  err_out: [P] mean error
 * of the chosen direction (host or device as flagged), or NULL.  When
 * per-pair weights are set, pairs with weight 0 are left out of the score
 * and the sign (unless an image pair has no other pair). */
fm_status fm_relative_translations(fm_problem* problem, float* err_out, int32_t err_on_device);

/* Relative poses of every image pair from its keypoint pairs (the setup step
 * standing in for the upstream two-view estimate the paper decomposes, Sec.
 * 3.3 "Global Rotation"): the eigenvector of W_n = sum_m w_m vec(x~2 x~1^T)
 * vec(x~2 x~1^T)^T with the smallest eigenvalue (the linear eight-point
 * estimate of E in calibrated coordinates; Eq. 17's W_n), irls_iters re-solves
 * with weights w_m = 1/max(|x~2^T E x~1|, delta) (0 <= irls_iters <= 16,
 * delta > 0), the projection onto the essential matrices (singular values
 * (1, 1, 0)), and of its four decompositions the one with the most keypoint
 * pairs in front of both cameras (the first on ties).  Writes the problem's
 * rel_R and unit rel_t (as fm_set_rel_poses would); image pairs with fewer
 * than 8 keypoint pairs get R = I, t = 0.  n_valid (or NULL) receives the
 * number of image pairs estimated.  Not robust to outliers by itself (a
 * linear least-squares estimate); synchronises. */
fm_status fm_relative_poses(fm_problem* problem, int32_t irls_iters, float delta, int32_t* n_valid);

/* Focal length interval search (Sec. 3.1 "Focal Length Estimation", Eq.
 * focal-vote; Appendix "Focal Length Estimation").  For every image pair, E0
 * = the eight-point estimate (as fm_relative_poses, irls_iters re-solves) in
 * the problem's current calibration (focal f0 per image, principal point
 * fixed); at focal ratios rho_i, rho_j (f = rho f0) its candidate essential
 * matrix is D_j E0 D_i, D = diag(rho, rho, 1), scored by
 * exp((1 - lambda1/lambda2)/tau) with lambda1 >= lambda2 its two largest
 * singular values.  Images form n_groups groups sharing intrinsics (group
 * [N] ids in [0, n_groups), or NULL with n_groups = 1: one focal length for
 * all).  Groups are estimated one at a time, the one with the most "ready"
 * image pairs first (both images in it, or one in it and the other's group
 * already estimated; the lowest id on ties), each by the candidate with the
 * highest summed score over its ready pairs (the first on ties), the other
 * side's ratio fixed where it is known.  Candidates: n_cand (2..65536) ratios
 * spaced evenly in log between rho_min and rho_max.  focal_out [N] (host)
 * receives f0 rho of each image's group, f0 where a group never became ready;
 * n_estimated (or NULL) the number of groups estimated.  Image pairs with
 * fewer than 8 keypoint pairs take no part.  Synchronises. */
fm_status fm_focal_search(fm_problem* problem, const int32_t* group, int32_t n_groups, float rho_min,
                          float rho_max, int32_t n_cand, float tau, int32_t irls_iters, float* focal_out,
                          int32_t* n_estimated);

/* Recalibrates the problem at new focal lengths focal [N] (host or device as
 * flagged; finite, > 0; principal points unchanged): every stored keypoint's
 * calibrated coordinates are rescaled by f_old / f_new of its image.  The
 * relative poses and every stage's parameters are kept (re-estimate them as
 * needed).  Synchronises. */
fm_status fm_set_focal(fm_problem* problem, const float* focal, int32_t on_device);

/* Distortion interval search (Sec. 3.1 "Distortion Estimation", Eq. 1;
 * Appendix "Distortion Estimation").  One-parameter division model about the
 * image centre (cx, cy): x_u = x_d / (1 + alpha r_d^2), x_d the observed
 * offset from the centre in units of the half diagonal h = |(cx, cy)|.  A
 * candidate alpha is scored on a set of image pairs by undistorting their
 * keypoints (homogeneous (x_u, y_u, 1)), re-estimating each pair's
 * fundamental matrix (Hartley-normalised linear eight-point: per image
 * y = T x_u with the centroid at the origin and RMS distance sqrt(2); F^
 * projected to rank 2, unit Frobenius norm) and averaging the epipolar error
 * |y_2^T F^ y_1| (scale-free) over all their keypoint pairs; the lowest
 * average wins (the first on ties).  The scores assume verified matches:
 * the eight-point fit is least squares, so gross outliers (more than a few
 * percent) bias the estimate.  Hierarchical: n_levels levels of
 * n_cand (2..32) candidates spaced evenly over the interval, [alpha_min,
 * alpha_max] at the first level and the winner's two neighbours (the end
 * candidate at an end) at the next.  Groups (cameras) as in fm_focal_search:
 * one at a time in the ready-pair order, an image of an estimated group
 * undistorted with its alpha.  Works on the stored keypoints as they are
 * (alpha of residual distortion once fm_set_distortion has been applied).
 * alpha_out [N] (host): each image's group's alpha, 0 where the group never
 * became ready; n_estimated (or NULL): groups estimated.  Image pairs with
 * fewer than 8 keypoint pairs take no part.  Synchronises. */
fm_status fm_distortion_search(fm_problem* problem, const int32_t* group, int32_t n_groups, float alpha_min,
                               float alpha_max, int32_t n_cand, int32_t n_levels, float* alpha_out,
                               int32_t* n_estimated);

/* The scores behind fm_distortion_search, per image pair: err_out [P*n_cand]
 * (pair-major; host or device as flagged) receives, for every image pair and
 * candidate alpha_cand[k] (n_cand in 1..32; host or device as flagged)
 * applied to both of its images, the sum of |y_2^T F^ y_1| over its keypoint
 * pairs with F^ its own normalised rank-2 eight-point estimate; 0 for image
 * pairs with fewer than 8 keypoint pairs.  Synchronises. */
fm_status fm_distortion_pair_errors(fm_problem* problem, const float* alpha_cand, int32_t n_cand,
                                    float* err_out, int32_t on_device);

/* Undistorts the stored keypoints in place with alpha [N] per image (host
 * or device as flagged; finite): x_c <- x_c / (1 + alpha r_d^2) in the
 * calibrated coordinates.  A keypoint with 1 + alpha r_d^2 <= 0 has no
 * undistorted point: its keypoint pair is left as it was and the call returns
 * FM_ERR_INVALID_ARG after undistorting all others.  Relative poses and stage
 * parameters are kept.  Synchronises. */
fm_status fm_set_distortion(fm_problem* problem, const float* alpha, int32_t on_device);

/* ------------------------------------------------ tracks and image pairs
 * Preprocessing of raw matches before a problem is built (Appendix "Tracks"
 * and "Filtering"). */

typedef struct fm_tracks fm_tracks;   /* opaque; results held on the device */

/* Track completion.  Keypoints are grouped by image: those of image c are
 * kp_off[c] .. kp_off[c+1]-1 (kp_off [n_images + 1], kp_off[0] = 0,
 * non-decreasing; n_images in 2..65535).  matches [n_matches * 2] holds
 * keypoint ids (u, v) of raw matches between two different images, in any
 * order and orientation.  A track is a connected component of the keypoint
 * graph with at least two keypoints; tracks are numbered by their smallest
 * keypoint id.  A consistent track (no two keypoints in one image) yields
 * every pair of its keypoints; an inconsistent one yields its raw matches as
 * given (duplicates included).  The keypoint pairs are oriented from the lower
 * to the higher image and grouped by image pair (i < j) in increasing (i, j);
 * inside an image pair the consistent tracks' pairs come first, by track,
 * then the raw matches of inconsistent tracks in input order.  Image pairs
 * with fewer than min_pairs (>= 1) keypoint pairs are dropped with their
 * pairs.  kp_px [K * 2] (or NULL): pixel coordinates, gathered into the
 * output pairs.  on_device: kp_off, matches and kp_px are device pointers,
 * complete when the call starts.  The labels, order and outputs are
 * deterministic.  Errors: FM_ERR_INVALID_ARG for a match outside [0, K) or
 * inside one image (checked on the device), FM_ERR_TIMEOUT if a union-find
 * step bound is reached.  *out is released with fm_tracks_destroy.  Device
 * memory (scratch and results) comes from a stream-ordered pool that the
 * library creates on first use and keeps for the process, so that later calls
 * reuse it without mapping memory.  Synchronises. */
fm_status fm_tracks_complete(int32_t n_images, const int32_t* kp_off, int64_t n_matches, const int32_t* matches,
                             const float* kp_px, int32_t min_pairs, int32_t on_device, fm_tracks** out);

/* Sizes of a completion: tracks, image pairs P, keypoint pairs Z and
 * inconsistent tracks; any pointer may be NULL. */
fm_status fm_tracks_info(const fm_tracks* tracks, int64_t* n_tracks, int64_t* n_img_pairs, int64_t* n_kp_pairs,
                         int64_t* n_inconsistent);

/* Copies the results (host or device buffers as flagged; any may be NULL):
 * pair_i, pair_j [P]; kp_img_pair, node1 (keypoint in image pair_i), node2,
 * kp_track [Z]; kp1_px, kp2_px [Z * 2] when kp_px was given.  The arrays feed
 * fm_problem_desc directly (kp_track as the track ids). */
fm_status fm_tracks_copy(const fm_tracks* tracks, int32_t* pair_i, int32_t* pair_j, int32_t* kp_img_pair,
                         int32_t* node1, int32_t* node2, int32_t* kp_track, float* kp1_px, float* kp2_px,
                         int32_t on_device);

void fm_tracks_destroy(fm_tracks* tracks);

/* Adaptive image-pair filtering (host).  An image pair is kept while its
 * count (e.g. its number of keypoint pairs) is above the threshold t; t
 * starts at t_start and becomes max(t / 2, t_min) while the kept pairs leave
 * the n_images images in more than one connected component and t > t_min.
 * At the final t, images outside the largest component (the one holding the
 * smallest image id on ties) are outliers: image_valid[c] = 0 (or NULL) and
 * every image pair touching one is dropped.  keep [n_pairs] receives 1 for
 * the kept pairs, *t_used (or NULL) the final threshold. */
fm_status fm_filter_image_pairs(int32_t n_images, int32_t n_pairs, const int32_t* pair_i, const int32_t* pair_j,
                                const int32_t* counts, double t_start, double t_min, int32_t* keep,
                                int32_t* image_valid, double* t_used);

/* Copies the current relative rotations [P*9] / translations [P*3]; either
 * may be NULL.  Synchronises for host outputs. */
fm_status fm_get_rel_poses(fm_problem* problem, float* rel_R, float* rel_t, int32_t out_on_device);

/* Random initial centres for every translation run (Sec. 3.3: the objective
 * is optimised from random starts): value k of the [m*N*3] array is
 * fmix32(k * 0x9E3779B9 + seed) >> 8, scaled by 2^-23, minus 1 (uniform in
 * [-1, 1); fmix32 is the MurmurHash3 32-bit finaliser).  Resets Adam. */
fm_status fm_translation_random_init(fm_problem* problem, uint32_t seed);

/* Merges the translation runs (Appendix "Multiple Initializations"): each run
 * is moved to zero centroid and unit mean norm, and every camera takes the
 * run with the lowest mean loss over its image pairs (lowest run on ties).
 * Afterwards the problem has one run holding the merged centres (Adam reset).
 * best_run_out: [N] host array of the chosen run per camera, or NULL.
 * Synchronises. */
fm_status fm_translation_merge(fm_problem* problem, int32_t* best_run_out);

/* Epipolar-stage parameters from the rotation stage (6D) and the merged
 * centres o: t_i = -R_i o_i.  Resets Adam and the compact matrices. */
fm_status fm_epipolar_init_from_stages(fm_problem* problem);

/* Sparse reconstruction (Appendix "Sparse Reconstruction") at the
 * epipolar-stage parameters: every keypoint pair of a track is triangulated
 * (two-ray midpoint), the points of a track are averaged, a keypoint is an
 * inlier if its reprojection error is <= max_err_px, and a point is valid if
 * its inlier keypoints span >= 3 cameras and its largest triangulation angle
 * (at the point, between two inlier keypoints' camera centres) is >=
 * min_angle_deg.  Needs kp_track at creation; tracks are the ids 0..T-1.
 * Outputs [T*3], [T], [T] (any may be NULL; host or device as flagged) and T. */
typedef struct {
  float max_err_px;
  float min_angle_deg;
} fm_tri_opts;

fm_status fm_triangulate(fm_problem* problem, const fm_tri_opts* opts, float* points,
                         int32_t* valid, int32_t* n_inlier_cams, int32_t out_on_device,
                         int32_t* n_tracks);

/* -------------------------------------------------------- end-to-end solve
 * The paper fixes no learning rate, iteration count or threshold; the
 * defaults of fm_solve_opts_default are this library's choices. */
typedef struct {
  int32_t rot_init_iters;     /* power iterations per column (2000) */
  int32_t rot_iters;          /* Adam steps on the rotation loss (2000) */
  float rot_lr;               /* (1e-3) */
  int32_t reestimate_rel_t;   /* 1: grid search; 0: keep the given rel_t (1) */
  int32_t trn_runs;           /* translation runs from random starts (4) */
  int32_t trn_iters;          /* Adam steps per run (2000) */
  float trn_lr;               /* (1e-2) */
  int32_t trn_final_iters;    /* after the merge (1000) */
  uint32_t seed;              /* of the random starts (0) */
  int32_t ea_rounds;          /* IRLS / filtering rounds (5) */
  int32_t ea_iters;           /* Adam steps per round on the compact form (500) */
  float ea_lr;                /* (1e-4) */
  float ea_tau0;              /* first filtering threshold, calibrated units (0.05) */
  float ea_tau_min;           /* halved each round down to this (0.005) */
  float ea_delta;             /* IRLS weight floor (1e-5) */
  float tri_max_err_px;       /* (4) */
  float tri_min_angle_deg;    /* (2) */
  float beta1, beta2, eps;    /* Adam (0.9, 0.999, 1e-8) */
  int32_t learned;            /* 1: the network prunes pairs after the first
                                 grid search (fm_mlp_prune, iteration
                                 fraction 0), the relative translations are
                                 re-estimated from the kept pairs, and every
                                 round filters with the network
                                 (fm_mlp_reweight, fraction (k+1)/(rounds+1))
                                 instead of the threshold tau_k; needs
                                 fm_mlp_set_params (0) */
  float learned_p_min;        /* inlier probability to keep a pair (0.5) */
  int32_t learned_prune_passes; /* prune + re-estimate passes before the
                                 translation stage (1): each pass sees the
                                 relative translations of the previous one */
  int32_t rot_given;          /* 1: start from the rotation-stage parameters
                                 set on the problem (fm_set_params), with no
                                 relative poses, rotation initialisation or
                                 rotation steps -- e.g. rotations aligned on
                                 the raw matches of another problem, the
                                 translation and epipolar stages then run on
                                 this problem's (completed) keypoint pairs
                                 (Appendix "Tracks"); needs reestimate_rel_t
                                 or rel_t; loss_rotation is then NaN (0) */
} fm_solve_opts;

void fm_solve_opts_default(fm_solve_opts* opts);

/* Caller-owned host buffers for the solution, and scalars filled in. */
typedef struct {
  float* R;                   /* [N*9] world-to-camera rotations (required) */
  float* t;                   /* [N*3] world-to-camera translations (required) */
  float* points;              /* [T*3] or NULL (needs kp_track) */
  int32_t* point_valid;       /* [T] or NULL */
  int32_t n_tracks;           /* out: T */
  int32_t n_points_valid;     /* out */
  float loss_rotation;        /* out: final losses of the three stages
                                 (summed over the scenes of a batch) */
  float loss_translation;
  float loss_epipolar;
  int64_t n_kept;             /* out: keypoint pairs kept by the last filtering
                                 (all scenes) */
  int32_t* cam_valid;         /* [N] or NULL: 1 for the cameras of the largest
                                 connected component of their scene's view
                                 graph (the connectivity filter, Appendix
                                 "Global Rotation"), 0 for the others, whose
                                 poses nothing constrains */
} fm_result;

/* Runs the whole first-order pipeline (from unit weights: weights left by an
 * earlier call are cleared): fm_relative_poses (irls_iters 0, ea_delta) when
 * no relative rotations were given, fm_rotation_init, Adam on the rotation
 * loss, fm_relative_translations (if asked), trn_runs translation runs from
 * fm_translation_random_init, fm_translation_merge, a final translation run,
 * fm_epipolar_init_from_stages, ea_rounds of {fm_ea_reweight(tau_k, delta),
 * Adam on FM_EA_COMPACT} with tau_k = max(tau0 / 2^k, tau_min), and
 * triangulation.  Each Adam loop runs in four equal phases with the learning
 * rate scaled by 1, 0.3, 0.1, 0.03.  Needs rel_t when reestimate_rel_t is 0
 * and rel_R was given.  The solution is defined up to a similarity of the
 * world frame; it is reported in a fixed gauge, per scene: the first valid
 * camera (cam_valid) has R = I, and the valid cameras' centres have their
 * centroid at the origin and unit mean norm (Appendix "Multiple
 * Initializations" normalises the centres the same way).  The epipolar-stage
 * parameters are left in that gauge and the points are triangulated in it.
 * Divergence: each stage's final per-scene losses are checked on the host; a
 * non-finite one ends the solve with FM_ERR_NAN (fm_last_error names the
 * stage and the scene), and so do non-finite output poses.
 * Synchronises. */
fm_status fm_solve(fm_problem* problem, const fm_solve_opts* opts, fm_result* result);

/* ------------------------------------------------- learned inlier weights
 *
 * The paper handles outlier keypoint pairs with IRLS weights and a periodic
 * filter whose threshold decreases (Sec. 3.3, Eq. 9).  These calls add a
 * learned filter: a network predicts, per keypoint pair, the probability that
 * it is an inlier.  The paper has no learned component; the definitions
 * below are this library's.
 *
 * Features of keypoint pair m of image pair n = (i, j) at epipolar-stage
 * parameters (r_m = x~2^T E_n x~1, the residual of Eq. 7):
 *   f0 |r_m| / (mean over the pairs of n of |r| + 1e-12)
 *   f1 log1p(d_m), d_m the epipolar (Sampson) distance in pixels:
 *      ((f_i + f_j)/2) |r_m| / sqrt(a0^2 + a1^2 + b0^2 + b1^2), a = E x~1,
 *      b = E^T x~2
 *   f2 log(k_m), k_m = (1 + sqrt(1 + 8 c_m))/2 the track length from the
 *      number c_m of keypoint pairs of the track (0 without kp_track)
 *   f3 the angle (radians) between the viewing rays R_i^T x~1, R_j^T x~2
 *   f4 (|x~1[0:2]| + |x~2[0:2]|)/2, the keypoint radius (calibrated units)
 *   f5 the iteration fraction (given)
 *   f6 log(Z_n)
 *   f7 log1p(w_m)/log1p(1/delta), w_m the current weight (1 without weights)
 * Network: h1 = GELU(x W1 + b1) [64], h2 = GELU(h1 W2 + b2) [64],
 * o = h2 . w3 + b3, p = sigmoid(o), GELU exact (erf).  Parameters, float32,
 * flat: W1 [8][64] (feature-major), b1 [64], W2 [64][64] (input-major),
 * b2 [64], w3 [64], b3 [1].  The products run on the tensor cores with
 * bfloat16 operands (x, W1, h1, W2; in training also dz2 and dz1) and
 * float32 accumulation, inference and training alike on tcgen05
 * (accumulators in tensor memory). */
#define FM_MLP_N_PARAMS 4801
#define FM_MLP_N_FEATURES 8

/* Sets the problem's network parameters (NULL clears them). */
fm_status fm_mlp_set_params(fm_problem* problem, const float* theta, int32_t on_device);

/* At epipolar-stage parameters params_dev [N*9] (NULL: the stage's own) and
 * the problem's current weights: features into feat_dev [Z*8], the signed
 * residuals r_m into resid_dev [Z], and the inlier probabilities p_m into
 * prob_dev [Z] (needs the network parameters); any output may be NULL.
 * Device pointers, in the order of the keypoint pairs given at creation.
 * delta: the IRLS floor of f7 (> 0).  Asynchronous without prob_dev; with
 * it, synchronises and returns FM_ERR_TIMEOUT if a bounded wait of the
 * tensor-core kernel ran out. */
fm_status fm_mlp_eval(fm_problem* problem, const float* params_dev, float iter_frac, float delta,
                      float* feat_dev, float* resid_dev, float* prob_dev);

/* The same at the rotation stage's global rotations and the current relative
 * translations (E_n = [t^{i->j}]_x R_j R_i^T), before any camera centre is
 * known. */
fm_status fm_mlp_eval_relative(fm_problem* problem, float iter_frac, float delta, float* feat_dev,
                               float* resid_dev, float* prob_dev);

/* Early pruning: the pairs whose inlier probability at the global rotations
 * and current relative translations is below p_min get weight 0, the others
 * weight 1 (per-scene normalisers 1/kept); the relative translations can then
 * be re-estimated from the kept pairs (fm_relative_translations).
 * Synchronises. */
fm_status fm_mlp_prune(fm_problem* problem, float iter_frac, float delta, float p_min, int64_t* n_kept);

/* The learned counterpart of fm_ea_reweight: at the current epipolar-stage
 * parameters, keeps a pair when its predicted inlier probability is >= p_min
 * (instead of |eps^| < tau) and weights it 1/max(|eps^|, delta) when
 * irls != 0, else 1; normalisers, W_n and *n_kept as fm_ea_reweight.
 * Synchronises. */
fm_status fm_mlp_reweight(fm_problem* problem, float iter_frac, float delta, float p_min, int32_t irls,
                          int64_t* n_kept);

/* Trainer: the network's parameters and Adam state on the device, trained
 * on feature rows x [B][8] and labels y [B] in {0, 1} (device pointers) with
 * the mean binary cross-entropy mean(softplus(o) - y o).  Errors are
 * reported by fm_last_error(NULL).  Gradients are deterministic (fixed-order
 * sums, no atomics).  The loss and gradient run asynchronously: when a
 * bounded wait of the tensor-core kernel runs out, the loss is NaN (and so
 * are the parameters after a step), and the next fm_mlp_trainer_get_params
 * to the host or fm_mlp_trainer_forward returns FM_ERR_TIMEOUT. */
typedef struct fm_mlp_trainer fm_mlp_trainer;
fm_status fm_mlp_trainer_create(int64_t max_batch, void* cuda_stream, fm_mlp_trainer** out);
void fm_mlp_trainer_destroy(fm_mlp_trainer* trainer);
/* Sets the parameters (host or device) and resets Adam. */
fm_status fm_mlp_trainer_set_params(fm_mlp_trainer* trainer, const float* theta, int32_t on_device);
fm_status fm_mlp_trainer_get_params(fm_mlp_trainer* trainer, float* theta, int32_t on_device);
/* Loss into loss_dev [1] and gradient into grad_dev [4801] (either may be
 * NULL) at the current parameters.  Asynchronous. */
fm_status fm_mlp_trainer_loss_grad(fm_mlp_trainer* trainer, const float* x_dev, const float* y_dev, int64_t B,
                                   float* loss_dev, float* grad_dev);
/* One Adam step on the batch; loss_dev [1] (or NULL) receives the loss before
 * the step.  Asynchronous. */
fm_status fm_mlp_trainer_step(fm_mlp_trainer* trainer, const float* x_dev, const float* y_dev, int64_t B,
                              const fm_adam_opts* opts, float* loss_dev);
/* Logits o of feature rows x [B][8] into logit_dev [B], on the tcgen05
 * tensor cores (bf16 operands in shared memory, fp32 accumulators in tensor
 * memory).  Synchronises; FM_ERR_TIMEOUT if a bounded wait ran out. */
fm_status fm_mlp_trainer_forward(fm_mlp_trainer* trainer, const float* x_dev, int64_t B, float* logit_dev);

/* Launch configuration of the direct epipolar kernel (k_ea_direct). */
typedef struct {
  int32_t pairs_per_lane;      /* keypoint pairs per thread at most: 11, 15
                                  or 21
                                  (a thread's pairs never cross an image-pair
                                  end; a warp run is 32 threads' pairs) */
  int32_t ctas_per_sm;         /* persistent CTAs per SM; 0 = as many as fit */
  float us_per_eval;           /* fm_autotune: mean time of one evaluation
                                  with the chosen one */
} fm_tuning;

/* Sets / reads the configuration (changing pairs_per_lane rebuilds the
 * kernel's tables; synchronises).  Defaults: 15, 0. */
fm_status fm_set_tuning(fm_problem* problem, const fm_tuning* tuning);
fm_status fm_get_tuning(const fm_problem* problem, fm_tuning* tuning);

/* Autotuner: times one gradient evaluation of the direct L1 objective as
 * fm_step chains it -- the E tables, the direct kernel and the per-camera
 * pass with the loss -- at the problem's current weights and epipolar
 * parameters (or generated parameters when none are set), for the three
 * tiles and every CTA count per SM that fits, `repeats` times each (CTA
 * counts in round robin), every sample after an L2 flush and a 0.2 ms device
 * idle, and keeps the configuration with the lowest mean time (event
 * timestamps come in steps of about 2 us on the B300, so single fastest
 * samples tie).  The whole chain is timed because the direct kernel's
 * configuration also sets how the next launch overlaps its end.  The loss
 * chosen by fm_ea_set_loss is left as it was.  The choice changes no result
 * beyond the order of additions inside an image pair's records.
 * Synchronises. */
fm_status fm_autotune(fm_problem* problem, int32_t repeats, fm_tuning* best);

/* fm_step replays captured CUDA graphs of 16 iterations (one graph launch
 * instead of every kernel launch of the 16 iterations) whenever per-kernel
 * timing and the loss trace are off; the results are identical either way.
 * enable = 0 launches every kernel from the host.  Default on. */
fm_status fm_graphs_enable(fm_problem* problem, int32_t enable);

/* Focal lengths inside epipolar adjustment (Sec. 3.3, last paragraph of
 * "Epipolar Adjustment": the focal lengths folded into the matrices, which
 * become fundamental matrices).  phi_dev [N]: a log focal ratio per camera,
 * f_c = f0_c exp(phi_c) with f0 the focal lengths the problem's keypoints are
 * calibrated at; the objective is the direct one (the problem's loss, L1 or
 * L2, and weights) at E'_n = S_j E_n S_i, S_c = diag(e^-phi_c, e^-phi_c, 1).
 * Forward: loss_dev as fm_ea_forward, dlde_saved [P*9] (16-byte aligned)
 * receives dL/dE'_n.  Backward: grad_dev [N*9] the poses' gradient (chain
 * rule through dL/dE_n = S_j dL/dE'_n S_i), grad_phi_dev [N]
 * dL/dphi_c = -s_c sum over the camera's image pairs of <dL/dE', S_j E D>
 * (camera i) or <dL/dE', D E S_i> (camera j), D = diag(1, 1, 0), summed in a
 * fixed order; grad_loss_dev [S] (or NULL) scales both.  All pointers are
 * device pointers; no synchronisation.  With free focal lengths this
 * objective drifts under pixel noise (smaller calibrated coordinates give
 * smaller algebraic residuals): an option, not the default solve. */
fm_status fm_ea_focal_forward(fm_problem* problem, const float* params_dev, const float* phi_dev, float* loss_dev,
                              float* dlde_saved);
fm_status fm_ea_focal_backward(fm_problem* problem, const float* params_dev, const float* phi_dev,
                               const float* dlde_saved, const float* grad_loss_dev, float* grad_dev,
                               float* grad_phi_dev);

/* ---------------------------------------------------------- observability
 * (no counterpart in the paper, which times whole stages by wall clock) */

/* Per-kernel device time: with timing on, the library records a CUDA event
 * pair around every kernel it launches (on its stream) and accumulates the
 * elapsed time per kernel name; timed kernels are launched without
 * programmatic dependent launch, so that each pair brackets exactly one
 * kernel (results are identical).  Enabling or disabling resets the
 * counters. */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
} fm_kernel_time;

fm_status fm_timing_enable(fm_problem* problem, int32_t enable);

/* Writes up to capacity entries (one per kernel name launched since timing
 * was enabled) and their count to *count.  Synchronises the stream. */
fm_status fm_timing_read(fm_problem* problem, fm_kernel_time* out, int32_t capacity,
                         int32_t* count);

/* Loss trace: with every > 0, fm_step also reduces the loss (fixed order, on
 * the device, no host synchronisation) every `every` iterations into a ring
 * of `capacity` values; every = 0 turns it off and clears the ring. */
fm_status fm_track_loss(fm_problem* problem, int32_t every, int32_t capacity);

/* Copies the most recent min(capacity, recorded) traced losses, oldest
 * first, into out and their number into *count (for the translation stage,
 * the loss of run 0).  Synchronises the stream. */
fm_status fm_loss_history(fm_problem* problem, float* out, int32_t capacity, int32_t* count);

/* ----------------------------------------------- allocation-free evaluation
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory when they evaluate -- code running under
 * another framework's allocator or memory pool that forbids cudaMalloc,
 * latency-critical loops where an allocation could block or fail, and
 * deployments that must keep a fixed, known footprint.
 *
 * fm_ea_loss_grad_static evaluates the direct epipolar loss of
 * fm_loss_grad's FM_STAGE_EPIPOLAR -- the mean over keypoint pairs of the
 * (optionally weighted) absolute algebraic epipolar error for FM_EA_L1, or of
 * its square for FM_EA_L2 -- and its gradient, with the same kernels as
 * fm_loss_grad, without creating a problem and without allocating anything:
 * its temporary tables live in one 16 MiB array of device memory that the
 * library holds on every GPU that loads it, until the process exits.
 *
 * Inputs (device pointers, read only; kp_dev and weights_dev 16-byte aligned):
 *   kp_dev       [Z] float4 (x1, y1, x2, y2): calibrated coordinates
 *                K^-1 [u, v, 1]^T of the keypoint in image i_n and in j_n,
 *                grouped by image pair in index order
 *   seg_off_dev  [P+1] first keypoint pair of each image pair: seg_off[0] =
 *                0, non-decreasing, seg_off[P] = Z (checked on the device,
 *                see Errors)
 *   pair_i_dev, pair_j_dev  [P] camera indices of each image pair, in
 *                [0, n_cams) (not checked: an index outside it reads outside
 *                params_dev)
 *   params_dev   [N*9] epipolar-stage parameters (6D rotation, t)
 *   weights_dev  [Z] per-pair weights, or NULL for unit weights
 * loss: FM_EA_L1 or FM_EA_L2; inv_z: the 1/Z normaliser.
 * Outputs (device pointers, caller-owned):
 *   loss_dev      [1] the loss
 *   pair_grad_dev [P*24] per image pair: dL/dR_i (9, row-major), dL/dt_i
 *                 (3), dL/dR_j (9), dL/dt_j (3) -- the caller sums them per
 *                 camera (and applies the 6D adjoint for rotations)
 * cuda_stream: the stream to enqueue on (NULL = default); the call returns
 * after enqueueing.
 *
 * Errors: arguments are checked on the host (FM_ERR_INVALID_ARG with a
 * message from fm_last_error(NULL), before any GPU work).  What only the
 * kernels can see is reported through the loss, since the call does not wait
 * for them: when seg_off_dev is not a CSR table of Z pairs (then no keypoint
 * pair is read and the gradient blocks are zero) or when a bounded wait of
 * the direct kernel runs out (the sums are then incomplete), *loss_dev is
 * NaN.  Check the loss before using the gradient.
 *
 * Limits and sharing: the tables need about 118 B per image pair plus 0.4 B
 * per keypoint pair; a problem that does not fit in 16 MiB (118 P + 0.4 Z
 * beyond 16.7M) is rejected with FM_ERR_INVALID_ARG before any GPU work.
 * Every call on a device shares the one array and leaves its contents
 * behind; each call clears the words that must start at zero (its error
 * word and an arrival counter) and writes every other entry before reading
 * it.  Calls whose GPU work
 * overlaps (two streams, or two host threads) race on the array: serialise
 * them.  The first call on each device looks up the array's device address
 * and sets the kernel's shared-memory limit on that device; make that first
 * call before any stream capture. */
fm_status fm_ea_loss_grad_static(const float* kp_dev, const int32_t* seg_off_dev,
                                 const int32_t* pair_i_dev, const int32_t* pair_j_dev,
                                 const float* params_dev, const float* weights_dev,
                                 int32_t n_cams, int32_t n_img_pairs, int64_t n_kp_pairs,
                                 int32_t loss, float inv_z, float* loss_dev,
                                 float* pair_grad_dev, void* cuda_stream);

#ifdef __cplusplus
}  /* extern "C" */
#endif

#endif /* FASTMAP_H */
