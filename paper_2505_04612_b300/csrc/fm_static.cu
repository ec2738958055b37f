// Allocation-free evaluation of the direct epipolar loss and gradient.
//
// Some callers cannot allocate device memory at the point where they need an
// evaluation: code running inside another framework's memory pool or a
// custom allocator that forbids cudaMalloc, real-time loops where an
// allocation could stall or fail, and callers that must keep a fixed memory
// footprint.  fm_ea_loss_grad_static serves them: it evaluates the same
// kernels as fm_loss_grad's direct path, but every temporary table lives in
// one fixed-size array of device memory that belongs to this library and
// exists on every GPU that loads it, from load until process exit.
//
// The array is shared by every call on a device and keeps whatever the last
// call wrote.  Each call writes every table entry it later reads, and clears
// the words that must start at zero (its error word and the loss slices'
// arrival counter) with a small kernel on the stream.  Two calls whose GPU
// work overlaps in time (different streams,
// or different host threads) race on the array and corrupt each other's
// results; order such calls on one stream or synchronise between them.
//
// The call never waits for the GPU, so it cannot return a status for what the
// kernels find: a keypoint-pair offset table that is not a CSR table of Z
// pairs (checked before any keypoint is read; the lane tables are then left
// empty, so nothing is read past the caller's arrays) or a bounded wait of
// the direct kernel that ran out.  Either one makes the loss NaN.
#include <mutex>

#include "fm_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;   // 16 MiB per GPU

static __device__ __align__(256) unsigned char g_ea_scratch[kStaticScratchBytes];

std::mutex g_addr_mutex;
void* g_addr[256] = {};   // device address of g_ea_scratch, per device ordinal

fm_status static_fail(fm_status st, const std::string& msg) {
  fm::set_thread_error(msg);   // reported by fm_last_error(NULL)
  return st;
}

// Looks up the array's device address once per device, with that device
// current.  In host code the name g_ea_scratch is only a host-side stand-in;
// kernels must be given this address instead.
cudaError_t scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_ea_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return cudaSuccess;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// clears the error word and the arrival counter, writes the slice table of
// one scene of P image pairs
__global__ void k_static_init(int* err, int* lsl, int P, int n_slices) {
  const int t = threadIdx.x;
  if (t == 0) {
    *err = 0;
    lsl[0] = 0;
    lsl[1] = P;
    lsl[2] = 0;
    lsl[3] = n_slices;
  }
  lsl[4 + t] = 0;   // the counter's line (32 ints)
}

// the loss becomes NaN when a kernel of the call raised an error bit
__global__ void k_nan_on_error(const int* err, float* loss) {
  if (*err != 0) *loss = __int_as_float(0x7fc00000);
}

}  // namespace

extern "C" {

fm_status fm_ea_loss_grad_static(const float* kp_dev, const int32_t* seg_off_dev,
                                 const int32_t* pair_i_dev, const int32_t* pair_j_dev,
                                 const float* params_dev, const float* weights_dev, int32_t n_cams,
                                 int32_t n_img_pairs, int64_t n_kp_pairs, int32_t loss, float inv_z,
                                 float* loss_dev, float* pair_grad_dev, void* cuda_stream) {
  if (!seg_off_dev || !pair_i_dev || !pair_j_dev || !params_dev || !loss_dev || !pair_grad_dev)
    return static_fail(FM_ERR_INVALID_ARG, "a required pointer is NULL");
  if (n_kp_pairs > 0 && !kp_dev) return static_fail(FM_ERR_INVALID_ARG, "kp_dev is NULL");
  if (n_cams < 2 || n_img_pairs < 1 || n_kp_pairs < 0 || n_kp_pairs >= (int64_t(1) << 31) - (int64_t(1) << 20))
    return static_fail(FM_ERR_INVALID_ARG, "sizes out of range");
  if (loss != FM_EA_L1 && loss != FM_EA_L2) return static_fail(FM_ERR_INVALID_ARG, "loss must be FM_EA_L1 or FM_EA_L2");
  if (!(inv_z >= 0.f)) return static_fail(FM_ERR_INVALID_ARG, "inv_z must be >= 0");
  if ((reinterpret_cast<uintptr_t>(kp_dev) | reinterpret_cast<uintptr_t>(weights_dev)) & 15u)
    return static_fail(FM_ERR_INVALID_ARG, "kp_dev and weights_dev must be 16-byte aligned");
  const int P = n_img_pairs;
  const int64_t Z = n_kp_pairs;
  // lanes in use <= sum_n max(1, ceil(m_n / U)) <= ceil(Z / U) + P; the warp
  // runs past the lanes in use are empty.  Records: at most one per (warp
  // run, image pair it touches) <= P - 1 + n_wruns
  constexpr int U = fm::kEaPairsPerLane;
  const int64_t lanes_max = (Z + U - 1) / U + P;
  const int n_wruns = Z > 0 ? (int)((lanes_max + 31) / 32) : 0;
  const size_t b_tab = align256(sizeof(float4) * 3 * (size_t)P);
  const size_t b_run = align256(sizeof(int) * 32 * (size_t)n_wruns);
  const size_t b_info = align256(sizeof(int4) * (size_t)n_wruns);
  const size_t b_srec = align256(sizeof(int) * 2 * (size_t)P);
  const size_t b_rec = align256(sizeof(float4) * 3 * ((size_t)P + (size_t)n_wruns));
  const size_t b_loss = align256(sizeof(float) * (size_t)P);
  const size_t b_g = align256(sizeof(int) * ((size_t)P + 2));
  const size_t b_total = align256(sizeof(long long) + sizeof(int));
  // the loss slices of one scene: slice table, slice sums, arrival counter
  const int n_slices = (P + fm::kLossSlice - 1) / fm::kLossSlice;
  const size_t b_lsl = align256(sizeof(int) * (4 + fm::kLossCntStride) + sizeof(float) * (size_t)n_slices);
  const size_t need = b_tab + b_run + b_info + b_srec + b_rec + b_loss + b_g + b_total + b_lsl;
  if (need > kStaticScratchBytes)
    return static_fail(FM_ERR_INVALID_ARG,
                       "problem needs " + std::to_string(need) + " bytes of scratch; the static array holds " +
                           std::to_string(kStaticScratchBytes) + " (use fm_problem_create for larger problems)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  void* base = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &base);
  if (e != cudaSuccess) return static_fail(FM_ERR_CUDA, std::string("scratch address: ") + cudaGetErrorString(e));
  unsigned char* p = static_cast<unsigned char*>(base);

  // a problem view whose tables point into the static array (no allocation)
  fm_problem v;
  v.device = dev;
  v.N = n_cams;
  v.P = P;
  v.Z = Z;
  v.stream = (cudaStream_t)cuda_stream;
  e = cudaDeviceGetAttribute(&v.sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return static_fail(FM_ERR_CUDA, cudaGetErrorString(e));
  v.kp = reinterpret_cast<float4*>(const_cast<float*>(kp_dev));
  v.seg_off = const_cast<int*>(seg_off_dev);
  v.pair_i = const_cast<int*>(pair_i_dev);
  v.pair_j = const_cast<int*>(pair_j_dev);
  v.seg_tab = reinterpret_cast<float4*>(p);
  p += b_tab;
  v.lane_desc = reinterpret_cast<int*>(p);
  p += b_run;
  v.wrun_info = reinterpret_cast<int4*>(p);
  p += b_info;
  v.seg_rec = reinterpret_cast<int*>(p);
  p += b_srec;
  v.rec = reinterpret_cast<float4*>(p);
  p += b_rec;
  v.seg_loss = reinterpret_cast<float*>(p);
  p += b_loss;
  int* G = reinterpret_cast<int*>(p);   // [P+1] lane scan, then the lanes in use
  int* T = G + P + 1;
  p += b_g;
  long long* total = reinterpret_cast<long long*>(p);
  v.d_err = reinterpret_cast<int*>(total + 1);   // error bits of this call (made a NaN loss at the end)
  p += b_total;
  int* lsl = reinterpret_cast<int*>(p);          // {0, P} {0, n_slices}, counter, slice sums
  fm::LossArgs la;
  la.sc_pair_off = lsl;
  la.sc_slice_off = lsl + 2;
  la.S = 1;
  la.n_slices = n_slices;
  la.cnt = lsl + 4;
  la.partial = reinterpret_cast<float*>(lsl + 4 + fm::kLossCntStride);
  la.out = loss_dev;
  la.out2 = nullptr;
  v.seg_grad = pair_grad_dev;
  v.n_wruns = n_wruns;
  cudaStream_t s = v.stream;

  // inside a caller's stream capture the launches must be plain ones (see
  // launch_pdl); the query is on the caller's own stream
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (s != nullptr && cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusNone;
  }
  const bool was = fm::g_capturing;
  fm::g_capturing = was || cap == cudaStreamCaptureStatusActive;
  fm::g_plain_once = true;
  // the words that must start at zero (error bits, arrival counter) and the
  // slice table of this call
  k_static_init<<<1, 32, 0, s>>>(v.d_err, lsl, P, n_slices);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    fm::g_capturing = was;
    return static_fail(FM_ERR_CUDA, std::string("initialising the array: ") + cudaGetErrorString(e));
  }
  fm::launch_ea_tables(params_dev, v.pair_i, v.pair_j, v.seg_off, P, v.seg_tab, nullptr, s);
  // the offsets are validated before any lane table is built from them
  fm::launch_lane_scan(v.seg_off, P, U, G, T, s, Z, v.d_err);
  if (n_wruns > 0) {
    fm::launch_lane_desc(v.seg_off, G, T, P, U, n_wruns, v.lane_desc, v.wrun_info, s);
    fm::launch_exclusive_scan_info(v.wrun_info, n_wruns, reinterpret_cast<int64_t*>(total), s);
  }
  fm::launch_seg_records(v.seg_off, G, v.wrun_info, P, v.seg_rec, s);
  if (n_wruns > 0) fm::launch_ea_direct(&v, weights_dev, loss, s);
  fm::SegArgs sa = fm::seg_args(&v, params_dev);
  sa.pair_scale = nullptr;   // one scene: the scalar normaliser
  sa.g_scale = (loss == FM_EA_L1) ? inv_z : 2.f * inv_z;
  sa.l_scale = inv_z;
  fm::launch_ea_segments(sa, s);
  fm::launch_sum_fixed(v.seg_loss, P, 1, la, s);
  k_nan_on_error<<<1, 1, 0, s>>>(v.d_err, loss_dev);
  fm::g_capturing = was;
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(FM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return FM_OK;
}

}  // extern "C"
