// The inlier network's forward pass on the fifth-generation tensor cores
// (tcgen05): bf16 operands in shared memory, fp32 accumulators in tensor
// memory (TMEM), one thread issuing the MMAs, completion through an mbarrier.
//
// A CTA of 128 threads evaluates tiles of 128 rows (M = 128) — feature rows
// from memory, or keypoint pairs whose features it computes itself:
//   layer 1   D1[128 x 64] = X[128 x 16] W1^T   (features padded to K = 16),
//   layer 2   D2[128 x 64] = H1[128 x 64] W2^T  (four K = 16 steps),
// each a tcgen05.mma.kind::f16 with M = 128, N = 64.  Thread t owns row t:
// it writes its features into the A tile, reads its row of D1 from TMEM
// (tcgen05.ld 32x32b: warp w reaches lanes 32w..32w+31), applies bias and
// GELU, writes its bf16 row of H1, and after layer 2 forms o = GELU(D2 + b2).w3
// + b3 in registers.  Operands use the K-major layout without swizzling:
// 8-row x 16-byte core matrices, LBO = stride between core matrices along K,
// SBO = stride between 8-row groups.  W1^T, W2^T are staged once per CTA.
//
// TMEM: 64 columns per CTA; D2 reuses D1's columns (every thread has read
// its row of D1 before the layer-2 MMA is issued).  The CTA's dynamic shared
// memory is sized so that at most seven CTAs share an SM (7 x 64 = 448 of the
// 512 columns), so an allocation never waits for another CTA.
// Waits on the mbarrier are bounded: past the bound the kernel records
// kErrMlpTimeout, skips the rest of its work, and still frees its TMEM.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>

#include "fm_device.cuh"
#include "fm_internal.h"
#include "fm_mlp.cuh"

namespace fm {
namespace {

constexpr int kRows = 128;   // M
constexpr int kN = 64;       // N of both layers
constexpr int kTmemCols = 64;
constexpr int kCtasPerSm = 7;
constexpr long kWaitBound = 1L << 22;   // polls of the mbarrier before giving up

// shared-memory layout (bytes), K-major no-swizzle core-matrix tiles
constexpr int kA1 = 0;                         // X   128 x 16: SBO 256, LBO 128      4 KB
constexpr int kB1 = kA1 + 4096;                // W1^T 64 x 16: SBO 256, LBO 128      2 KB
constexpr int kA2 = kB1 + 2048;                // H1  128 x 64: SBO 1024, LBO 128    16 KB
constexpr int kB2 = kA2 + 16384;               // W2^T 64 x 64: SBO 1024, LBO 128     8 KB
constexpr int kPar = kB2 + 8192;               // b1, b2, w3 (fp32), b3            772 B
constexpr int kBar = kPar + 1024;              // mbarrier (8 B) + TMEM address (4 B)
constexpr int kSmemUsed = kBar + 64;
// padded so that shared memory (227 KB per SM for CTAs, 1 KB reserved per
// CTA) admits at most kCtasPerSm CTAs per SM; registers (64 x 128 threads)
// admit at most 8 in any case, and 8 x 64 columns fit the 512 of TMEM
constexpr int kSmemDyn = 232448 / kCtasPerSm - 1024;
static_assert(8 * kTmemCols <= 512, "TMEM columns of the resident CTAs");

// byte offset of element (row r, k) in a K-major no-swizzle tile
__device__ __forceinline__ int core_off(int r, int k, int sbo) {
  return (r >> 3) * sbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// UMMA shared-memory descriptor: start >> 4 [0,14), LBO >> 4 [16,30),
// SBO >> 4 [32,46), version 1 [46,48), layout 0 (no swizzle) [61,64)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: D f32 [4,6) = 1, A bf16 [7,10) = 1,
// B bf16 [10,13) = 1, both K-major, N >> 3 at [17,23), M >> 4 at [24,29)
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate,
                                     uint32_t idesc = kIdesc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

// returns false when the bound runs out
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (long i = 0; i < kWaitBound; ++i) {
    uint32_t done = 0;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// v[0..15] into this warp's lanes, columns taddr .. taddr + 15; returns
// after the stores are done
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ float gelu_tc(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ void store_bf16x8(unsigned char* base, int off, const float* v) {
  __nv_bfloat162 h[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
  *reinterpret_cast<uint4*>(base + off) = *reinterpret_cast<const uint4*>(h);
}

// Forward pass of rows [0, a.Z): PAIRS computes each keypoint pair's features
// (written to a.feat / a.resid when given), otherwise rows come from a.x
// [Z][8]; logits and probabilities go to a.logit / a.prob when given.
// err: error bits.
template <bool PAIRS>
__global__ void __launch_bounds__(kRows, 1) k_mlp_forward_tc(InferArgs a, int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const float* theta = a.theta;
  const int64_t B = a.Z;
  const float* W1 = theta;          // [8][64]
  const float* b1 = theta + 512;
  const float* W2 = theta + 576;    // [64][64]
  const float* b2 = theta + 4672;
  const float* w3 = theta + 4736;
  float* par = reinterpret_cast<float*>(sm + kPar);
  // ---- stage W1^T (64 x 16, features 8..15 zero) and W2^T (64 x 64) as bf16
  for (int idx = tid; idx < kN * 16; idx += kRows) {
    const int n = idx >> 4, k = idx & 15;
    const float v = k < 8 ? W1[k * kN + n] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(sm + kB1 + core_off(n, k, 256)) = __float2bfloat16_rn(v);
  }
  for (int idx = tid; idx < kN * kN; idx += kRows) {
    const int n = idx >> 6, k = idx & 63;
    *reinterpret_cast<__nv_bfloat16*>(sm + kB2 + core_off(n, k, 1024)) = __float2bfloat16_rn(W2[k * kN + n]);
  }
  for (int k = tid; k < kN; k += kRows) {
    par[k] = b1[k];
    par[kN + k] = b2[k];
    par[2 * kN + k] = w3[k];
  }
  if (tid == 0) par[3 * kN] = theta[4800];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kBar + 8);
  const uint32_t bar_a = smem_u32(bar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");   // visible to the async proxy
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;   // TMEM lane field of this warp's rows
  const uint32_t a1 = smem_u32(sm + kA1), b1s = smem_u32(sm + kB1);
  const uint32_t a2 = smem_u32(sm + kA2), b2s = smem_u32(sm + kB2);
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t tile = blockIdx.x; tile * kRows < B; tile += gridDim.x) {
    const int64_t row = tile * kRows + tid;
    // ---- this thread's features into row tid of X (8 features + 8 zeros)
    float f[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) f[k] = 0.f;
    if (row < B) {
      if (PAIRS) {
        float r;
        pair_features(a, row, f, r);
        if (a.feat && ((uintptr_t)a.feat & 15) == 0) {
          float4* fo = reinterpret_cast<float4*>(a.feat + row * 8);
          fo[0] = make_float4(f[0], f[1], f[2], f[3]);
          fo[1] = make_float4(f[4], f[5], f[6], f[7]);
        } else if (a.feat) {
#pragma unroll
          for (int k = 0; k < 8; ++k) a.feat[row * 8 + k] = f[k];
        }
        if (a.resid) a.resid[row] = r;
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) f[k] = a.x[row * 8 + k];
      }
    }
    store_bf16x8(sm + kA1, core_off(tid, 0, 256), f);
    store_bf16x8(sm + kA1, core_off(tid, 8, 256), f + 8);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0 && ok) {
      umma(tmem, smem_desc(a1, 128, 256), smem_desc(b1s, 128, 256), 0u);
      umma_commit(bar_a);
    }
    ok = ok && bar_wait(bar_a, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) break;   // a wait ran out: stop, free TMEM below
    fence_after();
    // ---- row tid of D1 -> bias, GELU -> bf16 row of H1
#pragma unroll 1
    for (int c = 0; c < kN; c += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)c, v);
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = gelu_tc(v[k] + par[c + k]);
      store_bf16x8(sm + kA2, core_off(tid, c, 1024), v);
      store_bf16x8(sm + kA2, core_off(tid, c + 8, 1024), v + 8);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0 && ok) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        umma(tmem, smem_desc(a2 + 256 * kk, 128, 1024), smem_desc(b2s + 256 * kk, 128, 1024),
             kk > 0 ? 1u : 0u);
      umma_commit(bar_a);
    }
    ok = ok && bar_wait(bar_a, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) break;
    fence_after();
    // ---- row tid of D2 -> bias, GELU, . w3 + b3
    float o = 0.f;
#pragma unroll 1
    for (int c = 0; c < kN; c += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)c, v);
#pragma unroll
      for (int k = 0; k < 16; ++k) o = fmaf(gelu_tc(v[k] + par[kN + c + k]), par[2 * kN + c + k], o);
    }
    if (row < B) {
      o += par[3 * kN];
      if (a.logit) a.logit[row] = o;
      if (a.prob) a.prob[row] = 1.f / (1.f + expf(-o));
    }
    fence_before();
    __syncthreads();   // the tiles and TMEM columns are rewritten by the next tile
    fence_after();
  }
  if (!ok) {
    // a wait ran out: record it, give the MMAs in flight one more bounded
    // wait on the parity they complete, then free TMEM as usual
    atomicOr(err, kErrMlpTimeout);
    bar_wait(bar_a, phase ^ 1u);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

template <bool PAIRS>
void launch_tc(const InferArgs& a, int* err, int sm_count, cudaStream_t s) {
  if (a.Z == 0) return;
  // resident CTAs per SM, bound by shared memory; the shared-memory limit is
  // a per-device setting, so both are kept per device
  static std::atomic<int> per_sm_dev[64];
  int dev = 0;
  cudaGetDevice(&dev);
  const int slot = (dev >= 0 && dev < 64) ? dev : 0;
  int per_sm = per_sm_dev[slot].load();
  if (per_sm == 0) {
    cudaFuncSetAttribute(k_mlp_forward_tc<PAIRS>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDyn);
    int smem_sm = 0, reserved = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    per_sm = std::max(1, std::min(kCtasPerSm, smem_sm / (kSmemDyn + reserved)));
    per_sm_dev[slot].store(per_sm);
  }
  static_assert(kSmemUsed <= kSmemDyn, "shared memory layout");
  const int64_t tiles = (a.Z + kRows - 1) / kRows;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)sm_count * per_sm);
  k_mlp_forward_tc<PAIRS><<<(unsigned)grid, kRows, kSmemDyn, s>>>(a, err);
}

// ---------------------------------------------------------------- training
//
// k_mlp_grad_tc: the binary cross-entropy loss of a batch and its gradient
// with respect to the 4801 parameters, every contraction on tcgen05.  A
// persistent CTA of 128 threads takes tiles of 128 rows; thread t owns row t
// (TMEM lane t).  Per tile, five MMA groups, each completing on the CTA's
// mbarrier:
//   layer 1   D[0:64)    = X W1^T                  (M 128, N 64, K 16)
//   layer 2   D[64:128)  = H1 W2^T                 (M 128, N 64, K 64)
//   dh1       D[64:128)  = dZ2 W2                  (M 128, N 64, K 64)
//   weights   DW[0:128) += RT^T GT over the tile's rows  (M 128, N 128, K 128)
// RT and GT are the tile's two row-major bf16 tiles, 128 rows x 128 entries,
// 8-row groups 2048 B apart and 8-entry groups 128 B apart: RT holds h1
// (entries 0..63), x (64..71) and zeros (72..127), GT holds dz2 (0..63) and
// dz1 (64..127).  Read with K along a row (K-major: LBO 128, SBO 2048) they
// are the A operands of the forward and dh1 MMAs; read with K down the rows
// (MN-major: LBO 2048, SBO 128) they are both operands of the weight MMA,
// whose accumulator DW (128 TMEM columns, kept across the CTA's tiles) holds
// dW2 = h1^T dz2 in rows 0..63, columns 0..63 and dW1 = x^T dz1 in rows
// 64..71, columns 64..127; its other blocks are not used.
// The operands rounded to bf16 are those of the oracle's definition: x, W1,
// h1, W2 forward, dz2 and dz1 backward (with W2 and x, h1).  Each layer's
// pre-activations are read from TMEM once, and one erf and one exp per
// element give both GELU and GELU': h1 goes to RT and GELU'(z1) replaces z1
// in TMEM; h2 stays in registers (the logit, then dw3 once dl is known) and
// GELU'(z2) replaces z2 until dz2 = dl w3 GELU'(z2) is formed.  The bias gradients and dw3 are fp32 sums over the rows:
// per warp, a fixed butterfly that leaves column c of each 16-column chunk in
// lanes 2c, 2c + 1, accumulated over tiles per lane, then added over warps
// in warp order.  Per-CTA partials are summed in CTA order by k_mlp_reduce:
// the gradient is deterministic.
// Shared memory is sized for at most two CTAs per SM (2 x 256 TMEM columns).
constexpr int kTrCtasPerSm = 2;
constexpr int kTrTmemCols = 256;
constexpr int kTrRT = 0;                          // 32 KB
constexpr int kTrGT = kTrRT + 32768;              // 32 KB
constexpr int kTrW1T = kTrGT + 32768;             // W1^T 64 x 16, SBO 256     2 KB
constexpr int kTrW2T = kTrW1T + 2048;             // W2^T 64 x 64, SBO 1024    8 KB
constexpr int kTrW2 = kTrW2T + 8192;              // W2   64 x 64, SBO 1024    8 KB
constexpr int kTrPar = kTrW2 + 8192;              // b1, b2, w3, b3 (fp32)
constexpr int kTrRed = kTrPar + 1024;             // [4 warps][3][64] + [4][2] floats
constexpr int kTrBar = kTrRed + 4 * 3 * 64 * 4 + 64;
constexpr int kTrSmemUsed = kTrBar + 64;
constexpr int kTrSmemDyn = 232448 / kTrCtasPerSm - 1024;
static_assert(kTrSmemUsed <= kTrSmemDyn, "shared memory layout of the training kernel");
static_assert(kTrCtasPerSm * kTrTmemCols <= 512, "TMEM columns of the resident training CTAs");
constexpr int kTrPartStride = kMlpParams + 3;     // the layout of the per-CTA partials (+ loss)
constexpr int kTrMaxCtas = 148 * kTrCtasPerSm;
// weight MMA: M = 128, N = 128, A and B MN-major (transpose bits 15, 16)
constexpr uint32_t kIdescW = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                             ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);

// byte offset of entry (row r, e) in an RT / GT tile
__device__ __forceinline__ int rt_off(int r, int e) { return (r >> 3) * 2048 + (e >> 3) * 128 + (r & 7) * 16 + (e & 7) * 2; }

// GELU(z) = z Phi(z) (as gelu_tc) and GELU'(z) = Phi(z) + z phi(z), from one erf
__device__ __forceinline__ void gelu_both(float z, float& h, float& g) {
  const float e = erff(z * 0.70710678118654752f);
  h = 0.5f * z * (1.f + e);
  g = 0.5f * (1.f + e) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// the sum over the warp's lanes of v[0..15]; lane l returns the sum of
// v[(l >> 1) & 15] (a fixed tree: halves exchanged at lane distances 16, 8,
// 4, 2, then the pair at distance 1)
__device__ __forceinline__ float col_sum16(const float* v) {
  const int lane = threadIdx.x & 31;
  float a[8], b[4], c[2];
  bool hi = lane & 16;
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = (hi ? v[j + 8] : v[j]) + __shfl_xor_sync(0xffffffffu, hi ? v[j] : v[j + 8], 16);
  hi = lane & 8;
#pragma unroll
  for (int j = 0; j < 4; ++j) b[j] = (hi ? a[j + 4] : a[j]) + __shfl_xor_sync(0xffffffffu, hi ? a[j] : a[j + 4], 8);
  hi = lane & 4;
#pragma unroll
  for (int j = 0; j < 2; ++j) c[j] = (hi ? b[j + 2] : b[j]) + __shfl_xor_sync(0xffffffffu, hi ? b[j] : b[j + 2], 4);
  hi = lane & 2;
  const float d = (hi ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, hi ? c[0] : c[1], 2);
  return d + __shfl_xor_sync(0xffffffffu, d, 1);
}

struct TrainArgs {
  const float* theta;
  const float* x;   // [B][8]
  const float* y;   // [B]
  int64_t B;
  float inv_b;
  float* partial;   // [gridDim.x][kTrPartStride]
};

__global__ void __launch_bounds__(kRows, 1) k_mlp_grad_tc(TrainArgs a, int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float* theta = a.theta;
  float* par = reinterpret_cast<float*>(sm + kTrPar);   // b1 [0,64), b2 [64,128), w3 [128,192), b3 [192]
  // ---- weights as bf16 tiles, parameters, and the zero entries of RT
  for (int idx = tid; idx < kN * 16; idx += kRows) {
    const int n = idx >> 4, k = idx & 15;
    const float v = k < 8 ? theta[k * kN + n] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(sm + kTrW1T + core_off(n, k, 256)) = __float2bfloat16_rn(v);
  }
  for (int idx = tid; idx < kN * kN; idx += kRows) {
    const int n = idx >> 6, k = idx & 63;
    const float* W2 = theta + 576;
    *reinterpret_cast<__nv_bfloat16*>(sm + kTrW2T + core_off(n, k, 1024)) = __float2bfloat16_rn(W2[k * kN + n]);
    *reinterpret_cast<__nv_bfloat16*>(sm + kTrW2 + core_off(n, k, 1024)) = __float2bfloat16_rn(W2[n * kN + k]);
  }
  for (int k = tid; k < kN; k += kRows) {
    par[k] = theta[512 + k];
    par[kN + k] = theta[4672 + k];
    par[2 * kN + k] = theta[4736 + k];
  }
  if (tid == 0) par[3 * kN] = theta[4800];
  {
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int g = 9; g < 16; ++g) *reinterpret_cast<uint4*>(sm + kTrRT + rt_off(tid, 8 * g)) = z;
  }
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kTrBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kTrBar + 8);
  const uint32_t bar_a = smem_u32(bar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTrTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t rt = smem_u32(sm + kTrRT), gt = smem_u32(sm + kTrGT);
  const uint32_t w1t = smem_u32(sm + kTrW1T), w2t = smem_u32(sm + kTrW2T), w2 = smem_u32(sm + kTrW2);
  unsigned char* my_rt = sm + kTrRT + rt_off(tid, 0);   // entry group g of this row at + 128 g
  unsigned char* my_gt = sm + kTrGT + rt_off(tid, 0);
  float acc_b1[4] = {0.f, 0.f, 0.f, 0.f}, acc_b2[4] = {0.f, 0.f, 0.f, 0.f}, acc_w3[4] = {0.f, 0.f, 0.f, 0.f};
  float db3 = 0.f, lsum = 0.f;
  uint32_t phase = 0;
  bool ok = true;
  int n_tiles = 0;
  for (int64_t tile = blockIdx.x; tile * kRows < a.B; tile += gridDim.x, ++n_tiles) {
    const int64_t row = tile * kRows + tid;
    const bool valid = row < a.B;
    float f[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) f[k] = 0.f;
    float y = 0.f;
    if (valid) {
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] = a.x[row * 8 + k];
      y = a.y[row];
    }
    // the previous tile's weight MMA reads RT and GT: wait for it
    if (n_tiles > 0) {
      ok = ok && bar_wait(bar_a, phase);
      phase ^= 1u;
    }
    store_bf16x8(my_rt, 8 * 128, f);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0 && ok) {
      umma(tmem, smem_desc(rt + 8 * 128, 128, 2048), smem_desc(w1t, 128, 256), 0u);
      umma_commit(bar_a);
    }
    ok = ok && bar_wait(bar_a, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) break;
    fence_after();
    // ---- h1 = GELU(z1 + b1) into RT; GELU'(z1 + b1) replaces z1 in TMEM
#pragma unroll 1
    for (int c = 0; c < kN; c += 16) {
      float v[16], g[16];
      tmem_ld16(tmem + lane_base + (uint32_t)c, v);
#pragma unroll
      for (int k = 0; k < 16; ++k) gelu_both(v[k] + par[c + k], v[k], g[k]);
      store_bf16x8(my_rt, (c >> 3) * 128, v);
      store_bf16x8(my_rt, (c >> 3) * 128 + 128, v + 8);
      tmem_st16(tmem + lane_base + (uint32_t)c, g);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0 && ok) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        umma(tmem + 64, smem_desc(rt + 256 * kk, 128, 2048), smem_desc(w2t + 256 * kk, 128, 1024), kk > 0 ? 1u : 0u);
      umma_commit(bar_a);
    }
    ok = ok && bar_wait(bar_a, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) break;
    fence_after();
    // ---- the logit, then dl = dL/do; h2 stays in registers, GELU'(z2)
    // replaces z2 in TMEM
    float o = 0.f;
    float h2[kN];
#pragma unroll
    for (int c = 0; c < kN; c += 16) {
      float v[16], g[16];
      tmem_ld16(tmem + lane_base + 64 + (uint32_t)c, v);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        gelu_both(v[k] + par[kN + c + k], h2[c + k], g[k]);
        o = fmaf(h2[c + k], par[2 * kN + c + k], o);
      }
      tmem_st16(tmem + lane_base + 64 + (uint32_t)c, g);
    }
    o += par[3 * kN];
    const float dl = valid ? (1.f / (1.f + expf(-o)) - y) * a.inv_b : 0.f;
    if (valid) lsum += fmaxf(o, 0.f) + log1pf(expf(-fabsf(o))) - y * o;
    db3 += dl;
    // ---- dz2 = dl w3 GELU'(z2) into GT; db2, dw3 column sums (unrolled: the
    // per-chunk accumulators stay in registers)
#pragma unroll
    for (int c = 0; c < kN; c += 16) {
      float g[16], dz[16], hw[16];
      tmem_ld16(tmem + lane_base + 64 + (uint32_t)c, g);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        dz[k] = dl * par[2 * kN + c + k] * g[k];
        hw[k] = h2[c + k] * dl;
      }
      store_bf16x8(my_gt, (c >> 3) * 128, dz);
      store_bf16x8(my_gt, (c >> 3) * 128 + 128, dz + 8);
      acc_b2[c >> 4] += col_sum16(dz);
      acc_w3[c >> 4] += col_sum16(hw);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0 && ok) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        umma(tmem + 64, smem_desc(gt + 256 * kk, 128, 2048), smem_desc(w2 + 256 * kk, 128, 1024), kk > 0 ? 1u : 0u);
      umma_commit(bar_a);
    }
    ok = ok && bar_wait(bar_a, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) break;
    fence_after();
    // ---- dz1 = dh1 GELU'(z1) into GT; db1 column sums
#pragma unroll
    for (int c = 0; c < kN; c += 16) {
      float dh[16], g1[16];
      tmem_ld16(tmem + lane_base + 64 + (uint32_t)c, dh);
      tmem_ld16(tmem + lane_base + (uint32_t)c, g1);
#pragma unroll
      for (int k = 0; k < 16; ++k) dh[k] *= g1[k];
      store_bf16x8(my_gt, 8 * 128 + (c >> 3) * 128, dh);
      store_bf16x8(my_gt, 8 * 128 + (c >> 3) * 128 + 128, dh + 8);
      acc_b1[c >> 4] += col_sum16(dh);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    // ---- dW2, dW1 += RT^T GT over the tile's rows (K = 128: eight K = 16 steps)
    if (tid == 0 && ok) {
#pragma unroll
      for (int ks = 0; ks < 8; ++ks)
        umma(tmem + 128, smem_desc(rt + 4096 * ks, 2048, 128), smem_desc(gt + 4096 * ks, 2048, 128),
             (n_tiles > 0 || ks > 0) ? 1u : 0u, kIdescW);
      umma_commit(bar_a);
    }
  }
  if (ok && n_tiles > 0) {   // the last weight MMA
    ok = bar_wait(bar_a, phase);
    phase ^= 1u;
  }
  const bool all_ok = !__syncthreads_or(!ok);
  fence_after();
  float* P = a.partial + (size_t)blockIdx.x * kTrPartStride;
  // ---- dW2 (TMEM rows 0..63, columns 128..191), dW1 (rows 64..71, columns 192..255)
  if (warp < 3) {
    const uint32_t col = (warp < 2) ? 128u : 192u;
    float* dst = (warp < 2) ? P + 576 + tid * kN : P + (tid - 64) * kN;
    const bool mine = (warp < 2) || tid < 72;
#pragma unroll 1
    for (int c = 0; c < kN; c += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + col + (uint32_t)c, v);
      if (mine) {
#pragma unroll
        for (int k = 0; k < 16; ++k) dst[c + k] = (n_tiles > 0 && all_ok) ? v[k] : (all_ok ? 0.f : nanf(""));
      }
    }
  }
  // ---- bias gradients and dw3: warps in order
  float* red = reinterpret_cast<float*>(sm + kTrRed);   // [warp][3][64]
  if ((lane & 1) == 0) {
    const int col = (lane >> 1) & 15;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      red[(warp * 3 + 0) * kN + 16 * q + col] = acc_b1[q];
      red[(warp * 3 + 1) * kN + 16 * q + col] = acc_b2[q];
      red[(warp * 3 + 2) * kN + 16 * q + col] = acc_w3[q];
    }
  }
  db3 = warp_sum(db3);
  lsum = warp_sum(lsum);
  float* red1 = red + 4 * 3 * kN;
  if (lane == 0) {
    red1[2 * warp] = db3;
    red1[2 * warp + 1] = lsum;
  }
  __syncthreads();
  if (tid < kN) {
    float v0 = 0.f, v1 = 0.f, v2 = 0.f;
    for (int q = 0; q < 4; ++q) {
      v0 += red[(q * 3 + 0) * kN + tid];
      v1 += red[(q * 3 + 1) * kN + tid];
      v2 += red[(q * 3 + 2) * kN + tid];
    }
    P[512 + tid] = v0;
    P[4672 + tid] = v1;
    P[4736 + tid] = v2;
  }
  if (tid == 0) {
    float v0 = 0.f, v1 = 0.f;
    for (int q = 0; q < 4; ++q) {
      v0 += red1[2 * q];
      v1 += red1[2 * q + 1];
    }
    P[4800] = v0;
    P[kMlpParams] = all_ok ? v1 * a.inv_b : nanf("");
  }
  if (!all_ok) {
    // a wait ran out: record it, give the MMAs in flight one more bounded
    // wait, then free TMEM as usual
    if (tid == 0) atomicOr(err, kErrMlpTimeout);
    bar_wait(bar_a, phase);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTrTmemCols) : "memory");
}

}  // namespace

int mlp_grad_parts(int64_t B) {
  const int64_t tiles = (B + kRows - 1) / kRows;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, kTrMaxCtas));
}
int mlp_part_stride() { return kTrPartStride; }

void launch_mlp_grad_tc(const float* theta, const float* x, const float* y, int64_t B, float* partial, int* err,
                        cudaStream_t s) {
  static std::atomic<bool> attr_dev[64];   // the shared-memory limit is a per-device setting
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_dev[dev].load()) {
    cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrSmemDyn);
    if (dev >= 0 && dev < 64) attr_dev[dev].store(true);
  }
  TrainArgs a;
  a.theta = theta;
  a.x = x;
  a.y = y;
  a.B = B;
  a.inv_b = B > 0 ? (float)(1.0 / (double)B) : 0.f;
  a.partial = partial;
  k_mlp_grad_tc<<<mlp_grad_parts(B), kRows, kTrSmemDyn, s>>>(a, err);
}

void launch_mlp_forward_tc(const float* theta, const float* x, int64_t B, float* logit, int* err, int sm_count,
                           cudaStream_t s) {
  InferArgs a{};
  a.theta = theta;
  a.x = x;
  a.Z = B;
  a.logit = logit;
  launch_tc<false>(a, err, sm_count, s);
}

void launch_mlp_infer_tc(const InferArgs& a, int* err, int sm_count, cudaStream_t s) {
  launch_tc<true>(a, err, sm_count, s);
}

}  // namespace fm
