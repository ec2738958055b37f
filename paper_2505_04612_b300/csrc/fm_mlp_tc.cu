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

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
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
  static int per_sm = 0;   // resident CTAs per SM, bound by shared memory (one device per process)
  if (per_sm == 0) {
    cudaFuncSetAttribute(k_mlp_forward_tc<PAIRS>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDyn);
    int dev = 0, smem_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    per_sm = std::max(1, std::min(kCtasPerSm, smem_sm / (kSmemDyn + reserved)));
  }
  static_assert(kSmemUsed <= kSmemDyn, "shared memory layout");
  const int64_t tiles = (a.Z + kRows - 1) / kRows;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)sm_count * per_sm);
  k_mlp_forward_tc<PAIRS><<<(unsigned)grid, kRows, kSmemDyn, s>>>(a, err);
}

}  // namespace

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
