// Surrogate network on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Network: x (67) -> [Linear 128, ReLU] x 3 -> Linear 2 -> (v_hat, jam logit).
// BF16 weights and activations, FP32 accumulation (in tensor memory), FP32
// master weights and AdamW state.  The input dimension is padded to 80 and
// the output to 16 columns so every GEMM has K % 16 == 0 and N % 16 == 0;
// the batch is padded to a multiple of 128 (padding rows carry zero output
// gradients, so they add nothing to any weight gradient).
//
// GEMM kernel.  C[M x N] = A[M x K] * B[N x K]^T with A, B BF16 and K
// contiguous (K-major).  One CTA of 128 threads per 128-row tile of C and
// all N <= 128 columns, the FP32 accumulator in tensor memory.  Operands
// reach shared memory by TMA (cp.async.bulk.tensor) through a ring of up to
// four stages of one K chunk (64) each: thread 0 issues one copy per
// operand and stage (a box of 64 elements = 128 bytes of K x rows, written
// with the 128-byte swizzle: 8-row groups of 1024 bytes, the 16-byte chunks
// of row r permuted by r mod 8) and arms the stage's full barrier with the
// byte count; thread 32 waits for it, issues 4 tcgen05.mma (M=128, N, K=16;
// the matrix descriptors in the same swizzled K-major layout, advanced 32
// bytes per K step) and commits to the stage's empty
// barrier, which releases the stage to the producer; a last commit marks
// the accumulator complete.  Every wait is bounded by %globaltimer (on
// expiry an error flag is set, copies still in flight are waited for, again
// bounded, and the tensor memory is released).  The epilogue reads the
// accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = rows),
// applies bias / ReLU / conversion and stores row-major outputs through a
// per-warp shared-memory transpose so that a warp writes whole row segments.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched at run time)
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "../../include/bml.h"
#include "bml_internal.cuh"
#include "device_common.cuh"

namespace bml {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kIn = 67, kInPad = 80, kHid = 128, kOut = 2, kOutPad = 16;
// Blocks of the loss and bias-gradient kernels (grid-stride over the batch):
// few enough that the last block's ordered sum over their partials is short.
constexpr int kReluBlocks = 256, kLossBlocks = 256;
inline int relu_blocks(int Bp) {
  const int b = Bp / 8;
  return b < 1 ? 1 : (b > kReluBlocks ? kReluBlocks : b);
}
inline int loss_blocks(int Bp) {
  const int b = (Bp + 255) / 256;
  return b > kLossBlocks ? kLossBlocks : b;
}
constexpr int kKC = 64;                       // K per shared-memory stage
constexpr int kStageA = 128 * kKC * 2;        // A: 128 rows x 64 bf16
constexpr int kStageBytes = 2 * kStageA;      // + B: up to 128 rows x 64 bf16
constexpr int kMaxStages = 4;
constexpr int kBarBytes = 1024;               // barriers, TMEM slot, flags after the ring
constexpr int kMinSmem = 72 * 1024;           // caps residency at 3 CTAs per SM (TMEM)
constexpr int kMaxSmem = kMaxStages * kStageBytes + kBarBytes;
constexpr long long kWaitNs = 1000000000ll;   // 1 s bound on any wait

enum EpiMode { EPI_F32 = 0, EPI_RELU_BF16 = 1, EPI_F32_T = 2 };

struct Epi {
  int mode;
  const float *bias;  // per column, or nullptr
  float *out_f32;     // EPI_F32: [M][ldo]; EPI_F32_T: [N][ldo] (transposed)
  bf16 *out_bf16;     // EPI_RELU_BF16: [M][ldo]
  bf16 *out_bf16_t;   // EPI_RELU_BF16: optional [N][ldt] transposed copy
  int ldo, ldt;
  int *err;
  int test_stall;  // test hook: the producer issues no copy, so the first wait runs out
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}

// Shared-memory matrix descriptor of a K-major operand with the 128-byte
// swizzle: start address, leading offset 16 bytes (unused within one
// 128-byte swizzle row), stride 1024 bytes between 8-row groups, version
// field 1, layout type 2 (128-byte swizzle).  The tile base is 1024-byte
// aligned; a K step of 16 elements advances the start by 32 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = gtimer();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (gtimer() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               :: "r"(bar), "r"(bytes) : "memory");
}

// 2-D tiled TMA load of box {64 elements (128 bytes) of K, rows} at (x = k,
// y = row) into shared memory; completion is counted on the mbarrier in
// bytes (the whole box, zero-filled where it passes the matrix edge)
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];"
      :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(bar) : "memory");
}

__global__ void __launch_bounds__(128, 1)
    umma_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                     const __grid_constant__ CUtensorMap mapB, int M, int N, int K, int stages,
                     Epi epi) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *ring = smem;  // stages x [A 16 KB | B 16 KB]
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + stages * kStageBytes);
  // bars: full[kMaxStages], empty[kMaxStages], done; then the TMEM slot and flags
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kMaxStages + 1);
  volatile int *s_fail = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile int *s_issued = s_fail + 1, *s_consumed = s_fail + 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128;
  const int nk = (K + kKC - 1) / kKC;
  const uint32_t ncols = N <= 32 ? 32u : (N <= 64 ? 64u : 128u);
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int st) { return bar0 + 8u * (uint32_t)st; };
  auto empty = [&](int st) { return bar0 + 8u * (uint32_t)(kMaxStages + st); };
  const uint32_t done = bar0 + 8u * (uint32_t)(2 * kMaxStages);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(tmem_slot)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int st = 0; st < stages; ++st) {
      mbar_init(full(st), 1);
      mbar_init(empty(st), 1);
    }
    mbar_init(done, 1);
    *s_fail = 0;
    *s_issued = 0;
    *s_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *tmem_slot;

  if (tid == 0) {  // (the other lanes of warps 0 and 1 wait at __syncwarp below)
    // producer: stage c % stages takes K chunk c once the MMAs of chunk
    // c - stages have released it
    int c = 0;
    for (; c < nk && !epi.test_stall; ++c) {
      const int st = c % stages;
      if (c >= stages && !mbar_wait(empty(st), (uint32_t)((c / stages - 1) & 1))) {
        *s_fail = 1;
        break;
      }
      if (*s_fail) break;
      const int k0 = c * kKC;
      const uint32_t a = smem_u32(ring + st * kStageBytes), b = a + kStageA;
      mbar_expect_tx(full(st), (uint32_t)((128 + N) * kKC * 2));
      tma_load_2d(a, &mapA, k0, m0, full(st));
      tma_load_2d(b, &mapB, k0, 0, full(st));
    }
    *s_issued = c;
  } else if (tid == 32) {
    // MMA issuer
    const uint32_t idesc = idesc_bf16(128, N);
    int c = 0;
    for (; c < nk; ++c) {
      const int st = c % stages;
      if (!mbar_wait(full(st), (uint32_t)((c / stages) & 1))) {
        *s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int k0 = c * kKC;
      const int ksteps = (K - k0) >= kKC ? kKC / 16 : (K - k0) / 16;
      const uint32_t a = smem_u32(ring + st * kStageBytes), b = a + kStageA;
      for (int kk = 0; kk < ksteps; ++kk) {
        const uint64_t ad = smem_desc_sw128(a + (uint32_t)(kk * 32));
        const uint64_t bd = smem_desc_sw128(b + (uint32_t)(kk * 32));
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            :: "r"(taddr), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
      }
      umma_commit(empty(st));
    }
    *s_consumed = c;
    umma_commit(done);  // arrives once every MMA issued above has completed
  }
  if (warp < 2) __syncwarp();
  if (!mbar_wait(done, 0)) *s_fail = 1;
  __syncthreads();
  if (tid == 0) {
    // copies of stages the MMA thread never consumed (after a failed wait)
    for (int c = *s_consumed; c < *s_issued; ++c)
      if (!mbar_wait(full(c % stages), (uint32_t)((c / stages) & 1))) *s_fail = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (*s_fail) {
    if (tid == 0) atomicExch(epi.err, 1);
  } else {
    // epilogue: thread (warp w, lane l) owns row m0 + 32w + l; row-major
    // outputs go through this warp's 32 x 17 float tile in the (now idle) ring
    const int row0 = m0 + warp * 32, row = row0 + lane;
    float *stg = reinterpret_cast<float *>(ring) + warp * (32 * 17);
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        v[j] = __uint_as_float(r[j]) + (epi.bias ? epi.bias[c0 + j] : 0.f);
        if (epi.mode == EPI_RELU_BF16) v[j] = v[j] > 0.f ? v[j] : 0.f;
      }
      if (epi.mode == EPI_F32_T) {
        // transposed output: consecutive lanes write consecutive rows
        if (row < M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) epi.out_f32[(size_t)(c0 + j) * epi.ldo + row] = v[j];
        }
        continue;
      }
      if (epi.mode == EPI_RELU_BF16 && epi.out_bf16_t && row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          epi.out_bf16_t[(size_t)(c0 + j) * epi.ldt + row] = __float2bfloat16_rn(v[j]);
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) stg[lane * 17 + j] = v[j];
      __syncwarp();
      if (epi.mode == EPI_F32) {
        // two rows of 16 floats per instruction
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int rr = 2 * i + (lane >> 4), cc = lane & 15;
          if (row0 + rr < M) epi.out_f32[(size_t)(row0 + rr) * epi.ldo + c0 + cc] = stg[rr * 17 + cc];
        }
      } else {
        // four rows of 16 bf16 per instruction, two columns per lane
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int rr = 4 * i + (lane >> 3), cc = (lane & 7) * 2;
          if (row0 + rr < M) {
            __nv_bfloat162 h;
            h.x = __float2bfloat16_rn(stg[rr * 17 + cc]);
            h.y = __float2bfloat16_rn(stg[rr * 17 + cc + 1]);
            *reinterpret_cast<__nv_bfloat162 *>(epi.out_bf16 + (size_t)(row0 + rr) * epi.ldo +
                                                c0 + cc) = h;
          }
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(taddr), "r"(ncols) : "memory");
}

// ---- elementwise kernels ----

// x fp32 [B][67] -> X bf16 [Bp][80] and XT [80][Bp]; padding is zero
__global__ void prep_x_kernel(const float *__restrict__ x, int B, int Bp, bf16 *X, bf16 *XT) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Bp * kInPad;
       i += gridDim.x * blockDim.x) {
    const int b = i / kInPad, c = i - b * kInPad;
    const float v = (b < B && c < kIn) ? x[(size_t)b * kIn + c] : 0.f;
    const bf16 h = __float2bfloat16_rn(v);
    X[i] = h;
    if (XT) XT[(size_t)c * Bp + b] = h;
  }
}

// Sums over the blocks of a grid in a fixed order: block b has stored its n
// partial sums at part[b * n, (b + 1) * n) (and fenced them); the block that
// arrives last at the counter adds them up in a fixed association (ACC
// interleaved running sums, then those in order), so every sum is formed the
// same way whatever the blocks' timing (float atomics would make training
// runs differ from one another).  Returns true in that block, whose
// threads j < n then hold the total of entry j in *total; the counter is
// re-armed for the next launch on the stream.
template <int ACC>
__device__ __forceinline__ bool grid_sum_last(const float *part, int n, unsigned *count,
                                              float *total) {
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(count, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return false;
  if ((int)threadIdx.x < n) {
    // ACC running sums (block b into sum b % ACC), added in order at the end:
    // a fixed association with ACC loads in flight
    float t[ACC];
#pragma unroll
    for (int k = 0; k < ACC; ++k) t[k] = 0.f;
    const unsigned G = gridDim.x;
    for (unsigned b = 0; b < G; b += ACC) {
#pragma unroll
      for (int k = 0; k < ACC; ++k)
        if (b + k < G) t[k] += __ldcg(part + (size_t)(b + k) * n + threadIdx.x);
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < ACC; ++k) sum += t[k];
    *total = sum;
  }
  if (threadIdx.x == 0) *count = 0u;
  return true;
}

// outputs fp32 [Bp][16] -> loss (sum / B), dOut bf16 [Bp][16] and its
// transpose [16][Bp], and the output-bias gradient db4[0..1]; loss and db4
// are sums over the batch formed in a fixed order (per-warp shuffles, warps
// in order, blocks in order by the last block).  256 threads per block.
__global__ void loss_grad_kernel(const float *__restrict__ out, const float *__restrict__ v,
                                 const float *__restrict__ jam, int B, int Bp, bf16 *G,
                                 bf16 *GT, float *loss, float *db4, float *part,
                                 unsigned *count) {
  float l_sum = 0.f, g0 = 0.f, g1 = 0.f;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < Bp; b += gridDim.x * blockDim.x) {
    float d0 = 0.f, d1 = 0.f;
    if (b < B) {
      const float yv = out[(size_t)b * kOutPad + 0], z = out[(size_t)b * kOutPad + 1];
      const float e = expf(-fabsf(z));
      const float sig = z >= 0.f ? 1.f / (1.f + e) : e / (1.f + e);
      const float dv = yv - v[b];
      l_sum += dv * dv + fmaxf(z, 0.f) - z * jam[b] + log1pf(e);
      d0 = 2.f * dv / (float)B;
      d1 = (sig - jam[b]) / (float)B;
      g0 += d0;
      g1 += d1;
    }
    for (int c = 0; c < kOutPad; ++c) {
      const bf16 h = __float2bfloat16_rn(c == 0 ? d0 : (c == 1 ? d1 : 0.f));
      G[(size_t)b * kOutPad + c] = h;
      GT[(size_t)c * Bp + b] = h;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    l_sum += __shfl_down_sync(0xffffffffu, l_sum, o);
    g0 += __shfl_down_sync(0xffffffffu, g0, o);
    g1 += __shfl_down_sync(0xffffffffu, g1, o);
  }
  __shared__ float s_w[8][3];
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_w[warp][0] = l_sum;
    s_w[warp][1] = g0;
    s_w[warp][2] = g1;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w][threadIdx.x];
    part[(size_t)blockIdx.x * 3 + threadIdx.x] = t;
    __threadfence();
  }
  float total = 0.f;
  if (grid_sum_last<8>(part, 3, count, &total)) {
    if (threadIdx.x == 0) *loss = total / (float)B;
    if (threadIdx.x == 1) db4[0] = total;
    if (threadIdx.x == 2) db4[1] = total;
  }
}

// Mini-batch draw for bml_mlp_train: sample i of training step t takes row
// floor(u * n / 2^64) of the training set, u = SplitMix64(seed, t * B + i + 1)
// (uniform, with replacement); its features and labels are copied into xb,
// vb, jb.
__global__ void gather_batch_kernel(const float *__restrict__ x, const float *__restrict__ v,
                                    const float *__restrict__ jam, long long n, u64 seed,
                                    long long t, int B, float *xb, float *vb, float *jb) {
  for (int i = blockIdx.x; i < B; i += gridDim.x) {
    const u64 u = splitmix64_at(seed, (u64)t * (u64)B + (u64)i + 1ull);
    const long long r = (long long)__umul64hi(u, (u64)n);
    for (int c = threadIdx.x; c < kIn; c += blockDim.x) xb[(size_t)i * kIn + c] = x[r * kIn + c];
    if (threadIdx.x == 0) {
      vb[i] = v[r];
      jb[i] = jam[r];
    }
  }
}

// dZ = dH * (H > 0): bf16 [Bp][128] and transpose [128][Bp]; bias gradient
// db = column sums over the first B rows, formed in a fixed order (rows in
// order within a block, blocks in order by the last block).  128 threads per
// block, one per column.
__global__ void relu_bwd_kernel(const float *__restrict__ dH, const bf16 *__restrict__ H, int B,
                                int Bp, bf16 *__restrict__ dZ, bf16 *__restrict__ dZT,
                                float *__restrict__ db, float *__restrict__ part,
                                unsigned *count) {
  const int col = threadIdx.x;
  float s = 0.f;
#pragma unroll 8
  for (int b = blockIdx.x; b < Bp; b += gridDim.x) {
    const size_t i = (size_t)b * kHid + col;
    const float g = (b < B && __bfloat162float(H[i]) > 0.f) ? dH[i] : 0.f;
    s += g;
    const bf16 h = __float2bfloat16_rn(g);
    dZ[i] = h;
    dZT[(size_t)col * Bp + b] = h;
  }
  part[(size_t)blockIdx.x * kHid + col] = s;
  __threadfence();
  float total = 0.f;
  if (grid_sum_last<32>(part, kHid, count, &total)) db[col] = total;
}

// column sums of a bf16-free fp32 gradient are not needed for layer 4 (done
// in loss_grad_kernel).

// AdamW over the flat master parameters (oracle layout).  The gradient of
// entry i is read from the layer's padded gradient buffer; the updated
// weight is also written as BF16 into the padded forward copy and the
// transposed backward copy.
struct Layer {
  int out, in;        // true sizes
  int in_pad;         // padded row length of the forward copy
  int out_pad;        // padded rows of the forward copy
  long long w_off, b_off;   // offsets of W and b in the flat vector
  const float *gW;    // gradient [out_pad][in_pad]
  const float *gb;    // gradient [out]
  bf16 *W, *WT;       // [out_pad][in_pad], [in_pad][out_pad] (WT may be null)
};

struct Layers {
  Layer l[4];
};

__global__ void adamw_kernel(float *w, float *m, float *v, Layers Ls, long long n, float lr,
                             float wd, float b1, float b2, float eps, float c1, float c2,
                             const float *ext_grad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    // locate the layer and whether i is a weight or a bias
    int L = 3;
    while (L > 0 && i < Ls.l[L].w_off) --L;
    const Layer &ly = Ls.l[L];
    float g;
    int r = -1, c = -1;
    if (i < ly.b_off) {
      const long long j = i - ly.w_off;
      r = (int)(j / ly.in);
      c = (int)(j - (long long)r * ly.in);
      g = ext_grad ? ext_grad[i] : ly.gW[(size_t)r * ly.in_pad + c];
    } else {
      g = ext_grad ? ext_grad[i] : ly.gb[i - ly.b_off];
    }
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    const float wi = w[i] - lr * (mh / (sqrtf(vh) + eps) + wd * w[i]);
    w[i] = wi;
    if (r >= 0) {
      const bf16 h = __float2bfloat16_rn(wi);
      ly.W[(size_t)r * ly.in_pad + c] = h;
      if (ly.WT) ly.WT[(size_t)c * ly.out_pad + r] = h;
    }
  }
}

// master fp32 -> bf16 forward / transposed copies (after set_params)
__global__ void cast_params_kernel(const float *w, Layers Ls) {
  for (int L = 0; L < 4; ++L) {
    const Layer &ly = Ls.l[L];
    const int n = ly.out * ly.in;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
      const int r = j / ly.in, c = j - r * ly.in;
      const bf16 h = __float2bfloat16_rn(w[ly.w_off + j]);
      ly.W[(size_t)r * ly.in_pad + c] = h;
      if (ly.WT) ly.WT[(size_t)c * ly.out_pad + r] = h;
    }
  }
}

}  // namespace
}  // namespace bml

// =================================================================== C ABI ==
using namespace bml;

namespace {

int mfail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

#define MCUDA(expr)                                                                         \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return mfail(BML_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,   \
                   __LINE__);                                                               \
  } while (0)

// Set-up shared by all calls, under g_setup_mu: the tensor-map encoder
// (fetched from the driver once per process) and, per device, whether the
// GEMM kernel's dynamic shared-memory limit has been raised there.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
bool g_attr_done[kMaxDevices] = {};
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// Tensor map of a K-major bf16 matrix (rows x K, ld elements between rows)
// with a box of 64 elements of K x box_rows rows, 128-byte swizzle.
cudaError_t kmajor_map(CUtensorMap *map, const bf16 *p, int rows, int K, int ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_encode) {
      void *fn = nullptr;
      cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
      const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                             cudaEnableDefault, &q);
      if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    encode = g_encode;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)box_rows};
  const cuuint32_t elem[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(p), dims,
                              strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// A: M rows x K (lda), B: N rows x K (ldb); 16-byte aligned, lda, ldb % 8 == 0.
cudaError_t launch_gemm(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K,
                        const Epi &epi, cudaStream_t st) {
  {
    // the shared-memory limit is raised once on every device the GEMM runs on
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_attr_done[dev]) {
      e = cudaFuncSetAttribute(umma_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kMaxSmem);
      if (e != cudaSuccess) return e;
      g_attr_done[dev] = true;
    }
  }
  if (M < 1 || N < 16 || N > 128 || N % 16 || K < 16 || K % 16 || lda % 8 || ldb % 8 ||
      (uintptr_t)A % 16 || (uintptr_t)B % 16)
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  cudaError_t e = kmajor_map(&ma, A, M, K, lda, 128);
  if (e == cudaSuccess) e = kmajor_map(&mb, B, N, K, ldb, N);
  if (e != cudaSuccess) return e;
  const int nk = (K + kKC - 1) / kKC;
  const int stages = nk < kMaxStages ? nk : kMaxStages;
  int smem = stages * kStageBytes + kBarBytes;
  if (smem < kMinSmem) smem = kMinSmem;
  umma_gemm_kernel<<<(M + 127) / 128, 128, smem, st>>>(ma, mb, M, N, K, stages, epi);
  return cudaGetLastError();
}

}  // namespace

struct bml_mlp {
  cudaStream_t st = nullptr;
  long long n = 0;  // parameters
  float *w = nullptr, *m = nullptr, *v = nullptr;  // master, AdamW moments
  long long t = 0;
  // bf16 weights: forward [out_pad][in_pad], transposed [in_pad][out_pad]
  bf16 *W[4] = {}, *WT[4] = {};
  float *gW[4] = {}, *gb[4] = {};
  float *b[4] = {};  // views into w (biases)
  Layers layers;
  // activation buffers for a padded batch of up to cap rows
  int cap = 0;
  bf16 *X = nullptr, *XT = nullptr, *H[3] = {}, *HT[3] = {}, *G = nullptr, *GT = nullptr;
  bf16 *dZ = nullptr, *dZT = nullptr;
  float *out = nullptr, *dH = nullptr, *loss = nullptr;
  // fixed-order reductions: per-block partial sums and two arrival counters
  // (loss kernel, bias-gradient kernel)
  float *part = nullptr;
  unsigned *red_count = nullptr;
  float *bias4 = nullptr;  // padded output bias [16]
  int *err = nullptr;
  // bml_mlp_train: gathered mini-batch (features, labels) and per-step losses
  int train_cap = 0;
  float *xb = nullptr, *vb = nullptr, *jb = nullptr;
  long long loss_cap = 0;
  float *losses = nullptr;
};

namespace {

const int kOutDims[4] = {kHid, kHid, kHid, kOut};
const int kInDims[4] = {kIn, kHid, kHid, kHid};
const int kInPads[4] = {kInPad, kHid, kHid, kHid};
const int kOutPads[4] = {kHid, kHid, kHid, kOutPad};

void mlp_free_batch(bml_mlp *p) {
  cudaFree(p->X);
  cudaFree(p->XT);
  for (int i = 0; i < 3; ++i) {
    cudaFree(p->H[i]);
    cudaFree(p->HT[i]);
    p->H[i] = p->HT[i] = nullptr;
  }
  cudaFree(p->G);
  cudaFree(p->GT);
  cudaFree(p->dZ);
  cudaFree(p->dZT);
  cudaFree(p->out);
  cudaFree(p->dH);
  cudaFree(p->part);
  p->X = p->XT = p->G = p->GT = p->dZ = p->dZT = nullptr;
  p->out = p->dH = p->part = nullptr;
  p->cap = 0;
}

int ensure_batch(bml_mlp *p, int Bp) {
  if (Bp <= p->cap) return BML_OK;
  mlp_free_batch(p);
  MCUDA(cudaMalloc(&p->X, (size_t)Bp * kInPad * 2));
  MCUDA(cudaMalloc(&p->XT, (size_t)Bp * kInPad * 2));
  for (int i = 0; i < 3; ++i) {
    MCUDA(cudaMalloc(&p->H[i], (size_t)Bp * kHid * 2));
    MCUDA(cudaMalloc(&p->HT[i], (size_t)Bp * kHid * 2));
  }
  MCUDA(cudaMalloc(&p->G, (size_t)Bp * kOutPad * 2));
  MCUDA(cudaMalloc(&p->GT, (size_t)Bp * kOutPad * 2));
  MCUDA(cudaMalloc(&p->dZ, (size_t)Bp * kHid * 2));
  MCUDA(cudaMalloc(&p->dZT, (size_t)Bp * kHid * 2));
  MCUDA(cudaMalloc(&p->out, (size_t)Bp * kOutPad * 4));
  MCUDA(cudaMalloc(&p->dH, (size_t)Bp * kHid * 4));
  MCUDA(cudaMalloc(&p->part, (size_t)(kReluBlocks * kHid + kLossBlocks * 3) * 4));
  p->cap = Bp;
  return BML_OK;
}

int check_mlp_err(bml_mlp *p) {
  int h = 0;
  MCUDA(cudaMemcpyAsync(&h, p->err, sizeof h, cudaMemcpyDeviceToHost, p->st));
  MCUDA(cudaStreamSynchronize(p->st));
  if (h) return mfail(BML_ETIMEOUT, "a tensor-core completion wait timed out");
  return BML_OK;
}

// Forward pass of a padded batch Bp (X already staged).  keep_t: also write
// the transposed activations needed by the backward pass.
int forward_staged(bml_mlp *p, int Bp, bool keep_t) {
  const bf16 *in = p->X;
  int in_ld = kInPad;
  for (int l = 0; l < 3; ++l) {
    Epi e{};
    e.mode = EPI_RELU_BF16;
    e.bias = p->b[l];
    e.out_bf16 = p->H[l];
    e.out_bf16_t = keep_t ? p->HT[l] : nullptr;
    e.ldo = kHid;
    e.ldt = Bp;
    e.err = p->err;
    MCUDA(launch_gemm(in, in_ld, p->W[l], kInPads[l], Bp, kHid, in_ld, e, p->st));
    in = p->H[l];
    in_ld = kHid;
  }
  Epi e{};
  e.mode = EPI_F32;
  e.bias = p->bias4;
  e.out_f32 = p->out;
  e.ldo = kOutPad;
  e.err = p->err;
  MCUDA(launch_gemm(p->H[2], kHid, p->W[3], kHid, Bp, kOutPad, kHid, e, p->st));
  return BML_OK;
}

}  // namespace

extern "C" int bml_mlp_create(void *stream, bml_mlp **out) {
  if (!out) return mfail(BML_EINVAL, "out is NULL");
  bml_mlp *p = new (std::nothrow) bml_mlp;
  if (!p) return mfail(BML_ENOMEM, "host allocation failed");
  p->st = (cudaStream_t)stream;
  long long off = 0;
  for (int l = 0; l < 4; ++l) {
    Layer &ly = p->layers.l[l];
    ly.out = kOutDims[l];
    ly.in = kInDims[l];
    ly.in_pad = kInPads[l];
    ly.out_pad = kOutPads[l];
    ly.w_off = off;
    off += (long long)ly.out * ly.in;
    ly.b_off = off;
    off += ly.out;
  }
  p->n = off;
  int rc = BML_OK;
  cudaError_t e = cudaSuccess;
#define MTRY(expr)      \
  if (e == cudaSuccess) e = (expr)
  MTRY(cudaMalloc(&p->w, p->n * 4));
  MTRY(cudaMalloc(&p->m, p->n * 4));
  MTRY(cudaMalloc(&p->v, p->n * 4));
  MTRY(cudaMalloc(&p->err, 256));
  MTRY(cudaMalloc(&p->loss, 256));
  MTRY(cudaMalloc(&p->red_count, 256));
  MTRY(cudaMalloc(&p->bias4, kOutPad * 4));
  for (int l = 0; l < 4; ++l) {
    Layer &ly = p->layers.l[l];
    MTRY(cudaMalloc(&p->W[l], (size_t)ly.out_pad * ly.in_pad * 2));
    MTRY(cudaMalloc(&p->WT[l], (size_t)ly.out_pad * ly.in_pad * 2));
    MTRY(cudaMalloc(&p->gW[l], (size_t)ly.out_pad * ly.in_pad * 4));
    MTRY(cudaMalloc(&p->gb[l], (size_t)kOutPad * 8 * 4 + ly.out * 4));
    if (e == cudaSuccess) {
      e = cudaMemsetAsync(p->W[l], 0, (size_t)ly.out_pad * ly.in_pad * 2, p->st);
      MTRY(cudaMemsetAsync(p->WT[l], 0, (size_t)ly.out_pad * ly.in_pad * 2, p->st));
    }
    ly.gW = p->gW[l];
    ly.gb = p->gb[l];
    ly.W = p->W[l];
    ly.WT = p->WT[l];
  }
  MTRY(cudaMemsetAsync(p->w, 0, p->n * 4, p->st));
  MTRY(cudaMemsetAsync(p->m, 0, p->n * 4, p->st));
  MTRY(cudaMemsetAsync(p->v, 0, p->n * 4, p->st));
  MTRY(cudaMemsetAsync(p->err, 0, 256, p->st));
  MTRY(cudaMemsetAsync(p->red_count, 0, 256, p->st));
  MTRY(cudaMemsetAsync(p->bias4, 0, kOutPad * 4, p->st));
  MTRY(cudaStreamSynchronize(p->st));
#undef MTRY
  if (e != cudaSuccess) {
    rc = mfail(e == cudaErrorMemoryAllocation ? BML_ENOMEM : BML_ECUDA, "mlp create: %s",
               cudaGetErrorString(e));
    bml_mlp_destroy(p);
    return rc;
  }
  for (int l = 0; l < 3; ++l) p->b[l] = p->w + p->layers.l[l].b_off;
  *out = p;
  return BML_OK;
}

extern "C" void bml_mlp_destroy(bml_mlp *p) {
  if (!p) return;
  cudaStreamSynchronize(p->st);
  mlp_free_batch(p);
  cudaFree(p->w);
  cudaFree(p->m);
  cudaFree(p->v);
  cudaFree(p->err);
  cudaFree(p->loss);
  cudaFree(p->red_count);
  cudaFree(p->bias4);
  cudaFree(p->xb);
  cudaFree(p->vb);
  cudaFree(p->jb);
  cudaFree(p->losses);
  for (int l = 0; l < 4; ++l) {
    cudaFree(p->W[l]);
    cudaFree(p->WT[l]);
    cudaFree(p->gW[l]);
    cudaFree(p->gb[l]);
  }
  delete p;
}

extern "C" int64_t bml_mlp_num_params(const bml_mlp *p) { return p ? p->n : -1; }

extern "C" int bml_mlp_set_params(bml_mlp *p, const float *host) {
  if (!p || !host) return mfail(BML_EINVAL, "NULL argument");
  MCUDA(cudaMemcpyAsync(p->w, host, p->n * 4, cudaMemcpyHostToDevice, p->st));
  MCUDA(cudaMemsetAsync(p->m, 0, p->n * 4, p->st));
  MCUDA(cudaMemsetAsync(p->v, 0, p->n * 4, p->st));
  MCUDA(cudaMemcpyAsync(p->bias4, p->w + p->layers.l[3].b_off, kOut * 4,
                        cudaMemcpyDeviceToDevice, p->st));
  p->t = 0;
  cast_params_kernel<<<64, 256, 0, p->st>>>(p->w, p->layers);
  MCUDA(cudaGetLastError());
  MCUDA(cudaStreamSynchronize(p->st));
  return BML_OK;
}

extern "C" int bml_mlp_get_params(bml_mlp *p, float *host) {
  if (!p || !host) return mfail(BML_EINVAL, "NULL argument");
  MCUDA(cudaMemcpyAsync(host, p->w, p->n * 4, cudaMemcpyDeviceToHost, p->st));
  MCUDA(cudaStreamSynchronize(p->st));
  return BML_OK;
}

extern "C" int bml_mlp_forward(bml_mlp *p, const float *d_x, int64_t batch, float *d_out) {
  if (!p || !d_x || !d_out) return mfail(BML_EINVAL, "NULL argument");
  if (batch < 1 || batch > (1 << 24)) return mfail(BML_EINVAL, "batch must be in [1, 2^24]");
  const int B = (int)batch, Bp = (B + 127) / 128 * 128;
  int rc = ensure_batch(p, Bp);
  if (rc) return rc;
  prep_x_kernel<<<256, 256, 0, p->st>>>(d_x, B, Bp, p->X, nullptr);
  MCUDA(cudaGetLastError());
  if ((rc = forward_staged(p, Bp, false))) return rc;
  MCUDA(cudaMemcpy2DAsync(d_out, kOut * 4, p->out, kOutPad * 4, kOut * 4, B,
                          cudaMemcpyDeviceToDevice, p->st));
  return check_mlp_err(p);
}

// Gradients of the mean loss on a batch into gW / gb (no update).  wait:
// synchronise and report a timed-out tensor-core wait before returning.
static int compute_grads(bml_mlp *p, const float *d_x, const float *d_v, const float *d_jam,
                         int B, float *h_loss, bool wait) {
  const int Bp = (B + 127) / 128 * 128;
  int rc = ensure_batch(p, Bp);
  if (rc) return rc;
  // the loss and every bias gradient are written (not accumulated) below
  prep_x_kernel<<<256, 256, 0, p->st>>>(d_x, B, Bp, p->X, p->XT);
  MCUDA(cudaGetLastError());
  if ((rc = forward_staged(p, Bp, true))) return rc;
  loss_grad_kernel<<<loss_blocks(Bp), 256, 0, p->st>>>(p->out, d_v, d_jam, B, Bp, p->G, p->GT,
                                                       p->loss, p->gb[3], p->part,
                                                       p->red_count);
  MCUDA(cudaGetLastError());
  // layer 4: dW4^T [128][16] = H3^T (128 x Bp) . G^T (16 x Bp)^T, stored transposed
  {
    Epi e{};
    e.mode = EPI_F32_T;
    e.out_f32 = p->gW[3];
    e.ldo = kHid;
    e.err = p->err;
    MCUDA(launch_gemm(p->HT[2], Bp, p->GT, Bp, kHid, kOutPad, Bp, e, p->st));
    Epi d{};
    d.mode = EPI_F32;
    d.out_f32 = p->dH;
    d.ldo = kHid;
    d.err = p->err;
    MCUDA(launch_gemm(p->G, kOutPad, p->WT[3], kOutPad, Bp, kHid, kOutPad, d, p->st));
  }
  for (int l = 2; l >= 0; --l) {
    relu_bwd_kernel<<<relu_blocks(Bp), kHid, 0, p->st>>>(p->dH, p->H[l], B, Bp, p->dZ, p->dZT,
                                                         p->gb[l], p->part, p->red_count + 1);
    MCUDA(cudaGetLastError());
    const bf16 *prevT = l > 0 ? p->HT[l - 1] : p->XT;
    const int in_pad = kInPads[l];
    Epi e{};
    e.mode = EPI_F32;
    e.out_f32 = p->gW[l];
    e.ldo = in_pad;
    e.err = p->err;
    MCUDA(launch_gemm(p->dZT, Bp, prevT, Bp, kHid, in_pad, Bp, e, p->st));
    if (l > 0) {
      Epi d{};
      d.mode = EPI_F32;
      d.out_f32 = p->dH;
      d.ldo = kHid;
      d.err = p->err;
      MCUDA(launch_gemm(p->dZ, kHid, p->WT[l], kHid, Bp, kHid, kHid, d, p->st));
    }
  }
  if (h_loss) {
    MCUDA(cudaMemcpyAsync(h_loss, p->loss, 4, cudaMemcpyDeviceToHost, p->st));
  }
  return wait ? check_mlp_err(p) : BML_OK;
}

static int adamw(bml_mlp *p, float lr, float wd, const float *d_ext) {
  p->t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, (double)p->t));
  const float c2 = (float)(1.0 - std::pow(b2, (double)p->t));
  adamw_kernel<<<128, 256, 0, p->st>>>(p->w, p->m, p->v, p->layers, p->n, lr, wd, (float)b1,
                                       (float)b2, 1e-8f, c1, c2, d_ext);
  MCUDA(cudaGetLastError());
  MCUDA(cudaMemcpyAsync(p->bias4, p->w + p->layers.l[3].b_off, kOut * 4,
                        cudaMemcpyDeviceToDevice, p->st));
  return BML_OK;
}

extern "C" int bml_mlp_train_step(bml_mlp *p, const float *d_x, const float *d_v,
                                  const float *d_jam, int64_t batch, float lr,
                                  float weight_decay, float *h_loss) {
  if (!p || !d_x || !d_v || !d_jam) return mfail(BML_EINVAL, "NULL argument");
  if (batch < 1 || batch > (1 << 24)) return mfail(BML_EINVAL, "batch must be in [1, 2^24]");
  if (!(lr >= 0.f) || !(weight_decay >= 0.f)) return mfail(BML_EINVAL, "bad lr / weight_decay");
  // with a loss to return, the step waits for the gradients (and reports a
  // timed-out wait before anything is updated); without one it only enqueues
  // (the error flag is sticky: a failure in an enqueued step is reported by
  // the next call that waits)
  const bool wait = h_loss != nullptr;
  int rc = compute_grads(p, d_x, d_v, d_jam, (int)batch, h_loss, wait);
  if (rc) return rc;
  return adamw(p, lr, weight_decay, nullptr);
}

extern "C" int bml_mlp_train(bml_mlp *p, const float *d_x, const float *d_v, const float *d_jam,
                             int64_t n, int64_t steps, int64_t batch, float lr,
                             float weight_decay, uint64_t seed, float *h_losses) {
  if (!p || !d_x || !d_v || !d_jam) return mfail(BML_EINVAL, "NULL argument");
  if (n < 1 || n > (1ll << 40)) return mfail(BML_EINVAL, "n must be in [1, 2^40]");
  if (steps < 0 || steps > (1 << 30)) return mfail(BML_EINVAL, "steps must be in [0, 2^30]");
  if (batch < 1 || batch > (1 << 24)) return mfail(BML_EINVAL, "batch must be in [1, 2^24]");
  if (!(lr >= 0.f) || !(weight_decay >= 0.f)) return mfail(BML_EINVAL, "bad lr / weight_decay");
  if (steps == 0) return BML_OK;
  const int B = (int)batch;
  if (B > p->train_cap) {
    cudaFree(p->xb);
    cudaFree(p->vb);
    cudaFree(p->jb);
    p->xb = p->vb = p->jb = nullptr;
    p->train_cap = 0;
    MCUDA(cudaMalloc(&p->xb, (size_t)B * kIn * 4));
    MCUDA(cudaMalloc(&p->vb, (size_t)B * 4));
    MCUDA(cudaMalloc(&p->jb, (size_t)B * 4));
    p->train_cap = B;
  }
  if (h_losses && steps > p->loss_cap) {
    cudaFree(p->losses);
    p->losses = nullptr;
    p->loss_cap = 0;
    MCUDA(cudaMalloc(&p->losses, (size_t)steps * 4));
    p->loss_cap = steps;
  }
  const int gblocks = B < 1024 ? B : 1024;
  for (int64_t s = 0; s < steps; ++s) {
    gather_batch_kernel<<<gblocks, 64, 0, p->st>>>(d_x, d_v, d_jam, (long long)n, seed, p->t, B,
                                                   p->xb, p->vb, p->jb);
    MCUDA(cudaGetLastError());
    int rc = compute_grads(p, p->xb, p->vb, p->jb, B, nullptr, false);
    if (rc) return rc;
    if (h_losses)
      MCUDA(cudaMemcpyAsync(p->losses + s, p->loss, 4, cudaMemcpyDeviceToDevice, p->st));
    if ((rc = adamw(p, lr, weight_decay, nullptr))) return rc;
  }
  if (h_losses)
    MCUDA(cudaMemcpyAsync(h_losses, p->losses, (size_t)steps * 4, cudaMemcpyDeviceToHost, p->st));
  return check_mlp_err(p);
}

extern "C" int bml_mlp_grads(bml_mlp *p, const float *d_x, const float *d_v, const float *d_jam,
                             int64_t batch, float *host_grads, float *h_loss) {
  if (!p || !d_x || !d_v || !d_jam || !host_grads) return mfail(BML_EINVAL, "NULL argument");
  if (batch < 1 || batch > (1 << 24)) return mfail(BML_EINVAL, "batch must be in [1, 2^24]");
  int rc = compute_grads(p, d_x, d_v, d_jam, (int)batch, h_loss, true);
  if (rc) return rc;
  // gather the padded gradient buffers into the flat parameter layout
  for (int l = 0; l < 4; ++l) {
    const Layer &ly = p->layers.l[l];
    MCUDA(cudaMemcpy2DAsync(host_grads + ly.w_off, (size_t)ly.in * 4, p->gW[l],
                            (size_t)ly.in_pad * 4, (size_t)ly.in * 4, ly.out,
                            cudaMemcpyDeviceToHost, p->st));
    MCUDA(cudaMemcpyAsync(host_grads + ly.b_off, p->gb[l], (size_t)ly.out * 4,
                          cudaMemcpyDeviceToHost, p->st));
  }
  MCUDA(cudaStreamSynchronize(p->st));
  return BML_OK;
}

extern "C" int bml_mlp_apply_grads(bml_mlp *p, const float *host_grads, float lr,
                                   float weight_decay) {
  if (!p || !host_grads) return mfail(BML_EINVAL, "NULL argument");
  float *d = nullptr;
  MCUDA(cudaMalloc(&d, p->n * 4));
  cudaError_t e = cudaMemcpyAsync(d, host_grads, p->n * 4, cudaMemcpyHostToDevice, p->st);
  int rc = BML_OK;
  if (e == cudaSuccess) rc = adamw(p, lr, weight_decay, d);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  cudaFree(d);
  if (e != cudaSuccess) return mfail(BML_ECUDA, "apply grads: %s", cudaGetErrorString(e));
  return rc;
}

extern "C" int bml_mlp_get_layer(bml_mlp *p, int layer, float *host_W, float *host_WT,
                                 float *host_gW) {
  if (!p) return mfail(BML_EINVAL, "NULL argument");
  if (layer < 0 || layer > 3) return mfail(BML_EINVAL, "layer must be in [0, 3]");
  const Layer &ly = p->layers.l[layer];
  const size_t n = (size_t)ly.out_pad * ly.in_pad;
  std::vector<uint16_t> h(n);
  const bf16 *src[2] = {p->W[layer], p->WT[layer]};
  float *dst[2] = {host_W, host_WT};
  for (int k = 0; k < 2; ++k) {
    if (!dst[k]) continue;
    MCUDA(cudaMemcpyAsync(h.data(), src[k], n * 2, cudaMemcpyDeviceToHost, p->st));
    MCUDA(cudaStreamSynchronize(p->st));
    for (size_t i = 0; i < n; ++i) {  // a bf16 value is the top half of its float
      const uint32_t u = (uint32_t)h[i] << 16;
      std::memcpy(dst[k] + i, &u, 4);
    }
  }
  if (host_gW) {
    MCUDA(cudaMemcpyAsync(host_gW, p->gW[layer], n * 4, cudaMemcpyDeviceToHost, p->st));
    MCUDA(cudaStreamSynchronize(p->st));
  }
  return BML_OK;
}

extern "C" int bml_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, float *C,
                             int64_t ldc, int64_t M, int64_t N, int64_t K, void *stream) {
  return bml_gemm_bf16_ex(A, lda, B, ldb, C, ldc, M, N, K, 0u, stream);
}

extern "C" int bml_gemm_bf16_ex(const void *A, int64_t lda, const void *B, int64_t ldb, float *C,
                                int64_t ldc, int64_t M, int64_t N, int64_t K, unsigned flags,
                                void *stream) {
  if (!A || !B || !C) return mfail(BML_EINVAL, "NULL argument");
  if (flags & ~BML_GEMM_TEST_STALL) return mfail(BML_EINVAL, "unknown flags");
  if (M < 1 || M > (1 << 24) || N < 16 || N > 128 || N % 16 || K < 16 || K % 16 ||
      K > (1 << 24) || lda < K || ldb < K || ldc < N || lda % 8 || ldb % 8)
    return mfail(BML_EINVAL, "bml_gemm_bf16: need 16 <= N <= 128, N % 16 == 0, K % 16 == 0, "
                 "lda, ldb >= K and multiples of 8, ldc >= N");
  if ((uintptr_t)A % 16 || (uintptr_t)B % 16) return mfail(BML_EINVAL, "A, B not 16-byte aligned");
  // one completion-wait error flag per calling thread and device, allocated
  // on first use (the call waits for the stream, so a thread has at most one
  // call in flight)
  thread_local std::map<int, int *> err_flags;
  int dev = 0;
  MCUDA(cudaGetDevice(&dev));
  int *&err = err_flags[dev];
  if (!err) MCUDA(cudaMalloc(&err, 4));
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(err, 0, 4, st);
  Epi ep{};
  ep.mode = EPI_F32;
  ep.out_f32 = C;
  ep.ldo = (int)ldc;
  ep.err = err;
  ep.test_stall = (flags & BML_GEMM_TEST_STALL) ? 1 : 0;
  if (e == cudaSuccess)
    e = launch_gemm((const bf16 *)A, (int)lda, (const bf16 *)B, (int)ldb, (int)M, (int)N, (int)K,
                    ep, st);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return mfail(BML_ECUDA, "gemm: %s", cudaGetErrorString(e));
  if (h) return mfail(BML_ETIMEOUT, "a tensor-core completion wait timed out");
  return BML_OK;
}
