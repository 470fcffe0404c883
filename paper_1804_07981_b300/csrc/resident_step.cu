// Resident step for small lattices: one thread block keeps the whole lattice
// (both bitplanes, double buffered) in shared memory and runs every step of
// a bml_step call in one launch.  Small lattices are latency-bound: the
// streaming kernels need one launch per k <= 8 steps and a pipeline fill per
// band, while here a step costs two block barriers.
//
// Each step applies the Sec. 2 rules on whole words (the bitplane layout of
// bml_internal.cuh):
//   horizontal phase, word w of row i (right neighbour word wr, left wl,
//   wrapping within the row):
//     E = ~(L | T) & valid,  Er = E >> 1 with bit 0 of E(wr) at the last cell,
//     mvH = L & Er,  in = (mvH << 1 with the left word's moving last cell
//     at bit 0) & valid,  Lh = L ^ mvH ^ in
//   vertical phase, row i against rows i-1 and i+1 (wrapping):
//     E'_i = ~(Lh_i | T_i) & valid,  mvV_i = T_i & E'_{i+1},
//     T'_i = (T_i & ~mvV_i) | (T_{i-1} & E'_i)
// Thread t owns the words t, t + blockDim, ... (WPT of them): it keeps their
// L, T and Lh in registers, with the shared-memory offsets of their
// neighbours computed once.  The horizontal phase reads the neighbours' L, T
// and writes Lh to the other L buffer; the vertical phase reads the
// neighbours' Lh, T and writes T' to the other T buffer; a block barrier
// separates the phases.  Moved counts of a phase are summed per warp (redux)
// into a per-warp slot; after the phase's barrier warp 0 adds the slots into
// the step's counter (no atomics), and the counters are written once at the
// end.
#include <cooperative_groups.h>

#include "device_common.cuh"

namespace bml {

namespace cg = cooperative_groups;

// Split cluster barrier: arrive (release: this thread's earlier shared-memory
// writes become visible to the cluster) and wait (acquire).
__device__ __forceinline__ void barrier_cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void barrier_cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

namespace {

constexpr int kResThreads = 1024;
constexpr int kResMaxBlocks = 8;  // portable cluster size

struct ResGeom {
  int M, W, P, nb;
  u64 tail;
};

template <int WPT>
__global__ void __launch_bounds__(kResThreads, 1)
    resident_kernel(const u64 *__restrict__ Lin, const u64 *__restrict__ Tin,
                    u64 *__restrict__ Lout, u64 *__restrict__ Tout, ResGeom r, int K,
                    u64 *__restrict__ moved_lr, u64 *__restrict__ moved_tb) {
  extern __shared__ __align__(16) u64 sm[];
  const int words = r.M * r.P;
  u64 *sL[2] = {sm, sm + words};
  u64 *sT[2] = {sm + 2 * words, sm + 3 * words};
  unsigned int *cnt = (unsigned int *)(sm + 4 * words);  // [2][K]
  __shared__ unsigned int s_part[2][kResThreads / 32];   // per-warp partial counts, by phase
  for (int x = threadIdx.x; x < words; x += blockDim.x) {
    sL[0][x] = Lin[x];
    sT[0][x] = Tin[x];
    sL[1][x] = sT[1][x] = 0;  // padding words are never written by a step
  }
  for (int x = threadIdx.x; x < 2 * K; x += blockDim.x) cnt[x] = 0;

  // this thread's words: flat index, neighbour offsets, masks (x < 0: none)
  int xs[WPT], xr[WPT], xl[WPT], xu[WPT], xd[WPT], topl[WPT];
  u64 valid[WPT], topbit[WPT], L[WPT], T[WPT];
#pragma unroll
  for (int j = 0; j < WPT; ++j) {
    const int x = threadIdx.x + j * blockDim.x;
    const int i = x / r.P, w = x - i * r.P;
    const bool on = x < words && w < r.W;
    xs[j] = on ? x : -1;
    const int wr = w == r.W - 1 ? 0 : w + 1, wl = w == 0 ? r.W - 1 : w - 1;
    const int iu = i == 0 ? r.M - 1 : i - 1, id = i == r.M - 1 ? 0 : i + 1;
    xr[j] = i * r.P + wr;
    xl[j] = i * r.P + wl;
    xu[j] = iu * r.P + w;
    xd[j] = id * r.P + w;
    topl[j] = wl == r.W - 1 ? r.nb - 1 : 63;                    // left word's last cell
    valid[j] = w == r.W - 1 ? r.tail : ~0ull;
    topbit[j] = 1ull << (w == r.W - 1 ? r.nb - 1 : 63);        // this word's last cell
    L[j] = T[j] = 0;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < WPT; ++j)
    if (xs[j] >= 0) {
      L[j] = sL[0][xs[j]];
      T[j] = sT[0][xs[j]];
    }
  const int lane = threadIdx.x & 31;
  int a = 0;  // buffer holding the current state
  for (int t = 0; t < K; ++t) {
    // ---- horizontal phase: (L[a], T[a]) -> L[a^1] ----
    uint32_t c = 0;
    u64 Lh[WPT];
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      Lh[j] = 0;
      if (xs[j] >= 0) {
        const u64 E = ~(L[j] | T[j]) & valid[j];
        const u64 er0 = ~(sL[a][xr[j]] | sT[a][xr[j]]) & 1ull;
        const u64 mvH = L[j] & ((E >> 1) | (er0 ? topbit[j] : 0ull));
        // the left word's last LR car moves in iff this word's first cell is empty
        const u64 in_l = (sL[a][xl[j]] >> topl[j]) & E & 1ull;
        const u64 in = ((mvH << 1) | in_l) & valid[j];
        Lh[j] = L[j] ^ mvH ^ in;
        c += (uint32_t)__popcll(mvH);
        sL[a ^ 1][xs[j]] = Lh[j];
      }
    }
    c = __reduce_add_sync(BML_FULL_MASK, c);
    if (lane == 0) s_part[0][threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {  // the previous step's vertical slots were read before this barrier
      const uint32_t v = threadIdx.x < (blockDim.x >> 5) ? s_part[0][threadIdx.x] : 0u;
      const uint32_t tot = __reduce_add_sync(BML_FULL_MASK, v);
      if (threadIdx.x == 0) cnt[t] = tot;
    }
    // ---- vertical phase: (L[a^1], T[a]) -> T[a^1] ----
    c = 0;
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      if (xs[j] >= 0) {
        const u64 Ei = ~(Lh[j] | T[j]) & valid[j];
        const u64 Ed = ~(sL[a ^ 1][xd[j]] | sT[a][xd[j]]) & valid[j];
        const u64 mvV = T[j] & Ed;
        const u64 To = (T[j] & ~mvV) | (sT[a][xu[j]] & Ei);
        c += (uint32_t)__popcll(mvV);
        sT[a ^ 1][xs[j]] = To;
        T[j] = To;
        L[j] = Lh[j];
      }
    }
    c = __reduce_add_sync(BML_FULL_MASK, c);
    if (lane == 0) s_part[1][threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
      const uint32_t v = threadIdx.x < (blockDim.x >> 5) ? s_part[1][threadIdx.x] : 0u;
      const uint32_t tot = __reduce_add_sync(BML_FULL_MASK, v);
      if (threadIdx.x == 0) cnt[K + t] = tot;
    }
    a ^= 1;
  }
  __syncthreads();  // the last step's counters
  for (int x = threadIdx.x; x < words; x += blockDim.x) {
    Lout[x] = sL[a][x];
    Tout[x] = sT[a][x];
  }
  for (int x = threadIdx.x; x < K; x += blockDim.x) {
    if (cnt[x]) atomicAdd(moved_lr + x, (u64)cnt[x]);
    if (cnt[K + x]) atomicAdd(moved_tb + x, (u64)cnt[K + x]);
  }
}

// Resident step over a thread-block cluster: the lattice's rows are split
// into bands of R rows, one per block of the cluster (block c holds rows
// [c*R, min(M, (c+1)*R)) of both bitplanes, double buffered, in its shared
// memory), so a small lattice is stepped by several SMs instead of one.  The
// horizontal phase needs only the block's own rows.  The vertical phase
// reads the rows above and below a band's first and last rows from the
// neighbouring blocks' shared memory (distributed shared memory, through the
// generic addresses cluster.map_shared_rank gives).  One cluster barrier per
// step, between the phases, publishes every block's Lh; the vertical phase
// reads T of the current buffer and Lh of the other, and the next write of
// either happens only after the following step's cluster barrier, which a
// neighbour reaches only once its vertical phase is done; a block barrier
// after the vertical phase orders the block's own T' before the next
// horizontal phase.  A last cluster barrier keeps every block's shared
// memory alive until no neighbour reads it.  Each block adds its rows'
// counts of every step to the global counters at the end.
template <int WPT>
__global__ void __launch_bounds__(kResThreads, 1)
    resident_cluster_kernel(const u64 *__restrict__ Lin, const u64 *__restrict__ Tin,
                            u64 *__restrict__ Lout, u64 *__restrict__ Tout, ResGeom r, int R,
                            int K, u64 *__restrict__ moved_lr, u64 *__restrict__ moved_tb) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) u64 sm[];
  const int bw = R * r.P;  // words per buffer (R rows in every block)
  u64 *sL[2] = {sm, sm + bw};
  u64 *sT[2] = {sm + 2 * bw, sm + 3 * bw};
  unsigned int *cnt = (unsigned int *)(sm + 4 * bw);  // [2][K]
  const int row0 = rank * R;
  const int rows = r.M - row0 < R ? r.M - row0 : R;
  const int words = rows * r.P;
  const size_t g0 = (size_t)row0 * r.P;
  for (int x = threadIdx.x; x < bw; x += blockDim.x) {
    sL[0][x] = x < words ? Lin[g0 + x] : 0ull;
    sT[0][x] = x < words ? Tin[g0 + x] : 0ull;
    sL[1][x] = sT[1][x] = 0;  // padding words are never written by a step
  }
  for (int x = threadIdx.x; x < 2 * K; x += blockDim.x) cnt[x] = 0;

  // this thread's words: local index, horizontal neighbours (local), the
  // blocks holding the rows above and below and the word's offset there
  int xs[WPT], xr[WPT], xl[WPT], ou[WPT], od[WPT], topl[WPT];
  const u64 *bu[WPT], *bd[WPT];
  u64 valid[WPT], topbit[WPT], L[WPT], T[WPT];
#pragma unroll
  for (int j = 0; j < WPT; ++j) {
    const int x = threadIdx.x + j * blockDim.x;
    const int i = x / r.P, w = x - i * r.P;
    const bool on = x < words && w < r.W;
    xs[j] = on ? x : -1;
    const int wr = w == r.W - 1 ? 0 : w + 1, wl = w == 0 ? r.W - 1 : w - 1;
    xr[j] = i * r.P + wr;
    xl[j] = i * r.P + wl;
    const int gi = row0 + (on ? i : 0);
    const int giu = gi == 0 ? r.M - 1 : gi - 1, gid = gi == r.M - 1 ? 0 : gi + 1;
    const int ru = giu / R, rd = gid / R;
    ou[j] = (giu - ru * R) * r.P + w;
    od[j] = (gid - rd * R) * r.P + w;
    bu[j] = cluster.map_shared_rank(sm, ru);
    bd[j] = cluster.map_shared_rank(sm, rd);
    topl[j] = wl == r.W - 1 ? r.nb - 1 : 63;
    valid[j] = w == r.W - 1 ? r.tail : ~0ull;
    topbit[j] = 1ull << (w == r.W - 1 ? r.nb - 1 : 63);
    L[j] = T[j] = 0;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < WPT; ++j)
    if (xs[j] >= 0) {
      L[j] = sL[0][xs[j]];
      T[j] = sT[0][xs[j]];
    }
  const int lane = threadIdx.x & 31;
  int a = 0;
  for (int t = 0; t < K; ++t) {
    // ---- horizontal phase on the block's own rows ----
    uint32_t c = 0;
    u64 Lh[WPT];
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      Lh[j] = 0;
      if (xs[j] >= 0) {
        const u64 E = ~(L[j] | T[j]) & valid[j];
        const u64 er0 = ~(sL[a][xr[j]] | sT[a][xr[j]]) & 1ull;
        const u64 mvH = L[j] & ((E >> 1) | (er0 ? topbit[j] : 0ull));
        const u64 in_l = (sL[a][xl[j]] >> topl[j]) & E & 1ull;
        const u64 in = ((mvH << 1) | in_l) & valid[j];
        Lh[j] = L[j] ^ mvH ^ in;
        c += (uint32_t)__popcll(mvH);
        sL[a ^ 1][xs[j]] = Lh[j];
      }
    }
    // every block's Lh (and, at t = 0, its rows) becomes visible at the
    // cluster barrier; the count goes in while the barrier completes (a few
    // warps per block, so a shared atomic per warp costs little)
    barrier_cluster_arrive();
    c = __reduce_add_sync(BML_FULL_MASK, c);
    if (lane == 0 && c) atomicAdd(&cnt[t], c);
    barrier_cluster_wait();
    // ---- vertical phase: rows above and below, possibly in other blocks ----
    c = 0;
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      if (xs[j] >= 0) {
        const u64 Ei = ~(Lh[j] | T[j]) & valid[j];
        const u64 Ed = ~(bd[j][(a ^ 1) * bw + od[j]] | bd[j][(2 + a) * bw + od[j]]) & valid[j];
        const u64 mvV = T[j] & Ed;
        const u64 To = (T[j] & ~mvV) | (bu[j][(2 + a) * bw + ou[j]] & Ei);
        c += (uint32_t)__popcll(mvV);
        sT[a ^ 1][xs[j]] = To;
        T[j] = To;
        L[j] = Lh[j];
      }
    }
    c = __reduce_add_sync(BML_FULL_MASK, c);
    if (lane == 0 && c) atomicAdd(&cnt[K + t], c);
    __syncthreads();
    a ^= 1;
  }
  cluster.sync();  // no neighbour reads this block's shared memory any more
  for (int x = threadIdx.x; x < words; x += blockDim.x) {
    Lout[g0 + x] = sL[a][x];
    Tout[g0 + x] = sT[a][x];
  }
  for (int x = threadIdx.x; x < K; x += blockDim.x) {
    if (cnt[x]) atomicAdd(moved_lr + x, (u64)cnt[x]);
    if (cnt[K + x]) atomicAdd(moved_tb + x, (u64)cnt[K + x]);
  }
}

size_t resident_smem(const Geom &g, int K) {
  return (size_t)4 * (size_t)(g.M * g.P) * sizeof(u64) + (size_t)2 * K * sizeof(unsigned int);
}

template <int WPT>
cudaError_t launch_res(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const ResGeom &r,
                       int words, int k, size_t smem, u64 *moved_lr, u64 *moved_tb,
                       cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(resident_kernel<WPT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int threads = (words + WPT - 1) / WPT;
  threads = ((threads + 31) / 32) * 32;
  if (threads > kResThreads) threads = kResThreads;
  resident_kernel<WPT><<<1, threads, smem, st>>>(Lin, Tin, Lout, Tout, r, k, moved_lr, moved_tb);
  return cudaGetLastError();
}

size_t resident_cluster_smem(const Geom &g, int R, int K) {
  return (size_t)4 * (size_t)R * (size_t)g.P * sizeof(u64) + (size_t)2 * K * sizeof(unsigned int);
}

template <int WPT>
cudaError_t launch_res_cluster(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout,
                               const ResGeom &r, int R, int blocks, int k, size_t smem,
                               u64 *moved_lr, u64 *moved_tb, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(resident_cluster_kernel<WPT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int threads = (R * r.P + WPT - 1) / WPT;
  threads = ((threads + 31) / 32) * 32;
  if (threads > kResThreads) threads = kResThreads;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)blocks;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, resident_cluster_kernel<WPT>, Lin, Tin, Lout, Tout, r, R, k,
                            moved_lr, moved_tb);
}

}  // namespace

int resident_max_steps() { return 4096; }

int resident_blocks(const Geom &g, int64_t band_rows) {
  if (band_rows <= 0 || band_rows >= g.M) return 1;
  return (int)((g.M + band_rows - 1) / band_rows);
}

bool resident_applies(const Geom &g) {
  int dev = 0, cap = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return g.M * g.P <= 8 * kResThreads && resident_smem(g, resident_max_steps()) <= (size_t)cap;
}

cudaError_t launch_resident(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                            int k, int64_t band_rows, u64 *moved_lr, u64 *moved_tb,
                            cudaStream_t st) {
  if (k < 1 || k > resident_max_steps() || !resident_applies(g)) return cudaErrorInvalidValue;
  const ResGeom r{(int)g.M, (int)g.W, (int)g.P, g.nb, g.tail};
  const int blocks = resident_blocks(g, band_rows);
  if (blocks > 1) {
    if (blocks > kResMaxBlocks) return cudaErrorInvalidValue;
    const int R = (int)band_rows;
    const size_t smem = resident_cluster_smem(g, R, k);
    const int words = R * (int)g.P;
    if (words <= kResThreads)
      return launch_res_cluster<1>(Lin, Tin, Lout, Tout, r, R, blocks, k, smem, moved_lr,
                                   moved_tb, st);
    if (words <= 2 * kResThreads)
      return launch_res_cluster<2>(Lin, Tin, Lout, Tout, r, R, blocks, k, smem, moved_lr,
                                   moved_tb, st);
    if (words <= 4 * kResThreads)
      return launch_res_cluster<4>(Lin, Tin, Lout, Tout, r, R, blocks, k, smem, moved_lr,
                                   moved_tb, st);
    return launch_res_cluster<8>(Lin, Tin, Lout, Tout, r, R, blocks, k, smem, moved_lr,
                                 moved_tb, st);
  }
  const size_t smem = resident_smem(g, k);
  const int words = (int)(g.M * g.P);
  if (words <= kResThreads)
    return launch_res<1>(Lin, Tin, Lout, Tout, r, words, k, smem, moved_lr, moved_tb, st);
  if (words <= 2 * kResThreads)
    return launch_res<2>(Lin, Tin, Lout, Tout, r, words, k, smem, moved_lr, moved_tb, st);
  if (words <= 4 * kResThreads)
    return launch_res<4>(Lin, Tin, Lout, Tout, r, words, k, smem, moved_lr, moved_tb, st);
  return launch_res<8>(Lin, Tin, Lout, Tout, r, words, k, smem, moved_lr, moved_tb, st);
}

}  // namespace bml
