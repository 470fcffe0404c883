// Streaming bitplane step: k full steps per launch (k = 1 is the fused
// single-pass step; k > 1 is temporal blocking).
//
// Work decomposition.  A warp owns a tile = (column strip, band of rows).
// Lane l holds one 64-cell word of the strip; a row of the strip is one
// coalesced 256-byte access per plane.  The warp streams the rows of its band
// from top to bottom through a pipeline of k stages held in registers; stage
// s applies one full step (horizontal then vertical phase, Sec. 2) to the
// rows that stage s-1 emits.  With E = EMPTY before the horizontal phase:
//
//   receive row x (L_x, T_x) of state s:
//     in_x  = (L_x shifted one column right) & E_x   cells LR cars enter
//     Lh_x  = (L_x & ~Er_x) | in_x   horizontal rule on row x (Er[j] = E[j+1])
//     E'_x  = ~(Lh_x | T_x)          EMPTY after the horizontal phase
//     mvV_{x-1} = T_{x-1} & E'_x     TB cars of row x-1 that move down
//   emit row x-1 of state s+1:
//     L = Lh_{x-1},  T = (T_{x-1} & ~mvV_{x-1}) | mvV_{x-2}
//
// since the cars entering row x-1 from above are exactly mvV_{x-2}, computed
// one row earlier.  Each stage lags one row behind the previous one and keeps
// three words per lane (T_{x-1}, Lh_{x-1}, mvV_{x-2}).  The only horizontal
// communication per stage and row is two 32-bit warp shuffles, both issued at
// the start of the stage: the right neighbour's low half of E (its bit 0 is
// the cell right of this word) and the left neighbour's half of L holding its
// last cell, pre-aligned to bit 31; the receiver funnel-shifts them in.
//
// Halos.  Each step widens the dependency cone by one row up and down and one
// column left and right.  A band [r0, r1) therefore reads rows
// [r0 - k, r1 + k) (wrapping modulo M) and its stages compute redundant rows
// that are neither stored nor counted.  A strip that does not cover the whole
// periodic row carries `halo` redundant words on each side (one word covers a
// 64-column cone; two when the neighbouring word is the short last word of
// the row).  Rows that fit in one warp (W <= 32) are whole periodic rings:
// lane W-1's right neighbour is lane 0.
//
// Input rows of a lattice larger than half of L2 reach a warp through a ring
// of row slots in shared memory, filled a few rows ahead with cp.async
// (stage.cuh: a lane copies the aligned 16-byte word pair that holds its word
// and reads back its own half); a slot is refilled two rows after it was
// last read.  Rows of a smaller lattice come from L2, whose latency a
// prefetch of P rows into registers already hides, so the ring's extra
// instructions per row would only cost time there.  The row loop runs in chunks of PF rows (PF even: the stage
// state sets alternate by row).  Chunks that lie entirely in the steady part
// of the band (every stage counts its row and the last stage stores) run
// without per-row predicates.
//
// Counts.  Sub-step s counts LR moves of its row x and TB moves of its
// emitted row x-1, only for owned rows and words, in per-lane registers; at
// the end they are reduced per warp, then per block in shared memory, and
// added with one 64-bit atomic per block and sub-step.
#include "stage.cuh"

namespace bml {

namespace {

constexpr int kWarpsPerBlock = 4;

// rows per unrolled chunk of the row loop
template <int K>
struct PF {
  static constexpr int value = K >= 4 ? 2 : 4;
};

// Row slots per warp and rows in flight ahead of the row being consumed.  At
// depth 1 a smaller ring keeps more blocks resident (shared memory would
// otherwise bound the occupancy, not registers).
template <int K>
struct RingGeom {
  static constexpr int slots = K >= 2 ? 8 : 4;
  static constexpr int ahead = slots - 2;
};

template <int K>
struct Pipe {
  StageH st[K];
};

// One row through all K stages.  With PRED, stage s counts its moves only
// for band rows (band-relative row i - K - s horizontally, the row above it
// vertically).
template <int K, bool FULL, bool PRED, bool M3>
__device__ __forceinline__ void row_through(uint32_t (&L)[2], uint32_t (&T)[2], const Pipe<K> &src,
                                            Pipe<K> &dst, const LaneWord &lw, int i, int B,
                                            uint32_t (&c_lr)[K], uint32_t (&c_tb)[K]) {
#pragma unroll
  for (int s = 0; s < K; ++s) {
    uint32_t mvIn, mvV;
    stage_step_h<FULL, M3>(L, T, src.st[s], dst.st[s], lw, mvIn, mvV);
    if (!PRED || (unsigned)(i - K - s) < (unsigned)B) c_lr[s] += mvIn;
    if (!PRED || (unsigned)(i - K - s - 1) < (unsigned)B) c_tb[s] += mvV;
  }
}

// RING: input rows through the shared-memory ring, else a register prefetch.
// M3: Model III (see stage.cuh).
template <int K, bool FULL, bool RING, bool M3>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, K >= 8 ? 3 : 4)
    stream_kernel(const u64 *__restrict__ Lin, const u64 *__restrict__ Tin,
                  u64 *__restrict__ Lout, u64 *__restrict__ Tout, Geom g, StripPlan sp,
                  int band_rows, int n_bands, u64 *__restrict__ moved_lr,
                  u64 *__restrict__ moved_tb) {
  constexpr int P = PF<K>::value;
  constexpr int kRing = RING ? RingGeom<K>::slots : 1, kAhead = RingGeom<K>::ahead;
  static_assert(!RING || (kAhead <= kRing - 2 && (kRing & (kRing - 1)) == 0), "ring layout");
  __shared__ unsigned long long s_cnt[2 * K];
  __shared__ __align__(16) RingSlot s_ring[kWarpsPerBlock][kRing];
  for (int t = threadIdx.x; t < 2 * K; t += blockDim.x) s_cnt[t] = 0;
  pdl_wait();
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int tile = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  uint32_t c_lr[K], c_tb[K];
#pragma unroll
  for (int s = 0; s < K; ++s) c_lr[s] = c_tb[s] = 0;

  if (tile < sp.n_strips * n_bands) {  // warp-uniform
    const int strip = tile % sp.n_strips;
    const int band = tile / sp.n_strips;

    // ---- lane -> word of the periodic row ----
    bool on, own;
    int w;
    LaneWord lw;
    if (sp.whole) {
      const int W = (int)g.W;
      on = lane < W;
      own = on;
      w = on ? lane : 0;
      lw.src_l = lane == 0 ? W - 1 : lane - 1;
      lw.src_r = lane == W - 1 ? 0 : lane + 1;
      if (!on) lw.src_l = lw.src_r = lane;
    } else {
      const int owned = sp.base + (strip < sp.rem ? 1 : 0);
      const int first = strip * sp.base + (strip < sp.rem ? strip : sp.rem);
      const int span = owned + 2 * sp.halo;
      on = lane < span;
      own = on && lane >= sp.halo && lane < sp.halo + owned;
      int ww = (first - sp.halo + lane) % (int)g.W;
      if (ww < 0) ww += (int)g.W;
      w = on ? ww : 0;
      lw.src_l = lane > 0 ? lane - 1 : 0;
      lw.src_r = lane + 1 < span ? lane + 1 : lane;
      if (!on) lw.src_l = lw.src_r = lane;
    }
    lane_word_bits(lw, on, w == g.W - 1, g.nb, g.tail);

    // ---- band rows: unrolled input rows [r0 - K, r1 + K) ----
    const int r0 = band * band_rows;
    const int B = (r0 + band_rows < g.M ? band_rows : (int)g.M - r0);
    const int n_in = B + 2 * K;
    int ld_row = (r0 - K) % (int)g.M;
    if (ld_row < 0) ld_row += (int)g.M;
    const size_t pitch = (size_t)g.P;
    // ring: the 16-byte word pair that holds this lane's word
    const int pw = RING ? (w & ~1) : w;
    const u64 *Lbase = Lin + pw, *Tbase = Tin + pw;
    const u64 *Lp = Lbase + (size_t)ld_row * pitch;
    const u64 *Tp = Tbase + (size_t)ld_row * pitch;
    const int half = w & 1;
    const int M = (int)g.M;
    u64 *Lo = Lout + w + (size_t)r0 * pitch;
    u64 *To = Tout + w + (size_t)r0 * pitch;

    Pipe<K> pp[2];  // state sets, alternated row by row (P is even)
#pragma unroll
    for (int s = 0; s < K; ++s) pp[0].st[s] = pp[1].st[s] = StageH{};

    auto advance = [&]() {
      if (++ld_row == M) {
        ld_row = 0;
        Lp = Lbase;
        Tp = Tbase;
      } else {
        Lp += pitch;
        Tp += pitch;
      }
    };

    RingSlot *ring = s_ring[threadIdx.x >> 5];
    u64 bufL[P], bufT[P];  // register prefetch (no ring)
    if constexpr (RING) {
      // rows 0 .. kAhead-1 in flight, one commit group per row (empty past n_in)
#pragma unroll
      for (int u = 0; u < kAhead; ++u) {
        if (u < n_in) {
          if (on) ring_fill(ring, u, lane, Lp, Tp);
          advance();
        }
        cp_async_commit();
      }
    } else {
#pragma unroll
      for (int u = 0; u < P; ++u) {
        bufL[u] = bufT[u] = 0;
        if (u < n_in) {
          if (on) {
            bufL[u] = __ldg(Lp);
            bufT[u] = __ldg(Tp);
          }
          advance();
        }
      }
    }

    for (int i0 = 0; i0 < n_in; i0 += P) {
      // steady chunk: every row of it has all stages counting and a store
      const bool steady = i0 >= 2 * K && i0 + P <= B + K;
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int i = i0 + u;
        if (steady || i < n_in) {  // warp-uniform
          u64 inL, inT;
          if constexpr (RING) {
            if (i + kAhead < n_in) {
              if (on) ring_fill(ring, (i + kAhead) & (kRing - 1), lane, Lp, Tp);
              advance();
            }
            cp_async_commit();
            cp_async_wait<kAhead>();  // row i has landed (this lane's own copies)
            // lanes that are off read a stale slot: they are neither stored
            // nor counted, and no lane that is on reads their words
            ring_read(ring, i & (kRing - 1), lane, half, inL, inT);
          } else {
            inL = bufL[u];
            inT = bufT[u];
            if (i + P < n_in) {
              if (on) {
                bufL[u] = __ldg(Lp);
                bufT[u] = __ldg(Tp);
              }
              advance();
            }
          }
          uint32_t L2[2] = {lo32(inL), hi32(inL)}, T2[2] = {lo32(inT), hi32(inT)};
          if (steady)
            row_through<K, FULL, false, M3>(L2, T2, pp[u & 1], pp[(u & 1) ^ 1], lw, i, B, c_lr,
                                            c_tb);
          else
            row_through<K, FULL, true, M3>(L2, T2, pp[u & 1], pp[(u & 1) ^ 1], lw, i, B, c_lr,
                                           c_tb);
          // row i - 2K of the band leaves the last stage (rows in order)
          if (steady || i >= 2 * K) {
            if (own) {
              __stcs(Lo, mk64(L2[0], L2[1]));
              __stcs(To, mk64(T2[0], T2[1]));
            }
            Lo += pitch;
            To += pitch;
          }
        }
      }
    }
    if (!own) {
#pragma unroll
      for (int s = 0; s < K; ++s) c_lr[s] = c_tb[s] = 0;
    }
  }

  // ---- counts: warp -> block (shared) -> global ----
  pdl_release();  // this block's lattice work is done
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const uint32_t a = __reduce_add_sync(BML_FULL_MASK, c_lr[s]);
    const uint32_t b = __reduce_add_sync(BML_FULL_MASK, c_tb[s]);
    if (lane == 0) {
      if (a) atomicAdd(&s_cnt[s], (unsigned long long)a);
      if (b) atomicAdd(&s_cnt[K + s], (unsigned long long)b);
    }
  }
  __syncthreads();
  if (threadIdx.x < K) {
    if (s_cnt[threadIdx.x]) atomicAdd(moved_lr + threadIdx.x, s_cnt[threadIdx.x]);
  } else if (threadIdx.x < 2 * K) {
    const int s = threadIdx.x - K;
    if (s_cnt[K + s]) atomicAdd(moved_tb + s, s_cnt[K + s]);
  }
}

// The ring pays off when the step's rows come from DRAM: both buffers of the
// lattice (2 planes each) take more than half of L2.
bool use_ring(const Geom &g) {
  int dev = 0, l2_bytes = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l2_bytes, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
    cudaGetLastError();
    l2_bytes = 126 << 20;
  }
  const double footprint = 2.0 * 2.0 * (double)g.M * (double)g.P * 8.0;
  return footprint > 0.5 * (double)l2_bytes;
}

template <int K, bool FULL, bool RING, bool M3>
cudaError_t launch_kfr(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                       const StripPlan &sp, int64_t band_rows, int64_t n_bands, int64_t blocks,
                       u64 *moved_lr, u64 *moved_tb, cudaStream_t st) {
  return launch_pdl(stream_kernel<K, FULL, RING, M3>, dim3((unsigned)blocks),
                    dim3(kWarpsPerBlock * 32), 0, st, Lin, Tin, Lout, Tout, g, sp,
                    (int)band_rows, (int)n_bands, moved_lr, moved_tb);
}

template <int K, bool M3>
cudaError_t launch_k(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                     int64_t band_rows, u64 *moved_lr, u64 *moved_tb, cudaStream_t st) {
  const StripPlan sp = make_strip_plan(g, K);
  const int64_t n_bands = (g.M + band_rows - 1) / band_rows;
  const int64_t tiles = (int64_t)sp.n_strips * n_bands;
  if (tiles > INT32_MAX - kWarpsPerBlock) return cudaErrorInvalidValue;
  const int64_t blocks = (tiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const bool full = g.nb == 64, ring = use_ring(g);
  if (full && ring)
    return launch_kfr<K, true, true, M3>(Lin, Tin, Lout, Tout, g, sp, band_rows, n_bands, blocks,
                                     moved_lr, moved_tb, st);
  if (full)
    return launch_kfr<K, true, false, M3>(Lin, Tin, Lout, Tout, g, sp, band_rows, n_bands, blocks,
                                      moved_lr, moved_tb, st);
  if (ring)
    return launch_kfr<K, false, true, M3>(Lin, Tin, Lout, Tout, g, sp, band_rows, n_bands, blocks,
                                      moved_lr, moved_tb, st);
  return launch_kfr<K, false, false, M3>(Lin, Tin, Lout, Tout, g, sp, band_rows, n_bands, blocks,
                                     moved_lr, moved_tb, st);
}

template <int K, bool FULL, bool RING>
int occupancy_of() {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, stream_kernel<K, FULL, RING, false>,
                                                    kWarpsPerBlock * 32, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return blocks > 0 ? blocks : 1;
}

template <int K>
int occupancy_k(const Geom &g) {
  const bool full = g.nb == 64, ring = use_ring(g);
  if (full) return ring ? occupancy_of<K, true, true>() : occupancy_of<K, true, false>();
  return ring ? occupancy_of<K, false, true>() : occupancy_of<K, false, false>();
}

}  // namespace

int stream_occupancy(const Geom &g, int k, int *warps_per_block) {
  if (warps_per_block) *warps_per_block = kWarpsPerBlock;
  switch (k) {
    case 1: return occupancy_k<1>(g);
    case 2: return occupancy_k<2>(g);
    case 4: return occupancy_k<4>(g);
    default: return occupancy_k<8>(g);
  }
}

StripPlan make_strip_plan(const Geom &g, int k) {
  StripPlan sp;
  if (g.W <= 32) {
    sp.whole = 1;
    sp.n_strips = 1;
    sp.halo = 0;
    sp.base = (int32_t)g.W;
    sp.rem = 0;
    return sp;
  }
  sp.whole = 0;
  // a one-word halo holds a cone of up to 64 columns, unless the halo word
  // is the short last word of the row
  sp.halo = (g.nb == 64 || k <= g.nb) ? 1 : 2;
  const int64_t per = 32 - 2 * sp.halo;
  sp.n_strips = (int32_t)((g.W + per - 1) / per);
  sp.base = (int32_t)(g.W / sp.n_strips);
  sp.rem = (int32_t)(g.W % sp.n_strips);
  return sp;
}

template <bool M3>
cudaError_t launch_stream_m(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                            int k, int64_t band_rows, u64 *moved_lr, u64 *moved_tb,
                            cudaStream_t st) {
  switch (k) {
    case 1: return launch_k<1, M3>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, st);
    case 2: return launch_k<2, M3>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, st);
    case 4: return launch_k<4, M3>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, st);
    case 8: return launch_k<8, M3>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_stream(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                          int k, int64_t band_rows, u64 *moved_lr, u64 *moved_tb,
                          cudaStream_t st, bool model3) {
  if (band_rows < 1 || band_rows > INT32_MAX) return cudaErrorInvalidValue;
  if (model3)
    return launch_stream_m<true>(Lin, Tin, Lout, Tout, g, k, band_rows, moved_lr, moved_tb, st);
  return launch_stream_m<false>(Lin, Tin, Lout, Tout, g, k, band_rows, moved_lr, moved_tb, st);
}

}  // namespace bml
