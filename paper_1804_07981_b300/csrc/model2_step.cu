// Model II streaming step: the Sec. 2 variant in which every vehicle moves in
// one synchronous phase per step and an empty cell wanted by both an LR
// vehicle (from its left) and a TB vehicle (from above) goes to one of them
// at random; k steps per launch (temporal blocking, k in 1, 2, 4, 8).
//
// The rule on one 64-cell word w of row x at step t, every operand taken
// from the state at the start of the step:
//   E        = ~(L_x | T_x)                     empty cells
//   fromL    = L_x shifted one column right      an LR vehicle on the left
//   coin     = SplitMix64(tie_seed, n),  n = t*M*W + x*W + w + 1
//              (bit j set: the LR vehicle wins cell j if it is contested)
//   inLR_x   = E & fromL & (~T_{x-1} | coin)     LR vehicles that enter
//   inTB_x   = E & T_{x-1} & ~(fromL & coin)     TB vehicles that enter from x-1
//   mvH_x    = inLR_x shifted one column left    LR vehicles that leave
//   L'_x     = (L_x & ~mvH_x) | inLR_x
//   T'_{x-1} = (T_{x-1} & ~inTB_x) | inTB_{x-1}
// Row x-1 is final once row x has been seen, so the pipeline is that of the
// Model I streaming kernel (stream_step.cu): k register-resident stages,
// stage s one step behind stage s-1, each keeping T_{x-1}, L'_{x-1} and
// inTB_{x-1} per lane; the same strips, halos (one word per side covers the
// 1-column-per-step cone), bands (k rows above and below) and ping-pong
// state sets.  Two warp shuffles per stage and row: the left neighbour's
// last L cell, and bit 0 of the right neighbour's inLR.
//
// The moved counts are LR vehicles that left (popcount of mvH) and TB
// vehicles that left row x-1 (popcount of inTB_x), for owned words and band
// rows only, reduced per warp, per block, then one 64-bit atomic per block
// and step.
#include "stage.cuh"

namespace bml {

namespace {

constexpr int kWarpsM2 = 4;

template <int K>
struct M2Pipe {
  u64 curT[K], curL[K], prevIn[K];
};

template <bool FULL>
__device__ __forceinline__ void stage_m2(u64 &inL, u64 &inT, const u64 curT, const u64 curL,
                                         const u64 prevIn, u64 &nT, u64 &nL, u64 &nIn,
                                         const LaneWord &lw, const u64 coin, u64 &mvH,
                                         u64 &mvV) {
  // the left neighbour's last cell, moved to bit 31 of the shuffled half
  const uint32_t send_l = FULL ? hi32(inL) : ((lw.top_hi ? hi32(inL) : lo32(inL)) << lw.top_sh);
  const uint32_t rl = __shfl_sync(BML_FULL_MASK, send_l, lw.src_l);
  const u64 fromL =
      mk64(__funnelshift_l(rl, lo32(inL), 1), __funnelshift_l(lo32(inL), hi32(inL), 1));
  // entering LR: empty, LR on the left, and no TB above or the coin says LR;
  // entering TB: empty, TB above, and no LR on the left or the coin says TB
  const u64 wantLR = lop3<kAndOrNot>(fromL, curT, coin);
  const u64 wantTB = lop3<kAndNand>(curT, fromL, coin);
  u64 inLR, inTB;
  if (FULL) {
    inLR = lop3<kNorAnd>(inL, inT, wantLR);
    inTB = lop3<kNorAnd>(inL, inT, wantTB);
  } else {
    const u64 E = lop3<kNorAnd>(inL, inT, lw.valid);
    inLR = lop3<kAnd>(E, wantLR, 0ull);
    inTB = lop3<kAnd>(E, wantTB, 0ull);
  }
  // bit 0 of the right neighbour's inLR enters at this word's last cell
  const uint32_t rr = __shfl_sync(BML_FULL_MASK, lo32(inLR), lw.src_r);
  if (FULL) {
    mvH = mk64(__funnelshift_r(lo32(inLR), hi32(inLR), 1), __funnelshift_r(hi32(inLR), rr, 1));
  } else {
    const uint32_t m = 0u - (rr & 1u);
    mvH = mk64(__funnelshift_r(lo32(inLR), hi32(inLR), 1) | (lw.ins_lo & m),
               (hi32(inLR) >> 1) | (lw.ins_hi & m));
  }
  mvV = inTB;
  nT = inT;
  nL = lop3<kAndNotOr>(inL, mvH, inLR);
  nIn = inTB;
  inT = lop3<kAndNotOr>(curT, inTB, prevIn);
  inL = curL;
}

// One row through all K stages; stage s works on lattice row x_s at step
// t0 + s.  With PRED only band rows are counted.
template <int K, bool FULL, bool PRED>
__device__ __forceinline__ void m2_row(u64 &inL, u64 &inT, const M2Pipe<K> &src, M2Pipe<K> &dst,
                                       const LaneWord &lw, int i, int B, int x0, int M,
                                       u64 tie_seed, u64 nbase, u64 MW, u64 W,
                                       uint32_t (&c_lr)[K], uint32_t (&c_tb)[K]) {
#pragma unroll
  for (int s = 0; s < K; ++s) {
    int x = x0 - s;  // lattice row of this stage's row (x0 = row of stage 0)
    while (x < 0) x += M;
    const u64 coin = splitmix64_at(tie_seed, nbase + (u64)s * MW + (u64)x * W);
    u64 mvH, mvV;
    stage_m2<FULL>(inL, inT, src.curT[s], src.curL[s], src.prevIn[s], dst.curT[s],
                   dst.curL[s], dst.prevIn[s], lw, coin, mvH, mvV);
    if (!PRED || (unsigned)(i - K - s) < (unsigned)B) c_lr[s] += popc64(mvH);
    if (!PRED || (unsigned)(i - K - s - 1) < (unsigned)B) c_tb[s] += popc64(mvV);
  }
}

template <int K, bool FULL>
__global__ void __launch_bounds__(kWarpsM2 * 32, K >= 8 ? 2 : (K >= 4 ? 3 : 4))
    model2_kernel(const u64 *__restrict__ Lin, const u64 *__restrict__ Tin,
                  u64 *__restrict__ Lout, u64 *__restrict__ Tout, Geom g, StripPlan sp,
                  int band_rows, int n_bands, u64 tie_seed, u64 t0, u64 *__restrict__ moved_lr,
                  u64 *__restrict__ moved_tb) {
  constexpr int P = 2;  // rows per unrolled chunk (the state sets alternate by row)
  __shared__ unsigned long long s_cnt[2 * K];
  for (int t = threadIdx.x; t < 2 * K; t += blockDim.x) s_cnt[t] = 0;
  pdl_wait();
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int tile = blockIdx.x * kWarpsM2 + (threadIdx.x >> 5);
  uint32_t c_lr[K], c_tb[K];
#pragma unroll
  for (int s = 0; s < K; ++s) c_lr[s] = c_tb[s] = 0;

  if (tile < sp.n_strips * n_bands) {  // warp-uniform
    const int strip = tile % sp.n_strips;
    const int band = tile / sp.n_strips;

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

    const int M = (int)g.M;
    const int r0 = band * band_rows;
    const int B = (r0 + band_rows < M ? band_rows : M - r0);
    const int n_in = B + 2 * K;
    int ld_row = (r0 - K) % M;
    if (ld_row < 0) ld_row += M;
    const size_t pitch = (size_t)g.P;
    const u64 *Lp = Lin + w + (size_t)ld_row * pitch;
    const u64 *Tp = Tin + w + (size_t)ld_row * pitch;
    const u64 *Lbase = Lin + w, *Tbase = Tin + w;
    u64 *Lo = Lout + w + (size_t)r0 * pitch;
    u64 *To = Tout + w + (size_t)r0 * pitch;

    const u64 W64 = (u64)g.W, MW = (u64)g.M * W64;
    const u64 nbase = t0 * MW + (u64)w + 1;  // + s*M*W + x*W per stage and row
    int x0 = ld_row;                          // lattice row of the next input row

    M2Pipe<K> pp[2];
#pragma unroll
    for (int s = 0; s < K; ++s) {
      pp[0].curT[s] = pp[0].curL[s] = pp[0].prevIn[s] = 0;
      pp[1].curT[s] = pp[1].curL[s] = pp[1].prevIn[s] = 0;
    }

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

    u64 bufL[P], bufT[P];
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

    for (int i0 = 0; i0 < n_in; i0 += P) {
      const bool steady = i0 >= 2 * K && i0 + P <= B + K;
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int i = i0 + u;
        if (steady || i < n_in) {  // warp-uniform
          u64 inL = bufL[u], inT = bufT[u];
          if (i + P < n_in) {
            if (on) {
              bufL[u] = __ldg(Lp);
              bufT[u] = __ldg(Tp);
            }
            advance();
          }
          if (steady)
            m2_row<K, FULL, false>(inL, inT, pp[u & 1], pp[(u & 1) ^ 1], lw, i, B, x0, M,
                                   tie_seed, nbase, MW, W64, c_lr, c_tb);
          else
            m2_row<K, FULL, true>(inL, inT, pp[u & 1], pp[(u & 1) ^ 1], lw, i, B, x0, M,
                                  tie_seed, nbase, MW, W64, c_lr, c_tb);
          if (++x0 == M) x0 = 0;
          if ((steady || i >= 2 * K) && own) {
            const size_t off = (size_t)(i - 2 * K) * pitch;
            __stcs(Lo + off, inL);
            __stcs(To + off, inT);
          }
        }
      }
    }
    if (!own) {
#pragma unroll
      for (int s = 0; s < K; ++s) c_lr[s] = c_tb[s] = 0;
    }
  }

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

template <int K>
cudaError_t launch_m2_k(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                        int64_t band_rows, u64 tie_seed, u64 t0, u64 *moved_lr, u64 *moved_tb,
                        cudaStream_t st) {
  const StripPlan sp = make_strip_plan(g, K);
  const int64_t n_bands = (g.M + band_rows - 1) / band_rows;
  const int64_t tiles = (int64_t)sp.n_strips * n_bands;
  if (tiles > INT32_MAX - kWarpsM2) return cudaErrorInvalidValue;
  const int64_t blocks = (tiles + kWarpsM2 - 1) / kWarpsM2;
  if (g.nb == 64)
    return launch_pdl(model2_kernel<K, true>, dim3((unsigned)blocks), dim3(kWarpsM2 * 32), 0, st,
                      Lin, Tin, Lout, Tout, g, sp, (int)band_rows, (int)n_bands, tie_seed, t0,
                      moved_lr, moved_tb);
  return launch_pdl(model2_kernel<K, false>, dim3((unsigned)blocks), dim3(kWarpsM2 * 32), 0, st,
                    Lin, Tin, Lout, Tout, g, sp, (int)band_rows, (int)n_bands, tie_seed, t0,
                    moved_lr, moved_tb);
}

template <int K, bool FULL>
int m2_occupancy_of() {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, model2_kernel<K, FULL>,
                                                    kWarpsM2 * 32, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return blocks > 0 ? blocks : 1;
}

}  // namespace

int model2_occupancy(const Geom &g, int k) {
  const bool full = g.nb == 64;
  switch (k) {
    case 1: return full ? m2_occupancy_of<1, true>() : m2_occupancy_of<1, false>();
    case 2: return full ? m2_occupancy_of<2, true>() : m2_occupancy_of<2, false>();
    case 4: return full ? m2_occupancy_of<4, true>() : m2_occupancy_of<4, false>();
    default: return full ? m2_occupancy_of<8, true>() : m2_occupancy_of<8, false>();
  }
}

cudaError_t launch_model2(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                          int k, int64_t band_rows, u64 tie_seed, u64 t0, u64 *moved_lr,
                          u64 *moved_tb, cudaStream_t st) {
  if (band_rows < 1 || band_rows > INT32_MAX) return cudaErrorInvalidValue;
  switch (k) {
    case 1: return launch_m2_k<1>(Lin, Tin, Lout, Tout, g, band_rows, tie_seed, t0, moved_lr, moved_tb, st);
    case 2: return launch_m2_k<2>(Lin, Tin, Lout, Tout, g, band_rows, tie_seed, t0, moved_lr, moved_tb, st);
    case 4: return launch_m2_k<4>(Lin, Tin, Lout, Tout, g, band_rows, tie_seed, t0, moved_lr, moved_tb, st);
    case 8: return launch_m2_k<8>(Lin, Tin, Lout, Tout, g, band_rows, tie_seed, t0, moved_lr, moved_tb, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bml
