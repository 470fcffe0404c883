// Streaming bitplane step: k full steps per launch (k = 1 is the fused
// single-pass step; k > 1 is temporal blocking).
//
// Work decomposition.  A warp owns a tile = (column strip, band of rows).
// Lane l holds one 64-cell word of the strip; a row of the strip is one
// coalesced 256-byte access per plane.  The warp streams the rows of its band
// from top to bottom through a pipeline of k stages held in registers; stage
// s applies one full step (horizontal then vertical phase, Sec. 2) to the
// rows that stage s-1 emits:
//
//   receive row x (L_x, T_x) of state s:
//     E_x   = ~(L_x | T_x)                       (masked to real cells)
//     Lh_x  = (L_x & ~Er) | (Ll & E_x)           horizontal rule on row x
//     E'_x  = ~(Lh_x | T_x)
//     emit row x-1 of state s+1:
//       L = Lh_{x-1},  T = (T_{x-1} & ~E'_x) | (T_{x-2} & E'_{x-1})
//
// so each stage lags one row behind the previous one and keeps four words per
// lane (T_{x-2}, T_{x-1}, Lh_{x-1}, E'_{x-1}).  The only horizontal
// communication is one bit from each neighbouring lane per stage and row
// (two warp shuffles).
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
// Counts.  Sub-step s counts LR moves of its row x and TB moves of its
// emitted row x-1, only for owned rows and words, in per-lane registers;
// at the end they are reduced per warp, then per block in shared memory, and
// added with one 64-bit atomic per block and sub-step.
#include "device_common.cuh"

namespace bml {

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kPrefetch = 4;

template <int K>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    stream_kernel(const u64 *__restrict__ Lin, const u64 *__restrict__ Tin,
                  u64 *__restrict__ Lout, u64 *__restrict__ Tout, Geom g, StripPlan sp,
                  int64_t band_rows, int64_t n_bands, u64 *__restrict__ moved_lr,
                  u64 *__restrict__ moved_tb) {
  __shared__ unsigned long long s_cnt[2 * K];
  for (int t = threadIdx.x; t < 2 * K; t += blockDim.x) s_cnt[t] = 0;
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int64_t tile = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  uint32_t c_lr[K], c_tb[K];
#pragma unroll
  for (int s = 0; s < K; ++s) c_lr[s] = c_tb[s] = 0;

  if (tile < (int64_t)sp.n_strips * n_bands) {  // warp-uniform
    const int strip = (int)(tile % sp.n_strips);
    const int64_t band = tile / sp.n_strips;

    // ---- lane -> word of the periodic row ----
    bool on, own;
    int64_t w;
    int src_l, src_r;
    if (sp.whole) {
      on = lane < g.W;
      own = on;
      w = on ? lane : 0;
      src_l = lane == 0 ? (int)g.W - 1 : lane - 1;
      src_r = lane == (int)g.W - 1 ? 0 : lane + 1;
      if (!on) src_l = src_r = lane;
    } else {
      const int owned = sp.base + (strip < sp.rem ? 1 : 0);
      const int64_t first = (int64_t)strip * sp.base + (strip < sp.rem ? strip : sp.rem);
      const int span = owned + 2 * sp.halo;
      on = lane < span;
      own = on && lane >= sp.halo && lane < sp.halo + owned;
      int64_t ww = first - sp.halo + lane;
      ww %= g.W;
      if (ww < 0) ww += g.W;
      w = on ? ww : 0;
      src_l = lane > 0 ? lane - 1 : 0;
      src_r = lane + 1 < span ? lane + 1 : lane;
      if (!on) src_l = src_r = lane;
    }
    const u64 valid = on ? word_valid(w, g) : 0ull;
    const int top = word_top(w, g);

    // ---- band rows ----
    const int64_t r0 = band * band_rows;
    const int64_t r1 = r0 + band_rows < g.M ? r0 + band_rows : g.M;
    const int64_t xs = r0 - K, xe = r1 + K;  // unrolled input rows [xs, xe)
    int64_t ld_row = xs % g.M;
    if (ld_row < 0) ld_row += g.M;

    u64 prevT[K], curT[K], curLh[K], curE[K];
#pragma unroll
    for (int s = 0; s < K; ++s) prevT[s] = curT[s] = curLh[s] = curE[s] = 0;

    const u64 *Lp = Lin + w, *Tp = Tin + w;
    u64 bufL[kPrefetch], bufT[kPrefetch];
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      bufL[u] = bufT[u] = 0;
      if (xs + u < xe) {
        if (on) {
          bufL[u] = __ldg(Lp + ld_row * g.P);
          bufT[u] = __ldg(Tp + ld_row * g.P);
        }
        if (++ld_row == g.M) ld_row = 0;
      }
    }

    for (int64_t x0 = xs; x0 < xe; x0 += kPrefetch) {
#pragma unroll
      for (int u = 0; u < kPrefetch; ++u) {
        const int64_t x = x0 + u;
        if (x < xe) {  // warp-uniform
          u64 inL = bufL[u], inT = bufT[u];
          if (x + kPrefetch < xe) {
            if (on) {
              bufL[u] = __ldg(Lp + ld_row * g.P);
              bufT[u] = __ldg(Tp + ld_row * g.P);
            }
            if (++ld_row == g.M) ld_row = 0;
          }
#pragma unroll
          for (int s = 0; s < K; ++s) {
            // horizontal phase of step s+1 on unrolled row x - s
            const u64 E = ~(inL | inT) & valid;
            const uint32_t rb = __shfl_sync(BML_FULL_MASK, (uint32_t)E & 1u, src_r);
            const uint32_t lb = __shfl_sync(BML_FULL_MASK, (uint32_t)(inL >> top) & 1u, src_l);
            const u64 Er = (E >> 1) | ((u64)rb << top);
            const u64 Ll = (inL << 1) | (u64)lb;
            const u64 mvH = inL & Er;
            const u64 Lh = (inL & ~Er) | (Ll & E);
            const u64 Ep = ~(Lh | inT) & valid;
            // vertical phase of step s+1 on unrolled row x - s - 1
            const u64 mvV = curT[s] & Ep;
            const u64 oT = (curT[s] & ~Ep) | (prevT[s] & curE[s]);
            const u64 oL = curLh[s];
            const int64_t rh = x - s, rv = rh - 1;
            if (rh >= r0 && rh < r1) c_lr[s] += (uint32_t)__popcll(mvH);
            if (rv >= r0 && rv < r1) c_tb[s] += (uint32_t)__popcll(mvV);
            prevT[s] = curT[s];
            curT[s] = inT;
            curLh[s] = Lh;
            curE[s] = Ep;
            inL = oL;
            inT = oT;
          }
          const int64_t y = x - K;  // row of state K leaving the pipeline
          if (y >= r0 && own) {
            __stcs(Lout + y * g.P + w, inL);
            __stcs(Tout + y * g.P + w, inT);
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
cudaError_t launch_k(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                     int64_t band_rows, u64 *moved_lr, u64 *moved_tb, cudaStream_t st) {
  const StripPlan sp = make_strip_plan(g, K);
  const int64_t n_bands = (g.M + band_rows - 1) / band_rows;
  const int64_t tiles = (int64_t)sp.n_strips * n_bands;
  const int64_t blocks = (tiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  stream_kernel<K><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, st>>>(
      Lin, Tin, Lout, Tout, g, sp, band_rows, n_bands, moved_lr, moved_tb);
  return cudaGetLastError();
}

}  // namespace

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

cudaError_t launch_stream(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                          int k, int64_t band_rows, u64 *moved_lr, u64 *moved_tb,
                          cudaStream_t st) {
  if (band_rows < 1) return cudaErrorInvalidValue;
  switch (k) {
    case 1: return launch_k<1>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, st);
    case 2: return launch_k<2>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, st);
    case 4: return launch_k<4>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, st);
    case 8: return launch_k<8>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bml
