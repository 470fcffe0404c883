// Two-phase bitplane step: one horizontal-phase launch and one vertical-phase
// launch per step, on the two uint64 bitplanes L (LR) and T (TB).
//
// Horizontal phase (Sec. 2, first rule), on 64 cells of a row at a time:
//   E  = ~(L | T)              empty cells (tail bits masked)
//   Er = E shifted one cell toward lower columns: Er[j] = E[j+1 mod N]
//   Ll = L shifted one cell toward higher columns: Ll[j] = L[j-1 mod N]
//   moved = L & Er,  L' = (L & ~Er) | (Ll & E)
// Vertical phase (Sec. 2, second rule), row i against rows i-1 and i+1 of
// the horizontally updated lattice:
//   E_i = ~(L'_i | T_i),  moved = T_i & E_{i+1},
//   T'_i = (T_i & ~E_{i+1}) | (T_{i-1} & E_i)
// The cross-word shifts are 32-bit funnel shifts; the word holding column
// N-1 takes its right neighbour from bit 0 of word 0 and word 0 takes its
// left neighbour from column N-1, whatever N mod 64 is.
#include "device_common.cuh"

namespace bml {

namespace {

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 148;
  }
  return sms;
}

// Horizontal phase on the word pair (a, a+1) of one row: returns the updated
// L of both words, the pre-phase EMPTY masks and the number of LR cars that
// moved out of the pair.
struct HPair {
  u64 La, Lb, Ea, Eb;
  uint32_t moved;
};

__device__ __forceinline__ HPair h_pair(const u64 *__restrict__ Lr, const u64 *__restrict__ Tr,
                                        int64_t a, const Geom &g, u64 La, u64 Lb, u64 Ta,
                                        u64 Tb) {
  const int64_t b = a + 1;
  HPair r;
  r.Ea = ~(La | Ta) & word_valid(a, g);
  r.Eb = ~(Lb | Tb) & word_valid(b, g);
  // left neighbour of column 64a: the last cell of word a-1 (or of word W-1)
  const int64_t wl = a == 0 ? g.W - 1 : a - 1;
  const u64 lbit = (__ldg(Lr + wl) >> word_top(wl, g)) & 1ull;
  u64 Era, Erb, Llb;
  if (b < g.W) {
    // right neighbour of word b: bit 0 of word b+1, or of word 0 after N-1
    const int64_t wr = b == g.W - 1 ? 0 : b + 1;
    const u64 e0 = ~(__ldg(Lr + wr) | __ldg(Tr + wr)) & 1ull;
    Era = funnel_r1(r.Ea, r.Eb);
    Erb = (r.Eb >> 1) | (e0 << word_top(b, g));
    Llb = funnel_l1(La, Lb);
  } else {
    // word a is the last word of the row; b is padding
    const u64 e0 = ~(__ldg(Lr) | __ldg(Tr)) & 1ull;
    Era = (r.Ea >> 1) | (e0 << word_top(a, g));
    Erb = 0;
    Llb = 0;
  }
  const u64 Lla = (La << 1) | lbit;
  r.La = (La & ~Era) | (Lla & r.Ea);
  r.Lb = (Lb & ~Erb) | (Llb & r.Eb);
  r.moved = (uint32_t)(__popcll(La & Era) + __popcll(Lb & Erb));
  return r;
}

// A warp takes 32 consecutive word pairs of one row (a row segment), one pair
// per lane, with 128-bit loads of L and T.  The left neighbour's last L cell
// and the right neighbour's first E cell come from the adjacent lanes by
// shuffle, and from memory (loaded beside the pair) only at the segment's
// ends and at the row's wrap.  The (row, segment) of a warp advances by the
// number of warps in the grid, without a division per item.
__global__ void __launch_bounds__(256) plane_h_kernel(const u64 *__restrict__ L,
                                                      const u64 *__restrict__ T,
                                                      u64 *__restrict__ Lh, Geom g, u64 *moved) {
  const int np = (int)(g.P / 2), segs = (np + 31) / 32;
  const int W = (int)g.W;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t di = nwarps / segs;
  const int dseg = (int)(nwarps - di * segs);
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t i = w0 / segs;
  int seg = (int)(w0 - i * segs);
  uint32_t cnt = 0;
  pdl_wait();
  for (; i < g.M; i += di, seg += dseg) {
    if (seg >= segs) {
      seg -= segs;
      ++i;
      if (i >= g.M) break;
    }
    const int q = seg * 32 + lane;
    const bool on = q < np;
    const int a = 2 * q, b = a + 1;
    const bool a_last = a == W - 1, b_last = b == W - 1;
    // word whose first E cell is right of b (or of a when a ends the row),
    // and word whose last L cell is left of a, when they are not in the
    // neighbouring lanes
    const bool mem_r = on && (a_last || b_last || lane == 31);
    const bool mem_l = on && lane == 0;
    const int wr = (a_last || b_last) ? 0 : b + 1;
    const int wl = a == 0 ? W - 1 : a - 1;
    const u64 *Lr = L + i * g.P, *Tr = T + i * g.P;
    u64 La = 0, Lb = 0, Ta = 0, Tb = 0, Lrr = 0, Trr = 0, Lll = 0;
    if (on) {
      ld2(Lr + a, La, Lb);
      ld2(Tr + a, Ta, Tb);
    }
    if (mem_r) {
      Lrr = __ldg(Lr + wr);
      Trr = __ldg(Tr + wr);
    }
    if (mem_l) Lll = __ldg(Lr + wl);
    // only the pair holding the row's last word has cells to mask
    const bool full = b < W - 1;
    const u64 Ea = full ? ~(La | Ta) : (~(La | Ta) & word_valid(a, g));
    const u64 Eb = full ? ~(Lb | Tb) : (~(Lb | Tb) & word_valid(b, g));
    const uint32_t nxt_e = __shfl_down_sync(BML_FULL_MASK, (uint32_t)Ea, 1);
    const uint32_t prv_l = __shfl_up_sync(BML_FULL_MASK, (uint32_t)(Lb >> 32), 1);
    if (on) {
      const u64 e0 = mem_r ? (~(Lrr | Trr) & 1ull) : (u64)(nxt_e & 1u);
      const u64 lbit = mem_l ? ((Lll >> (a == 0 ? g.nb - 1 : 63)) & 1ull) : (u64)(prv_l >> 31);
      u64 Era, Erb, Llb;
      if (full) {
        Era = funnel_r1(Ea, Eb);
        Erb = (Eb >> 1) | (e0 << 63);
        Llb = funnel_l1(La, Lb);
      } else if (!a_last) {  // b ends the row
        Era = funnel_r1(Ea, Eb);
        Erb = (Eb >> 1) | (e0 << (g.nb - 1));
        Llb = funnel_l1(La, Lb);
      } else {  // a ends the row, b is padding
        Era = (Ea >> 1) | (e0 << (g.nb - 1));
        Erb = 0;
        Llb = 0;
      }
      const u64 Lla = (La << 1) | lbit;
      st2(Lh + i * g.P + a, (La & ~Era) | (Lla & Ea), (Lb & ~Erb) | (Llb & Eb));
      cnt += (uint32_t)(__popcll(La & Era) + __popcll(Lb & Erb));
    }
  }
  pdl_release();  // this block's lattice work is done
  block_count_add(cnt, moved);
}

// Fused one-pass step without bands: one thread per (group of R rows, pair
// of words).  It loads rows i0-1 .. i0+R of both planes at once (all loads
// independent, so many bytes are in flight), applies the horizontal rule to
// rows i0 .. i0+R (the vertical rule of row i0+R-1 needs E' of row i0+R) and
// the vertical rule to rows i0 .. i0+R-1.  Neighbouring threads share rows
// through L1/L2, so DRAM sees each row about once.
template <int R>
__global__ void __launch_bounds__(128) fused_rows_kernel(const u64 *__restrict__ L,
                                                         const u64 *__restrict__ T,
                                                         u64 *__restrict__ Lo,
                                                         u64 *__restrict__ To, Geom g,
                                                         u64 *moved_lr, u64 *moved_tb) {
  const int np = (int)(g.P / 2);
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int groups = (int)((g.M + R - 1) / R);
  uint32_t clr = 0, ctb = 0;
  pdl_wait();
  if (p < np) {
    const int64_t a = 2 * (int64_t)p;
    const u64 va = word_valid(a, g), vb = word_valid(a + 1, g);
    for (int grp = blockIdx.y; grp < groups; grp += gridDim.y) {
      const int64_t i0 = (int64_t)grp * R;
      u64 La[R + 1], Lb[R + 1], Ta[R + 1], Tb[R + 1], Tua, Tub;
      ld2(T + (i0 > 0 ? i0 - 1 : g.M - 1) * g.P + a, Tua, Tub);
      int64_t rows[R + 1];
#pragma unroll
      for (int r = 0; r <= R; ++r) {
        int64_t i = i0 + r;
        while (i >= g.M) i -= g.M;
        rows[r] = i;
        ld2(L + i * g.P + a, La[r], Lb[r]);
        ld2(T + i * g.P + a, Ta[r], Tb[r]);
      }
      u64 Ea[R + 1], Eb[R + 1], Ha[R + 1], Hb[R + 1];
#pragma unroll
      for (int r = 0; r <= R; ++r) {
        const HPair h = h_pair(L + rows[r] * g.P, T + rows[r] * g.P, a, g, La[r], Lb[r], Ta[r],
                               Tb[r]);
        Ha[r] = h.La;
        Hb[r] = h.Lb;
        Ea[r] = ~(h.La | Ta[r]) & va;
        Eb[r] = ~(h.Lb | Tb[r]) & vb;
        if (r < R && i0 + r < g.M) clr += h.moved;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (i0 + r < g.M) {
          const u64 upa = r == 0 ? Tua : Ta[r - 1], upb = r == 0 ? Tub : Tb[r - 1];
          st2(Lo + rows[r] * g.P + a, Ha[r], Hb[r]);
          st2(To + rows[r] * g.P + a, (Ta[r] & ~Ea[r + 1]) | (upa & Ea[r]),
              (Tb[r] & ~Eb[r + 1]) | (upb & Eb[r]));
          ctb += (uint32_t)(__popcll(Ta[r] & Ea[r + 1]) + __popcll(Tb[r] & Eb[r + 1]));
        }
      }
    }
  }
  pdl_release();  // this block's lattice work is done
  block_count_add(clr, moved_lr);
  block_count_add(ctb, moved_tb);
}

// One thread per (band of rows, pair of words): marches down the band with
// the previous row's T and the current row's E in registers.  Padding words
// (past column N) hold no TB car, so no move involves them and the vertical
// rule needs no column mask.
__global__ void __launch_bounds__(256) plane_v_kernel(const u64 *__restrict__ Lh,
                                                         const u64 *__restrict__ T,
                                                         u64 *__restrict__ Tv, Geom g,
                                                         int64_t band, u64 *moved) {
  const int64_t np = g.P / 2, nbands = (g.M + band - 1) / band, total = nbands * np;
  uint32_t cnt = 0;
  pdl_wait();
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bnd = idx / np, p = idx - bnd * np;
    const int64_t r0 = bnd * band;
    const int len = (int)(r0 + band < g.M ? band : g.M - r0);
    const bool wraps = r0 + len == g.M;  // the band's last row reads row 0 below it
    const int64_t off0 = 2 * p;
    const u64 *lp = Lh + r0 * g.P + off0, *tp = T + r0 * g.P + off0;
    u64 *op = Tv + r0 * g.P + off0;
    u64 Tpa, Tpb, x0, x1, Ta, Tb;
    ld2(r0 > 0 ? tp - g.P : T + (g.M - 1) * g.P + off0, Tpa, Tpb);
    ld2(lp, x0, x1);
    ld2(tp, Ta, Tb);
    u64 Ea = ~(x0 | Ta), Eb = ~(x1 | Tb);
#pragma unroll 1
    for (int k = 0; k < len; ++k) {
      lp += g.P;
      tp += g.P;
      const bool w = k + 1 == len && wraps;
      u64 Lna, Lnb, Tna, Tnb;
      ld2(w ? Lh + off0 : lp, Lna, Lnb);
      ld2(w ? T + off0 : tp, Tna, Tnb);
      const u64 Ena = ~(Lna | Tna), Enb = ~(Lnb | Tnb);
      const u64 mva = Ta & Ena, mvb = Tb & Enb;
      st2(op, (Ta & ~Ena) | (Tpa & Ea), (Tb & ~Enb) | (Tpb & Eb));
      op += g.P;
      cnt += (uint32_t)(__popcll(mva) + __popcll(mvb));
      Tpa = Ta;
      Tpb = Tb;
      Ta = Tna;
      Tb = Tnb;
      Ea = Ena;
      Eb = Enb;
    }
  }
  pdl_release();  // this block's lattice work is done
  block_count_add(cnt, moved);
}

int grid_cap(int64_t items, int threads, int per_sm) {
  int64_t blocks = (items + threads - 1) / threads;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

// Blocks of `threads` threads of kernel f resident per SM (at least 1): the
// grid-stride kernels launch exactly one wave of them, so that every block's
// equal share of the items runs concurrently.
template <typename F>
int resident_per_sm(F f, int threads) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return b > 0 ? b : 1;
}

}  // namespace

cudaError_t launch_plane_h(const u64 *L, const u64 *T, u64 *Lh, const Geom &g, u64 *moved,
                           cudaStream_t st) {
  const int64_t items = g.M * ((g.P / 2 + 31) / 32) * 32;
  static const int per_sm = resident_per_sm(plane_h_kernel, 256);
  return launch_pdl(plane_h_kernel, dim3(grid_cap(items, 256, per_sm)), dim3(256), 0, st, L, T,
                    Lh, g, moved);
}

cudaError_t launch_fused_direct(const u64 *L, const u64 *T, u64 *Lo, u64 *To, const Geom &g,
                                u64 *moved_lr, u64 *moved_tb, cudaStream_t st) {
  constexpr int R = 4;
  const int64_t np = g.P / 2;
  const int64_t groups = (g.M + R - 1) / R;
  dim3 grid((unsigned)((np + 127) / 128), (unsigned)(groups < 65535 ? groups : 65535));
  return launch_pdl(fused_rows_kernel<R>, grid, dim3(128), 0, st, L, T, Lo, To, g, moved_lr,
                    moved_tb);
}

cudaError_t launch_plane_v(const u64 *Lh, const u64 *T, u64 *Tv, const Geom &g, u64 *moved,
                           cudaStream_t st) {
  // Band height: as short as one resident wave of threads allows, so that
  // every thread marches down exactly one band (no tail of threads doing one
  // band more than the others) and the re-read row above each band is 1/band
  // of the traffic; at least 8 rows, at most 1024.
  static const int per_sm = resident_per_sm(plane_v_kernel, 256);
  const int64_t np = g.P / 2;
  const int64_t threads = (int64_t)sm_count() * per_sm * 256;
  int64_t band = (g.M * np + threads - 1) / threads;
  band = band < 8 ? 8 : (band > 1024 ? 1024 : band);
  const int64_t items = ((g.M + band - 1) / band) * np;
  return launch_pdl(plane_v_kernel, dim3(grid_cap(items, 256, per_sm)), dim3(256), 0, st, Lh, T,
                    Tv, g, band, moved);
}

}  // namespace bml
