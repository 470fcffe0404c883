// Streaming bitplane step with two words per lane (rows whose every word holds
// 64 cells, N % 64 == 0, and wider than one warp strip).
//
// Same pipeline as stream_step.cu (k stages in registers, the Sec. 2 rules
// per stage, the TB cars entering a row being the previous row's TB move
// mask), but a lane holds one aligned pair of ring words (128 columns), read
// and written with 128-bit accesses.  For the paper's model the planes are
// kept in the interleaved layout (launch_pair_layout: every word's even
// columns in its low half, its odd columns in its high half), so that a
// cell's right neighbour is mostly the same bit of the other half and the
// horizontal rule needs half the shifts of the plain layout.  Per stage and
// row a lane makes two 32-bit shuffles for two words: the right lane's even
// columns of E and the left lane's odd columns of the LR move mask.
//
// Lane groups.  A row of WP <= 32 pairs is one cyclic group of WP lanes (the
// whole ring, no halo).  Wider rows are cut into segments of 31 pairs and a
// remainder segment; a segment's group is its lanes plus one halo lane that
// holds the first 64 columns right of the segment (its first word) and the
// last 64 columns left of it (its second word), and the group's shuffles are
// cyclic.  The halo lane's two words are not neighbours in the lattice, but
// a cell d columns away from a wrong neighbour is still exact after d steps
// (a car moves one cell per phase and a phase reads only neighbours), so the
// segment's cells, 64 columns from that junction, stay exact at every depth
// the kernel runs (k <= 8).  Remainder groups of several bands share a
// warp (up to 32 lanes), so a row of 256 pairs costs 8 + 1/3 warp tiles per
// band instead of 9 with a halo lane on each side of 30 pairs.  At depth 1
// (bound by HBM) rows of more than 32 pairs keep that strip form instead:
// see PairPlan.
//
// Moved-car counts: one 32-bit register per stage and lane holds the LR moves
// in its low 16 bits and the TB moves in its high 16 bits (a lane moves at
// most 128 cars of each kind per row, so a field cannot overflow within 511
// rows); the kernel flushes both fields to the block's counters every 256
// rows.  This keeps the depth-8 kernel within 255 registers without spills.
//
// Input rows reach the warp through a ring of kRing row slots in shared
// memory, filled kAhead rows ahead with cp.async (see fetch_row); a slot is
// refilled at least two rows after it was last read.  The
// prefetch holds no registers and its wait is explicit.  In the steady part
// of a band two rows are read from the ring before either runs its stages,
// so that the second row's early stages can overlap the first row's late
// ones.
//
// MODEL = 3 runs Model III (one synchronous phase; a cell may hold one
// vehicle of each kind) in the interleaved layout: the same stage as the
// paper's model with the TB moves read from the state at the step's start.
//
// MODEL = 2 runs the Model II rule of model2_step.cu (one synchronous phase,
// tie-break words from the step, row and word indices) on the same
// structure, in the plain layout: per stage and row a lane draws the two tie-break words of its
// pair, shuffles the left lane's last L cell and bit 0 of the right lane's
// inLR, and the state word handed on is inTB instead of mvV.
#include <type_traits>

#include "stage.cuh"

namespace bml {

namespace {

constexpr int kWarps2 = 4;
constexpr int kRing = 8;   // row slots per warp
constexpr int kAhead = 5;  // rows in flight ahead of the row being consumed
// a slot is refilled at least two rows after it was last read, also when the
// steady loop fetches two rows at once
static_assert(kAhead + 1 <= kRing - 2 && (kRing & (kRing - 1)) == 0, "ring layout");

__device__ __forceinline__ uint32_t fsr(uint32_t lo, uint32_t hi) { return __funnelshift_r(lo, hi, 1); }
__device__ __forceinline__ uint32_t fsl(uint32_t lo, uint32_t hi) { return __funnelshift_l(lo, hi, 1); }

// A lane's 128 columns as four 32-bit halves: a.lo, a.hi, b.lo, b.hi, where
// a is the pair's 64 even columns (bit i = column 2i of the pair's 128) and b
// its 64 odd columns.  In the interleaved layout a.lo and b.lo are the low
// and high halves of the pair's first word, a.hi and b.hi those of its
// second.  Model I keeps every value of a stage as separate 32-bit halves (no
// 64-bit register pairs to form), which measured 3-7% faster than the same
// logic on u64.
typedef uint32_t Quad[4];

// Stage state of the paper's model: T_{x-1}, Lh_{x-1}, mvV_{x-2} (halves).
struct StateI {
  Quad T, L, M;
};

// One Model I stage on the lane's 128 columns (a: even columns, b: odd
// columns; see Quad); see stage.cuh for the rule.  The right neighbour of even column 2i is odd column 2i + 1, the
// same bit of b, so the even cells' move mask needs no shift:
// mHa = La & ~(Lb | Tb), and the cars entering the odd cells are exactly
// mHa.  Only the odd cells' right neighbours (a shifted one bit, the right
// lane's column 0 entering at bit 63) and the even cells' entering cars (mHb
// shifted one bit, the left lane's column 127 entering at bit 0) need
// shifts: 4 funnel shifts per pair and stage instead of 8 in the plain
// layout, 22 logic operations instead of 28.  Every rule line is one lop3
// per half (18 of the 22), so the count holds in the compiled kernel.
//
// M3: Model III (one synchronous phase; a cell may hold one vehicle of each
// kind): a TB vehicle moves iff the cell below held no vehicle at the start
// of the step, so mV reads the row's input L instead of Lh.
template <bool M3>
__device__ __forceinline__ void stage_i(Quad &L, Quad &T, const StateI &st, StateI &nx,
                                        int src_l, int src_r, uint32_t &cnt, bool cnt_h,
                                        bool cnt_v) {
  const uint32_t Ea0 = lop3<kNor>(L[0], T[0], 0u), Ea1 = lop3<kNor>(L[1], T[1], 0u);
  const uint32_t rr = __shfl_sync(BML_FULL_MASK, Ea0, src_r);
  const uint32_t mHa0 = lop3<kAndNor>(L[0], L[2], T[2]), mHa1 = lop3<kAndNor>(L[1], L[3], T[3]);
  const uint32_t mHb0 = lop3<kAnd>(L[2], fsr(Ea0, Ea1), 0u),
                 mHb1 = lop3<kAnd>(L[3], fsr(Ea1, rr), 0u);
  const uint32_t rl = __shfl_sync(BML_FULL_MASK, mHb1, src_l);
  const Quad Lh = {lop3<kXor3>(L[0], mHa0, fsl(rl, mHb0)), lop3<kXor3>(L[1], mHa1, fsl(mHb0, mHb1)),
                   lop3<kXor3>(L[2], mHb0, mHa0), lop3<kXor3>(L[3], mHb1, mHa1)};
  Quad mV;
#pragma unroll
  for (int h = 0; h < 4; ++h) mV[h] = lop3<kAndNor>(st.T[h], M3 ? L[h] : Lh[h], T[h]);
  // a car cannot move while the cell to its right holds a car, so the cars of
  // columns 2i and 2i + 1 never both move: mHa and mHb share no bit, and one
  // popcount per half pair counts both (the popcounts' pipe, not the logic,
  // was the busiest unit before)
  if (cnt_h) cnt += __popc(mHa0 | mHb0) + __popc(mHa1 | mHb1);
  if (cnt_v) cnt += (__popc(mV[0]) + __popc(mV[1]) + __popc(mV[2]) + __popc(mV[3])) << 16;
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    nx.T[h] = T[h];
    nx.L[h] = Lh[h];
    nx.M[h] = mV[h];
    T[h] = lop3<kAndNotOr>(st.T[h], mV[h], st.M[h]);
    L[h] = st.L[h];
  }
}

// Stage state of Model II (plain layout): T_{x-1}, L'_{x-1}, inTB_{x-1}.
struct StateII {
  u64 Ta, Tb, La, Lb, Ma, Mb;
};

// One Model II stage on the word pair (a, b); st.M is inTB of the row above.
__device__ __forceinline__ void stage_ii(u64 &La, u64 &Lb, u64 &Ta, u64 &Tb, const StateII &st,
                                         StateII &nx, int src_l, int src_r, uint32_t &cnt,
                                         bool cnt_h, bool cnt_v, u64 coinA, u64 coinB) {
  const uint32_t rl = __shfl_sync(BML_FULL_MASK, hi32(Lb), src_l);
  const u64 fLa = mk64(fsl(rl, lo32(La)), fsl(lo32(La), hi32(La)));
  const u64 fLb = mk64(fsl(hi32(La), lo32(Lb)), fsl(lo32(Lb), hi32(Lb)));
  // entering LR: empty, LR on the left, and no TB above or the coin says LR;
  // entering TB: empty, TB above, and no LR on the left or the coin says TB
  const u64 iLa = lop3<kNorAnd>(La, Ta, lop3<kAndOrNot>(fLa, st.Ta, coinA)),
            iLb = lop3<kNorAnd>(Lb, Tb, lop3<kAndOrNot>(fLb, st.Tb, coinB));
  const u64 iTa = lop3<kNorAnd>(La, Ta, lop3<kAndNand>(st.Ta, fLa, coinA)),
            iTb = lop3<kNorAnd>(Lb, Tb, lop3<kAndNand>(st.Tb, fLb, coinB));
  const uint32_t rr = __shfl_sync(BML_FULL_MASK, lo32(iLa), src_r);
  const u64 mHa = mk64(fsr(lo32(iLa), hi32(iLa)), fsr(hi32(iLa), lo32(iLb)));
  const u64 mHb = mk64(fsr(lo32(iLb), hi32(iLb)), fsr(hi32(iLb), rr));
  const u64 oTa = lop3<kAndNotOr>(st.Ta, iTa, st.Ma), oTb = lop3<kAndNotOr>(st.Tb, iTb, st.Mb);
  if (cnt_h) cnt += popc64(mHa) + popc64(mHb);
  if (cnt_v) cnt += (popc64(iTa) + popc64(iTb)) << 16;
  nx.Ta = Ta;
  nx.Tb = Tb;
  nx.La = lop3<kAndNotOr>(La, mHa, iLa);
  nx.Lb = lop3<kAndNotOr>(Lb, mHb, iLb);
  nx.Ma = iTa;
  nx.Mb = iTb;
  La = st.La;
  Lb = st.Lb;
  Ta = oTa;
  Tb = oTb;
}

// Adds the packed per-lane counts of every stage (lanes that own no pair
// contribute nothing) to the block's counters and clears them.
template <int K>
__device__ __forceinline__ void flush_counts(uint32_t (&cnt)[K], bool own, int lane,
                                             unsigned long long *s_cnt) {
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const uint32_t c = own ? cnt[s] : 0u;
    const uint32_t a = __reduce_add_sync(BML_FULL_MASK, c & 0xffffu);
    const uint32_t b = __reduce_add_sync(BML_FULL_MASK, c >> 16);
    if (lane == 0) {
      if (a) atomicAdd(&s_cnt[s], (unsigned long long)a);
      if (b) atomicAdd(&s_cnt[K + s], (unsigned long long)b);
    }
    cnt[s] = 0;
  }
}

// Store a lane's pair (the inverse of read_row's order).
template <int MODEL>
__device__ __forceinline__ void st_quad(u64 *p, const Quad &v) {
  __stcs(reinterpret_cast<uint4 *>(p), MODEL == 2 ? make_uint4(v[0], v[1], v[2], v[3])
                                                  : make_uint4(v[0], v[2], v[1], v[3]));
}

// Per-lane constants and running positions of a tile.
struct PairTile {
  const u64 *Lin;  // this lane's first word in row 0 of the input L plane
  const u64 *fL;   // this lane's first word in the next row to fetch (L plane)
  int64_t dT;      // T plane minus L plane, in words (input and output)
  int64_t dH;      // this lane's second word minus its first (1, except the halo lane)
  bool split;      // the tile has a two-sided halo lane: 8-byte copies (warp-uniform)
  u64 *sL;         // this lane's pair in the next row to store (L plane)
  size_t pitch;    // row pitch in words
  int ld_row, M;   // lattice row of the next row to fetch
  int wa;          // first word of this lane's (owned) pair
  int r0, B, n_in; // band start, band rows, input rows (B + 2K); B = 0 off a band
  int src_l, src_r;
  bool own;
  u64 W64, MW, nbase, tie_seed;  // Model II tie-break counters
  int x0;                        // lattice row of the current input row (Model II)
};

// Fetch the next input row into ring slot `slot` (one commit group).  In a
// tile with a two-sided halo lane every lane makes two 8-byte copies per
// plane (the halo lane's words come from two pairs; copies chosen per lane
// made the warp diverge on every row and measured 3% slower at depth 8),
// otherwise one 16-byte copy per plane.
__device__ __forceinline__ void fetch_row(PairTile &t, RingSlot *ring, int lane, int slot) {
  u64 *dL = reinterpret_cast<u64 *>(&ring[slot][0][lane]);
  u64 *dT = reinterpret_cast<u64 *>(&ring[slot][1][lane]);
  const u64 *fT = t.fL + t.dT;
  if (t.split) {
    cp_async8(dL, t.fL);
    cp_async8(dL + 1, t.fL + t.dH);
    cp_async8(dT, fT);
    cp_async8(dT + 1, fT + t.dH);
  } else {
    cp_async16(dL, t.fL);
    cp_async16(dT, fT);
  }
  if (++t.ld_row == t.M) {
    t.ld_row = 0;
    t.fL = t.Lin;
  } else {
    t.fL += t.pitch;
  }
}

// Ring slot of input row i as four halves per plane: in memory order for
// Model II (plain layout: first word, second word), as (a.lo, a.hi, b.lo,
// b.hi) for the interleaved layout (see Quad).
template <int MODEL>
__device__ __forceinline__ void read_row(const RingSlot *ring, int lane, int i, Quad &L, Quad &T) {
  const uint4 vL = *reinterpret_cast<const uint4 *>(&ring[i & (kRing - 1)][0][lane]);
  const uint4 vT = *reinterpret_cast<const uint4 *>(&ring[i & (kRing - 1)][1][lane]);
  if (MODEL == 2) {
    L[0] = vL.x, L[1] = vL.y, L[2] = vL.z, L[3] = vL.w;
    T[0] = vT.x, T[1] = vT.y, T[2] = vT.z, T[3] = vT.w;
  } else {
    L[0] = vL.x, L[1] = vL.z, L[2] = vL.y, L[3] = vL.w;
    T[0] = vT.x, T[1] = vT.z, T[2] = vT.y, T[3] = vT.w;
  }
}

// Input row i (already in registers) through the K stages; U selects the
// state set the row reads (the other receives the row's new state).  GUARD:
// a stage's row may lie outside the band (then it is not counted).
template <int K, int MODEL, bool GUARD, int U, typename ST>
__device__ __forceinline__ void run_stages(PairTile &t, int i, int x0, Quad &L, Quad &T,
                                           ST (&st)[2][K], uint32_t (&cnt)[K]) {
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const bool ch = !GUARD || (unsigned)(i - K - s) < (unsigned)t.B;
    const bool cv = !GUARD || (unsigned)(i - K - s - 1) < (unsigned)t.B;
    if constexpr (MODEL == 2) {
      int x = x0 - s;  // lattice row of this stage's row
      while (x < 0) x += t.M;
      const u64 n = t.nbase + (u64)s * t.MW + (u64)x * t.W64;
      u64 La = mk64(L[0], L[1]), Lb = mk64(L[2], L[3]), Ta = mk64(T[0], T[1]),
          Tb = mk64(T[2], T[3]);
      stage_ii(La, Lb, Ta, Tb, st[U][s], st[U ^ 1][s], t.src_l, t.src_r, cnt[s], ch, cv,
               splitmix64_at(t.tie_seed, n), splitmix64_at(t.tie_seed, n + (u64)t.dH));
      L[0] = lo32(La), L[1] = hi32(La), L[2] = lo32(Lb), L[3] = hi32(Lb);
      T[0] = lo32(Ta), T[1] = hi32(Ta), T[2] = lo32(Tb), T[3] = hi32(Tb);
    } else {
      stage_i<MODEL == 3>(L, T, st[U][s], st[U ^ 1][s], t.src_l, t.src_r, cnt[s], ch, cv);
    }
  }
}

// Store the next emitted row (band rows in order); `in_band`: the row lies
// in the lane's band.
template <int MODEL>
__device__ __forceinline__ void store_row(PairTile &t, const Quad &L, const Quad &T,
                                          bool in_band = true) {
  if (t.own && in_band) {
    st_quad<MODEL>(t.sL, L);
    st_quad<MODEL>(t.sL + t.dT, T);
  }
  t.sL += t.pitch;
}

// One input row near the band's ends (pipeline fill and drain), run by the
// whole warp while any of its lanes has input rows left (the bands of a
// warp's lane groups may differ in height): a lane fetches only its own input
// rows, stages whose row lies outside the lane's band are not counted, and a
// lane stores only rows of its band, from row 2K on (lanes past their input
// run on stale slots and keep nothing).
template <int K, int MODEL, int U, typename ST>
__device__ __forceinline__ void guarded_row(PairTile &t, RingSlot *ring, int lane, int i,
                                            ST (&st)[2][K], uint32_t (&cnt)[K]) {
  if (i + kAhead < t.n_in) fetch_row(t, ring, lane, (i + kAhead) & (kRing - 1));
  cp_async_commit();
  cp_async_wait<kAhead>();  // row i has landed
  Quad L, T;
  read_row<MODEL>(ring, lane, i, L, T);
  run_stages<K, MODEL, true, U>(t, i, t.x0, L, T, st, cnt);
  if (++t.x0 == t.M) t.x0 = 0;
  if (i >= 2 * K) store_row<MODEL>(t, L, T, i - 2 * K < t.B);
}

// One input row of the band's steady part (below the smallest B + K of the
// warp's lanes): every stage's row lies in the lane's band and the emitted
// row is stored.
template <int K, int MODEL, int U, typename ST>
__device__ __forceinline__ void steady_row1(PairTile &t, RingSlot *ring, int lane, int i,
                                            ST (&st)[2][K], uint32_t (&cnt)[K]) {
  if (K >= kAhead || i + kAhead < t.n_in) fetch_row(t, ring, lane, (i + kAhead) & (kRing - 1));
  cp_async_commit();
  cp_async_wait<kAhead>();  // row i has landed
  Quad L, T;
  read_row<MODEL>(ring, lane, i, L, T);
  run_stages<K, MODEL, false, U>(t, i, t.x0, L, T, st, cnt);
  if (++t.x0 == t.M) t.x0 = 0;
  store_row<MODEL>(t, L, T);
}

// Two input rows i, i + 1 of the band's steady part (both below the
// smallest B + K of the warp's lanes):
// every stage's row lies in the band and both emitted rows are stored.  Both
// rows are fetched from the ring before any stage runs, so the stages of row
// i + 1 can overlap the later stages of row i (no memory operation of row i
// sits between them).
template <int K, int MODEL, typename ST>
__device__ __forceinline__ void steady_rows(PairTile &t, RingSlot *ring, int lane, int i,
                                            ST (&st)[2][K], uint32_t (&cnt)[K]) {
  if constexpr (MODEL == 2) {
    // Model II: one row at a time (reading both rows first measured 4% slower:
    // its longer stage already fills the schedule)
    steady_row1<K, MODEL, 0>(t, ring, lane, i, st, cnt);
    steady_row1<K, MODEL, 1>(t, ring, lane, i + 1, st, cnt);
    return;
  }
  // rows i + kAhead and i + kAhead + 1 exist when K > kAhead (i + 1 < B + K)
  if (K > kAhead || i + kAhead < t.n_in) fetch_row(t, ring, lane, (i + kAhead) & (kRing - 1));
  cp_async_commit();
  if (K > kAhead || i + kAhead + 1 < t.n_in)
    fetch_row(t, ring, lane, (i + kAhead + 1) & (kRing - 1));
  cp_async_commit();
  cp_async_wait<kAhead>();  // rows i and i + 1 have landed
  Quad L0, T0, L1, T1;
  read_row<MODEL>(ring, lane, i, L0, T0);
  read_row<MODEL>(ring, lane, i + 1, L1, T1);
  const int x0 = t.x0;
  int x1 = x0 + 1;
  if (x1 == t.M) x1 = 0;
  run_stages<K, MODEL, false, 0>(t, i, x0, L0, T0, st, cnt);
  run_stages<K, MODEL, false, 1>(t, i + 1, x1, L1, T1, st, cnt);
  t.x0 = x1 + 1 == t.M ? 0 : x1 + 1;
  store_row<MODEL>(t, L0, T0);
  store_row<MODEL>(t, L1, T1);
}

// Tile plan of a launch (see the lane groups above).  Bands come in runs of
// gpw: a run's tiles are its bands' full segments (band-major), then one
// tile with the run's remainder groups, so that a remainder group runs near
// the full segments of its band (their halo rows are then still in L2 when a
// launch takes several waves).
//
// two_sided (depth 1 on rows of more than 32 pairs): strips of up to 30
// pairs with a whole-pair halo lane on each side and one 16-byte copy per
// plane for every lane (tile = band * n_strips + strip).  At depth 1 the
// launch is bound by HBM, not by the logic, and this form reads the planes
// at 97% of the copy peak against 77% with the 8-byte copies of the
// two-sided halo lane (90% with 16-byte copies off the halo lane).
struct PairPlan {
  int n_full;      // segments of kSegOwn owned pairs (groups of 32 lanes)
  int rem_own;     // owned pairs of the remainder segment (0: none)
  int rem_g;       // lanes of a remainder group
  int rem_halo;    // 1: remainder groups have a halo lane; 0: a group is the whole row ring
  int gpw;         // remainder groups per warp tile
  int band_rows, n_bands;
  int per_run;     // tiles of a run of gpw bands: gpw * n_full, plus 1 with a remainder
  int n_tiles;
  int two_sided;   // the strip form below
  int n_strips, s_base, s_rem;  // strips; owned pairs: s_base, one more in the first s_rem
};

constexpr int kSegOwn = 31;  // owned pairs of a full segment (plus one halo lane)

template <int K, int MODEL>
__global__ void __launch_bounds__(kWarps2 * 32, K >= 8 ? 2 : 3)
    stream2_kernel(const u64 *__restrict__ Lin, const u64 *__restrict__ Tin,
                   u64 *__restrict__ Lout, u64 *__restrict__ Tout, Geom g, PairPlan pp,
                   u64 *__restrict__ moved_lr, u64 *__restrict__ moved_tb, u64 tie_seed,
                   u64 t0) {
  using ST = typename std::conditional<MODEL == 2, StateII, StateI>::type;
  __shared__ unsigned long long s_cnt[2 * K];
  __shared__ __align__(16) ulonglong2 s_ring[kWarps2][kRing][2][32];  // [warp][slot][plane][lane]
  for (int t = threadIdx.x; t < 2 * K; t += blockDim.x) s_cnt[t] = 0;
  pdl_wait();
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int tile = blockIdx.x * kWarps2 + (threadIdx.x >> 5);
  uint32_t cnt[K];  // per stage: LR moves (bits 0-15), TB moves (bits 16-31)
#pragma unroll
  for (int s = 0; s < K; ++s) cnt[s] = 0;
  bool own = false;

  if (tile < pp.n_tiles) {
    // this lane's group: its band, first owned pair, owned pairs, lanes,
    // position and first lane in the warp, halo lane or not
    const int WP = (int)(g.W / 2);
    int band, p_lo, p_hi;
    bool on = true, halo_lane = false;
    PairTile t;
    if (pp.two_sided) {
      // a strip of up to 30 pairs, its halo lanes 0 and owned + 1 (whole pairs)
      const int strip = tile % pp.n_strips;
      band = tile / pp.n_strips;
      const int owned = pp.s_base + (strip < pp.s_rem ? 1 : 0);
      const int first = strip * pp.s_base + (strip < pp.s_rem ? strip : pp.s_rem);
      p_lo = (first - 1 + lane) % WP;
      if (p_lo < 0) p_lo += WP;
      p_hi = p_lo;
      own = lane >= 1 && lane <= owned;
      t.src_l = lane > 0 ? lane - 1 : 0;
      t.src_r = lane < 31 ? lane + 1 : 31;
      t.split = false;
    } else {
      int first, n_own, gs, gl, gbase, halo;
      const int run = tile / pp.per_run, r = tile - run * pp.per_run;
      const int b0 = run * pp.gpw;
      const int run_bands = pp.n_bands - b0 < pp.gpw ? pp.n_bands - b0 : pp.gpw;
      if (r < run_bands * pp.n_full) {  // a full segment
        const int bi = r / pp.n_full;
        band = b0 + bi;
        first = (r - bi * pp.n_full) * kSegOwn;
        n_own = kSegOwn;
        gs = 32;
        gl = lane;
        gbase = 0;
        halo = 1;
      } else {  // the run's remainder groups, one band each
        const int grp = lane / pp.rem_g;
        band = b0 + grp;
        first = pp.n_full * kSegOwn;
        n_own = pp.rem_own;
        gs = pp.rem_g;
        gbase = grp * gs;
        gl = lane - gbase;
        halo = pp.rem_halo;
        on = grp < run_bands;
      }
      // the pairs whose first and second words this lane holds (the halo lane:
      // the first word of the pair right of the segment and the second word of
      // the pair left of it); lanes in no group take pair 0 of band 0 and keep
      // nothing
      p_lo = first + gl - halo;
      p_hi = p_lo;
      halo_lane = halo && gl == 0;
      if (halo_lane) {
        p_lo = first + n_own;
        if (p_lo >= WP) p_lo -= WP;
        p_hi = first > 0 ? first - 1 : WP - 1;
      }
      if (!on) band = p_lo = p_hi = 0;
      own = on && !halo_lane;
      t.src_l = on ? gbase + (gl == 0 ? gs - 1 : gl - 1) : lane;
      t.src_r = on ? gbase + (gl == gs - 1 ? 0 : gl + 1) : lane;
      t.split = halo != 0;  // the same for every lane of the tile
    }
    t.wa = 2 * p_lo;
    t.own = own;
    t.r0 = band * pp.band_rows;
    t.B = !on ? 0 : (t.r0 + pp.band_rows < g.M ? pp.band_rows : (int)g.M - t.r0);
    t.n_in = t.B + 2 * K;
    t.M = (int)g.M;
    t.ld_row = (t.r0 - K) % t.M;
    if (t.ld_row < 0) t.ld_row += t.M;
    t.pitch = (size_t)g.P;
    // the T planes follow the L planes at the same distance in both buffers
    t.dT = Tin - Lin;
    t.dH = (int64_t)(2 * p_hi + 1) - 2 * p_lo;
    t.Lin = Lin + t.wa;
    t.fL = t.Lin + (size_t)t.ld_row * t.pitch;
    t.sL = Lout + (size_t)t.r0 * t.pitch + t.wa;
    // Model II tie-break counters: n = t*M*W + x*W + w + 1 for word w of row x
    t.W64 = (u64)g.W;
    t.MW = (u64)g.M * t.W64;
    t.nbase = t0 * t.MW + (u64)t.wa + 1;
    t.tie_seed = tie_seed;
    t.x0 = t.ld_row;  // lattice row of input row i (stage 0)
    // rows of the warp: the steady part ends at the smallest band's end, the
    // drain at the tallest band's input
    const int minB = (int)__reduce_min_sync(BML_FULL_MASK, on ? (unsigned)t.B : 0x7fffffffu);
    const int n_max = (int)__reduce_max_sync(BML_FULL_MASK, (unsigned)t.B) + 2 * K;

    ST st[2][K];  // state sets, alternated row by row
#pragma unroll
    for (int s = 0; s < K; ++s) st[0][s] = st[1][s] = ST{};

    RingSlot *ring = s_ring[threadIdx.x >> 5];
    // rows 0 .. kAhead-1 in flight, one commit group per row (empty past n_in)
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      if (u < t.n_in) fetch_row(t, ring, lane, u);
      cp_async_commit();
    }
    // rows [0, 2K): the pipeline fills (guarded); rows [2K, minB + K): every
    // stage's row lies in every lane's band and a row is emitted (unguarded,
    // two rows a turn); the rest: the pipeline drains (guarded).  Counts are
    // flushed every 256 rows (a 16-bit field holds at most 511 rows of moves).
    int i = 0;
    for (; i < 2 * K; i += 2) {
      guarded_row<K, MODEL, 0>(t, ring, lane, i, st, cnt);
      guarded_row<K, MODEL, 1>(t, ring, lane, i + 1, st, cnt);
    }
    const int steady_end = minB + K;
    for (; i + 2 <= steady_end; i += 2) {
      if ((i & 255) == 0) flush_counts<K>(cnt, own, lane, s_cnt);
      steady_rows<K, MODEL>(t, ring, lane, i, st, cnt);
    }
    for (; i < n_max; i += 2) {
      if ((i & 255) == 0) flush_counts<K>(cnt, own, lane, s_cnt);
      guarded_row<K, MODEL, 0>(t, ring, lane, i, st, cnt);
      if (i + 1 < n_max) guarded_row<K, MODEL, 1>(t, ring, lane, i + 1, st, cnt);
    }
  }
  pdl_release();  // this block's lattice work is done
  flush_counts<K>(cnt, own, lane, s_cnt);
  __syncthreads();
  if (threadIdx.x < K) {
    if (s_cnt[threadIdx.x]) atomicAdd(moved_lr + threadIdx.x, s_cnt[threadIdx.x]);
  } else if (threadIdx.x < 2 * K) {
    const int s = threadIdx.x - K;
    if (s_cnt[K + s]) atomicAdd(moved_tb + s, s_cnt[K + s]);
  }
}

// The tile plan for depth k and bands of band_rows rows (see PairPlan);
// false if the tile count does not fit an int.
bool pair_plan(const Geom &g, int k, int64_t band_rows, PairPlan &pp) {
  const int64_t WP = g.W / 2;
  const int64_t n_bands = (g.M + band_rows - 1) / band_rows;
  pp = PairPlan{};
  int64_t tiles;
  if (k == 1 && WP > 32) {
    pp.two_sided = 1;
    pp.n_strips = (int)((WP + 29) / 30);
    pp.s_base = (int)(WP / pp.n_strips);
    pp.s_rem = (int)(WP % pp.n_strips);
    tiles = (int64_t)pp.n_strips * n_bands;
  } else {
    if (WP <= 32) {  // the whole row ring in one group
      pp.n_full = 0;
      pp.rem_own = (int)WP;
      pp.rem_g = (int)WP;
      pp.rem_halo = 0;
    } else {
      pp.n_full = (int)(WP / kSegOwn);
      pp.rem_own = (int)(WP % kSegOwn);
      pp.rem_g = pp.rem_own + 1;
      pp.rem_halo = 1;
    }
    pp.gpw = pp.rem_own ? 32 / pp.rem_g : 1;
    pp.per_run = pp.gpw * pp.n_full + (pp.rem_own ? 1 : 0);
    tiles = pp.n_full * n_bands + (pp.rem_own ? (n_bands + pp.gpw - 1) / pp.gpw : 0);
  }
  if (tiles > INT32_MAX - kWarps2 || band_rows > INT32_MAX) return false;
  pp.band_rows = (int)band_rows;
  pp.n_bands = (int)n_bands;
  pp.n_tiles = (int)tiles;
  return true;
}

template <int K, int MODEL>
cudaError_t launch2_k(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                      int64_t band_rows, u64 *moved_lr, u64 *moved_tb, u64 tie_seed, u64 t0,
                      cudaStream_t st) {
  PairPlan pp;
  if (!pair_plan(g, K, band_rows, pp)) return cudaErrorInvalidValue;
  const int64_t blocks = ((int64_t)pp.n_tiles + kWarps2 - 1) / kWarps2;
  return launch_pdl(stream2_kernel<K, MODEL>, dim3((unsigned)blocks), dim3(kWarps2 * 32), 0, st,
                    Lin, Tin, Lout, Tout, g, pp, moved_lr, moved_tb, tie_seed, t0);
}

template <int K, int MODEL>
int occupancy2() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, stream2_kernel<K, MODEL>, kWarps2 * 32,
                                                    0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return b > 0 ? b : 1;
}

// Even bits of x to bits 0..31, odd bits to bits 32..63 (the outer perfect
// unshuffle by five delta swaps, Warren, Hacker's Delight, Sec. 7-2), and
// its inverse.
__device__ __forceinline__ u64 delta_swap(u64 x, u64 m, int s) {
  const u64 t = (x ^ (x >> s)) & m;
  return x ^ t ^ (t << s);
}
__device__ __forceinline__ u64 unshuffle64(u64 x) {
  x = delta_swap(x, 0x2222222222222222ull, 1);
  x = delta_swap(x, 0x0C0C0C0C0C0C0C0Cull, 2);
  x = delta_swap(x, 0x00F000F000F000F0ull, 4);
  x = delta_swap(x, 0x0000FF000000FF00ull, 8);
  return delta_swap(x, 0x00000000FFFF0000ull, 16);
}
__device__ __forceinline__ u64 shuffle64(u64 x) {
  x = delta_swap(x, 0x00000000FFFF0000ull, 16);
  x = delta_swap(x, 0x0000FF000000FF00ull, 8);
  x = delta_swap(x, 0x00F000F000F000F0ull, 4);
  x = delta_swap(x, 0x0C0C0C0C0C0C0C0Cull, 2);
  return delta_swap(x, 0x2222222222222222ull, 1);
}

// In place, every word of both planes: plain -> interleaved (to_pair) puts
// the word's even columns in its low half and its odd columns in its high
// half; interleaved -> plain undoes it.
// One thread per aligned word pair (16-byte accesses) of either plane.
__global__ void pair_layout_kernel(u64 *__restrict__ L, u64 *__restrict__ T, int64_t pairs,
                                   int to_pair) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 2 * pairs;
       q += (int64_t)gridDim.x * blockDim.x) {
    u64 *p = (q < pairs ? L : T) + 2 * (q < pairs ? q : q - pairs);
    const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p);
    ulonglong2 o;
    o.x = to_pair ? unshuffle64(v.x) : shuffle64(v.x);
    o.y = to_pair ? unshuffle64(v.y) : shuffle64(v.y);
    *reinterpret_cast<ulonglong2 *>(p) = o;
  }
}

}  // namespace

cudaError_t launch_pair_layout(u64 *L, u64 *T, const Geom &g, bool to_pair, cudaStream_t st) {
  if (!stream2_applies(g)) return cudaErrorInvalidValue;
  const int64_t pairs = g.M * g.P / 2;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 148;
  }
  int64_t blocks = (2 * pairs + 255) / 256;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  pair_layout_kernel<<<(unsigned)blocks, 256, 0, st>>>(L, T, pairs, to_pair ? 1 : 0);
  return cudaGetLastError();
}

bool stream2_applies(const Geom &g) { return g.nb == 64 && g.W % 2 == 0 && g.W > 32; }

int64_t stream2_bands_for_tiles(const Geom &g, int k, int64_t tiles) {
  // the tile count grows with the band count n: the largest n that fits
  PairPlan pp;
  if (!pair_plan(g, k, g.M, pp)) return 0;
  int64_t lo = 0, hi = g.M;
  while (lo < hi) {
    const int64_t n = (lo + hi + 1) / 2;
    const int64_t t = pp.two_sided ? (int64_t)pp.n_strips * n
                                   : (int64_t)pp.n_full * n +
                                         (pp.rem_own ? (n + pp.gpw - 1) / pp.gpw : 0);
    if (t <= tiles) lo = n; else hi = n - 1;
  }
  return lo;
}

int stream2_occupancy(int k, int model) {
  if (model == 2) {
    switch (k) {
      case 1: return occupancy2<1, 2>();
      case 2: return occupancy2<2, 2>();
      case 4: return occupancy2<4, 2>();
      default: return occupancy2<8, 2>();
    }
  }
  switch (k) {
    case 1: return occupancy2<1, 1>();
    case 2: return occupancy2<2, 1>();
    case 4: return occupancy2<4, 1>();
    default: return occupancy2<8, 1>();
  }
}

cudaError_t launch_stream2(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                           int k, int64_t band_rows, u64 *moved_lr, u64 *moved_tb,
                           cudaStream_t st, int model, u64 tie_seed, u64 t0) {
  if (!stream2_applies(g) || band_rows < 1 || band_rows > INT32_MAX || Tin - Lin != Tout - Lout)
    return cudaErrorInvalidValue;
  if (model == 3) {
    switch (k) {
      case 1: return launch2_k<1, 3>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, 0, 0, st);
      case 2: return launch2_k<2, 3>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, 0, 0, st);
      case 4: return launch2_k<4, 3>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, 0, 0, st);
      case 8: return launch2_k<8, 3>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, 0, 0, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (model == 2) {
    switch (k) {
      case 1: return launch2_k<1, 2>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, tie_seed, t0, st);
      case 2: return launch2_k<2, 2>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, tie_seed, t0, st);
      case 4: return launch2_k<4, 2>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, tie_seed, t0, st);
      case 8: return launch2_k<8, 2>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, tie_seed, t0, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (k) {
    case 1: return launch2_k<1, 1>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, 0, 0, st);
    case 2: return launch2_k<2, 1>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, 0, 0, st);
    case 4: return launch2_k<4, 1>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, 0, 0, st);
    case 8: return launch2_k<8, 1>(Lin, Tin, Lout, Tout, g, band_rows, moved_lr, moved_tb, 0, 0, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bml
