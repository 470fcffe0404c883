// Batched ensemble: many independent lattices of uneven sizes and densities
// advanced together by one persistent, cooperative launch per call (replayed
// from a CUDA graph).
//
// Layout.  Every lattice has two bitplane buffers (ping-pong), each L then T,
// M x P words (P = W rounded up to even), in one device pool; within a word
// the even columns sit in the low half and the odd ones in the high half
// (ens_bit).  Per-lattice moved-count traces are [lattice][step] int64
// arrays (LR and TB).
//
// Tiles.  Every lattice row fits one warp (N <= 2048, W <= 32 words).  A
// lattice is cut into row bands; a warp tile packs bands of any word widths
// side by side (first fit over the bands sorted by length; a band of W words
// takes W consecutive lanes, one whole periodic row), so narrow lattices do
// not leave lanes idle.  Each band streams through the same k-stage register
// pipeline as the single-lattice streaming kernel (the rule of stage.cuh,
// here on interleaved words: stage_step_x), with k-row halos read modulo M.  Tiles are ordered longest first
// and warps draw them from a dispenser (one atomic per tile), so the work is
// spread by longest-processing-time-first list scheduling; the band height
// is chosen on the host by a model of that schedule and confirmed by timing.
//
// Chunks.  One launch runs n chunks of k steps.  There is no grid-wide
// barrier between chunks: a tile of chunk c waits only until every band of
// its own lattices has finished chunk c - 1 (a per-lattice count of finished
// bands, released by each band after its stores; the waits are bounded by
// %globaltimer, on expiry the kernel sets an error flag and returns and the
// host reports BML_ETIMEOUT).  The tiles of a chunk are all handed out
// before those of the next, so the warps a tile waits for are running.  A
// barrier made every warp wait for the slowest tile of the whole chunk
// (about 6% of the warps' time in stalls at the barrier, plus the idle tail
// of every chunk).  Data written in one chunk is read by other blocks in the
// next, so lattice words move through L2 only (cp.async.cg into a per-warp
// shared-memory ring, st.cg), never through L1 or the non-coherent
// read-only path.
//
// Jam early exit (optional).  A step in which no car moves leaves the lattice
// unchanged, so every later step does too (an absorbing fixed point).  At the
// start of each chunk a group checks the previous chunk's counts of its
// lattice; after a zero-move step the lattice is frozen: its buffer index is
// recorded and its tiles are skipped.  Later counts stay zero, which is what
// the automaton would produce.  A retired lattice (bml_ensemble_retire) is
// frozen the same way at the step of its retirement.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/bml.h"
#include "bml_internal.cuh"
#include "stage.cuh"

namespace bml {

struct EnsLattice {
  int M, N, W, P;
  int nb, pad;
  u64 tail;
  u64 off[2];  // word offset of buffer 0 / 1 (L plane; T plane at + M*P)
};

struct EnsGroup {
  int lat, r0, len, lane0;  // lattice, band rows [r0, r0+len), first lane in its tile
};

// A warp's work: up to 32 lanes holding the rows of one or more bands (groups)
// of possibly different word widths; lane_grp[l] = group slot of lane l
// (0xff: idle lane).
struct EnsTile {
  int G, first_group, max_len, min_len;
  unsigned char lane_grp[32];
};

struct EnsCtrl {
  long long steps;       // steps completed
  long long last_depth;  // depth of the last chunk run (for jam checks)
  int parity;            // buffer holding the state of lattices not frozen
  int err;               // set by a wait between chunks that timed out
  unsigned tile_next;    // tile dispenser (0 between launches)
};

struct EnsParams {
  const EnsLattice *lat;
  const EnsTile *tiles;
  const EnsGroup *groups;
  int n_tiles;
  int n_chunks;
  u64 *pool;
  u64 *tr_lr, *tr_tb;  // traces, [lattice][cap]
  long long cap;
  long long *frozen;   // first zero-move step of a frozen lattice, else -1
  int *frozen_buf;     // buffer index holding a frozen lattice
  EnsCtrl *ctrl;
  int commit;          // 0: tuning launch: every chunk reads the current buffer, counts
                       // go to scratch, nothing frozen
  int early_exit;
  const unsigned *lat_groups;  // bands (groups) of every lattice in the tile plan
  unsigned *lat_done;  // bands of every lattice finished in this launch (0 at its start)
  unsigned stall_extra;  // test hook: 1 makes the first wait between chunks never end
  long long timeout_ns;
  u64 *scratch;        // tuning counts
};

namespace {

constexpr int kEnsWarps = 4;

__device__ __forceinline__ long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *q) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(q) : "memory");
  return v;
}

// Wait until lattice l's count of finished bands reaches `target`, bounded by
// p.timeout_ns; on expiry (or when another wait gave up) the error flag is
// set and false is returned.
__device__ bool wait_lattice(const EnsParams &p, int l, unsigned target) {
  const unsigned *cnt = p.lat_done + l;
  if (ld_acquire_u32(cnt) >= target) return true;
  volatile int *err = &p.ctrl->err;
  const long long t0 = globaltimer_ns();
  while (ld_acquire_u32(cnt) < target) {
    if (*err) return false;
    if (globaltimer_ns() - t0 > p.timeout_ns) {
      atomicExch(&p.ctrl->err, 1);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

// Input rows reach a warp through a ring of kEnsRing row slots in shared
// memory (stage.cuh), filled kEnsAhead rows ahead with cp.async.cg: through
// L2, so the words other blocks wrote in the previous chunk are seen.  A slot
// is refilled two rows after it was last read.
constexpr int kEnsRing = 8;
constexpr int kEnsAhead = 5;
// a slot is refilled at least two rows after it was last read, also when the
// steady loop fetches two rows at once
static_assert(kEnsAhead + 1 <= kEnsRing - 2 && (kEnsRing & (kEnsRing - 1)) == 0, "ring layout");
using EnsRing = RingSlot[kEnsRing];

// Running position of a lane in its band: the next input row to fetch (with
// wrap-around at the lattice's last row) and the next output row to store.
struct EnsCursor {
  const u64 *Lp;     // next row to fetch (L plane; T plane at + plane)
  const u64 *inbase; // row 0
  u64 *Lo;           // next row to store (L plane)
  size_t pitch, plane;
  int ld_row, M;
};

__device__ __forceinline__ void ens_fetch(EnsCursor &c, EnsRing &ring, int slot, int lane) {
  ring_fill(ring, slot, lane, c.Lp, c.Lp + c.plane);
  if (++c.ld_row == c.M) {
    c.ld_row = 0;
    c.Lp = c.inbase;
  } else {
    c.Lp += c.pitch;
  }
}

__device__ __forceinline__ void ens_store(EnsCursor &c, u64 L, u64 T) {
  __stcg(c.Lo, L);
  __stcg(c.Lo + c.plane, T);
  c.Lo += c.pitch;
}

// Interleaved word layout of the ensemble's planes: column 64w + b of a row
// is bit ens_bit(b) of word w, the word's even columns in its low half and
// its odd columns in its high half (so a cell's right neighbour is mostly
// the same bit of the other half, and the stage needs half the shifts).
__host__ __device__ __forceinline__ int ens_bit(int b) { return (b >> 1) | ((b & 1) << 5); }

// Per-lane constants of the interleaved stage; half a = even columns (low
// 32 bits), half b = odd columns (high 32 bits).  A word with n cells (64
// except a row's last word) has ne = ceil(n/2) even and no = floor(n/2) odd
// cells.  The right neighbour of its last cell is the right lane's column 0,
// inserted by a multiply-add: for n odd the last cell is even (a bit no), the
// neighbour's E enters the even cells' right-neighbour word at bit no
// (ins_a); for n even it is odd (b bit no - 1, bit 31 of a full word) and
// enters at bit no - 1 of the odd cells' one (ins_b).  The last cell sent
// to the left lane's neighbour is placed at bit 31 by a * mul_a + b * mul_b.
struct LaneWordX {
  uint32_t va, vb;        // valid cells of each half (0 for a lane that is off)
  uint32_t ins_a, ins_b;  // bit that receives the right neighbour's column 0
  uint32_t mul_a, mul_b;
  int src_l, src_r;       // lanes holding the left / right neighbour words
};

__device__ __forceinline__ void lane_word_bits_x(LaneWordX &lw, bool on, bool last, int nb) {
  const int n = last ? nb : 64;
  const int ne = (n + 1) >> 1, no = n >> 1;
  lw.va = on ? (ne >= 32 ? ~0u : (1u << ne) - 1u) : 0u;
  lw.vb = on ? (no >= 32 ? ~0u : (1u << no) - 1u) : 0u;
  lw.ins_a = (n & 1) ? 1u << no : 0u;
  lw.ins_b = (n & 1) ? 0u : 1u << (no - 1);
  lw.mul_a = (n & 1) ? 1u << (31 - no) : 0u;
  lw.mul_b = (n & 1) ? 0u : 1u << (32 - no);
}

// One stage (the rule of stage.cuh, "who enters" form) on a word in the
// interleaved layout; L, T: {a, b}.  Even cell 2i: right neighbour odd cell
// 2i + 1 (b bit i), left neighbour odd cell 2i - 1 (b bit i - 1, the left
// word's last cell for i = 0).  Odd cell 2i + 1: right neighbour even cell
// 2i + 2 (a bit i + 1, the right word's column 0 for the last one), left
// neighbour even cell 2i (a bit i).  So the cars entering the odd cells are
// La & Eb with no shift, and only Er_b and the cars entering the even cells
// need a shift: 2 shifts per word instead of 4.  A car never enters an even
// and the odd cell right of it in the same step (the even cell would have to
// be empty and hold the leaving car), so one popcount of in_a | in_b counts
// the LR moves.
__device__ __forceinline__ void stage_step_x(uint32_t (&L)[2], uint32_t (&T)[2], const StageH &st,
                                             StageH &nx, const LaneWordX &lw, uint32_t &mvIn,
                                             uint32_t &mvV) {
  const uint32_t Ea = lop3<kNorAnd>(L[0], T[0], lw.va);
  const uint32_t Eb = lop3<kNorAnd>(L[1], T[1], lw.vb);
  const uint32_t send_l = L[1] * lw.mul_b + L[0] * lw.mul_a;
  const uint32_t rl = __shfl_sync(BML_FULL_MASK, send_l, lw.src_l);
  const uint32_t rr = __shfl_sync(BML_FULL_MASK, Ea, lw.src_r);
  // the right neighbours' E (no carry: the inserted bit is past the valid ones)
  const uint32_t Era = Eb + rr * lw.ins_a;
  const uint32_t Erb = (Ea >> 1) + rr * lw.ins_b;
  const uint32_t ina = lop3<kAnd>(__funnelshift_l(rl, L[1], 1), Ea, 0u);
  const uint32_t inb = lop3<kAnd>(L[0], Eb, 0u);
  const uint32_t Lha = lop3<kAndNotOr>(L[0], Era, ina), Lhb = lop3<kAndNotOr>(L[1], Erb, inb);
  const uint32_t mva = lop3<kAndNor>(st.T[0], Lha, T[0]);
  const uint32_t mvb = lop3<kAndNor>(st.T[1], Lhb, T[1]);
  mvIn = __popc(ina | inb);
  mvV = __popc(mva) + __popc(mvb);
  nx.T[0] = T[0];
  nx.T[1] = T[1];
  nx.Lh[0] = Lha;
  nx.Lh[1] = Lhb;
  nx.M[0] = mva;
  nx.M[1] = mvb;
  T[0] = lop3<kAndNotOr>(st.T[0], mva, st.M[0]);
  T[1] = lop3<kAndNotOr>(st.T[1], mvb, st.M[1]);
  L[0] = st.Lh[0];
  L[1] = st.Lh[1];
}

// The K stages on one input row i (already read); A selects the state set
// the row reads.  GUARD: a stage's row may lie outside the band.
template <int K, bool GUARD, int A>
__device__ __forceinline__ void ens_stages(uint32_t (&L)[2], uint32_t (&T)[2],
                                           StageH (&st)[2][K], uint32_t (&c_lr)[K],
                                           uint32_t (&c_tb)[K], const LaneWordX &lw, int i,
                                           int len) {
  constexpr int B = A ^ 1;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    uint32_t mvIn, mvV;
    stage_step_x(L, T, st[A][s], st[B][s], lw, mvIn, mvV);
    if (!GUARD || (unsigned)(i - K - s) < (unsigned)len) c_lr[s] += mvIn;
    if (!GUARD || (unsigned)(i - K - s - 1) < (unsigned)len) c_tb[s] += mvV;
  }
}

template <int K>
__device__ void process_tile(const EnsParams &p, int t, long long step0, int par,
                             long long prev_depth, int lane, EnsRing &ring) {
  const EnsTile &tile = p.tiles[t];
  const int grp = tile.lane_grp[lane];
  bool on = grp != 0xff;
  EnsGroup gr{0, 0, 0, 0};
  EnsLattice L{};
  if (on) {
    gr = p.groups[tile.first_group + grp];
    L = p.lat[gr.lat];
  }
  const int W = on ? L.W : 1;           // words per row of this lane's lattice
  const int wi = on ? lane - gr.lane0 : 0;  // this lane's word of the row
  if (on) {  // frozen: jammed (early exit) or retired
    long long fz = __ldcg(p.frozen + gr.lat);
    if (p.early_exit && fz < 0 && step0 > 0) {
      const u64 *a = p.tr_lr + (long long)gr.lat * p.cap, *b = p.tr_tb + (long long)gr.lat * p.cap;
      for (long long s = step0 - prev_depth; s < step0; ++s) {
        if (s >= 0 && __ldcg(a + s) + __ldcg(b + s) == 0ull) {
          fz = s;
          break;
        }
      }
      if (fz >= 0) {
        p.frozen[gr.lat] = fz;  // every group of the lattice writes the same values
        p.frozen_buf[gr.lat] = par;
      }
    }
    if (fz >= 0) on = false;
  }
  if (!__any_sync(BML_FULL_MASK, on)) return;

  LaneWordX lw;
  if (on) {
    lw.src_l = gr.lane0 + (wi == 0 ? W - 1 : wi - 1);
    lw.src_r = gr.lane0 + (wi == W - 1 ? 0 : wi + 1);
  } else {
    lw.src_l = lw.src_r = lane;
  }
  lane_word_bits_x(lw, on, on && wi == L.W - 1, on ? L.nb : 64);

  const int M = on ? L.M : 1;
  const size_t pitch = on ? (size_t)L.P : 0;
  // the 16-byte word pair that holds this lane's word (buffers picked by a
  // select: a runtime index into the copied lattice record would put it in
  // local memory)
  const u64 off_in = par ? L.off[1] : L.off[0], off_out = par ? L.off[0] : L.off[1];
  EnsCursor cur;
  cur.inbase = p.pool + (on ? off_in : 0) + (wi & ~1);
  cur.pitch = pitch;
  cur.plane = (size_t)M * pitch;
  cur.M = M;
  const int len = gr.len, n_in = len + 2 * K;
  cur.ld_row = on ? (gr.r0 - K) % M : 0;
  if (cur.ld_row < 0) cur.ld_row += M;
  cur.Lp = cur.inbase + (size_t)cur.ld_row * pitch;
  cur.Lo = p.pool + (on ? off_out : 0) + wi + (size_t)gr.r0 * pitch;
  const int half = wi & 1;

  // two state sets, alternated row by row, so no value is copied
  StageH st[2][K];
  uint32_t c_lr[K], c_tb[K];
#pragma unroll
  for (int s = 0; s < K; ++s) {
    st[0][s] = st[1][s] = StageH{};
    c_lr[s] = c_tb[s] = 0;
  }

  // rows 0 .. kEnsAhead-1 in flight, one commit group per row (empty past n_in)
#pragma unroll
  for (int u = 0; u < kEnsAhead; ++u) {
    if (on && u < n_in) ens_fetch(cur, ring, u, lane);
    cp_async_commit();
  }
  // One input row near the band ends (guarded: rows past a lane's input,
  // stages outside its band and rows before 2K are neither counted nor
  // stored; lanes past their band's input rows, or off, read stale slots).
  auto guarded_row = [&](int i, auto a_tag) {
    constexpr int A = decltype(a_tag)::value;
    if (on && i + kEnsAhead < n_in) ens_fetch(cur, ring, (i + kEnsAhead) & (kEnsRing - 1), lane);
    cp_async_commit();
    cp_async_wait<kEnsAhead>();  // row i has landed (this lane's own copies)
    u64 inL, inT;
    ring_read(ring, i & (kEnsRing - 1), lane, half, inL, inT);
    uint32_t L[2] = {lo32(inL), hi32(inL)}, T[2] = {lo32(inT), hi32(inT)};
    ens_stages<K, true, A>(L, T, st, c_lr, c_tb, lw, i, len);
    if (on && i >= 2 * K && i - 2 * K < len) ens_store(cur, mk64(L[0], L[1]), mk64(T[0], T[1]));
  };
  using A0 = std::integral_constant<int, 0>;
  using A1 = std::integral_constant<int, 1>;
  const int n_max = tile.max_len + 2 * K;
  // rows [0, 2K): the pipeline fills; rows [2K, min_len + K): every lane's
  // stage rows lie in its band and every on-lane stores (two rows a turn,
  // both read from the ring before either runs its stages); the rest drains
  int i = 0;
  for (; i < 2 * K; i += 2) {
    guarded_row(i, A0{});
    guarded_row(i + 1, A1{});
  }
  const int steady_end = tile.min_len + K;
  for (; i + 2 <= steady_end; i += 2) {
    // rows i + kEnsAhead (+1) exist when K > kEnsAhead (i + 1 < min_len + K)
    if (on && (K > kEnsAhead || i + kEnsAhead < n_in))
      ens_fetch(cur, ring, (i + kEnsAhead) & (kEnsRing - 1), lane);
    cp_async_commit();
    if (on && (K > kEnsAhead || i + kEnsAhead + 1 < n_in))
      ens_fetch(cur, ring, (i + kEnsAhead + 1) & (kEnsRing - 1), lane);
    cp_async_commit();
    cp_async_wait<kEnsAhead>();  // rows i and i + 1 have landed
    u64 a0, b0, a1, b1;
    ring_read(ring, i & (kEnsRing - 1), lane, half, a0, b0);
    ring_read(ring, (i + 1) & (kEnsRing - 1), lane, half, a1, b1);
    uint32_t L0[2] = {lo32(a0), hi32(a0)}, T0[2] = {lo32(b0), hi32(b0)};
    uint32_t L1[2] = {lo32(a1), hi32(a1)}, T1[2] = {lo32(b1), hi32(b1)};
    ens_stages<K, false, 0>(L0, T0, st, c_lr, c_tb, lw, i, len);
    ens_stages<K, false, 1>(L1, T1, st, c_lr, c_tb, lw, i + 1, len);
    if (on) {
      ens_store(cur, mk64(L0[0], L0[1]), mk64(T0[0], T0[1]));
      ens_store(cur, mk64(L1[0], L1[1]), mk64(T1[0], T1[1]));
    }
  }
  for (; i < n_max; i += 2) {
    guarded_row(i, A0{});
    if (i + 1 < n_max) guarded_row(i + 1, A1{});  // warp-uniform
  }
  // per-group reduction of the counts, then one atomic per group and step
#pragma unroll
  for (int s = 0; s < K; ++s) {
    uint32_t a = on ? c_lr[s] : 0u, b = on ? c_tb[s] : 0u;
    // segmented sum over each group's lanes [lane0, lane0 + W): every lane
    // shuffles, a lane adds only a partner of its own group
    for (int off = 16; off > 0; off >>= 1) {
      const uint32_t ua = __shfl_down_sync(BML_FULL_MASK, a, off);
      const uint32_t ub = __shfl_down_sync(BML_FULL_MASK, b, off);
      if (wi + off < W) {
        a += ua;
        b += ub;
      }
    }
    if (on && wi == 0) {
      if (p.commit) {
        const long long slot = (long long)gr.lat * p.cap + step0 + s;
        if (a) atomicAdd(p.tr_lr + slot, (unsigned long long)a);
        if (b) atomicAdd(p.tr_tb + slot, (unsigned long long)b);
      } else {
        if (a) atomicAdd(p.scratch + s, (unsigned long long)a);
        if (b) atomicAdd(p.scratch + K + s, (unsigned long long)b);
      }
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kEnsWarps * 32, K >= 8 ? 3 : 4) ens_kernel(EnsParams p) {
  __shared__ __align__(16) EnsRing s_ring[kEnsWarps];
  __shared__ unsigned s_ticket[kEnsWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = gridDim.x * kEnsWarps;
  const long long base = __ldcg(&p.ctrl->steps);
  const long long last_depth = __ldcg(&p.ctrl->last_depth);
  const int par0 = *(volatile int *)&p.ctrl->parity;
  // Ticket v is tile v % n_tiles of chunk v / n_tiles: every tile of a chunk
  // is drawn before any tile of the next one, and tiles are ordered longest
  // first (longest-processing-time-first list scheduling within a chunk).
  // Every warp draws until it gets a ticket past the last tile, so a launch
  // draws n_chunks * n_tiles + nwarps tickets; the draw of the last one
  // resets the dispenser for the next launch (no later draw exists).  (The
  // host keeps that count below 2^32.)
  const unsigned total = (unsigned)p.n_tiles * (unsigned)p.n_chunks;
  const unsigned last_ticket = total + (unsigned)nwarps - 1u;
  for (;;) {
    if (lane == 0) {
      const unsigned v = atomicAdd(&p.ctrl->tile_next, 1u);
      if (v == last_ticket) atomicExch(&p.ctrl->tile_next, 0u);
      s_ticket[warp] = v;
    }
    __syncwarp();
    const unsigned v = s_ticket[warp];
    __syncwarp();
    if (v >= total) break;
    const int c = (int)(v / (unsigned)p.n_tiles);
    const int t = (int)(v - (unsigned)c * (unsigned)p.n_tiles);
    const long long step0 = base + (long long)c * K;
    // a tuning launch (not committed) runs every chunk from the current
    // buffer into the other one, so the lattices' state is left as it was
    const int par = p.commit ? (par0 + c) & 1 : par0;
    const long long prev_depth = c == 0 ? last_depth : K;
    // A band of chunk c reads its lattice's rows written in chunk c - 1 (its
    // own and k rows of each neighbour band) and overwrites the buffer chunk
    // c - 1 read; the jam check reads the lattice's counts of chunk c - 1.
    // So before its tile runs, the lane leading each of the tile's bands
    // waits until every band of that lattice has finished chunk c - 1 (a
    // count of finished bands, released after their stores).  Tiles of
    // chunk c - 1 were all drawn before this one, by warps that are running
    // them, so every wait ends (within the time bound, else an error).
    const EnsTile &tile = p.tiles[t];
    const int grp = tile.lane_grp[lane];
    int lat = -1;
    if (grp != 0xff) {
      const EnsGroup g = p.groups[tile.first_group + grp];
      if (g.lane0 == lane) lat = g.lat;
    }
    if (c > 0) {
      const bool ok =
          lat < 0 || wait_lattice(p, lat, p.lat_groups[lat] * (unsigned)c + p.stall_extra);
      if (!__all_sync(BML_FULL_MASK, ok)) return;
    }
    process_tile<K>(p, t, step0, par, prev_depth, lane, s_ring[warp]);
    // the tile's rows and counts are written: each band leader publishes
    // (the warp's stores are ordered before the leader's fence and atomic)
    __syncwarp();
    if (lat >= 0) {
      __threadfence();
      atomicAdd(p.lat_done + lat, 1u);
    }
  }
}

// Stream-ordered after ens_kernel: advance the step counter and parity.
__global__ void ens_advance_kernel(EnsCtrl *ctrl, int n_chunks, int depth) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && ctrl->err == 0) {
    ctrl->steps += (long long)n_chunks * depth;
    ctrl->parity ^= (n_chunks & 1);
    ctrl->last_depth = depth;
  }
}

// ---- set-up kernels (not on the step path) ----
__device__ __forceinline__ u64 sm64_at(u64 seed, u64 n) {
  u64 z = seed + n * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// seeded placement of every lattice into buffer 0
__global__ void ens_init_kernel(const EnsLattice *lat, int count, const u64 *seed,
                                const u64 *t_lr, const u64 *t_tb, u64 *pool) {
  for (int l = blockIdx.x; l < count; l += gridDim.x) {
    const EnsLattice L = lat[l];
    const long long words = (long long)L.M * L.P;
    u64 *Lp = pool + L.off[0], *Tp = Lp + words;
    for (long long idx = threadIdx.x; idx < words; idx += blockDim.x) {
      const int i = (int)(idx / L.P), w = (int)(idx - (long long)i * L.P);
      u64 lv = 0, tv = 0;
      if (w < L.W) {
        const int nbits = w == L.W - 1 ? L.nb : 64;
        const u64 base = (u64)((long long)i * L.N + 64ll * w) + 1ull;
        for (int b = 0; b < nbits; ++b) {
          const u64 u = sm64_at(seed[l], base + (u64)b);
          if (u < t_lr[l])
            lv |= 1ull << ens_bit(b);
          else if (u - t_lr[l] < t_tb[l])
            tv |= 1ull << ens_bit(b);
        }
      }
      Lp[idx] = lv;
      Tp[idx] = tv;
    }
  }
}

// bytes (each lattice M*N, back to back at byte_off[l]) -> buffer `buf` of
// every lattice; with pool == nullptr only the values are checked.
__global__ void ens_pack_kernel(const EnsLattice *lat, int count, const long long *byte_off,
                                const uint8_t *bytes, int buf, u64 *pool, int *bad) {
  int badl = 0;
  for (int l = blockIdx.x; l < count; l += gridDim.x) {
    const EnsLattice L = lat[l];
    const long long words = (long long)L.M * L.P;
    const uint8_t *src = bytes + byte_off[l];
    for (long long idx = threadIdx.x; idx < words; idx += blockDim.x) {
      const int i = (int)(idx / L.P), w = (int)(idx - (long long)i * L.P);
      u64 lv = 0, tv = 0;
      if (w < L.W) {
        const int nbits = w == L.W - 1 ? L.nb : 64;
        const uint8_t *row = src + (long long)i * L.N + 64ll * w;
        for (int b = 0; b < nbits; ++b) {
          const uint32_t x = row[b];
          badl |= x > 2u;
          lv |= (u64)(x & 1u) << ens_bit(b);
          tv |= (u64)((x >> 1) & 1u) << ens_bit(b);
        }
      }
      if (pool) {
        u64 *Lp = pool + L.off[buf];
        Lp[idx] = lv;
        Lp[words + idx] = tv;
      }
    }
  }
  if (badl) atomicOr(bad, 1);
}

// buffer of each lattice -> bytes, back to back
__global__ void ens_unpack_kernel(const EnsLattice *lat, int count, const long long *byte_off,
                                  const int *buf_of, const u64 *pool, uint8_t *bytes) {
  for (int l = blockIdx.x; l < count; l += gridDim.x) {
    const EnsLattice L = lat[l];
    const long long words = (long long)L.M * L.P;
    const u64 *Lp = pool + L.off[buf_of[l]], *Tp = Lp + words;
    uint8_t *dst = bytes + byte_off[l];
    const long long cells = (long long)L.M * L.N;
    for (long long idx = threadIdx.x; idx < cells; idx += blockDim.x) {
      const int i = (int)(idx / L.N), j = (int)(idx - (long long)i * L.N);
      const long long wi = (long long)i * L.P + (j >> 6);
      const int b = ens_bit(j & 63);
      dst[idx] = (uint8_t)(((Lp[wi] >> b) & 1ull) | (((Tp[wi] >> b) & 1ull) << 1));
    }
  }
}

// one lattice's bitplanes -> its bytes (the whole grid on one lattice)
__global__ void ens_unpack_one_kernel(const EnsLattice *lat, int l, const int *buf_of,
                                      const u64 *pool, uint8_t *dst) {
  const EnsLattice L = lat[l];
  const long long words = (long long)L.M * L.P;
  const u64 *Lp = pool + L.off[buf_of[l]], *Tp = Lp + words;
  const long long cells = (long long)L.M * L.N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < cells;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / L.N), j = (int)(idx - (long long)i * L.N);
    const long long wi = (long long)i * L.P + (j >> 6);
    const int b = ens_bit(j & 63);
    dst[idx] = (uint8_t)(((Lp[wi] >> b) & 1ull) | (((Tp[wi] >> b) & 1ull) << 1));
  }
}

// first step (0-based entry) with no move, per lattice, over [0, steps)
__global__ void ens_first_zero_kernel(const u64 *tr_lr, const u64 *tr_tb, long long cap,
                                      int count, long long steps, const long long *retired,
                                      long long *out) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < count; l += gridDim.x * blockDim.x) {
    long long r = -1;
    const u64 *a = tr_lr + (long long)l * cap, *b = tr_tb + (long long)l * cap;
    const long long end = retired[l] >= 0 && retired[l] < steps ? retired[l] : steps;
    for (long long s = 0; s < end; ++s)
      if (a[s] + b[s] == 0ull) {
        r = s;
        break;
      }
    out[l] = r;
  }
}

// current buffer index of every lattice
__global__ void ens_buf_of_kernel(const long long *frozen, const int *frozen_buf,
                                  const EnsCtrl *ctrl, int count, int *buf_of) {
  const int par = ctrl->parity;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < count; l += gridDim.x * blockDim.x)
    buf_of[l] = frozen[l] >= 0 ? frozen_buf[l] : par;
}

// number of cars of every lattice in buffer `buf` (conserved by the dynamics)
__global__ void ens_cars_kernel(const EnsLattice *lat, int count, const u64 *pool, int buf,
                                long long *cars) {
  __shared__ unsigned long long s;
  for (int l = blockIdx.x; l < count; l += gridDim.x) {
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const EnsLattice L = lat[l];
    const long long words = 2ll * L.M * L.P;  // both planes
    const u64 *p = pool + L.off[buf];
    unsigned long long c = 0;
    for (long long i = threadIdx.x; i < words; i += blockDim.x) c += __popcll(p[i]);
    atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0) cars[l] = (long long)s;
    __syncthreads();
  }
}

// Surrogate inputs: [cars/(M N), M/2048, N/2048, mean velocity of each of
// `points` windows of steps first .. first+n-1]; velocity = moved / cars.
__global__ void ens_features_kernel(const EnsLattice *lat, const long long *cars,
                                    const u64 *tr_lr, const u64 *tr_tb, long long cap,
                                    int count, long long first, long long n, int points,
                                    float *out) {
  const int stride = 3 + points;
  const long long per = n / points;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       idx < (long long)count * points; idx += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(idx / points), p = (int)(idx - (long long)l * points);
    const EnsLattice L = lat[l];
    const double c = (double)cars[l];
    const u64 *a = tr_lr + (long long)l * cap + first + p * per;
    const u64 *b = tr_tb + (long long)l * cap + first + p * per;
    double sum = 0.0;
    for (long long t = 0; t < per; ++t) sum += (double)(a[t] + b[t]);
    out[(long long)l * stride + 3 + p] = c > 0 ? (float)(sum / (c * (double)per)) : 0.f;
    if (p == 0) {
      out[(long long)l * stride + 0] = (float)(c / ((double)L.M * (double)L.N));
      out[(long long)l * stride + 1] = (float)L.M / 2048.f;
      out[(long long)l * stride + 2] = (float)L.N / 2048.f;
    }
  }
}

// Labels: mean velocity over steps steps-window .. steps-1, and jam = some
// step in 0 .. steps-1 moved no car.
__global__ void ens_labels_kernel(const long long *cars, const u64 *tr_lr, const u64 *tr_tb,
                                  long long cap, int count, long long steps, long long window,
                                  const long long *retired, float *v, float *jam) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < count; l += gridDim.x * blockDim.x) {
    const u64 *a = tr_lr + (long long)l * cap, *b = tr_tb + (long long)l * cap;
    // a retired lattice's trajectory ends at its retirement
    const long long end = retired[l] >= 0 && retired[l] < steps ? retired[l] : steps;
    const long long win = window < end ? window : end;
    double sum = 0.0;
    int j = 0;
    for (long long t = 0; t < end; ++t) {
      const u64 m = a[t] + b[t];
      if (m == 0) j = 1;
      if (t >= end - win) sum += (double)m;
    }
    const double c = (double)cars[l];
    v[l] = c > 0 && win > 0 ? (float)(sum / (c * (double)win)) : 0.f;
    jam[l] = (float)j;
  }
}

__global__ void ens_fill_kernel(long long *a, int count, long long v) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < count; l += gridDim.x * blockDim.x)
    a[l] = v;
}

// Stream-ordered after the steps taken so far: freeze the listed lattices
// where they are (a jammed lattice is frozen already) and record the step.
__global__ void ens_retire_kernel(const long long *idx, int n, const EnsCtrl *ctrl,
                                  long long *frozen, int *frozen_buf, long long *retired) {
  const long long now = ctrl->steps;
  const int par = ctrl->parity;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long l = idx[i];
    if (retired[l] < 0) retired[l] = now;
    if (frozen[l] < 0) {
      frozen[l] = now;
      frozen_buf[l] = par;
    }
  }
}

template <int K>
int ens_occupancy() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ens_kernel<K>, kEnsWarps * 32, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return b > 0 ? b : 1;
}

// The grid is one resident wave (SMs x blocks per SM); the launch is
// cooperative so that it fails rather than run part of the grid later.  The
// waits between chunks do not rely on that: a tile waits only for tiles that
// running warps have already drawn.
template <int K>
cudaError_t launch_ens(const EnsParams &p, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kEnsWarps * 32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, ens_kernel<K>, p);
}

}  // namespace
}  // namespace bml

// =================================================================== C ABI ==
using namespace bml;

namespace {

int efail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

}  // namespace

#define ECUDA(expr)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return efail(BML_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                   __LINE__);                                                             \
  } while (0)

struct bml_ens {
  int count = 0;
  std::vector<EnsLattice> lat;  // host copy
  cudaStream_t st = nullptr;
  int block_k = 0;
  int64_t band_rows = 0;
  unsigned flags = 0;
  long long timeout_ns = 2000000000ll;
  EnsLattice *d_lat = nullptr;
  EnsTile *d_tiles = nullptr;
  EnsGroup *d_groups = nullptr;
  int n_tiles = 0;
  u64 *pool = nullptr;
  size_t pool_words = 0;
  u64 *tr = nullptr;  // lr then tb, count * cap each
  long long cap = 0;
  long long *frozen = nullptr;
  long long *retired = nullptr;  // step at which a lattice was retired, else -1
  std::vector<char> unplanned;   // lattices left out of the tile plan (retired); empty: none
  bool band_fixed = false;       // band height given at creation (kept when re-planning)
  long long *cars = nullptr;
  int *frozen_buf = nullptr;
  int *buf_of = nullptr;
  long long *byte_off_d = nullptr;
  std::vector<long long> byte_off;
  long long total_bytes = 0;
  EnsCtrl *ctrl = nullptr;
  unsigned *lat_groups = nullptr;  // bands of every lattice in the current tile plan
  unsigned *lat_done = nullptr;    // bands finished per lattice, cleared before each launch
  unsigned max_groups = 1;         // most bands of one lattice
  u64 *scratch = nullptr;
  int *flag = nullptr;
  int grid[4] = {0, 0, 0, 0};  // persistent grid per depth index (k = 1, 2, 4, 8)
  int64_t steps_done = 0;
  bool failed = false;
  std::map<int64_t, cudaGraphExec_t> graphs;
  bool graphs_ok = true;
};

namespace {

int kidx(int k) { return k == 1 ? 0 : k == 2 ? 1 : k == 4 ? 2 : 3; }

void drop_graphs(bml_ens *e) {
  for (auto &kv : e->graphs) cudaGraphExecDestroy(kv.second);
  e->graphs.clear();
}

void ens_free(bml_ens *e) {
  cudaStreamSynchronize(e->st);
  drop_graphs(e);
  cudaFree(e->d_lat);
  cudaFree(e->d_tiles);
  cudaFree(e->d_groups);
  cudaFree(e->pool);
  cudaFree(e->tr);
  cudaFree(e->frozen);
  cudaFree(e->retired);
  cudaFree(e->cars);
  cudaFree(e->frozen_buf);
  cudaFree(e->buf_of);
  cudaFree(e->byte_off_d);
  cudaFree(e->ctrl);
  cudaFree(e->lat_groups);
  cudaFree(e->lat_done);
  cudaFree(e->scratch);
  cudaFree(e->flag);
}

struct TilePlan {
  std::vector<EnsTile> tiles;
  std::vector<EnsGroup> groups;
};

// Plan tiles for target band height `band`: every lattice is cut into
// round(M / band) bands (at least one) of near-equal length; groups of equal
// word width are packed 32 / W to a warp tile, longest bands first, and the
// tiles are ordered longest first for the kernel's dynamic assignment.
void plan_tiles(const bml_ens *e, int64_t band, TilePlan &plan) {
  // bands of every lattice, longest first
  struct Band {
    EnsGroup g;
    int W;
  };
  std::vector<Band> all;
  for (int l = 0; l < e->count; ++l) {
    if (!e->unplanned.empty() && e->unplanned[(size_t)l]) continue;  // retired: no tiles
    const int M = e->lat[l].M;
    int64_t nb = (int64_t)std::llround((double)M / (double)band);
    if (nb < 1) nb = 1;
    if (nb > M) nb = M;
    // keep every band below 65536 rows (per-lane counters are 32-bit)
    while ((M + nb - 1) / nb > 65535) ++nb;
    const int base = (int)(M / nb), rem = (int)(M % nb);
    int r0 = 0;
    for (int64_t b = 0; b < nb; ++b) {
      const int len = base + (b < rem ? 1 : 0);
      all.push_back(Band{EnsGroup{l, r0, len, 0}, e->lat[l].W});
      r0 += len;
    }
  }
  std::sort(all.begin(), all.end(), [](const Band &a, const Band &b) {
    if (a.g.len != b.g.len) return a.g.len > b.g.len;
    if (a.W != b.W) return a.W > b.W;
    return a.g.lat != b.g.lat ? a.g.lat < b.g.lat : a.g.r0 < b.g.r0;
  });
  // first fit into warps of 32 lanes: a band joins the first open warp (in
  // creation order) with room for its W lanes; a warp closes once the bands
  // reaching it are more than 1/8 shorter than its longest (every band runs
  // the warp's longest band's rows), or when it is full.  Open warps are kept
  // in ordered sets by free lanes; since bands arrive longest first, the
  // warps that have closed by age are the oldest of each set.
  std::vector<std::vector<EnsGroup>> tg;
  std::vector<int> used, maxlen, minlen;
  std::vector<std::set<size_t>> open_by_room(33);
  for (const Band &x : all) {
    size_t chosen = SIZE_MAX;
    for (int r = x.W; r <= 32; ++r) {
      std::set<size_t> &q = open_by_room[r];
      while (!q.empty() && (int64_t)maxlen[*q.begin()] * 7 > (int64_t)x.g.len * 8) q.erase(q.begin());
      if (!q.empty() && *q.begin() < chosen) chosen = *q.begin();
    }
    if (chosen == SIZE_MAX) {
      chosen = tg.size();
      tg.emplace_back();
      used.push_back(0);
      maxlen.push_back(x.g.len);
      minlen.push_back(x.g.len);
    } else {
      open_by_room[32 - used[chosen]].erase(chosen);
    }
    EnsGroup g = x.g;
    g.lane0 = used[chosen];
    tg[chosen].push_back(g);
    used[chosen] += x.W;
    minlen[chosen] = std::min(minlen[chosen], x.g.len);
    if (used[chosen] < 32) open_by_room[32 - used[chosen]].insert(chosen);
  }
  std::vector<EnsGroup> &groups = plan.groups;
  std::vector<EnsTile> &tiles = plan.tiles;
  groups.clear();
  tiles.clear();
  for (size_t ti = 0; ti < tg.size(); ++ti) {
    EnsTile t{};
    t.G = (int)tg[ti].size();
    t.first_group = (int)groups.size();
    t.max_len = maxlen[ti];
    t.min_len = minlen[ti];
    for (int l = 0; l < 32; ++l) t.lane_grp[l] = 0xff;
    for (int j = 0; j < t.G; ++j) {
      const EnsGroup &g = tg[ti][j];
      for (int l = g.lane0; l < g.lane0 + e->lat[g.lat].W; ++l) t.lane_grp[l] = (unsigned char)j;
      groups.push_back(g);
    }
    tiles.push_back(t);
  }
  std::stable_sort(tiles.begin(), tiles.end(),
                   [](const EnsTile &a, const EnsTile &b) { return a.max_len > b.max_len; });
}

// Predicted time of a launch of kTuneChunks chunks of depth k for a plan, in
// rows per warp.  A tile costs its longest band plus the 2k halo rows.  With
// no barrier between chunks a chunk costs the mean work per warp (total /
// warps), unless one lattice's longest band comes close: a lattice's chunk c
// waits for all of its bands' chunk c - 1, so the longest tile bounds a
// chunk from below (counted with a margin of 1.2: near the mean that chain
// already makes the time vary from run to run); the makespan of the
// longest-first assignment (list scheduling, simulated) beyond the mean is
// paid once, at the launch's end.
// On the bench ensemble (4096 lattices, depth 8) the measured times follow
// it: bands of 336 / 448 / 576 / 768 / 1024 rows, mean 1379 / 1363 / 1357 /
// 1359 / 1348 rows per warp, longest tile 519 / 687 / 879 / 1167 / 1551,
// 1.063 / 1.054 / 1.041 / 1.043 / 1.128 s for 10^4 steps.
constexpr int kTuneChunks = 32;
double plan_score(const TilePlan &plan, int k, int warps) {
  if (plan.tiles.empty() || warps < 1) return 0.0;
  std::vector<long long> heap((size_t)warps, 0);  // min-heap of warp finish times
  long long total = 0, makespan = 0, longest = 0;
  for (const EnsTile &t : plan.tiles) {
    const long long c = (long long)t.max_len + 2ll * k;
    total += c;
    longest = std::max(longest, c);
    std::pop_heap(heap.begin(), heap.end(), std::greater<long long>());
    heap.back() += c;
    makespan = std::max(makespan, heap.back());
    std::push_heap(heap.begin(), heap.end(), std::greater<long long>());
  }
  const double mean = (double)total / warps;
  return kTuneChunks * std::max(mean, 1.2 * (double)longest) + ((double)makespan - mean);
}

int upload_tiles(bml_ens *e, const TilePlan &plan, int64_t band) {
  const std::vector<EnsTile> &tiles = plan.tiles;
  const std::vector<EnsGroup> &groups = plan.groups;
  cudaFree(e->d_tiles);
  cudaFree(e->d_groups);
  e->d_tiles = nullptr;
  e->d_groups = nullptr;
  ECUDA(cudaMalloc(&e->d_tiles, std::max<size_t>(1, tiles.size()) * sizeof(EnsTile)));
  ECUDA(cudaMalloc(&e->d_groups, std::max<size_t>(1, groups.size()) * sizeof(EnsGroup)));
  ECUDA(cudaMemcpyAsync(e->d_tiles, tiles.data(), tiles.size() * sizeof(EnsTile),
                        cudaMemcpyHostToDevice, e->st));
  ECUDA(cudaMemcpyAsync(e->d_groups, groups.data(), groups.size() * sizeof(EnsGroup),
                        cudaMemcpyHostToDevice, e->st));
  // bands per lattice: what a wait between chunks counts to
  std::vector<unsigned> per((size_t)e->count, 0u);
  for (const EnsGroup &g : groups) ++per[(size_t)g.lat];
  e->max_groups = std::max(1u, *std::max_element(per.begin(), per.end()));
  ECUDA(cudaMemcpyAsync(e->lat_groups, per.data(), per.size() * sizeof(unsigned),
                        cudaMemcpyHostToDevice, e->st));
  ECUDA(cudaStreamSynchronize(e->st));
  e->n_tiles = (int)tiles.size();
  e->band_rows = band;
  drop_graphs(e);
  return BML_OK;
}

int build_tiles(bml_ens *e, int64_t band) {
  TilePlan plan;
  plan_tiles(e, band, plan);
  return upload_tiles(e, plan, band);
}

// Candidate band heights of the planner: 32 to 1024 rows in steps of 16,
// then powers of two up to the tallest lattice.
std::vector<int64_t> band_candidates(const bml_ens *e) {
  int max_m = 1;
  for (const EnsLattice &l : e->lat) max_m = std::max(max_m, l.M);
  std::vector<int64_t> bands;
  for (int64_t b = 32; b <= 1024; b += 16) bands.push_back(b);
  for (int64_t b = 2048; b / 2 < max_m; b *= 2) bands.push_back(b);
  return bands;
}

double plan_score(const TilePlan &plan, int k, int warps);
int grid_for(bml_ens *e, int k);

// New tile plan for the lattices still in it (after a retirement), at the
// current depth, with the band height given at creation, else the one of the
// best plan score (host only; no timing: the lattices' state must not move).
int replan_ens(bml_ens *e) {
  if (e->band_fixed) return build_tiles(e, e->band_rows);
  const int k = e->block_k;
  const int warps = grid_for(e, k) * kEnsWarps;
  double best = 1e300;
  int64_t best_b = e->band_rows;
  TilePlan plan;
  for (int64_t b : band_candidates(e)) {
    plan_tiles(e, b, plan);
    if (plan.tiles.empty()) {
      best_b = b;
      break;
    }
    const double sc = plan_score(plan, k, warps);
    if (sc < best) {
      best = sc;
      best_b = b;
    }
  }
  return build_tiles(e, best_b);
}

EnsParams make_params(bml_ens *e, int n_chunks, int commit) {
  EnsParams p{};
  p.lat = e->d_lat;
  p.tiles = e->d_tiles;
  p.groups = e->d_groups;
  p.n_tiles = e->n_tiles;
  p.n_chunks = n_chunks;
  p.pool = e->pool;
  p.tr_lr = e->tr;
  p.tr_tb = e->tr + (size_t)e->count * e->cap;
  p.cap = e->cap;
  p.frozen = e->frozen;
  p.frozen_buf = e->frozen_buf;
  p.ctrl = e->ctrl;
  p.commit = commit;
  p.early_exit = commit && (e->flags & BML_ENS_EARLY_EXIT) ? 1 : 0;
  p.lat_groups = e->lat_groups;
  p.lat_done = e->lat_done;
  p.stall_extra = (e->flags & BML_ENS_TEST_STALL) ? 1u : 0u;
  p.timeout_ns = e->timeout_ns;
  p.scratch = e->scratch;
  return p;
}

int grid_for(bml_ens *e, int k) {
  int &g = e->grid[kidx(k)];
  if (!g) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int occ = k == 1 ? ens_occupancy<1>() : k == 2 ? ens_occupancy<2>()
                  : k == 4 ? ens_occupancy<4>() : ens_occupancy<8>();
    g = sms * occ;
  }
  return g;
}

// Enqueue one persistent launch of n_chunks chunks of depth k.
int enqueue_ens(bml_ens *e, int k, int n_chunks, int commit) {
  if (n_chunks <= 0) return BML_OK;
  if (e->n_tiles == 0) {  // every lattice retired: nothing moves, the steps still count
    if (commit) {
      ens_advance_kernel<<<1, 32, 0, e->st>>>(e->ctrl, n_chunks, k);
      ECUDA(cudaGetLastError());
    }
    return BML_OK;
  }
  EnsParams p = make_params(e, n_chunks, commit);
  const int grid = grid_for(e, k);
  ECUDA(cudaMemsetAsync(e->lat_done, 0, (size_t)e->count * sizeof(unsigned), e->st));
  cudaError_t rc;
  switch (k) {
    case 1: rc = launch_ens<1>(p, grid, e->st); break;
    case 2: rc = launch_ens<2>(p, grid, e->st); break;
    case 4: rc = launch_ens<4>(p, grid, e->st); break;
    default: rc = launch_ens<8>(p, grid, e->st); break;
  }
  if (rc != cudaSuccess) return efail(BML_ECUDA, "ensemble launch: %s", cudaGetErrorString(rc));
  if (commit) {
    ens_advance_kernel<<<1, 32, 0, e->st>>>(e->ctrl, n_chunks, k);
    ECUDA(cudaGetLastError());
  }
  return BML_OK;
}

// k steps: full chunks at block_k, then the remainder by powers of two.
int enqueue_steps_ens(bml_ens *e, int64_t k) {
  const int64_t full = k / e->block_k;
  int64_t left = k - full * e->block_k;
  int64_t done = 0;
  // one launch draws n_chunks * n_tiles + warps 32-bit tickets, and a
  // lattice's count of finished bands reaches n_chunks * its bands
  const int64_t per_chunk = (int64_t)e->n_tiles + 4ll * grid_for(e, e->block_k);
  const int64_t max_chunks = std::max<int64_t>(
      1, std::min<int64_t>({1 << 20, 0xffffffffll / per_chunk,
                            (0xffffffffll - 1) / (int64_t)e->max_groups}));
  while (done < full) {
    const int n = (int)std::min<int64_t>(full - done, max_chunks);
    int rc = enqueue_ens(e, e->block_k, n, 1);
    if (rc) return rc;
    done += n;
  }
  for (int d = 4; d >= 1; d >>= 1)
    if (d < e->block_k && left >= d) {
      int rc = enqueue_ens(e, d, 1, 1);
      if (rc) return rc;
      left -= d;
    }
  return BML_OK;
}

int grow_traces(bml_ens *e, long long need) {
  if (need <= e->cap) return BML_OK;
  long long ncap = e->cap > 0 ? e->cap : 1024;
  while (ncap < need) ncap *= 2;
  u64 *ntr = nullptr;
  ECUDA(cudaMalloc(&ntr, (size_t)e->count * ncap * 2 * sizeof(u64)));
  ECUDA(cudaMemsetAsync(ntr, 0, (size_t)e->count * ncap * 2 * sizeof(u64), e->st));
  if (e->tr && e->steps_done > 0) {
    for (int half = 0; half < 2; ++half)
      ECUDA(cudaMemcpy2DAsync(ntr + (size_t)half * e->count * ncap, (size_t)ncap * 8,
                              e->tr + (size_t)half * e->count * e->cap, (size_t)e->cap * 8,
                              (size_t)e->steps_done * 8, (size_t)e->count,
                              cudaMemcpyDeviceToDevice, e->st));
  }
  ECUDA(cudaStreamSynchronize(e->st));
  cudaFree(e->tr);
  e->tr = ntr;
  e->cap = ncap;
  drop_graphs(e);  // captured launches hold the old pointers
  return BML_OK;
}

int check_err(bml_ens *e) {
  EnsCtrl c;
  ECUDA(cudaMemcpyAsync(&c, e->ctrl, sizeof c, cudaMemcpyDeviceToHost, e->st));
  ECUDA(cudaStreamSynchronize(e->st));
  if (c.err) {
    e->failed = true;
    return efail(BML_ETIMEOUT, "a wait between chunks of the ensemble kernel timed out; the "
                 "ensemble state is undefined");
  }
  return BML_OK;
}

// Autotune (depth, band).  Every band height from 32 to 1024 rows in steps of
// 16 (and powers of two up to the tallest lattice) is planned on the host
// and scored for depth 8 (plan_score); the four best distinct plans are
// timed at depth 8 and the best-scored one also at depths 1, 2 and 4, each
// on launches of kTuneChunks chunks (as long calls run them: the end-of-launch
// tail is paid once, not once per chunk).
int autotune_ens(bml_ens *e) {
  const std::vector<int64_t> bands = band_candidates(e);
  const int warps8 = grid_for(e, 8) * kEnsWarps;
  struct Cand {
    double score;
    int64_t band;
    size_t n_tiles;
  };
  std::vector<Cand> cands;
  {
    TilePlan plan;
    for (int64_t b : bands) {
      plan_tiles(e, b, plan);
      cands.push_back(Cand{plan_score(plan, 8, warps8), b, plan.tiles.size()});
    }
  }
  std::stable_sort(cands.begin(), cands.end(),
                   [](const Cand &x, const Cand &y) { return x.score < y.score; });
  // drop repeats of the same plan (bands above every lattice's height)
  std::vector<Cand> top;
  for (const Cand &c : cands) {
    bool dup = false;
    for (const Cand &t : top) dup = dup || (t.n_tiles == c.n_tiles && t.score == c.score);
    if (!dup) top.push_back(c);
    if (top.size() == 4) break;
  }
  std::vector<std::pair<int64_t, int>> trials;  // (band, depth)
  for (const Cand &c : top) trials.emplace_back(c.band, 8);
  for (int k : {4, 2, 1}) trials.emplace_back(top[0].band, k);

  cudaEvent_t a, b;
  ECUDA(cudaEventCreate(&a));
  ECUDA(cudaEventCreate(&b));
  double best = 1e30;
  int best_k = 8;
  int64_t best_b = top[0].band;
  int64_t built = -1;
  int rc = BML_OK;
  for (const auto &tr : trials) {
    const int64_t band = tr.first;
    const int k = tr.second;
    if (band != built) {
      if ((rc = build_tiles(e, band))) break;
      built = band;
    }
    if ((rc = enqueue_ens(e, k, kTuneChunks, 0))) break;  // warm-up, not committed
    cudaEventRecord(a, e->st);
    const int reps = 2;
    for (int r = 0; r < reps && !rc; ++r) rc = enqueue_ens(e, k, kTuneChunks, 0);
    cudaEventRecord(b, e->st);
    if (rc) break;
    if (cudaEventSynchronize(b) != cudaSuccess) {
      rc = efail(BML_ECUDA, "ensemble autotune: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    const double per = ms / ((double)reps * kTuneChunks * k);
    if (per < best) {
      best = per;
      best_k = k;
      best_b = band;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  if ((rc = check_err(e))) return rc;
  e->block_k = best_k;
  return build_tiles(e, best_b);
}

// Autotuned (depth, band) per device and multiset of lattice shapes: an
// ensemble of the same shapes (another seed set or density mix, say) reuses
// the choice instead of timing the candidates again.
struct EnsTuneKey {
  int dev;
  int count;
  unsigned long long shapes;  // FNV-1a hash of the sorted (M, N) pairs
  bool operator<(const EnsTuneKey &o) const {
    if (dev != o.dev) return dev < o.dev;
    if (count != o.count) return count < o.count;
    return shapes < o.shapes;
  }
};
std::mutex g_ens_tune_mu;
std::map<EnsTuneKey, std::pair<int, int64_t>> g_ens_tune;

EnsTuneKey tune_key(const bml_ens *e) {
  std::vector<std::pair<int, int>> sh;
  sh.reserve(e->lat.size());
  for (const EnsLattice &l : e->lat) sh.emplace_back(l.M, l.N);
  std::sort(sh.begin(), sh.end());
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&h](unsigned long long v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xffull;
      h *= 1099511628211ull;
    }
  };
  for (const auto &x : sh) {
    mix((unsigned long long)x.first);
    mix((unsigned long long)x.second);
  }
  int dev = 0;
  cudaGetDevice(&dev);
  return EnsTuneKey{dev, e->count, h};
}

int tune_or_reuse(bml_ens *e) {
  const EnsTuneKey key = tune_key(e);
  {
    std::lock_guard<std::mutex> lock(g_ens_tune_mu);
    auto it = g_ens_tune.find(key);
    if (it != g_ens_tune.end()) {
      e->block_k = it->second.first;
      return build_tiles(e, it->second.second);
    }
  }
  int rc = autotune_ens(e);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_ens_tune_mu);
  g_ens_tune[key] = std::make_pair(e->block_k, e->band_rows);
  return BML_OK;
}

}  // namespace

extern "C" int bml_ensemble_create_ex(int64_t count, const int64_t *M, const int64_t *N,
                                      const uint64_t *seed, const double *p_lr,
                                      const double *p_tb, int block_k, int64_t band_rows,
                                      unsigned flags, void *stream, int64_t reserve_steps,
                                      bml_ens **out) {
  if (!out || !M || !N || !seed || !p_lr || !p_tb) return efail(BML_EINVAL, "NULL argument");
  if (count < 1 || count > (1 << 30)) return efail(BML_EINVAL, "count must be in [1, 2^30]");
  if (block_k != 0 && block_k != 1 && block_k != 2 && block_k != 4 && block_k != 8)
    return efail(BML_EINVAL, "block_k must be 0 (autotune), 1, 2, 4 or 8");
  if (band_rows < 0) return efail(BML_EINVAL, "band_rows < 0");
  if ((block_k == 0) != (band_rows == 0))
    return efail(BML_EINVAL, "block_k and band_rows are both 0 (autotune) or both set");
  if (reserve_steps < 0) return efail(BML_EINVAL, "reserve_steps < 0");
  double total_cells = 0;
  for (int64_t l = 0; l < count; ++l) {
    if (M[l] < 1 || N[l] < 1 || N[l] > 2048 || M[l] > (1 << 24))
      return efail(BML_EINVAL, "lattice %lld: need 1 <= N <= 2048 and 1 <= M <= 2^24",
                   (long long)l);
    if (!(p_lr[l] >= 0.0 && p_tb[l] >= 0.0 && p_lr[l] + p_tb[l] <= 1.0))
      return efail(BML_EINVAL, "lattice %lld: bad p_lr/p_tb", (long long)l);
    total_cells += (double)M[l] * (double)N[l];
  }
  if (total_cells > 68719476736.0) return efail(BML_EINVAL, "ensemble larger than 2^36 cells");

  bml_ens *e = new (std::nothrow) bml_ens;
  if (!e) return efail(BML_ENOMEM, "host allocation failed");
  e->count = (int)count;
  e->st = (cudaStream_t)stream;
  e->flags = flags;
  if (flags & BML_ENS_TEST_STALL) e->timeout_ns = 20000000ll;  // 20 ms
  e->lat.resize(count);
  e->byte_off.resize(count);
  size_t words = 0;
  long long bytes = 0;
  for (int64_t l = 0; l < count; ++l) {
    EnsLattice &L = e->lat[l];
    L.M = (int)M[l];
    L.N = (int)N[l];
    L.W = (L.N + 63) / 64;
    L.P = (L.W + 1) & ~1;
    L.nb = L.N - 64 * (L.W - 1);
    L.tail = L.nb == 64 ? ~0ull : ((1ull << L.nb) - 1ull);
    L.pad = 0;
    const size_t per = (size_t)2 * L.M * L.P;  // L and T
    L.off[0] = words;
    L.off[1] = words + per;
    words += 2 * per;
    e->byte_off[l] = bytes;
    bytes += (long long)L.M * L.N;
  }
  e->pool_words = words;
  e->total_bytes = bytes;
  int rc = BML_OK;
  std::vector<u64> tl(count), tt(count);
  for (int64_t l = 0; l < count; ++l) {
    tl[l] = placement_threshold(p_lr[l]);
    tt[l] = placement_threshold(p_tb[l]);
  }
  u64 *d_seed = nullptr, *d_tl = nullptr, *d_tt = nullptr;
#define ETRY(expr)                                                                          \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      rc = efail(e_ == cudaErrorMemoryAllocation ? BML_ENOMEM : BML_ECUDA, "%s: %s", #expr, \
                 cudaGetErrorString(e_));                                                   \
      goto fail_;                                                                           \
    }                                                                                       \
  } while (0)
  ETRY(cudaMalloc(&e->d_lat, count * sizeof(EnsLattice)));
  ETRY(cudaMalloc(&e->pool, words * sizeof(u64)));
  ETRY(cudaMalloc(&e->frozen, count * sizeof(long long)));
  ETRY(cudaMalloc(&e->retired, count * sizeof(long long)));
  ETRY(cudaMalloc(&e->cars, count * sizeof(long long)));
  ETRY(cudaMalloc(&e->frozen_buf, count * sizeof(int)));
  ETRY(cudaMalloc(&e->buf_of, count * sizeof(int)));
  ETRY(cudaMalloc(&e->byte_off_d, count * sizeof(long long)));
  ETRY(cudaMalloc(&e->ctrl, sizeof(EnsCtrl)));
  ETRY(cudaMalloc(&e->lat_groups, count * sizeof(unsigned)));
  ETRY(cudaMalloc(&e->lat_done, count * sizeof(unsigned)));
  ETRY(cudaMalloc(&e->scratch, 16 * sizeof(u64)));
  ETRY(cudaMalloc(&e->flag, 256));
  ETRY(cudaMalloc(&d_seed, count * 8));
  ETRY(cudaMalloc(&d_tl, count * 8));
  ETRY(cudaMalloc(&d_tt, count * 8));
  ETRY(cudaMemcpyAsync(e->d_lat, e->lat.data(), count * sizeof(EnsLattice),
                       cudaMemcpyHostToDevice, e->st));
  ETRY(cudaMemcpyAsync(e->byte_off_d, e->byte_off.data(), count * 8, cudaMemcpyHostToDevice,
                       e->st));
  ETRY(cudaMemcpyAsync(d_seed, seed, count * 8, cudaMemcpyHostToDevice, e->st));
  ETRY(cudaMemcpyAsync(d_tl, tl.data(), count * 8, cudaMemcpyHostToDevice, e->st));
  ETRY(cudaMemcpyAsync(d_tt, tt.data(), count * 8, cudaMemcpyHostToDevice, e->st));
  ETRY(cudaMemsetAsync(e->pool, 0, words * sizeof(u64), e->st));
  ETRY(cudaMemsetAsync(e->ctrl, 0, sizeof(EnsCtrl), e->st));
  ETRY(cudaMemsetAsync(e->scratch, 0, 16 * sizeof(u64), e->st));
  ETRY(cudaMemsetAsync(e->frozen_buf, 0, count * sizeof(int), e->st));
  ens_fill_kernel<<<256, 256, 0, e->st>>>(e->frozen, (int)count, -1);
  ens_fill_kernel<<<256, 256, 0, e->st>>>(e->retired, (int)count, -1);
  ETRY(cudaGetLastError());
  ens_init_kernel<<<(unsigned)std::min<int64_t>(count, 148 * 16), 256, 0, e->st>>>(
      e->d_lat, (int)count, d_seed, d_tl, d_tt, e->pool);
  ETRY(cudaGetLastError());
  ens_cars_kernel<<<(unsigned)std::min<int64_t>(count, 148 * 16), 256, 0, e->st>>>(
      e->d_lat, (int)count, e->pool, 0, e->cars);
  ETRY(cudaGetLastError());
  ETRY(cudaStreamSynchronize(e->st));
  cudaFree(d_seed);
  cudaFree(d_tl);
  cudaFree(d_tt);
  d_seed = d_tl = d_tt = nullptr;
  if ((rc = grow_traces(e, reserve_steps > 0 ? reserve_steps : 1024))) goto fail_;
  if (block_k == 0) {
    if ((rc = tune_or_reuse(e))) goto fail_;
  } else {
    e->block_k = block_k;
    e->band_fixed = true;
    if ((rc = build_tiles(e, band_rows))) goto fail_;
  }
  *out = e;
  return BML_OK;
fail_:
#undef ETRY
  cudaFree(d_seed);
  cudaFree(d_tl);
  cudaFree(d_tt);
  ens_free(e);
  delete e;
  return rc;
}

extern "C" int bml_ensemble_create(int64_t count, const int64_t *M, const int64_t *N,
                                   const uint64_t *seed, const double *p_lr, const double *p_tb,
                                   void *stream, bml_ens **out) {
  return bml_ensemble_create_ex(count, M, N, seed, p_lr, p_tb, 0, 0, 0, stream, 0, out);
}

extern "C" void bml_ensemble_destroy(bml_ens *e) {
  if (!e) return;
  ens_free(e);
  delete e;
}

extern "C" int bml_ensemble_step(bml_ens *e, int64_t k) {
  if (!e) return efail(BML_EINVAL, "ensemble is NULL");
  if (e->failed) return efail(BML_ESTATE, "ensemble failed earlier (a wait between chunks timed out)");
  if (k < 0) return efail(BML_EINVAL, "k < 0");
  if (k == 0) return BML_OK;
  int rc = grow_traces(e, e->steps_done + k);
  if (rc) return rc;
  const bool use_graph = e->graphs_ok && !(e->flags & BML_ENS_NO_GRAPH);
  if (use_graph) {
    auto it = e->graphs.find(k);
    if (it == e->graphs.end()) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      bool ok = cudaStreamBeginCapture(e->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const int erc = enqueue_steps_ens(e, k);
        ok = cudaStreamEndCapture(e->st, &g) == cudaSuccess && erc == BML_OK;
      }
      if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
      if (!ok) {
        cudaGetLastError();
        e->graphs_ok = false;  // fall back to direct launches from now on
      } else {
        it = e->graphs.emplace(k, ge).first;
      }
    }
    if (e->graphs_ok) {
      ECUDA(cudaGraphLaunch(it->second, e->st));
      e->steps_done += k;
      if (e->flags & BML_ENS_TEST_STALL) return check_err(e);
      return BML_OK;
    }
  }
  if ((rc = enqueue_steps_ens(e, k))) return rc;
  e->steps_done += k;
  if (e->flags & BML_ENS_TEST_STALL) return check_err(e);
  return BML_OK;
}

extern "C" int bml_ensemble_synchronize(bml_ens *e) {
  if (!e) return efail(BML_EINVAL, "ensemble is NULL");
  ECUDA(cudaStreamSynchronize(e->st));
  return check_err(e);
}

extern "C" int64_t bml_ensemble_steps_done(const bml_ens *e) { return e ? e->steps_done : -1; }

extern "C" int bml_ensemble_plan(int64_t count, const int64_t *M, const int64_t *N,
                                 int64_t band, int depth, int warps, int64_t *out_tiles,
                                 double *out_score, int64_t *out_rows) {
  if (!M || !N || !out_tiles || !out_score) return efail(BML_EINVAL, "NULL argument");
  if (count < 1 || count > (1 << 30)) return efail(BML_EINVAL, "count must be in [1, 2^30]");
  if (band < 1 || depth < 1 || depth > 64 || warps < 1)
    return efail(BML_EINVAL, "need band >= 1, 1 <= depth <= 64, warps >= 1");
  bml_ens e;  // host fields only: no device memory is touched
  e.count = (int)count;
  e.lat.resize((size_t)count);
  for (int64_t l = 0; l < count; ++l) {
    if (M[l] < 1 || N[l] < 1 || N[l] > 2048 || M[l] > (1 << 24))
      return efail(BML_EINVAL, "lattice %lld: need 1 <= N <= 2048 and 1 <= M <= 2^24",
                   (long long)l);
    EnsLattice &L = e.lat[(size_t)l];
    L.M = (int)M[l];
    L.N = (int)N[l];
    L.W = (L.N + 63) / 64;
    L.P = L.W + (L.W & 1);
    L.nb = L.N - 64 * (L.W - 1);
  }
  TilePlan plan;
  plan_tiles(&e, band, plan);
  *out_tiles = (int64_t)plan.tiles.size();
  *out_score = plan_score(plan, depth, warps);
  if (out_rows) {
    for (int64_t l = 0; l < count; ++l) out_rows[l] = 0;
    for (const EnsTile &t : plan.tiles)
      for (int j = 0; j < t.G; ++j) {
        const EnsGroup &g = plan.groups[(size_t)(t.first_group + j)];
        // a group's lanes must lie inside the warp and match the lattice's width
        int lanes = 0;
        for (int l = 0; l < 32; ++l) lanes += t.lane_grp[l] == j;
        if (g.lane0 + e.lat[(size_t)g.lat].W > 32 || lanes != e.lat[(size_t)g.lat].W ||
            g.len > t.max_len || g.len < t.min_len)
          return efail(BML_ESTATE, "inconsistent tile plan");
        out_rows[g.lat] += g.len;
      }
  }
  return BML_OK;
}

extern "C" int bml_ensemble_retire(bml_ens *e, int64_t n, const int64_t *lattices) {
  if (!e || (n > 0 && !lattices)) return efail(BML_EINVAL, "NULL argument");
  if (n < 0 || n > INT32_MAX) return efail(BML_EINVAL, "n outside [0, 2^31)");
  if (e->failed) return efail(BML_ESTATE, "ensemble failed earlier (a wait between chunks timed out)");
  for (int64_t i = 0; i < n; ++i)
    if (lattices[i] < 0 || lattices[i] >= e->count)
      return efail(BML_EINVAL, "lattice index %lld out of range", (long long)lattices[i]);
  if (n == 0) return BML_OK;
  long long *d = nullptr;
  ECUDA(cudaMalloc(&d, (size_t)n * sizeof(long long)));
  cudaError_t r = cudaMemcpyAsync(d, lattices, (size_t)n * sizeof(long long),
                                  cudaMemcpyHostToDevice, e->st);
  if (r == cudaSuccess) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
    ens_retire_kernel<<<blocks, 256, 0, e->st>>>(d, (int)n, e->ctrl, e->frozen, e->frozen_buf,
                                                 e->retired);
    r = cudaGetLastError();
  }
  if (r == cudaSuccess) r = cudaStreamSynchronize(e->st);
  cudaFree(d);
  if (r != cudaSuccess) return efail(BML_ECUDA, "retire: %s", cudaGetErrorString(r));
  int rc = check_err(e);
  if (rc) return rc;
  // the retired lattices leave the tile plan, and the band height is chosen
  // again for the lattices that go on (fewer lattices: shorter bands keep the
  // warps busy)
  if (e->unplanned.empty()) e->unplanned.assign((size_t)e->count, 0);
  for (int64_t i = 0; i < n; ++i) e->unplanned[(size_t)lattices[i]] = 1;
  return replan_ens(e);
}

extern "C" int bml_ensemble_get_config(const bml_ens *e, int *block_k, int64_t *band_rows,
                                       int *graphs) {
  if (!e) return efail(BML_EINVAL, "ensemble is NULL");
  if (block_k) *block_k = e->block_k;
  if (band_rows) *band_rows = e->band_rows;
  if (graphs) *graphs = e->graphs_ok && !(e->flags & BML_ENS_NO_GRAPH) ? 1 : 0;
  return BML_OK;
}

extern "C" int bml_ensemble_traces(bml_ens *e, int64_t first, int64_t n, int64_t *out_lr,
                                   int64_t *out_tb) {
  if (!e) return efail(BML_EINVAL, "ensemble is NULL");
  if (first < 0 || n < 0 || first + n > e->steps_done)
    return efail(BML_EINVAL, "step range outside [0, steps_done)");
  if (n == 0) return BML_OK;
  int rc = check_err(e);
  if (rc) return rc;
  for (int half = 0; half < 2; ++half) {
    int64_t *dst = half ? out_tb : out_lr;
    if (!dst) continue;
    ECUDA(cudaMemcpy2DAsync(dst, (size_t)n * 8,
                            e->tr + (size_t)half * e->count * e->cap + first, (size_t)e->cap * 8,
                            (size_t)n * 8, (size_t)e->count, cudaMemcpyDeviceToHost, e->st));
  }
  ECUDA(cudaStreamSynchronize(e->st));
  return BML_OK;
}

extern "C" int bml_ensemble_moved_counts(bml_ens *e, int64_t lattice, int64_t first, int64_t n,
                                         int64_t *out_total, int64_t *out_lr, int64_t *out_tb) {
  if (!e) return efail(BML_EINVAL, "ensemble is NULL");
  if (lattice < 0 || lattice >= e->count) return efail(BML_EINVAL, "lattice out of range");
  if (first < 0 || n < 0 || first + n > e->steps_done)
    return efail(BML_EINVAL, "step range outside [0, steps_done)");
  if (n == 0) return BML_OK;
  int rc = check_err(e);
  if (rc) return rc;
  std::vector<int64_t> a((size_t)n), b((size_t)n);
  ECUDA(cudaMemcpyAsync(a.data(), e->tr + (size_t)lattice * e->cap + first, (size_t)n * 8,
                        cudaMemcpyDeviceToHost, e->st));
  ECUDA(cudaMemcpyAsync(b.data(),
                        e->tr + (size_t)e->count * e->cap + (size_t)lattice * e->cap + first,
                        (size_t)n * 8, cudaMemcpyDeviceToHost, e->st));
  ECUDA(cudaStreamSynchronize(e->st));
  for (int64_t t = 0; t < n; ++t) {
    if (out_lr) out_lr[t] = a[(size_t)t];
    if (out_tb) out_tb[t] = b[(size_t)t];
    if (out_total) out_total[t] = a[(size_t)t] + b[(size_t)t];
  }
  return BML_OK;
}

extern "C" int bml_ensemble_jam_steps(bml_ens *e, int64_t *out) {
  if (!e || !out) return efail(BML_EINVAL, "NULL argument");
  int rc = check_err(e);
  if (rc) return rc;
  long long *d = nullptr;
  ECUDA(cudaMalloc(&d, (size_t)e->count * 8));
  ens_first_zero_kernel<<<(e->count + 255) / 256, 256, 0, e->st>>>(
      e->tr, e->tr + (size_t)e->count * e->cap, e->cap, e->count, e->steps_done, e->retired, d);
  cudaError_t r = cudaGetLastError();
  if (r == cudaSuccess)
    r = cudaMemcpyAsync(out, d, (size_t)e->count * 8, cudaMemcpyDeviceToHost, e->st);
  if (r == cudaSuccess) r = cudaStreamSynchronize(e->st);
  cudaFree(d);
  if (r != cudaSuccess) return efail(BML_ECUDA, "jam steps: %s", cudaGetErrorString(r));
  return BML_OK;
}

extern "C" int bml_ensemble_read_lattices(bml_ens *e, uint8_t *out) {
  if (!e || !out) return efail(BML_EINVAL, "NULL argument");
  int rc = check_err(e);
  if (rc) return rc;
  uint8_t *d = nullptr;
  ECUDA(cudaMalloc(&d, (size_t)std::max<long long>(1, e->total_bytes)));
  ens_buf_of_kernel<<<(e->count + 255) / 256, 256, 0, e->st>>>(e->frozen, e->frozen_buf, e->ctrl,
                                                              e->count, e->buf_of);
  ens_unpack_kernel<<<(unsigned)std::min(e->count, 148 * 16), 256, 0, e->st>>>(
      e->d_lat, e->count, e->byte_off_d, e->buf_of, e->pool, d);
  cudaError_t r = cudaGetLastError();
  if (r == cudaSuccess)
    r = cudaMemcpyAsync(out, d, (size_t)e->total_bytes, cudaMemcpyDeviceToHost, e->st);
  if (r == cudaSuccess) r = cudaStreamSynchronize(e->st);
  cudaFree(d);
  if (r != cudaSuccess) return efail(BML_ECUDA, "read lattices: %s", cudaGetErrorString(r));
  return BML_OK;
}

extern "C" int bml_ensemble_read_lattice(bml_ens *e, int64_t lattice, uint8_t *out) {
  if (!e || !out) return efail(BML_EINVAL, "NULL argument");
  if (lattice < 0 || lattice >= e->count) return efail(BML_EINVAL, "lattice out of range");
  int rc = check_err(e);
  if (rc) return rc;
  // unpack only this lattice (reading every lattice would move the whole
  // ensemble for one of them)
  const EnsLattice &L = e->lat[(size_t)lattice];
  const size_t cells = (size_t)L.M * (size_t)L.N;
  uint8_t *d = nullptr;
  ECUDA(cudaMalloc(&d, std::max<size_t>(1, cells)));
  ens_buf_of_kernel<<<(e->count + 255) / 256, 256, 0, e->st>>>(e->frozen, e->frozen_buf, e->ctrl,
                                                              e->count, e->buf_of);
  const size_t blocks = std::min<size_t>((cells + 255) / 256, 148 * 8);
  ens_unpack_one_kernel<<<(unsigned)std::max<size_t>(1, blocks), 256, 0, e->st>>>(
      e->d_lat, (int)lattice, e->buf_of, e->pool, d);
  cudaError_t r = cudaGetLastError();
  if (r == cudaSuccess) r = cudaMemcpyAsync(out, d, cells, cudaMemcpyDeviceToHost, e->st);
  if (r == cudaSuccess) r = cudaStreamSynchronize(e->st);
  cudaFree(d);
  if (r != cudaSuccess) return efail(BML_ECUDA, "read lattice: %s", cudaGetErrorString(r));
  return BML_OK;
}

extern "C" int bml_ensemble_write_lattices(bml_ens *e, const uint8_t *in) {
  if (!e || !in) return efail(BML_EINVAL, "NULL argument");
  if (e->failed) return efail(BML_ESTATE, "ensemble failed earlier (a wait between chunks timed out)");
  uint8_t *d = nullptr;
  ECUDA(cudaMalloc(&d, (size_t)std::max<long long>(1, e->total_bytes)));
  int hbad = 0;
  EnsCtrl c0{};
  const unsigned blocks = (unsigned)std::min(e->count, 148 * 16);
  cudaError_t r = cudaMemcpyAsync(d, in, (size_t)e->total_bytes, cudaMemcpyHostToDevice, e->st);
  if (r == cudaSuccess) r = cudaMemsetAsync(e->flag, 0, sizeof(int), e->st);
  // check every value first, so that a rejected input leaves the state as it
  // was; then pack into buffer 0 and restart all trajectories
  if (r == cudaSuccess) {
    ens_pack_kernel<<<blocks, 256, 0, e->st>>>(e->d_lat, e->count, e->byte_off_d, d, 0, nullptr,
                                               e->flag);
    r = cudaGetLastError();
  }
  if (r == cudaSuccess)
    r = cudaMemcpyAsync(&hbad, e->flag, sizeof(int), cudaMemcpyDeviceToHost, e->st);
  if (r == cudaSuccess) r = cudaStreamSynchronize(e->st);
  if (r == cudaSuccess && !hbad) {
    ens_pack_kernel<<<blocks, 256, 0, e->st>>>(e->d_lat, e->count, e->byte_off_d, d, 0, e->pool,
                                               e->flag);
    r = cudaGetLastError();
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(e->ctrl, &c0, sizeof c0, cudaMemcpyHostToDevice, e->st);
    if (r == cudaSuccess)
      r = cudaMemsetAsync(e->tr, 0, (size_t)e->count * e->cap * 2 * sizeof(u64), e->st);
    if (r == cudaSuccess) {
      ens_fill_kernel<<<256, 256, 0, e->st>>>(e->frozen, e->count, -1);
      ens_fill_kernel<<<256, 256, 0, e->st>>>(e->retired, e->count, -1);
      r = cudaGetLastError();
    }
    if (r == cudaSuccess) {
      ens_cars_kernel<<<blocks, 256, 0, e->st>>>(e->d_lat, e->count, e->pool, 0, e->cars);
      r = cudaGetLastError();
    }
    if (r == cudaSuccess) r = cudaStreamSynchronize(e->st);
    if (r == cudaSuccess) e->steps_done = 0;
  }
  cudaFree(d);
  if (r != cudaSuccess) return efail(BML_ECUDA, "write lattices: %s", cudaGetErrorString(r));
  if (hbad) return efail(BML_EINVAL, "a lattice holds a value other than 0, 1, 2");
  if (!e->unplanned.empty()) {  // no lattice is retired any more: plan them all again
    e->unplanned.clear();
    return replan_ens(e);
  }
  return BML_OK;
}

extern "C" int bml_ensemble_car_counts(bml_ens *e, int64_t *out) {
  if (!e || !out) return efail(BML_EINVAL, "NULL argument");
  ECUDA(cudaMemcpyAsync(out, e->cars, (size_t)e->count * 8, cudaMemcpyDeviceToHost, e->st));
  ECUDA(cudaStreamSynchronize(e->st));
  return BML_OK;
}

extern "C" int bml_ensemble_features(bml_ens *e, int64_t first, int64_t n, int points,
                                     float *d_out) {
  if (!e || !d_out) return efail(BML_EINVAL, "NULL argument");
  if (points < 1 || n < points || n % points || first < 0 || first + n > e->steps_done)
    return efail(BML_EINVAL, "need points >= 1, n a multiple of points, and steps "
                 "[first, first+n) already taken");
  int rc = check_err(e);
  if (rc) return rc;
  const long long items = (long long)e->count * points;
  ens_features_kernel<<<(unsigned)std::min<long long>((items + 255) / 256, 4096), 256, 0, e->st>>>(
      e->d_lat, e->cars, e->tr, e->tr + (size_t)e->count * e->cap, e->cap, e->count, first, n,
      points, d_out);
  ECUDA(cudaGetLastError());
  ECUDA(cudaStreamSynchronize(e->st));
  return BML_OK;
}

extern "C" int bml_ensemble_labels(bml_ens *e, int64_t window, float *d_v, float *d_jam) {
  if (!e || !d_v || !d_jam) return efail(BML_EINVAL, "NULL argument");
  if (window < 1 || window > e->steps_done)
    return efail(BML_EINVAL, "need 1 <= window <= steps_done");
  int rc = check_err(e);
  if (rc) return rc;
  ens_labels_kernel<<<(e->count + 255) / 256, 256, 0, e->st>>>(
      e->cars, e->tr, e->tr + (size_t)e->count * e->cap, e->cap, e->count, e->steps_done, window,
      e->retired, d_v, d_jam);
  ECUDA(cudaGetLastError());
  ECUDA(cudaStreamSynchronize(e->st));
  return BML_OK;
}
