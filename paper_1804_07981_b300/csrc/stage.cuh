// One pipeline stage of the streaming bitplane step, shared by the
// single-lattice streaming kernel and the ensemble kernel.
//
// With E = EMPTY before the horizontal phase (Sec. 2 rules):
//   Er_x  = E_x shifted one column left (Er[j] = E[j+1], the cell ahead)
//   in_x  = (L_x shifted one column right) & E_x   the cells LR cars enter
//   Lh_x  = (L_x & ~Er_x) | in_x   horizontal rule on row x (cars that stay,
//                                  plus cars that enter)
//   E'_x  = ~(Lh_x | T_x)          EMPTY after the horizontal phase (TB cars
//                                  do not move in it)
//   mvV_{x-1} = T_{x-1} & E'_x     TB cars of row x-1 that move down
//   emitted row x-1: L = Lh_{x-1}, T = (T_{x-1} & ~mvV_{x-1}) | mvV_{x-2}
// (the cars entering row x-1 from above are mvV_{x-2}, computed one row
// earlier).  Written this way E' is never formed: mvV and the emitted T are
// one three-input logic operation each.  Every LR car that moves enters
// exactly one cell, so the row's LR count is the popcount of in.  Horizontal
// neighbours come from two 32-bit warp shuffles, both issued at the start of
// the stage: the right neighbour's low half of E (bit 0 = the cell right of
// this word) and the left neighbour's half of L holding its last cell,
// pre-aligned to bit 31.
#pragma once

#include "device_common.cuh"

namespace bml {

// Per-lane constants of the word a lane holds.
struct LaneWord {
  u64 valid;                // valid-cell mask (all ones for a full word, 0 if the lane is off)
  uint32_t ins_lo, ins_hi;  // bit that receives the right neighbour's first cell
  uint32_t mul_lo, mul_hi;  // lo * mul_lo + hi * mul_hi has the word's last cell at bit 31
  int top_hi;               // the word's last cell lies in the high half
  int top_sh;               // left shift that moves the last cell to bit 31 of its half
  int src_l, src_r;         // lanes holding the left / right neighbour words
};

__device__ __forceinline__ void lane_word_bits(LaneWord &lw, bool on, bool last, int nb,
                                               u64 tail) {
  const int top = last ? nb - 1 : 63;
  lw.valid = on ? (last ? tail : ~0ull) : 0ull;
  lw.ins_lo = top < 32 ? (1u << top) : 0u;
  lw.ins_hi = top >= 32 ? (1u << (top - 32)) : 0u;
  lw.mul_lo = top < 32 ? (1u << (31 - top)) : 0u;
  lw.mul_hi = top >= 32 ? (1u << (63 - top)) : 0u;
  lw.top_hi = top >= 32;
  lw.top_sh = 31 - (top & 31);
}

// Stage state: T_{x-1}, Lh_{x-1}, mvV_{x-2}, every value as two 32-bit
// halves (index 0: bits 0-31, 1: bits 32-63; halves need no 64-bit register
// pairs, which saves the compiler copies).  Consumes row x (L, T) of its
// input state, replaces them with row x-1 of the next state, and returns the
// row's moved-car counts.  The state is read from one set and written to
// another (callers alternate two sets from row to row, so no value is
// copied).  FULL: every word of the row holds 64 cells.
//
// The horizontal rule in the "who enters" form: Ll = L shifted one column
// right (the left neighbour's last cell enters bit 0), in = Ll & E (the cells
// an LR car enters), Lh = (L & ~Er) | in (cars that stay, plus cars that
// enter).  Every moving car enters exactly one cell, so the row's LR move
// count is the popcount of `in` (returned as mvIn).  The left shuffle needs
// only L, so both shuffles issue at the start of the stage.  Each rule line is
// one lop3 per half.
//
// Words with fewer cells (the last word of a row whose N is not a multiple of
// 64): E is masked to the valid cells, so `in` never sets a cell past the
// row's end; the right neighbour's E enters at this word's last cell as a
// multiply-add on the FMA pipe (the shifted E is zero from that bit on, so
// the add carries nothing; the neighbour's higher bits land past the end,
// where L is zero and Er is not read); the last cell sent to the left
// neighbour is placed at bit 31 by two multiply-adds.
//
// M3 (Model III, one synchronous phase, a cell may hold one vehicle of each
// kind): a TB vehicle moves iff the cell below held no vehicle at the start
// of the step, so mvV reads the row's input L instead of Lh; the rest is
// unchanged (an empty cell may then receive an LR and a TB vehicle).
struct StageH {
  uint32_t T[2], Lh[2], M[2];
};

template <bool FULL, bool M3 = false>
__device__ __forceinline__ void stage_step_h(uint32_t (&L)[2], uint32_t (&T)[2], const StageH &st,
                                             StageH &nx, const LaneWord &lw, uint32_t &mvIn,
                                             uint32_t &mvV) {
  const uint32_t E0 =
      FULL ? lop3<kNor>(L[0], T[0], 0u) : lop3<kNorAnd>(L[0], T[0], lo32(lw.valid));
  const uint32_t E1 =
      FULL ? lop3<kNor>(L[1], T[1], 0u) : lop3<kNorAnd>(L[1], T[1], hi32(lw.valid));
  const uint32_t send_l = FULL ? L[1] : L[1] * lw.mul_hi + L[0] * lw.mul_lo;
  const uint32_t rl = __shfl_sync(BML_FULL_MASK, send_l, lw.src_l);
  const uint32_t rr = __shfl_sync(BML_FULL_MASK, E0, lw.src_r);
  uint32_t Er0, Er1;
  if (FULL) {
    Er0 = __funnelshift_r(E0, E1, 1);
    Er1 = __funnelshift_r(E1, rr, 1);
  } else {
    Er0 = __funnelshift_r(E0, E1, 1) + rr * lw.ins_lo;
    Er1 = (E1 >> 1) + rr * lw.ins_hi;
  }
  const uint32_t in0 = lop3<kAnd>(__funnelshift_l(rl, L[0], 1), E0, 0u);
  const uint32_t in1 = lop3<kAnd>(__funnelshift_l(L[0], L[1], 1), E1, 0u);
  const uint32_t Lh0 = lop3<kAndNotOr>(L[0], Er0, in0), Lh1 = lop3<kAndNotOr>(L[1], Er1, in1);
  const uint32_t mv0 = lop3<kAndNor>(st.T[0], M3 ? L[0] : Lh0, T[0]);
  const uint32_t mv1 = lop3<kAndNor>(st.T[1], M3 ? L[1] : Lh1, T[1]);
  mvIn = __popc(in0) + __popc(in1);
  mvV = __popc(mv0) + __popc(mv1);
  nx.T[0] = T[0];
  nx.T[1] = T[1];
  nx.Lh[0] = Lh0;
  nx.Lh[1] = Lh1;
  nx.M[0] = mv0;
  nx.M[1] = mv1;
  T[0] = lop3<kAndNotOr>(st.T[0], mv0, st.M[0]);
  T[1] = lop3<kAndNotOr>(st.T[1], mv1, st.M[1]);
  L[0] = st.Lh[0];
  L[1] = st.Lh[1];
}

// Input-row ring of a warp in shared memory, [slot][plane][lane], 16 bytes
// per lane and plane.  A lane copies (cp.async, through L2) the aligned
// 16-byte pair of words that holds its own word (rows start 16-byte aligned:
// the pitch is even) and reads back only its own half (half = word & 1); the
// two lanes of a pair request the same bytes, so a warp's requests cover the
// same sectors as one word per lane.
using RingSlot = ulonglong2[2][32];

__device__ __forceinline__ void ring_fill(RingSlot *ring, int slot, int lane, const u64 *Lpair,
                                          const u64 *Tpair) {
  cp_async16(&ring[slot][0][lane], Lpair);
  cp_async16(&ring[slot][1][lane], Tpair);
}

__device__ __forceinline__ void ring_read(const RingSlot *ring, int slot, int lane, int half,
                                          u64 &L, u64 &T) {
  const u64 *q = reinterpret_cast<const u64 *>(&ring[slot][0][lane]) + half;
  L = q[0];
  T = q[64];  // the same lane's entry of plane 1
}

__device__ __forceinline__ uint32_t popc64(u64 x) {
  return (uint32_t)(__popc(lo32(x)) + __popc(hi32(x)));
}

}  // namespace bml
