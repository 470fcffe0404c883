// Device helpers shared by the kernels of libbml.
#pragma once

#include <stdint.h>

#include "bml_internal.cuh"

namespace bml {

#define BML_FULL_MASK 0xffffffffu

// Valid-cell mask of word w of a row: all ones for full words, the tail mask
// for word W-1, zero for padding words.
__device__ __forceinline__ u64 word_valid(int64_t w, const Geom &g) {
  return w < g.W - 1 ? ~0ull : (w == g.W - 1 ? g.tail : 0ull);
}

// Bit position of the last cell of word w (the one whose right neighbour is
// in the next word, or wraps to column 0).
__device__ __forceinline__ int word_top(int64_t w, const Geom &g) {
  return w == g.W - 1 ? g.nb - 1 : 63;
}

__device__ __forceinline__ uint32_t lo32(u64 x) { return (uint32_t)x; }
__device__ __forceinline__ uint32_t hi32(u64 x) { return (uint32_t)(x >> 32); }
__device__ __forceinline__ u64 mk64(uint32_t lo, uint32_t hi) {
  return (u64)lo | ((u64)hi << 32);
}

// One three-input logic instruction (PTX lop3.b32): bit i of the result is
// bit (a_i b_i c_i) of the truth table LUT, whose operand patterns are
// a = 0xF0, b = 0xCC, c = 0xAA.  The stage rules are written with it, one
// instruction per rule line and 32-bit half: left to the compiler, algebraic
// rewriting (L ^ (L & ~X) into L & X, for one) makes operands shared between
// lines, and a line that then needs four inputs costs two instructions (26
// instead of 18 logic instructions per pair-stage of the pair kernel).
template <unsigned LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
}
template <unsigned LUT>
__device__ __forceinline__ u64 lop3(u64 a, u64 b, u64 c) {
  return mk64(lop3<LUT>(lo32(a), lo32(b), lo32(c)), lop3<LUT>(hi32(a), hi32(b), hi32(c)));
}
constexpr unsigned kNor = 0x03;       // ~(a | b)          (c unused)
constexpr unsigned kNorAnd = 0x02;    // ~(a | b) & c
constexpr unsigned kAnd = 0xC0;       // a & b             (c unused)
constexpr unsigned kAndNor = 0x10;    // a & ~(b | c)
constexpr unsigned kXor3 = 0x96;      // a ^ b ^ c
constexpr unsigned kAndNotOr = 0xBA;  // (a & ~b) | c
constexpr unsigned kAndOrNot = 0xB0;  // a & (~b | c)
constexpr unsigned kAndNand = 0x70;   // a & ~(b & c)

// Programmatic dependent launch: a kernel launched with launch_pdl may start
// (and run its set-up) while the previous kernel on the stream finishes;
// pdl_wait() returns once that kernel has completed and its memory writes are
// visible, so it comes before the first global access (the ping-pong buffers
// the previous kernel read are written after it).  pdl_release(), once a
// block's lattice work is done, lets the next kernel launch when every block
// has released or exited (releasing at the start let the next kernel's
// waiting blocks take the free slots of a partial wave and unbalance it).
// Both are no-ops for a normal launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// n-th output (n >= 1) of SplitMix64 (Steele, Lea, Flood 2014) started from
// state `seed`: the placement's and the Model II tie-break's generator.
__device__ __forceinline__ u64 splitmix64_at(u64 seed, u64 n) {
  u64 z = seed + n * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Asynchronous 16-byte copy global -> shared (bypassing L1), its commit and
// its wait (all but the N most recent committed groups complete; the copied
// bytes are then visible to the issuing thread).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
// 8-byte form (through L1: the .cg form takes only 16 bytes).
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 128-bit read-only load / streaming store of two consecutive words.
__device__ __forceinline__ void ld2(const u64 *p, u64 &a, u64 &b) {
  const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void st2(u64 *p, u64 a, u64 b) {
  ulonglong2 v;
  v.x = a;
  v.y = b;
  __stcs(reinterpret_cast<ulonglong2 *>(p), v);
}

// Cross-word right shift by one cell: bit b of the result is bit b+1 of lo,
// bit 63 is bit 0 of hi.  Written as two 32-bit funnel shifts.
__device__ __forceinline__ u64 funnel_r1(u64 lo, u64 hi) {
  const uint32_t l0 = (uint32_t)lo, l1 = (uint32_t)(lo >> 32), h0 = (uint32_t)hi;
  const uint32_t r0 = __funnelshift_r(l0, l1, 1);
  const uint32_t r1 = __funnelshift_r(l1, h0, 1);
  return (u64)r0 | ((u64)r1 << 32);
}
// Cross-word left shift by one cell: bit 0 of the result is bit 63 of lo.
__device__ __forceinline__ u64 funnel_l1(u64 lo, u64 hi) {
  const uint32_t l1 = (uint32_t)(lo >> 32), h0 = (uint32_t)hi, h1 = (uint32_t)(hi >> 32);
  const uint32_t r0 = __funnelshift_l(l1, h0, 1);
  const uint32_t r1 = __funnelshift_l(h0, h1, 1);
  return (u64)r0 | ((u64)r1 << 32);
}

// Add a per-thread count to a global 64-bit counter: warp reduction, then
// one shared-memory add per warp, then one global atomic per block.  Every
// thread of the block must call it (it contains __syncthreads).
__device__ __forceinline__ void block_count_add(uint32_t v, u64 *dst) {
  __shared__ unsigned long long s_sum;
  if (threadIdx.x == 0) s_sum = 0;
  __syncthreads();
  const uint32_t w = __reduce_add_sync(BML_FULL_MASK, v);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(&s_sum, (unsigned long long)w);
  __syncthreads();
  if (threadIdx.x == 0 && s_sum) atomicAdd(dst, s_sum);
}

}  // namespace bml
