// Byte-per-cell step: the plain GPU form (Sec. 6 of the paper turns the
// serial phase functions into kernels).  One horizontal and one vertical
// launch per step, each reading and writing one byte per cell.
//
// A thread handles a 16-byte chunk (16 cells) with one 128-bit load and
// computes the rules branch-free on byte lanes, the selection-by-mask idea
// of Sec. 5 (pick one of two values per lane through a condition mask and its
// complement instead of a branch): with per-byte bit masks of
// LR, TB and EMPTY (1 in bit 0 of a byte), a moving LR car and the cell it
// enters both flip bit 0, a moving TB car and its destination flip bit 1.
//   horizontal: out = x ^ ((L & Er) | (Ll & E))          (Sec. 2 rule 1)
//   vertical:   out = x ^ (((T & Eb) | (Tt & E)) << 1)   (Sec. 2 rule 2)
// where Er / Ll are the right / left neighbours' masks (with wrap) and
// Eb / Tt the lower / upper row's.
#include "device_common.cuh"

namespace bml {

namespace {

constexpr u64 kLsb = 0x0101010101010101ull;

struct Chunk {
  u64 lo, hi;
};

__device__ __forceinline__ Chunk load_chunk(const uint8_t *p) {
  const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
  return Chunk{v.x, v.y};
}
__device__ __forceinline__ void store_chunk(uint8_t *p, Chunk c) {
  ulonglong2 v;
  v.x = c.lo;
  v.y = c.hi;
  __stcs(reinterpret_cast<ulonglong2 *>(p), v);
}

// per-byte masks (bit 0 of each byte) of the first n cells of a chunk
__device__ __forceinline__ Chunk valid_bytes(int n) {
  Chunk m;
  m.lo = n >= 8 ? kLsb : (kLsb & ((1ull << (8 * n)) - 1ull));
  m.hi = n >= 16 ? kLsb : (n <= 8 ? 0ull : (kLsb & ((1ull << (8 * (n - 8))) - 1ull)));
  return m;
}

__device__ __forceinline__ Chunk lr_mask(Chunk x) { return Chunk{x.lo & kLsb, x.hi & kLsb}; }
__device__ __forceinline__ Chunk tb_mask(Chunk x) {
  return Chunk{(x.lo >> 1) & kLsb, (x.hi >> 1) & kLsb};
}
__device__ __forceinline__ Chunk empty_mask(Chunk x, Chunk valid) {
  return Chunk{~(x.lo | (x.lo >> 1)) & valid.lo, ~(x.hi | (x.hi >> 1)) & valid.hi};
}

// number of set bits of a chunk whose bits are all at bit 0 of bytes (the
// high word's bits move to bit 1 of its bytes, so one 64-bit count suffices)
__device__ __forceinline__ uint32_t popc_chunk(Chunk c) {
  return (uint32_t)__popcll(c.lo | (c.hi << 1));
}

// A warp takes 32 consecutive chunks of one row (a row segment), one per lane;
// the cells just past a chunk's ends come from the neighbouring lanes'
// chunks by shuffle, and from memory only at the segment's and the row's ends.
__global__ void byte_h_kernel(const uint8_t *__restrict__ cur, uint8_t *__restrict__ nxt, Geom g,
                              u64 *moved) {
  const int nq = (int)(g.PB / 16), segs = (nq + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t di = nwarps / segs;
  const int dseg = (int)(nwarps - di * segs);
  // (row, segment) of this warp's first item, advanced by nwarps items a turn
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
    const bool on = q < nq;
    const uint8_t *row = cur + i * g.PB;
    const int64_t c0 = 16 * (int64_t)q;
    const int nv = on ? (int)(g.N - c0 < 16 ? g.N - c0 : 16) : 16;
    // cell c0 + 16 is byte 0 of the next lane's chunk unless this chunk ends
    // the row (wrap to column 0) or the segment; cell c0 - 1 is byte 15 of the
    // previous lane's chunk (every chunk but a row's last is full).  The few
    // cells read from memory are loaded together with the chunk.
    const bool row_end = c0 + nv >= g.N;
    const bool mem_r = on && (lane == 31 || row_end), mem_l = on && lane == 0;
    Chunk x{0, 0};
    uint8_t right = 0, left = 0;
    if (on) x = load_chunk(row + c0);
    if (mem_r) right = __ldg(row + (row_end ? 0 : c0 + nv));
    if (mem_l) left = __ldg(row + (c0 > 0 ? c0 - 1 : g.N - 1));
    const uint32_t nxt_b0 = __shfl_down_sync(BML_FULL_MASK, (uint32_t)x.lo, 1);
    const uint32_t prv_b15 = __shfl_up_sync(BML_FULL_MASK, (uint32_t)(x.hi >> 32), 1);
    if (on) {
      if (!mem_r) right = (uint8_t)(nxt_b0 & 0xffu);
      if (!mem_l) left = (uint8_t)(prv_b15 >> 24);
      const Chunk L = lr_mask(x);
      const u64 rE = right == 0 ? 1ull : 0ull;
      const u64 lL = left == 1 ? 1ull : 0ull;
      Chunk E, Er, Ll;
      if (nv == 16) {  // every chunk but a row's last
        E = empty_mask(x, Chunk{kLsb, kLsb});
        Er.lo = (E.lo >> 8) | (E.hi << 56);
        Er.hi = (E.hi >> 8) | (rE << 56);
      } else {
        E = empty_mask(x, valid_bytes(nv));
        Er.lo = (E.lo >> 8) | (E.hi << 56);
        Er.hi = E.hi >> 8;
        if (nv > 8)
          Er.hi |= rE << (8 * (nv - 9));
        else
          Er.lo |= rE << (8 * (nv - 1));
      }
      Ll.lo = (L.lo << 8) | lL;
      Ll.hi = (L.hi << 8) | (L.lo >> 56);
      const Chunk mv{L.lo & Er.lo, L.hi & Er.hi};
      Chunk out;
      out.lo = x.lo ^ (mv.lo | (Ll.lo & E.lo));
      out.hi = x.hi ^ (mv.hi | (Ll.hi & E.hi));
      store_chunk(nxt + i * g.PB + c0, out);
      cnt += popc_chunk(mv);
    }
  }
  pdl_release();  // this block's lattice work is done
  block_count_add(cnt, moved);
}

// One thread per (band of rows, chunk column); marches down the band keeping
// the upper row's TB mask and the current row's EMPTY mask.  The library's
// own byte lattices keep their padding bytes (columns N..PB-1) at 0, so no
// move involves them and the rule needs no column mask.  PAD_ANY (the
// allocation-free entry point, which steps caller-owned rows whose padding
// may hold anything): the EMPTY mask of a row's last chunk is limited to the
// columns < N, so no TB move involves a padding byte, and padding bytes are
// copied unchanged and never counted.
template <bool PAD_ANY>
__global__ void __launch_bounds__(256, 8)
    byte_v_kernel(const uint8_t *__restrict__ cur, uint8_t *__restrict__ nxt, Geom g,
                  int64_t band, u64 *moved) {
  const int64_t nq = g.PB / 16, nbands = (g.M + band - 1) / band, total = nbands * nq;
  uint32_t cnt = 0;
  pdl_wait();
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = idx / nq, q = idx - b * nq;
    const int64_t r0 = b * band;
    const int len = (int)(r0 + band < g.M ? band : g.M - r0);
    const bool wraps = r0 + len == g.M;  // the band's last row reads row 0 below it
    const uint8_t *col = cur + 16 * q;
    const uint8_t *src = col + r0 * g.PB;
    uint8_t *dst = nxt + r0 * g.PB + 16 * q;
    Chunk vm{kLsb, kLsb};
    if (PAD_ANY && g.N - 16 * q < 16) vm = valid_bytes((int)(g.N - 16 * q));
    const Chunk up = load_chunk(r0 > 0 ? src - g.PB : col + (g.M - 1) * g.PB);
    Chunk Tt = tb_mask(up);
    Chunk x = load_chunk(src);
    Chunk E = empty_mask(x, vm);
#pragma unroll 1
    for (int k = 0; k < len; ++k) {
      src += g.PB;
      const Chunk xn = load_chunk(k + 1 == len && wraps ? col : src);
      const Chunk En = empty_mask(xn, vm);
      const Chunk T = tb_mask(x);
      const Chunk mv{T.lo & En.lo, T.hi & En.hi};
      Chunk out;
      out.lo = x.lo ^ ((mv.lo | (Tt.lo & E.lo)) << 1);
      out.hi = x.hi ^ ((mv.hi | (Tt.hi & E.hi)) << 1);
      store_chunk(dst, out);
      dst += g.PB;
      cnt += popc_chunk(mv);
      Tt = T;
      x = xn;
      E = En;
    }
  }
  pdl_release();  // this block's lattice work is done
  block_count_add(cnt, moved);
}

int grid_cap(int64_t items, int threads) {
  int64_t blocks = (items + threads - 1) / threads;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = (int64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

}  // namespace

cudaError_t launch_byte_h(const uint8_t *cur, uint8_t *nxt, const Geom &g, u64 *moved,
                          cudaStream_t st) {
  const int64_t items = g.M * ((g.PB / 16 + 31) / 32) * 32;
  return launch_pdl(byte_h_kernel, dim3(grid_cap(items, 256)), dim3(256), 0, st, cur, nxt, g,
                    moved);
}

cudaError_t launch_byte_v(const uint8_t *cur, uint8_t *nxt, const Geom &g, u64 *moved,
                          cudaStream_t st, bool pad_any) {
  // Band height: as short as one wave of the launched threads allows (every
  // thread marches down one band; the rows re-read above and below a band
  // are 2/band of the traffic), at least 32 rows, at most 4096.
  const int64_t nq = g.PB / 16;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 148;
  }
  const int64_t threads = (int64_t)sms * 8 * 256;
  int64_t band = (g.M * nq + threads - 1) / threads;
  band = band < 32 ? 32 : (band > 4096 ? 4096 : band);
  const int64_t items = ((g.M + band - 1) / band) * nq;
  if (pad_any)
    return launch_pdl(byte_v_kernel<true>, dim3(grid_cap(items, 256)), dim3(256), 0, st, cur,
                      nxt, g, band, moved);
  return launch_pdl(byte_v_kernel<false>, dim3(grid_cap(items, 256)), dim3(256), 0, st, cur,
                    nxt, g, band, moved);
}

}  // namespace bml
