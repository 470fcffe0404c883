// Internal declarations shared by the CUDA translation units of libbml.
//
// Bit-packed layout: two bitplanes per lattice, L (LR occupancy) and T (TB
// occupancy).  Row i is P 64-bit words; column j is bit (j % 64) of word
// (j / 64) (LSB first).  W = ceil(N / 64) words carry cells; the last one
// holds nb = N - 64 (W - 1) cells and its bits >= nb are always 0; words
// W .. P-1 (P = W rounded up to even, for 16-byte vector access) are always
// 0.  EMPTY is implicit: not L and not T.
//
// Byte layout (the plain form): one byte per cell, row pitch PB = N rounded
// up to 16; padding bytes are always 0.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bml {

typedef unsigned long long u64;

struct Geom {
  int64_t M;   // rows
  int64_t N;   // columns
  int64_t W;   // words per row holding cells
  int64_t P;   // plane pitch in words (even)
  int64_t PB;  // byte-layout pitch in bytes (multiple of 16)
  int32_t nb;  // cells in word W-1 (1..64)
  u64 tail;    // mask of the valid bits of word W-1
};

Geom make_geom(int64_t M, int64_t N);

// Record the message returned by bml_last_error() on this thread.
void set_last_error(const char *msg);

// Seeded placement thresholds: floor(p * 2^64) clamped to 2^64 - 1.
u64 placement_threshold(double p);

// How the streaming kernel cuts a row into warp-wide column strips.  When the
// row fits in one warp (W <= 32) the strip is the whole periodic row and
// needs no halo; otherwise each strip carries `halo` redundant words on each
// side (1, or 2 when the last word is too short to hold a k-step cone).
struct StripPlan {
  int32_t whole;
  int32_t n_strips;
  int32_t halo;
  int32_t base;  // owned words per strip: base + (strip < rem)
  int32_t rem;
};

StripPlan make_strip_plan(const Geom &g, int k);

// ---- launchers (all asynchronous on `st`; return cudaGetLastError()) ----
cudaError_t launch_init_planes(u64 *L, u64 *T, const Geom &g, u64 seed, u64 t_lr,
                               u64 t_tb, cudaStream_t st);
cudaError_t launch_init_bytes(uint8_t *c, const Geom &g, u64 seed, u64 t_lr, u64 t_tb,
                              cudaStream_t st);
// bytes (pitch PB) -> planes; sets *bad (device int) if a byte is above
// max_value (2; 3 where a cell may hold one vehicle of each kind).
cudaError_t launch_pack(const uint8_t *c, u64 *L, u64 *T, const Geom &g, int *bad,
                        cudaStream_t st, int max_value = 2);
// Sets *flag (device int) if some cell holds both an LR and a TB vehicle.
cudaError_t launch_find_overlap(const u64 *L, const u64 *T, const Geom &g, int *flag,
                                cudaStream_t st);
// planes -> bytes (pitch PB).
cudaError_t launch_unpack(const u64 *L, const u64 *T, uint8_t *c, const Geom &g,
                          cudaStream_t st);
// bytes (pitch PB) -> validity check only.
cudaError_t launch_check_bytes(const uint8_t *c, const Geom &g, int *bad, cudaStream_t st);
// n moved counts (device) -> host arrays given by their device-mapped
// addresses (either may be NULL)
cudaError_t launch_copy_counts(const u64 *lr, const u64 *tb, int64_t n, int64_t *dlr,
                               int64_t *dtb, cudaStream_t st);

// Byte-per-cell phases: cur -> nxt, moved cars added to *moved.
cudaError_t launch_byte_h(const uint8_t *cur, uint8_t *nxt, const Geom &g, u64 *moved,
                          cudaStream_t st);
// pad_any: the padding bytes of a row may hold any value (caller-owned
// rows); they are then excluded from the rule and left unchanged.
cudaError_t launch_byte_v(const uint8_t *cur, uint8_t *nxt, const Geom &g, u64 *moved,
                          cudaStream_t st, bool pad_any = false);

// Bitplane phases.  H: (L, T) -> Lh; V: (Lh, T) -> Tv.  Moved cars added to
// *moved.
cudaError_t launch_plane_h(const u64 *L, const u64 *T, u64 *Lh, const Geom &g, u64 *moved,
                           cudaStream_t st);
cudaError_t launch_plane_v(const u64 *Lh, const u64 *T, u64 *Tv, const Geom &g, u64 *moved,
                           cudaStream_t st);

// Fused one-pass step (both phases, one launch, no bands): (L, T) -> (Lo, To).
cudaError_t launch_fused_direct(const u64 *L, const u64 *T, u64 *Lo, u64 *To, const Geom &g,
                                u64 *moved_lr, u64 *moved_tb, cudaStream_t st);

// Resident blocks per SM and warps per block of the streaming kernel at depth k.
int stream_occupancy(const Geom &g, int k, int *warps_per_block);

// Streaming kernel: k full steps (k in 1, 2, 4, 8) from (Lin, Tin) to
// (Lout, Tout); the counts of sub-step s are added to moved_lr[s],
// moved_tb[s].  band_rows: rows per warp tile.  model3: Model III steps
// (one synchronous phase; a cell may hold one vehicle of each kind).
cudaError_t launch_stream(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                          int k, int64_t band_rows, u64 *moved_lr, u64 *moved_tb,
                          cudaStream_t st, bool model3 = false);

// Model II streaming kernel (one synchronous phase, random tie-break of
// contested cells; k in 1, 2, 4, 8): t0 = index of the launch's first step.
int model2_occupancy(const Geom &g, int k);
cudaError_t launch_model2(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                          int k, int64_t band_rows, u64 tie_seed, u64 t0, u64 *moved_lr,
                          u64 *moved_tb, cudaStream_t st);

// Resident kernel: the whole lattice in shared memory, k <=
// resident_max_steps() steps per launch; band_rows >= M: one block holds it,
// else the rows are split into bands of band_rows over the blocks of one
// thread-block cluster (resident_blocks of them, at most 8).
bool resident_applies(const Geom &g);
int resident_max_steps();
int resident_blocks(const Geom &g, int64_t band_rows);
cudaError_t launch_resident(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                            int k, int64_t band_rows, u64 *moved_lr, u64 *moved_tb,
                            cudaStream_t st);

// Two-words-per-lane streaming kernel (rows of full words, W even, W > 32);
// model 1 (the paper's model), 2 (Model II, with tie_seed and the index t0
// of the launch's first step) or 3 (Model III).  Models 1 and 3 run on the
// interleaved layout of the planes (see launch_pair_layout), Model II on the
// plain one.  stream2_bands_for_tiles: the largest band count whose warp
// tiles number at most `tiles` at depth k.
bool stream2_applies(const Geom &g);
int64_t stream2_bands_for_tiles(const Geom &g, int k, int64_t tiles);
int stream2_occupancy(int k, int model = 1);
cudaError_t launch_stream2(const u64 *Lin, const u64 *Tin, u64 *Lout, u64 *Tout, const Geom &g,
                           int k, int64_t band_rows, u64 *moved_lr, u64 *moved_tb,
                           cudaStream_t st, int model = 1, u64 tie_seed = 0, u64 t0 = 0);

// Interleaved layout (rows of full words, W even): word w of a row holds
// its 64 columns' even ones in its low half (bit i = column 64w + 2i) and
// the odd ones in its high half (bit 32 + i = column 64w + 2i + 1).
// Converts both planes in place between the plain layout and this one
// (to_pair: plain -> interleaved).
cudaError_t launch_pair_layout(u64 *L, u64 *T, const Geom &g, bool to_pair, cudaStream_t st);

// Launch `kern` with programmatic stream serialization: it may be scheduled
// while the previous kernel on the stream finishes; the kernel calls
// pdl_wait() before its first global memory access.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace bml
