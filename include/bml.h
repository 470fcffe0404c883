/*
 * bml.h -- C ABI of the B300 (sm_103a) Biham-Middleton-Levine traffic CA.
 *
 * The automaton (Marzolla 2018, "Parallel Implementations of Cellular
 * Automata for Traffic Models", Sec. 2): a periodic lattice of M rows and
 * N columns; each cell is EMPTY (0), LR (1, moves one column right) or
 * TB (2, moves one row down).  One step is a horizontal phase (every LR car
 * whose right neighbour is EMPTY moves into it) followed by a vertical phase
 * (every TB car whose lower neighbour is EMPTY moves into it), both applied
 * synchronously with wrap-around.  The paper states the model for square
 * N x N lattices; this library takes any M x N.
 *
 * Lattice format at the boundary (Sec. 3): one byte per cell, values 0/1/2,
 * row-major, cell (i, j) at byte i*N + j, no padding (Model III, below,
 * adds the value 3 for a cell holding one vehicle of each kind).
 *
 * Moved counts (not defined in the paper): for step t (1-based), moved_lr[t-1]
 * is the number of LR cars that moved in its horizontal phase and
 * moved_tb[t-1] the number of TB cars that moved in its vertical phase;
 * total = lr + tb.  Counts are exact int64.
 *
 * Seeded placement (Sec. 2 says only that cars are placed at random): cell
 * (i, j) takes u = SplitMix64 output number i*N + j + 1 from state `seed`
 * (Steele, Lea, Flood 2014); with t_x = floor(p_x * 2^64) (clamped to
 * 2^64 - 1) the cell is LR if u < t_lr, else TB if u - t_lr < t_tb, else
 * EMPTY.  bml_create's `density` means p_lr = p_tb = density / 2.
 *
 * Conventions for every call:
 *   - the return value is a status code (BML_OK or a negative BML_E*);
 *     on failure the object is left unchanged and bml_last_error() returns a
 *     message (thread-local, valid until the next call on that thread);
 *   - host buffers are owned by the caller and only read/written during the
 *     call; device memory is owned by the library (or by the allocator that
 *     bml_set_allocator installed);
 *   - work is enqueued on the simulation's CUDA stream (the caller's stream
 *     given at creation, or the legacy default stream); calls that return
 *     host data synchronise that stream first;
 *   - a bml_sim is not thread-safe: one thread at a time per object.
 */
#ifndef BML_H
#define BML_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define BML_OK 0
#define BML_EINVAL (-1)   /* invalid argument                                  */
#define BML_ENOMEM (-2)   /* device or host allocation failed                  */
#define BML_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed       */
#define BML_ETIMEOUT (-4) /* a bounded device-side wait gave up               */
#define BML_ESTATE (-5)   /* call not valid in the object's state (e.g. count
                             capacity exhausted)                              */

/* Step kernels. */
#define BML_KERNEL_AUTO 0     /* autotuned: streaming bitplane kernel with the
                                 fastest (temporal depth k, band height)      */
#define BML_KERNEL_BYTE 1     /* one byte per cell; one horizontal and one
                                 vertical launch per step (the plain GPU form
                                 of Sec. 6)                                   */
#define BML_KERNEL_BITPLANE 2 /* two uint64 bitplanes; one horizontal and one
                                 vertical launch per step                     */
#define BML_KERNEL_FUSED 3    /* two bitplanes; one launch per step (both
                                 phases in one pass, no bands)                */
#define BML_KERNEL_TBLOCK 4   /* two bitplanes; k full steps per launch       */
#define BML_KERNEL_RESIDENT 5 /* two bitplanes kept in one thread block's
                                 shared memory; every step of a bml_step
                                 call (up to 4096 per launch) in one launch.
                                 Small lattices only: 4*M*P*8 bytes plus
                                 32 KiB must fit the block's shared memory
                                 (P = ceil(N/64) rounded up to even; about
                                 M*P <= 5000 words on B300), else BML_EINVAL */

typedef struct bml_sim bml_sim;

/* Optional device allocator (e.g. a framework's caching allocator).
 * alloc returns a device pointer of at least `bytes` bytes usable on
 * `stream`, or NULL; free releases it.  Pointers must be 256-byte aligned. */
typedef void *(*bml_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*bml_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);

/* Install (or, with NULLs, remove) the process-wide device allocator used by
 * objects created afterwards.  Objects remember the allocator they were
 * created with.  Returns BML_EINVAL if exactly one of alloc/free is NULL. */
int bml_set_allocator(bml_alloc_fn alloc, bml_free_fn free_fn, void *ctx);

/* Create an M x N lattice with the seeded placement above at `density`
 * (p_lr = p_tb = density/2), kernel BML_KERNEL_AUTO, legacy default stream.
 * M, N >= 1, M*N <= 2^37; 0 <= density <= 1.  *out receives the object. */
int bml_create(int64_t M, int64_t N, uint64_t seed, double density, bml_sim **out);

/* Full form.  p_lr, p_tb >= 0, p_lr + p_tb <= 1.  kernel is a BML_KERNEL_*.
 * block_k is the temporal depth for BML_KERNEL_TBLOCK (1, 2, 4 or 8; 0 picks
 * 4) and is ignored otherwise.  stream is a cudaStream_t (NULL = legacy
 * default stream).  reserve_steps preallocates the moved-count history (0
 * picks 4096; it grows on demand in bml_step).  With BML_KERNEL_AUTO the call
 * times the candidate configurations on this lattice (the lattice itself is
 * not advanced) and keeps the fastest; results are cached per (M, N, device)
 * for the process. */
int bml_create_ex(int64_t M, int64_t N, uint64_t seed, double p_lr, double p_tb,
                  int kernel, int block_k, void *stream, int64_t reserve_steps,
                  bml_sim **out);

/* Ensure room for the moved counts of at least K steps in total. */
int bml_reserve_steps(bml_sim *sim, int64_t K);

/* Enqueue k >= 0 full steps (horizontal then vertical phase each) on the
 * object's stream; asynchronous.  Grows the count history if needed. */
int bml_step(bml_sim *sim, int64_t k);

/* Copy the moved counts of steps first+1 .. first+n (0-based entries
 * first .. first+n-1) to host arrays of n int64 each.  Any of the three
 * outputs may be NULL.  Requires 0 <= first, first + n <= bml_steps_done().
 * Synchronises the stream. */
int bml_moved_counts(bml_sim *sim, int64_t first, int64_t n, int64_t *out_total,
                     int64_t *out_lr, int64_t *out_tb);

/* Enqueue copies of the LR and TB moved counts of steps first+1 ..
 * first+n into host arrays of n int64 each (either may be NULL; the total
 * is their sum) on the object's stream and return without waiting: a
 * caller can read every step's result while the steps run.  The values are
 * valid once the stream has been synchronised (bml_synchronize, or any call
 * documented to synchronise).  Page-locked arrays that the current device
 * can address (cudaHostAlloc / pinned tensors under unified addressing) are
 * written by a small kernel ordered after the steps, so no copy-engine round
 * trip sits between two step launches; other page-locked arrays take
 * cudaMemcpyAsync; pageable arrays make the copy wait for the stream.  Same
 * range rule as bml_moved_counts. */
int bml_moved_counts_async(bml_sim *sim, int64_t first, int64_t n, int64_t *out_lr,
                           int64_t *out_tb);

/* Copy the current lattice (M*N bytes, format above) to host memory `out`.
 * Synchronises the stream. */
int bml_read_lattice(bml_sim *sim, uint8_t *out);

/* Replace the lattice with M*N bytes from host memory `in` (values 0, 1, 2;
 * any other value gives BML_EINVAL and leaves the object unchanged).  This
 * starts a new trajectory: bml_steps_done() becomes 0 and the count history
 * is cleared.  Synchronises the stream. */
int bml_write_lattice(bml_sim *sim, const uint8_t *in);

/* Device-memory forms of the two calls above: `d_out` / `d_in` are device
 * pointers to M*N bytes (for example a framework tensor); enqueued on the
 * object's stream without synchronising.  bml_write_lattice_device checks
 * the values on the device and synchronises to report BML_EINVAL. */
int bml_read_lattice_device(bml_sim *sim, uint8_t *d_out);
int bml_write_lattice_device(bml_sim *sim, const uint8_t *d_in);

/* Number of steps taken since creation (or the last bml_write_lattice). */
int64_t bml_steps_done(const bml_sim *sim);

/* Kernel actually used (BML_KERNEL_*; AUTO reports the one it picked), its
 * temporal depth and band height (rows per warp tile; 0 for kernels without
 * bands: BYTE, BITPLANE and the one-pass FUSED kernel). */
int bml_get_config(const bml_sim *sim, int *kernel, int *block_k, int64_t *band_rows);

/* Override the tiling of the bitplane step of a BML_KERNEL_AUTO or TBLOCK
 * object: temporal depth block_k in {1, 2, 4, 8} and band height band_rows
 * >= 1 (rows per warp tile of the streaming kernel), or band_rows = 0 with
 * block_k = 1 for the one-pass fused kernel.  BML_EINVAL for other kernels
 * or values. */
int bml_set_tiling(bml_sim *sim, int block_k, int64_t band_rows);

/* As bml_set_tiling, choosing also the 64-cell words each lane of the
 * streaming kernel holds: 1, or 2 (rows of full words only: N % 64 == 0, an
 * even number > 32 of words per row; band_rows >= 1).  bml_set_tiling
 * selects 1. */
int bml_set_tiling_ex(bml_sim *sim, int block_k, int64_t band_rows, int lane_words);

/* For an object that runs the resident kernel (created with
 * BML_KERNEL_RESIDENT, or BML_KERNEL_AUTO when the autotuner chose it): hold
 * the lattice in `blocks` thread blocks of one cluster (1, 2, 4 or 8; at most
 * M), each keeping ceil(M / blocks) rows in its shared memory and reading
 * the rows next to its band from its neighbours' shared memory; 1 keeps the
 * whole lattice in one block.  The choice is reported by bml_get_tiling as
 * band_rows = ceil(M / blocks).  BML_EINVAL for other objects or values. */
int bml_set_resident_blocks(bml_sim *sim, int blocks);

/* Current tiling of the bitplane kernels (band_rows 0: one-pass kernel;
 * lane_words 0 with block_k 0: the resident kernel). */
int bml_get_tiling(const bml_sim *sim, int *block_k, int64_t *band_rows, int *lane_words);

/* ------------------------------------------------------------------------
 * Model II (Sec. 2: a variation of the original model).  Every vehicle
 * moves in one synchronous phase per step, from the state at the start of
 * the step, into its target cell (right for LR, below for TB, wrap-around)
 * if that cell is EMPTY; an EMPTY cell wanted by both an LR vehicle (from
 * its left) and a TB vehicle (from above) goes to one of them at random.
 * The paper does not fix the random choice: the LR vehicle wins cell (i,j)
 * at step t (t = 0 for the first step after bml_create_ex or
 * bml_write_lattice, i.e. t = bml_steps_done() before the step) iff bit
 * (j mod 64) of the SplitMix64 output n = t*M*W + i*W + floor(j/64) + 1
 * from state tie_seed is 1 (W = ceil(N/64)).  Moved counts: LR and TB
 * vehicles that changed cell in the step.
 *
 * Model III (Sec. 2: the same cell may contain both an LR and a TB
 * vehicle).  The paper gives only that sentence; the reading here: every
 * vehicle moves in one synchronous phase per step, from the state at the
 * start of the step, into its target cell if that cell holds no vehicle;
 * an EMPTY cell wanted by both an LR and a TB vehicle receives both and
 * then holds one of each.  At the boundary such a cell is the byte 3 (LR
 * bit 0 plus TB bit 1): bml_read_lattice may return it and
 * bml_write_lattice accepts it while the object runs Model III.  (This
 * reading keeps flowing at densities where Model I jams; the paper states
 * that Model III behaves like Model I.)
 * ---------------------------------------------------------------------- */
#define BML_MODEL_I 1   /* the paper's model: H phase then V phase (default) */
#define BML_MODEL_II 2  /* one synchronous phase, random tie-break */
#define BML_MODEL_III 3 /* one synchronous phase, a cell may hold one of each kind */

/* Select the update rule for the following steps (the lattice and the
 * count history are kept).  Models II and III run on the streaming
 * bitplane kernels (k steps per launch; two words per lane on rows of full
 * words, else one; any N): the object must have been created with
 * BML_KERNEL_TBLOCK or BML_KERNEL_AUTO (and a TBLOCK object must have bands,
 * band_rows >= 1), otherwise BML_EINVAL.  Leaving Model III while the
 * lattice holds a doubly occupied cell gives BML_ESTATE.  On a
 * BML_KERNEL_AUTO object selecting a model autotunes the tiling for it
 * (cached per shape, model and device); a BML_KERNEL_TBLOCK object keeps its
 * tiling (bml_set_tiling_ex may change either).  Synchronises the object's
 * stream.  BML_EINVAL for an unknown model; the object is unchanged on
 * failure. */
int bml_set_model(bml_sim *sim, int model, uint64_t tie_seed);

/* Current model and tie-break seed. */
int bml_get_model(const bml_sim *sim, int *model, uint64_t *tie_seed);

/* Wait for all work enqueued by the object. */
int bml_synchronize(bml_sim *sim);

/* Release the object and its device memory (synchronises first).  NULL is
 * allowed. */
void bml_destroy(bml_sim *sim);

/* Message describing the last failure on this thread ("" if none); covers
 * the single-lattice and the ensemble calls. */
const char *bml_last_error(void);

/* ------------------------------------------------------------------------
 * Surrogate network (no counterpart in the paper; it serves the sweep budget
 * allocator): x (67 features) -> [Linear 128, ReLU] x 3 -> Linear 2 ->
 * (v_hat = predicted steady-state velocity, z = jam logit).  BF16 weights
 * and activations on the tcgen05 tensor cores, FP32 accumulation, FP32
 * master weights and AdamW (beta1 0.9, beta2 0.999, eps 1e-8, decoupled
 * weight decay).  Loss per sample (v_hat - v)^2 + BCE-with-logits(z, jam),
 * mean over the batch.  Parameters are a flat float array of
 * bml_mlp_num_params() entries: W1 (128 x 67), b1 (128), W2 (128 x 128), b2,
 * W3 (128 x 128), b3, W4 (2 x 128), b4 (2), each W row-major [out][in].
 * d_* pointers are device memory, read in stream order on the network's
 * stream; the calls synchronise that stream, except bml_mlp_train_step
 * without a loss to return.
 * ------------------------------------------------------------------------ */
typedef struct bml_mlp bml_mlp;

int bml_mlp_create(void *stream, bml_mlp **out);
int64_t bml_mlp_num_params(const bml_mlp *mlp);
/* Upload parameters (host float array) and reset the AdamW state. */
int bml_mlp_set_params(bml_mlp *mlp, const float *host_params);
int bml_mlp_get_params(bml_mlp *mlp, float *host_params);
/* d_x: batch x 67 floats; d_out: batch x 2 floats (v_hat, z). */
int bml_mlp_forward(bml_mlp *mlp, const float *d_x, int64_t batch, float *d_out);
/* One AdamW step on the mean loss of the batch (d_v, d_jam: batch floats;
 * jam is 0 or 1).  *h_loss (host, may be NULL) receives the loss before the
 * update; the call then waits for the gradients and returns BML_ETIMEOUT,
 * with nothing updated, if a tensor-core wait timed out.  With h_loss NULL
 * the step is only enqueued (d_x, d_v, d_jam must stay valid until the
 * stream reaches it), and a timed-out wait inside it is reported by the
 * next call that waits (forward, get_params, grads, a train step with a
 * loss); the weights are then undefined. */
int bml_mlp_train_step(bml_mlp *mlp, const float *d_x, const float *d_v, const float *d_jam,
                       int64_t batch, float lr, float weight_decay, float *h_loss);
/* `steps` AdamW steps, each on a mini-batch of `batch` samples drawn with
 * replacement from the n training samples (d_x: n x 67 floats, d_v, d_jam: n
 * floats, device memory): sample i of the network's training step t (t =
 * AdamW steps taken so far) is row floor(u * n / 2^64), u = SplitMix64 of
 * (seed, t * batch + i + 1), the generator of the seeded placement.  The
 * draw, the gather and every step run on the device, enqueued on the
 * network's stream; the call waits at the end.  h_losses (host, NULL or
 * `steps` floats) receives each step's loss before its update.  Errors:
 * BML_EINVAL (NULL pointer, n < 1, steps < 0, batch outside [1, 2^24], bad
 * lr / weight_decay), BML_ENOMEM / BML_ECUDA, BML_ETIMEOUT (a tensor-core
 * wait timed out; the weights are then undefined). */
int bml_mlp_train(bml_mlp *mlp, const float *d_x, const float *d_v, const float *d_jam,
                  int64_t n, int64_t steps, int64_t batch, float lr, float weight_decay,
                  uint64_t seed, float *h_losses);
/* Gradients of the mean loss (host array in the parameter layout), no
 * update. */
int bml_mlp_grads(bml_mlp *mlp, const float *d_x, const float *d_v, const float *d_jam,
                  int64_t batch, float *host_grads, float *h_loss);
/* One AdamW step with caller-supplied gradients (host array). */
int bml_mlp_apply_grads(bml_mlp *mlp, const float *host_grads, float lr, float weight_decay);
/* Inspection of one layer's device buffers in their padded layouts (layer
 * 0..3; out_pad x in_pad = 128 x 80, 128 x 128, 128 x 128, 16 x 128): host_W
 * receives the BF16 forward copy of W [out_pad][in_pad] (as floats),
 * host_WT its transposed copy [in_pad][out_pad], host_gW the weight gradient
 * of the last gradient computation [out_pad][in_pad] (fp32).  Any of the
 * three may be NULL.  Entries outside [out][in] are padding: the forward and
 * transposed copies keep them 0, and so does every gradient computation.
 * Synchronises the network's stream.  Errors: BML_EINVAL (NULL mlp, layer
 * out of range), BML_ECUDA. */
int bml_mlp_get_layer(bml_mlp *mlp, int layer, float *host_W, float *host_WT, float *host_gW);
void bml_mlp_destroy(bml_mlp *mlp);

/* The tensor-core GEMM the network runs on: C (M x N, fp32, row-major, ldc)
 * = A (M x K) * B (N x K)^T, A and B bf16 row-major with K contiguous (lda,
 * ldb elements; multiples of 8, 16-byte aligned).  16 <= N <= 128,
 * N % 16 == 0, K % 16 == 0.  Device pointers; synchronises the stream. */
int bml_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, float *C, int64_t ldc,
                  int64_t M, int64_t N, int64_t K, void *stream);

/* bml_gemm_bf16 with flags.  BML_GEMM_TEST_STALL (test hook): no operand copy
 * is issued, so the kernel's first completion wait runs out after its 1 s
 * bound; the kernel sets its error flag, releases its tensor memory and
 * returns, and the call reports BML_ETIMEOUT (C is then undefined; the
 * context stays usable).  Unknown flags: BML_EINVAL. */
#define BML_GEMM_TEST_STALL 1u
int bml_gemm_bf16_ex(const void *A, int64_t lda, const void *B, int64_t ldb, float *C,
                     int64_t ldc, int64_t M, int64_t N, int64_t K, unsigned flags, void *stream);

/* ------------------------------------------------------------------------
 * Byte-per-cell step that allocates nothing (no counterpart in the paper).
 *
 * For callers that cannot allocate device memory when they step a lattice:
 * code that runs inside a framework whose own pool owns every allocation,
 * code being recorded into a pipeline in which an allocation would
 * synchronise the device, or embedded users whose memory budget is fixed at
 * start-up.  The caller owns the lattice and the count arrays; the one extra
 * buffer the step needs (the lattice between its two phases) is a 16 MiB
 * array compiled into the library, which every GPU that loads the library's
 * device code holds until the process exits.
 *
 * d_cells: device pointer, 16-byte aligned, M rows of PB bytes each, PB = N
 *   rounded up to a multiple of 16; cell (i, j) is byte i*PB + j (0/1/2);
 *   bytes j >= N of a row (the row padding) may hold any value: they are
 *   not cells, take no part in any move or count, and are left exactly as
 *   they were.  Stepped k times in place.
 * d_moved_lr, d_moved_tb: device arrays of k int64; set to the counts of the
 *   k steps (they are cleared first).
 * stream: cudaStream_t (NULL = legacy default stream); the call only
 *   enqueues work.
 * Limits and errors: M * PB <= BML_NOALLOC_MAX_BYTES (else BML_EINVAL, use
 *   bml_create_ex with BML_KERNEL_BYTE); NULL pointers, M < 1, N < 1, k < 0
 *   or a misaligned d_cells give BML_EINVAL.  No cudaMalloc, cudaFree or any
 *   other allocating routine is called.
 * The first call on a device looks up the device address of the built-in
 *   array (cudaGetSymbolAddress) and keeps it for the life of the process;
 *   make that first call before any stream capture.  A device reset
 *   (cudaDeviceReset) between calls is not supported: the array may be
 *   reloaded at another address while the kept one stays in use.  All calls share the one array: calls whose work overlaps on
 *   the GPU (different streams, or other threads) race and corrupt each
 *   other; order them on one stream.
 * ------------------------------------------------------------------------ */
#define BML_NOALLOC_MAX_BYTES (16u * 1024u * 1024u)

int bml_step_bytes_noalloc(uint8_t *d_cells, int64_t M, int64_t N, int64_t k,
                           int64_t *d_moved_lr, int64_t *d_moved_tb, void *stream);

/* ------------------------------------------------------------------------
 * Batched ensemble: `count` independent lattices of uneven shapes and
 * densities advanced together.  Every lattice follows the model and the
 * placement rule above (lattice l: M[l] x N[l], seed[l], p_lr[l], p_tb[l]).
 * Each lattice row must fit one warp: 1 <= N[l] <= 2048; 1 <= M[l] <= 2^24;
 * at most 2^36 cells in total.  One bml_ensemble_step call runs as one
 * persistent cooperative launch per temporal depth used (replayed from a
 * cached CUDA graph when the stream can be captured).  Lattices are numbered
 * 0..count-1; "concatenated" byte buffers hold lattice 0's M*N bytes, then
 * lattice 1's, and so on.  Steps of all lattices advance together.
 * ------------------------------------------------------------------------ */
typedef struct bml_ens bml_ens;

/* Flags of bml_ensemble_create_ex. */
#define BML_ENS_EARLY_EXIT 1u /* skip lattices that reached an absorbing fixed
                                 point (a step with no move); their later
                                 counts are 0 and their lattice stays as it is,
                                 exactly as the automaton would evolve        */
#define BML_ENS_NO_GRAPH 2u   /* launch directly instead of replaying graphs  */
#define BML_ENS_TEST_STALL 4u /* test hook: the first wait between chunks
                                 waits for one band more than its lattice
                                 has and gives up after 20 ms (a call of at
                                 least two chunks); bml_ensemble_step returns
                                 BML_ETIMEOUT and the ensemble becomes
                                 unusable (BML_ESTATE afterwards)             */

/* Create with autotuned tiling, no flags.  Arrays hold `count` entries and
 * are read during the call only. */
int bml_ensemble_create(int64_t count, const int64_t *M, const int64_t *N, const uint64_t *seed,
                        const double *p_lr, const double *p_tb, void *stream, bml_ens **out);

/* Full form: block_k in {1, 2, 4, 8} and band_rows >= 1 fix the temporal
 * depth and the target band height; both 0 autotune them on this ensemble
 * (the lattices are not advanced; the choice is kept per device and multiset
 * of lattice shapes, and a later ensemble of the same shapes reuses it).  reserve_steps preallocates the traces
 * (0 picks 1024; they grow on demand). */
int bml_ensemble_create_ex(int64_t count, const int64_t *M, const int64_t *N,
                           const uint64_t *seed, const double *p_lr, const double *p_tb,
                           int block_k, int64_t band_rows, unsigned flags, void *stream,
                           int64_t reserve_steps, bml_ens **out);

/* Enqueue k >= 0 steps of every lattice; asynchronous. */
int bml_ensemble_step(bml_ens *ens, int64_t k);

/* Moved counts of one lattice for steps first+1 .. first+n (host arrays of n
 * int64; any may be NULL).  Synchronises. */
int bml_ensemble_moved_counts(bml_ens *ens, int64_t lattice, int64_t first, int64_t n,
                              int64_t *out_total, int64_t *out_lr, int64_t *out_tb);

/* Counts of all lattices for steps first+1 .. first+n: out_lr / out_tb are
 * host arrays of count * n int64, lattice-major (either may be NULL). */
int bml_ensemble_traces(bml_ens *ens, int64_t first, int64_t n, int64_t *out_lr,
                        int64_t *out_tb);

/* Per lattice, the 0-based index t of the first step t+1 in which no car
 * moved (the lattice is at a fixed point from then on), or -1. */
int bml_ensemble_jam_steps(bml_ens *ens, int64_t *out);

/* Read one lattice (M[l]*N[l] bytes) or all lattices (concatenated). */
int bml_ensemble_read_lattice(bml_ens *ens, int64_t lattice, uint8_t *out);
int bml_ensemble_read_lattices(bml_ens *ens, uint8_t *out);

/* Replace all lattices with concatenated bytes (values 0, 1, 2, else
 * BML_EINVAL and no change); restarts every trajectory (steps_done = 0). */
int bml_ensemble_write_lattices(bml_ens *ens, const uint8_t *in);

int64_t bml_ensemble_steps_done(const bml_ens *ens);

/* Number of cars of every lattice (host array of count int64; conserved by
 * the dynamics, recounted by bml_ensemble_write_lattices). */
int bml_ensemble_car_counts(bml_ens *ens, int64_t *out);

/* Surrogate inputs from the traces: d_out (device, count x (3 + points)
 * floats, lattice-major) = [cars / (M N), M / 2048, N / 2048, mean velocity
 * of each of `points` equal windows of steps first+1 .. first+n], velocity =
 * moved cars / cars (0 without cars).  n must be a multiple of points and the
 * steps already taken.  Synchronises. */
int bml_ensemble_features(bml_ens *ens, int64_t first, int64_t n, int points, float *d_out);

/* Labels over the steps taken so far: d_v[l] = mean velocity over the last
 * `window` steps, d_jam[l] = 1 if some step moved no car (the lattice is at
 * a fixed point), else 0 (device arrays of count floats).  Synchronises. */
int bml_ensemble_labels(bml_ens *ens, int64_t window, float *d_v, float *d_jam);

/* The ensemble's tile plan for lattices M[l] x N[l] (host arrays of count
 * entries) at target band height `band`, computed on the host without any
 * CUDA call: *out_tiles = warp tiles; *out_score = the autotuner's predicted
 * cost of a launch of 32 chunks of depth `depth` on `warps` warps, in rows
 * per warp: each tile costs its longest band plus 2 * depth halo rows, a
 * chunk costs the larger of the mean tile rows per warp and 1.2 times the
 * longest tile, and the makespan of the longest-first assignment beyond the
 * mean is added once (32 * max(mean, 1.2 * longest) + makespan - mean);
 * out_rows (NULL or count entries) = rows of each lattice covered by the
 * plan's bands (M[l] when every row is in exactly one band).  BML_EINVAL on
 * bad arguments. */
int bml_ensemble_plan(int64_t count, const int64_t *M, const int64_t *N, int64_t band, int depth,
                      int warps, int64_t *out_tiles, double *out_score, int64_t *out_rows);

/* Stop advancing the n listed lattices (host array of indices; repeats and
 * lattices already retired or jammed are allowed): from the next step on
 * they keep their current state, their per-step counts are 0 and they leave
 * the tile plan, while the other lattices go on; the tiles are planned again
 * for the lattices that go on (with the band height given at creation, else
 * the one the autotuner's plan score prefers for them).  Their jam
 * steps and labels are computed over the steps before the retirement.  For
 * budget allocation: runs that have had their budget stop, the others
 * continue in the same ensemble.  bml_ensemble_write_lattices makes every
 * lattice active again.  Synchronises.  Errors: BML_EINVAL (NULL with n > 0,
 * an index outside [0, count)), BML_ESTATE (the ensemble failed earlier). */
int bml_ensemble_retire(bml_ens *ens, int64_t n, const int64_t *lattices);

/* Temporal depth, band height and whether graph replay is in use. */
int bml_ensemble_get_config(const bml_ens *ens, int *block_k, int64_t *band_rows, int *graphs);

/* Wait for the ensemble's work; reports BML_ETIMEOUT if a barrier gave up. */
int bml_ensemble_synchronize(bml_ens *ens);

void bml_ensemble_destroy(bml_ens *ens);

#ifdef __cplusplus
}
#endif

#endif /* BML_H */
