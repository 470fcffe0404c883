/*
 * BML traffic CA oracle: plain, slow, obviously correct CPU implementation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA library.
 *
 * Model (Biham-Middleton-Levine Model I, Marzolla 2018, Sec. 2):
 *   - a periodic M x N lattice of cells, each EMPTY, LR (moves right) or
 *     TB (moves down);
 *   - one step = a horizontal phase then a vertical phase (Sec. 2; the
 *     Fig. 1 caption counts both phases as one step);
 *   - horizontal rule (Sec. 2, first case analysis):
 *       center' = LR     if left == LR and center == EMPTY
 *                 EMPTY  if center == LR and right == EMPTY
 *                 center otherwise
 *   - vertical rule (Sec. 2, second case analysis): the same with
 *     top/bottom and TB;
 *   - neighbours wrap around (periodic boundary, Sec. 2);
 *   - synchronous update through two grids cur/next (Sec. 3);
 *   - one byte per cell, EMPTY=0, LR=1, TB=2, cell (i,j) at i*N+j (Sec. 3).
 * The paper states the model for square N x N grids; this oracle takes
 * M rows and N columns, LR moving along j (+1) and TB along i (+1).
 *
 * "Moved count" (not defined by the paper): the number of vehicles that
 * changed cell in a phase.  An LR car at (i,j) moves in the horizontal
 * phase iff cell (i,(j+1) mod N) is EMPTY before that phase; likewise for TB
 * in the vertical phase with ((i+1) mod M, j).
 *
 * Initial placement (the paper only says vehicles are "placed randomly",
 * Sec. 2): every cell independently, from SplitMix64 (Steele, Lea, Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014):
 *   z_n = seed + n * 0x9E3779B97F4A7C15 (mod 2^64), u_n = mix(z_n),
 *   n = i*N + j + 1;
 *   cell = LR if u < t_lr, else TB if u - t_lr < t_tb, else EMPTY,
 *   t_x = floor(p_x * 2^64) clamped to 2^64 - 1.
 *
 * Models II and III: oracle_run_model below (readings stated there).
 *
 * Threaded mode: the row loop of each phase may be split across OpenMP
 * threads exactly as Sec. 4 describes ("parallel for" over rows).  Every
 * cell is computed by the same expression from the same inputs, so the
 * result is identical for any thread count; moved counts are integer sums.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { EMPTY = 0, LR = 1, TB = 2 };

/* SplitMix64 output function ("mix64" variant 13 of Stafford), as
 * published with the generator. */
static uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* n-th output (n >= 1) of SplitMix64 started from state `seed`. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t n)
{
    return sm64_mix(seed + n * 0x9E3779B97F4A7C15ULL);
}

/* floor(p * 2^64), clamped to [0, 2^64 - 1]. */
uint64_t oracle_threshold(double p)
{
    double x = ldexp(p, 64);
    if (!(x > 0.0)) return 0;
    if (x >= 18446744073709551616.0) return UINT64_MAX;
    return (uint64_t)x;
}

/* Fill g (M*N bytes, row-major) with the seeded random placement. */
int oracle_init(uint8_t *g, int64_t M, int64_t N, uint64_t seed,
                double p_lr, double p_tb)
{
    if (!g || M <= 0 || N <= 0) return -1;
    if (!(p_lr >= 0.0 && p_tb >= 0.0 && p_lr + p_tb <= 1.0)) return -1;
    const uint64_t t_lr = oracle_threshold(p_lr);
    const uint64_t t_tb = oracle_threshold(p_tb);
    for (int64_t i = 0; i < M; i++) {
        for (int64_t j = 0; j < N; j++) {
            const uint64_t u = oracle_splitmix64(seed, (uint64_t)(i * N + j) + 1);
            uint8_t c;
            if (u < t_lr)
                c = LR;
            else if (u - t_lr < t_tb)
                c = TB;
            else
                c = EMPTY;
            g[i * N + j] = c;
        }
    }
    return 0;
}

/* Fill w (R*C bytes, row-major) with the cells of rows i0..i0+R-1 and
 * columns j0..j0+C-1 (both mod M, N) of the seeded placement of an M x N
 * lattice: the same cells oracle_init would write there, for a window of a
 * lattice too large to hold whole. */
int oracle_init_window(uint8_t *w, int64_t R, int64_t C, int64_t i0, int64_t j0,
                       int64_t M, int64_t N, uint64_t seed, double p_lr, double p_tb)
{
    if (!w || M <= 0 || N <= 0 || R <= 0 || C <= 0 || i0 < 0 || j0 < 0) return -1;
    if (!(p_lr >= 0.0 && p_tb >= 0.0 && p_lr + p_tb <= 1.0)) return -1;
    const uint64_t t_lr = oracle_threshold(p_lr);
    const uint64_t t_tb = oracle_threshold(p_tb);
    for (int64_t a = 0; a < R; a++) {
        const int64_t i = (i0 + a) % M;
        for (int64_t b = 0; b < C; b++) {
            const int64_t j = (j0 + b) % N;
            const uint64_t u = oracle_splitmix64(seed, (uint64_t)(i * N + j) + 1);
            uint8_t c;
            if (u < t_lr)
                c = LR;
            else if (u - t_lr < t_tb)
                c = TB;
            else
                c = EMPTY;
            w[a * C + b] = c;
        }
    }
    return 0;
}

/* Horizontal phase over all rows: next = H(cur); returns LR cars moved. */
static int64_t horizontal_phase(const uint8_t *cur, uint8_t *next,
                                int64_t M, int64_t N, int threads)
{
    int64_t moved = 0;
#pragma omp parallel for reduction(+ : moved) num_threads(threads) schedule(static)
    for (int64_t i = 0; i < M; i++) {
        for (int64_t j = 0; j < N; j++) {
            const uint8_t left = cur[i * N + (j - 1 + N) % N];
            const uint8_t center = cur[i * N + j];
            const uint8_t right = cur[i * N + (j + 1) % N];
            uint8_t out;
            if (left == LR && center == EMPTY)
                out = LR;
            else if (center == LR && right == EMPTY)
                out = EMPTY;
            else
                out = center;
            next[i * N + j] = out;
            if (center == LR && right == EMPTY) moved++;
        }
    }
    return moved;
}

/* Vertical phase over all rows: next = V(cur); returns TB cars moved. */
static int64_t vertical_phase(const uint8_t *cur, uint8_t *next,
                              int64_t M, int64_t N, int threads)
{
    int64_t moved = 0;
#pragma omp parallel for reduction(+ : moved) num_threads(threads) schedule(static)
    for (int64_t i = 0; i < M; i++) {
        for (int64_t j = 0; j < N; j++) {
            const uint8_t top = cur[((i - 1 + M) % M) * N + j];
            const uint8_t center = cur[i * N + j];
            const uint8_t bottom = cur[((i + 1) % M) * N + j];
            uint8_t out;
            if (top == TB && center == EMPTY)
                out = TB;
            else if (center == TB && bottom == EMPTY)
                out = EMPTY;
            else
                out = center;
            next[i * N + j] = out;
            if (center == TB && bottom == EMPTY) moved++;
        }
    }
    return moved;
}

/*
 * Advance g (M*N bytes, in place from the caller's view) by K full steps.
 * moved_lr[t], moved_tb[t] (t = 0..K-1, either may be NULL) receive the
 * counts of step t+1.  threads <= 1 runs serially.
 * Returns 0, or -1 on bad arguments, -2 if scratch cannot be allocated.
 */
int oracle_run(uint8_t *g, int64_t M, int64_t N, int64_t K,
               int64_t *moved_lr, int64_t *moved_tb, int threads)
{
    if (!g || M <= 0 || N <= 0 || K < 0) return -1;
    if (threads < 1) threads = 1;
    uint8_t *tmp = (uint8_t *)malloc((size_t)(M * N));
    if (!tmp) return -2;
    for (int64_t t = 0; t < K; t++) {
        /* cur = g, next = tmp; then cur = tmp, next = g (Sec. 3 swap). */
        const int64_t mlr = horizontal_phase(g, tmp, M, N, threads);
        const int64_t mtb = vertical_phase(tmp, g, M, N, threads);
        if (moved_lr) moved_lr[t] = mlr;
        if (moved_tb) moved_tb[t] = mtb;
    }
    free(tmp);
    return 0;
}

/* One phase only (phase 0 = horizontal, 1 = vertical), for tests of the
 * individual rules.  cur and next must not overlap. */
int64_t oracle_phase(const uint8_t *cur, uint8_t *next, int64_t M, int64_t N,
                     int phase)
{
    if (phase == 0) return horizontal_phase(cur, next, M, N, 1);
    return vertical_phase(cur, next, M, N, 1);
}

/*
 * Model II (Sec. 2: a variation of the original BML paper).  Every vehicle
 * moves in one synchronous phase per step, from the state at the start of
 * the step; a vehicle's target cell (right for LR, below for TB, with
 * wrap-around) must be EMPTY at that time.  If an LR vehicle (from the left)
 * and a TB vehicle (from above) both target the same empty cell, one of
 * them, chosen at random, moves and the other stands still.  The paper does
 * not fix the random choice; here the LR vehicle wins the cell (i,j) at step
 * t iff bit (j mod 64) of SplitMix64 output n = t*M*W + i*W + floor(j/64) + 1
 * from state tie_seed is 1 (W = ceil(N/64)); t counts steps from 0.
 */
static int lr_wins(uint64_t tie_seed, int64_t t, int64_t M, int64_t N,
                   int64_t i, int64_t j)
{
    const uint64_t W = (uint64_t)((N + 63) / 64);
    const uint64_t n = (uint64_t)t * (uint64_t)M * W + (uint64_t)i * W +
                       (uint64_t)(j / 64) + 1;
    return (int)((oracle_splitmix64(tie_seed, n) >> (j % 64)) & 1u);
}

/* Whether an LR vehicle from the left may enter cell (i,j) of cur, and
 * whether a TB vehicle from above may (both need the cell empty). */
static void entries(const uint8_t *cur, int64_t M, int64_t N, int model,
                    uint64_t tie_seed, int64_t t, int64_t i, int64_t j,
                    int *lr_in, int *tb_in)
{
    *lr_in = *tb_in = 0;
    if (cur[i * N + j] != EMPTY) return;
    const int from_left = cur[i * N + (j - 1 + N) % N] == LR;
    const int from_top = cur[((i - 1 + M) % M) * N + j] == TB;
    if (model == 2 && from_left && from_top) {
        const int lr = lr_wins(tie_seed, t, M, N, i, j);
        *lr_in = lr;
        *tb_in = !lr;
    } else {
        *lr_in = from_left;
        *tb_in = from_top;
    }
}

static void model_step(const uint8_t *cur, uint8_t *next, int64_t M, int64_t N,
                       int model, uint64_t tie_seed, int64_t t, int threads,
                       int64_t *mlr, int64_t *mtb)
{
    int64_t a = 0, b = 0;
#pragma omp parallel for reduction(+ : a, b) num_threads(threads) schedule(static)
    for (int64_t i = 0; i < M; i++) {
        for (int64_t j = 0; j < N; j++) {
            const uint8_t c = cur[i * N + j];
            uint8_t out = EMPTY;
            int lr_in, tb_in;
            if (c == LR) {
                /* the right neighbour accepts this LR vehicle? */
                entries(cur, M, N, model, tie_seed, t, i, (j + 1) % N, &lr_in, &tb_in);
                if (lr_in) a++;
                else out = LR;
            }
            if (c == TB) {
                entries(cur, M, N, model, tie_seed, t, (i + 1) % M, j, &lr_in, &tb_in);
                if (tb_in) b++;
                else out = TB;
            }
            entries(cur, M, N, model, tie_seed, t, i, j, &lr_in, &tb_in);
            if (lr_in) out = LR;
            if (tb_in) out = TB;
            next[i * N + j] = out;
        }
    }
    *mlr = a;
    *mtb = b;
}

/*
 * Model III (Sec. 2: the same cell may contain both an LR and a TB
 * vehicle).  The paper gives only that sentence; the reading here: every
 * vehicle moves in one synchronous phase per step, from the state at its
 * start; a vehicle moves iff its target cell (right for LR, below for TB,
 * wrap-around) holds no vehicle at that time; an empty cell wanted by an LR
 * and a TB vehicle receives both, and then holds one vehicle of each kind.
 * A cell byte has bit 0 for an LR vehicle and bit 1 for a TB vehicle, so a
 * doubly occupied cell is 3.  (With alternating phases, or with targets
 * that need only be free of the vehicle's own kind, no cell could become
 * doubly occupied or the two kinds would never interact.)
 */
static void model3_step(const uint8_t *cur, uint8_t *next, int64_t M, int64_t N,
                        int threads, int64_t *mlr, int64_t *mtb)
{
    int64_t a = 0, b = 0;
#pragma omp parallel for reduction(+ : a, b) num_threads(threads) schedule(static)
    for (int64_t i = 0; i < M; i++) {
        for (int64_t j = 0; j < N; j++) {
            const uint8_t c = cur[i * N + j];
            const uint8_t right = cur[i * N + (j + 1) % N];
            const uint8_t below = cur[((i + 1) % M) * N + j];
            const uint8_t left = cur[i * N + (j - 1 + N) % N];
            const uint8_t above = cur[((i - 1 + M) % M) * N + j];
            uint8_t out = 0;
            /* the vehicles in this cell: each stays unless its target is empty */
            if (c & LR) {
                if (right == EMPTY) a++;
                else out |= LR;
            }
            if (c & TB) {
                if (below == EMPTY) b++;
                else out |= TB;
            }
            /* an empty cell receives the LR vehicle on its left and the TB
               vehicle above it, both of whose targets it is */
            if (c == EMPTY) {
                if (left & LR) out |= LR;
                if (above & TB) out |= TB;
            }
            next[i * N + j] = out;
        }
    }
    *mlr = a;
    *mtb = b;
}

/*
 * Advance g by K steps of Model II (model = 2) or Model III (model = 3); the
 * first step has index t0 (for Model II it selects the tie-break bits).
 * Counts as in oracle_run.  Returns 0, -1 on bad arguments (another model,
 * or for Model III a cell byte above 3), -2 on no memory.
 */
int oracle_run_model(uint8_t *g, int64_t M, int64_t N, int64_t K, int model,
                     uint64_t tie_seed, int64_t t0, int64_t *moved_lr,
                     int64_t *moved_tb, int threads)
{
    if (!g || M <= 0 || N <= 0 || K < 0 || t0 < 0 || (model != 2 && model != 3))
        return -1;
    if (model == 3)
        for (int64_t q = 0; q < M * N; q++)
            if (g[q] > (LR | TB)) return -1;
    if (threads < 1) threads = 1;
    uint8_t *tmp = (uint8_t *)malloc((size_t)(M * N));
    if (!tmp) return -2;
    for (int64_t t = 0; t < K; t++) {
        int64_t a, b;
        if (model == 3)
            model3_step(g, tmp, M, N, threads, &a, &b);
        else
            model_step(g, tmp, M, N, model, tie_seed, t0 + t, threads, &a, &b);
        memcpy(g, tmp, (size_t)(M * N));
        if (moved_lr) moved_lr[t] = a;
        if (moved_tb) moved_tb[t] = b;
    }
    free(tmp);
    return 0;
}

/*
 * Run `count` independent M x N lattices stored back to back in g, each for
 * K steps; counts go to moved_lr[l*K + t], moved_tb[l*K + t].  A plain loop
 * over oracle_run, used for exhaustive enumeration of tiny lattices.
 */
int oracle_run_batch(uint8_t *g, int64_t count, int64_t M, int64_t N,
                     int64_t K, int64_t *moved_lr, int64_t *moved_tb)
{
    for (int64_t l = 0; l < count; l++) {
        const int rc = oracle_run(g + l * M * N, M, N, K,
                                  moved_lr ? moved_lr + l * K : NULL,
                                  moved_tb ? moved_tb + l * K : NULL, 1);
        if (rc) return rc;
    }
    return 0;
}
