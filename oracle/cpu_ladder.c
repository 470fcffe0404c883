/*
 * The paper's CPU implementations of the BML step, as timed baselines
 * beside the oracle -- TEST / BASELINE INFRASTRUCTURE.
 *
 * Only the tests and the benchmark's CPU-baseline leg load this file's
 * library; it shares nothing with the CUDA library.  The oracle
 * (bml_oracle.c) is the serial form with modulo indexing (Sec. 3); here are
 * the faster forms the paper measures against it (Sec. 7, Fig. 3), written
 * from their descriptions:
 *
 *   1  serial with ghost cells (Sec. 3): the lattice is stored with one
 *      extra row above and below and one extra column left and right; the
 *      ghost columns are copied from the opposite side before each
 *      horizontal phase and the ghost rows before each vertical phase, so
 *      the rules need no modulo;
 *   2  the same with the row loops shared among threads (Sec. 4);
 *   3  SIMD (Sec. 5): 32 adjacent cells per vector, the rules computed by
 *      selection with masks instead of branches (GCC vector types, compiled
 *      for AVX-512, AVX2 and the baseline x86-64 set, the widest the host
 *      supports chosen at run time; one thread);
 *   4  SIMD with the row loops shared among threads (Sec. 7, OpenMP+SIMD);
 *   5  beyond the paper: two bitplanes of 64 cells per 64-bit word (its
 *      Sec. 3 remark that two bits per cell suffice), the rules as bit logic
 *      on whole words, rows shared among threads.
 *
 * Every form computes exactly the rules of Sec. 2 (horizontal phase, then
 * vertical phase, wrap-around, synchronous double buffer); the tests compare
 * each with the oracle bit for bit.  None counts moved cars (the paper's
 * programs do not).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

enum { EMPTY = 0, LR = 1, TB = 2 };

static double now_s(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* ---------------------------------------------------------- ghost grid --
 * (M + 2) rows of `pitch` bytes; cell (i, j) of the lattice at row i + 1,
 * column j + 1.  The pitch leaves room for whole vectors past column N + 1. */
#define VBYTES 32
typedef signed char vbytes __attribute__((vector_size(VBYTES)));

typedef struct {
    uint8_t *cur, *nxt;
    int64_t M, N, pitch;
} ghost_t;

static int ghost_alloc(ghost_t *g, int64_t M, int64_t N)
{
    g->M = M;
    g->N = N;
    g->pitch = ((N + 2 + VBYTES - 1) / VBYTES + 1) * VBYTES;
    const size_t bytes = (size_t)(M + 2) * (size_t)g->pitch;
    g->cur = (uint8_t *)calloc(bytes, 1);
    g->nxt = (uint8_t *)calloc(bytes, 1);
    if (!g->cur || !g->nxt) {
        free(g->cur);
        free(g->nxt);
        return -2;
    }
    return 0;
}

static void ghost_free(ghost_t *g)
{
    free(g->cur);
    free(g->nxt);
}

#define AT(buf, p, i, j) ((buf)[(i) * (p) + (j)])

/* left ghost column = the lattice's last column, right ghost = its first */
static void fill_ghost_columns(uint8_t *c, int64_t M, int64_t N, int64_t p, int threads)
{
#pragma omp parallel for num_threads(threads) schedule(static) if (threads > 1)
    for (int64_t i = 1; i <= M; i++) {
        AT(c, p, i, 0) = AT(c, p, i, N);
        AT(c, p, i, N + 1) = AT(c, p, i, 1);
    }
}

/* top ghost row = the lattice's last row, bottom ghost = its first */
static void fill_ghost_rows(uint8_t *c, int64_t M, int64_t N, int64_t p)
{
    memcpy(&AT(c, p, 0, 1), &AT(c, p, M, 1), (size_t)N);
    memcpy(&AT(c, p, M + 1, 1), &AT(c, p, 1, 1), (size_t)N);
}

/* the rules on one cell from its neighbours along the phase's direction */
static inline __attribute__((always_inline)) uint8_t rule(uint8_t before, uint8_t c,
                                                           uint8_t after, uint8_t kind)
{
    if (before == kind && c == EMPTY) return kind;
    if (c == kind && after == EMPTY) return EMPTY;
    return c;
}

static void scalar_h(const uint8_t *cur, uint8_t *nxt, int64_t M, int64_t N, int64_t p,
                     int threads)
{
#pragma omp parallel for num_threads(threads) schedule(static) if (threads > 1)
    for (int64_t i = 1; i <= M; i++)
        for (int64_t j = 1; j <= N; j++)
            AT(nxt, p, i, j) =
                rule(AT(cur, p, i, j - 1), AT(cur, p, i, j), AT(cur, p, i, j + 1), LR);
}

static void scalar_v(const uint8_t *cur, uint8_t *nxt, int64_t M, int64_t N, int64_t p,
                     int threads)
{
#pragma omp parallel for num_threads(threads) schedule(static) if (threads > 1)
    for (int64_t i = 1; i <= M; i++)
        for (int64_t j = 1; j <= N; j++)
            AT(nxt, p, i, j) =
                rule(AT(cur, p, i - 1, j), AT(cur, p, i, j), AT(cur, p, i + 1, j), TB);
}

/* The rules on VBYTES adjacent cells by selection with masks: a lane of a
 * comparison is all ones where it holds, so
 *   enter = (before == kind) & (c == EMPTY)    the cell receives a vehicle
 *   leave = (c == kind) & (after == EMPTY)     its vehicle moves on
 *   out   = (enter & kind) | (~(enter | leave) & c)
 * (a leaving vehicle leaves EMPTY = 0, which needs no term).  The cells past
 * the last whole vector of a row take the scalar rule. */
static inline __attribute__((always_inline)) vbytes vload(const uint8_t *p)
{
    vbytes v;
    memcpy(&v, p, sizeof v);
    return v;
}

static inline __attribute__((always_inline)) void vstore(uint8_t *p, vbytes v)
{
    memcpy(p, &v, sizeof v);
}

static inline __attribute__((always_inline)) vbytes vrule(vbytes before, vbytes c,
                                                          vbytes after, signed char kind)
{
    const vbytes enter = (vbytes)((before == kind) & (c == EMPTY));
    const vbytes leave = (vbytes)((c == kind) & (after == EMPTY));
    return (enter & kind) | (~(enter | leave) & c);
}

/* one row of each phase, compiled three times: with AVX-512 (BW), with AVX2
   and for the baseline instruction set; the widest the host supports runs */
#define SIMD_ROWS(SUFFIX, ATTR)                                                          \
    ATTR static void simd_h_row_##SUFFIX(const uint8_t *r, uint8_t *o, int64_t N)       \
    {                                                                                    \
        int64_t j = 1;                                                                   \
        for (; j + VBYTES - 1 <= N; j += VBYTES)                                         \
            vstore(o + j, vrule(vload(r + j - 1), vload(r + j), vload(r + j + 1), LR));  \
        for (; j <= N; j++) o[j] = rule(r[j - 1], r[j], r[j + 1], LR);                   \
    }                                                                                    \
    ATTR static void simd_v_row_##SUFFIX(const uint8_t *up, const uint8_t *r,            \
                                         const uint8_t *dn, uint8_t *o, int64_t N)       \
    {                                                                                    \
        int64_t j = 1;                                                                   \
        for (; j + VBYTES - 1 <= N; j += VBYTES)                                         \
            vstore(o + j, vrule(vload(up + j), vload(r + j), vload(dn + j), TB));        \
        for (; j <= N; j++) o[j] = rule(up[j], r[j], dn[j], TB);                         \
    }

SIMD_ROWS(avx512, __attribute__((target("avx512bw"))))
SIMD_ROWS(avx2, __attribute__((target("avx2"))))
SIMD_ROWS(base, )

typedef void (*h_row_fn)(const uint8_t *, uint8_t *, int64_t);
typedef void (*v_row_fn)(const uint8_t *, const uint8_t *, const uint8_t *, uint8_t *, int64_t);

static void pick_simd(h_row_fn *h, v_row_fn *v)
{
    __builtin_cpu_init();
    if (__builtin_cpu_supports("avx512bw")) {
        *h = simd_h_row_avx512;
        *v = simd_v_row_avx512;
    } else if (__builtin_cpu_supports("avx2")) {
        *h = simd_h_row_avx2;
        *v = simd_v_row_avx2;
    } else {
        *h = simd_h_row_base;
        *v = simd_v_row_base;
    }
}

static void simd_h(const uint8_t *cur, uint8_t *nxt, int64_t M, int64_t N, int64_t p,
                   int threads)
{
    h_row_fn h;
    v_row_fn v;
    pick_simd(&h, &v);
#pragma omp parallel for num_threads(threads) schedule(static) if (threads > 1)
    for (int64_t i = 1; i <= M; i++) h(cur + i * p, nxt + i * p, N);
}

static void simd_v(const uint8_t *cur, uint8_t *nxt, int64_t M, int64_t N, int64_t p,
                   int threads)
{
    h_row_fn h;
    v_row_fn v;
    pick_simd(&h, &v);
#pragma omp parallel for num_threads(threads) schedule(static) if (threads > 1)
    for (int64_t i = 1; i <= M; i++)
        v(cur + (i - 1) * p, cur + i * p, cur + (i + 1) * p, nxt + i * p, N);
}

static double run_ghost(uint8_t *g, int64_t M, int64_t N, int64_t K, int threads, int simd,
                        int *rc)
{
    ghost_t G;
    *rc = ghost_alloc(&G, M, N);
    if (*rc) return 0.0;
    const int64_t p = G.pitch;
    for (int64_t i = 0; i < M; i++) memcpy(&AT(G.cur, p, i + 1, 1), g + i * N, (size_t)N);
    const double t0 = now_s();
    for (int64_t t = 0; t < K; t++) {
        fill_ghost_columns(G.cur, M, N, p, threads);
        if (simd)
            simd_h(G.cur, G.nxt, M, N, p, threads);
        else
            scalar_h(G.cur, G.nxt, M, N, p, threads);
        fill_ghost_rows(G.nxt, M, N, p);
        if (simd)
            simd_v(G.nxt, G.cur, M, N, p, threads);
        else
            scalar_v(G.nxt, G.cur, M, N, p, threads);
    }
    const double dt = now_s() - t0;
    for (int64_t i = 0; i < M; i++) memcpy(g + i * N, &AT(G.cur, p, i + 1, 1), (size_t)N);
    ghost_free(&G);
    return dt;
}

/* ----------------------------------------------------------- bitplanes --
 * Row i is W = ceil(N / 64) words per plane; cell j is bit j % 64 of word
 * j / 64; the last word holds nb = N - 64 (W - 1) cells and zeros above. */
typedef struct {
    uint64_t *L, *T, *L2, *T2;
    int64_t M, N, W;
    int nb;
    uint64_t tail;
} planes_t;

static int planes_alloc(planes_t *q, int64_t M, int64_t N)
{
    q->M = M;
    q->N = N;
    q->W = (N + 63) / 64;
    q->nb = (int)(N - 64 * (q->W - 1));
    q->tail = q->nb == 64 ? ~0ull : ((1ull << q->nb) - 1ull);
    const size_t words = (size_t)(M * q->W);
    q->L = (uint64_t *)calloc(words, 8);
    q->T = (uint64_t *)calloc(words, 8);
    q->L2 = (uint64_t *)calloc(words, 8);
    q->T2 = (uint64_t *)calloc(words, 8);
    if (!q->L || !q->T || !q->L2 || !q->T2) return -2;
    return 0;
}

static void planes_free(planes_t *q)
{
    free(q->L);
    free(q->T);
    free(q->L2);
    free(q->T2);
}

/* horizontal phase on every row: L2 from (L, T) */
static void bits_h(planes_t *q, int threads)
{
    const int64_t W = q->W;
    const int top = q->nb - 1;
#pragma omp parallel for num_threads(threads) schedule(static) if (threads > 1)
    for (int64_t i = 0; i < q->M; i++) {
        const uint64_t *L = q->L + i * W, *T = q->T + i * W;
        uint64_t *Lo = q->L2 + i * W;
        /* E of the first word (the right neighbour of the last cell) and the
           move mask of the last word (the left neighbour of the first cell) */
        const uint64_t E0 = ~(L[0] | T[0]) & (W == 1 ? q->tail : ~0ull);
        uint64_t Elast = ~(L[W - 1] | T[W - 1]) & q->tail;
        uint64_t Er_last = (Elast >> 1) | ((E0 & 1ull) << top);
        const uint64_t mv_last = L[W - 1] & Er_last;
        uint64_t carry = (mv_last >> top) & 1ull; /* moving car entering cell 0 */
        for (int64_t w = 0; w < W; w++) {
            const uint64_t valid = w == W - 1 ? q->tail : ~0ull;
            const uint64_t E = ~(L[w] | T[w]) & valid;
            uint64_t Er;
            if (w == W - 1) {
                Er = Er_last;
            } else {
                const uint64_t En = ~(L[w + 1] | T[w + 1]) & (w + 1 == W - 1 ? q->tail : ~0ull);
                Er = (E >> 1) | ((En & 1ull) << 63);
            }
            const uint64_t mv = L[w] & Er;
            const uint64_t in = (mv << 1) | carry;
            carry = mv >> 63;
            Lo[w] = (L[w] ^ mv ^ in) & valid;
        }
    }
}

/* vertical phase on every row: T2 from (L2, T) */
static void bits_v(planes_t *q, int threads)
{
    const int64_t W = q->W, M = q->M;
#pragma omp parallel for num_threads(threads) schedule(static) if (threads > 1)
    for (int64_t i = 0; i < M; i++) {
        const int64_t up = (i + M - 1) % M, dn = (i + 1) % M;
        for (int64_t w = 0; w < W; w++) {
            const uint64_t E_dn = ~(q->L2[dn * W + w] | q->T[dn * W + w]);
            const uint64_t E_here = ~(q->L2[i * W + w] | q->T[i * W + w]);
            const uint64_t leave = q->T[i * W + w] & E_dn;
            const uint64_t enter = q->T[up * W + w] & E_here;
            q->T2[i * W + w] = (q->T[i * W + w] & ~leave) | enter;
        }
    }
}

static double run_bits(uint8_t *g, int64_t M, int64_t N, int64_t K, int threads, int *rc)
{
    planes_t q;
    *rc = planes_alloc(&q, M, N);
    if (*rc) {
        planes_free(&q);
        return 0.0;
    }
    for (int64_t i = 0; i < M; i++)
        for (int64_t j = 0; j < N; j++) {
            const uint8_t c = g[i * N + j];
            if (c == LR) q.L[i * q.W + j / 64] |= 1ull << (j % 64);
            if (c == TB) q.T[i * q.W + j / 64] |= 1ull << (j % 64);
        }
    const double t0 = now_s();
    for (int64_t t = 0; t < K; t++) {
        bits_h(&q, threads);
        bits_v(&q, threads);
        uint64_t *x = q.L;
        q.L = q.L2;
        q.L2 = x;
        x = q.T;
        q.T = q.T2;
        q.T2 = x;
    }
    const double dt = now_s() - t0;
    for (int64_t i = 0; i < M; i++)
        for (int64_t j = 0; j < N; j++) {
            const uint64_t b = 1ull << (j % 64);
            const int64_t w = i * q.W + j / 64;
            g[i * N + j] = (q.L[w] & b) ? LR : ((q.T[w] & b) ? TB : EMPTY);
        }
    planes_free(&q);
    return dt;
}

/*
 * Advance g (M*N bytes, 0/1/2, row-major) by K steps with form `impl`
 * (1..5 above) on `threads` threads (forms 1 and 3 use one).  *seconds
 * receives the time of the K steps alone (layout conversions excluded).
 * Returns 0, -1 on bad arguments, -2 if memory is short.
 */
int ladder_run(int impl, uint8_t *g, int64_t M, int64_t N, int64_t K, int threads,
               double *seconds)
{
    if (!g || M <= 0 || N <= 0 || K < 0 || impl < 1 || impl > 5) return -1;
    for (int64_t q = 0; q < M * N; q++)
        if (g[q] > TB) return -1;
    if (threads < 1) threads = 1;
    int rc = 0;
    double dt;
    switch (impl) {
    case 1: dt = run_ghost(g, M, N, K, 1, 0, &rc); break;
    case 2: dt = run_ghost(g, M, N, K, threads, 0, &rc); break;
    case 3: dt = run_ghost(g, M, N, K, 1, 1, &rc); break;
    case 4: dt = run_ghost(g, M, N, K, threads, 1, &rc); break;
    default: dt = run_bits(g, M, N, K, threads, &rc); break;
    }
    if (seconds) *seconds = dt;
    return rc;
}
