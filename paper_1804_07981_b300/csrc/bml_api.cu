// C ABI of the single-lattice simulator (declared in include/bml.h).
//
// Host-side logic only: argument checks, device memory, the count history,
// dispatch of the step kernels and the autotuner.  Every step of the
// automaton runs in the kernels of the other translation units.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/bml.h"
#include "bml_internal.cuh"

using namespace bml;

// ---------------------------------------------------------------- errors --
static thread_local std::string g_last_error;

static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(BML_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,    \
                  __LINE__);                                                                 \
  } while (0)

extern "C" const char *bml_last_error(void) { return g_last_error.c_str(); }

void bml::set_last_error(const char *msg) { g_last_error = msg; }

// ------------------------------------------------------------- allocator --
namespace {

struct Allocator {
  bml_alloc_fn alloc = nullptr;
  bml_free_fn free_fn = nullptr;
  void *ctx = nullptr;
};

std::mutex g_alloc_mu;
Allocator g_alloc;

struct DevBuf {
  void *ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace

extern "C" int bml_set_allocator(bml_alloc_fn alloc, bml_free_fn free_fn, void *ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(BML_EINVAL, "bml_set_allocator: alloc and free must both be set or both NULL");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.free_fn = free_fn;
  g_alloc.ctx = ctx;
  return BML_OK;
}

// ------------------------------------------------------------------ sim --
// Longest launch (in steps) the autotuner times; its count scratch holds
// this many LR and TB counts.
constexpr int kTuneSteps = 64;

struct bml_sim {
  Geom g;
  int kernel = BML_KERNEL_AUTO;
  int block_k = 1;
  int64_t band_rows = 0;
  int lane_words = 1;  // streaming kernel: 64-cell words per lane (1 or 2); 0: resident kernel
  int model = BML_MODEL_I;
  u64 tie_seed = 0;  // Model II tie-break generator state
  cudaStream_t st = nullptr;
  Allocator alloc;
  // state: bitplane kernels use L[cur], T[cur]; the byte kernel uses c[0]
  // (c[1] holds the lattice between the two phases of a step)
  DevBuf planes[2];  // each: L then T, M*P words apiece
  DevBuf bytes[2];
  int cur = 0;
  bool pair_layout = false;  // planes[cur] in the interleaved layout (else plain)
  DevBuf counts;  // cap u64 LR counts, then cap u64 TB counts
  int64_t cap = 0;
  int64_t steps_done = 0;
  DevBuf flag;     // one int for value checks
  DevBuf scratch;  // kTuneSteps LR then kTuneSteps TB counts for autotuning launches
};

namespace {

int dev_alloc(bml_sim *s, DevBuf &b, size_t bytes) {
  b.bytes = bytes;
  b.ptr = nullptr;
  if (bytes == 0) return BML_OK;
  if (s->alloc.alloc) {
    b.ptr = s->alloc.alloc(bytes, (void *)s->st, s->alloc.ctx);
    if (!b.ptr) return fail(BML_ENOMEM, "allocator returned NULL for %zu bytes", bytes);
    if ((uintptr_t)b.ptr % 256)
      return fail(BML_EINVAL, "allocator returned a pointer not aligned to 256 bytes");
  } else {
    cudaError_t e = cudaMalloc(&b.ptr, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b.ptr = nullptr;
      return fail(BML_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
  }
  cudaError_t e = cudaMemsetAsync(b.ptr, 0, bytes, s->st);
  if (e != cudaSuccess) return fail(BML_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  return BML_OK;
}

void dev_free(bml_sim *s, DevBuf &b) {
  if (!b.ptr) return;
  if (s->alloc.free_fn)
    s->alloc.free_fn(b.ptr, b.bytes, (void *)s->st, s->alloc.ctx);
  else
    cudaFree(b.ptr);
  b.ptr = nullptr;
  b.bytes = 0;
}

void free_all(bml_sim *s) {
  cudaStreamSynchronize(s->st);
  for (int i = 0; i < 2; ++i) {
    dev_free(s, s->planes[i]);
    dev_free(s, s->bytes[i]);
  }
  dev_free(s, s->counts);
  dev_free(s, s->flag);
  dev_free(s, s->scratch);
}

inline u64 *plane_L(bml_sim *s, int i) { return (u64 *)s->planes[i].ptr; }
inline u64 *plane_T(bml_sim *s, int i) { return (u64 *)s->planes[i].ptr + s->g.M * s->g.P; }
inline u64 *cnt_lr(bml_sim *s) { return (u64 *)s->counts.ptr; }
inline u64 *cnt_tb(bml_sim *s) { return (u64 *)s->counts.ptr + s->cap; }

bool uses_planes(int kernel) { return kernel != BML_KERNEL_BYTE; }

int check_shape(int64_t M, int64_t N) {
  if (M < 1 || N < 1) return fail(BML_EINVAL, "M and N must be >= 1 (got %lld x %lld)",
                                  (long long)M, (long long)N);
  if (M > INT32_MAX || N > INT32_MAX || (double)M * (double)N > 137438953472.0)
    return fail(BML_EINVAL, "lattice %lld x %lld too large (M, N < 2^31, M*N <= 2^37)",
                (long long)M, (long long)N);
  return BML_OK;
}

int grow_counts(bml_sim *s, int64_t need) {
  if (need <= s->cap) return BML_OK;
  int64_t ncap = s->cap > 0 ? s->cap : 4096;
  while (ncap < need) ncap *= 2;
  DevBuf nb;
  int rc = dev_alloc(s, nb, (size_t)ncap * 2 * sizeof(u64));
  if (rc) return rc;
  if (s->counts.ptr && s->steps_done > 0) {
    const size_t n = (size_t)s->steps_done * sizeof(u64);
    CUDA_TRY(cudaMemcpyAsync(nb.ptr, cnt_lr(s), n, cudaMemcpyDeviceToDevice, s->st));
    CUDA_TRY(cudaMemcpyAsync((u64 *)nb.ptr + ncap, cnt_tb(s), n, cudaMemcpyDeviceToDevice, s->st));
  }
  dev_free(s, s->counts);
  s->counts = nb;
  s->cap = ncap;
  return BML_OK;
}

// Bring the current planes into the layout the next kernel reads: the
// interleaved one for the two-words-per-lane kernel of Models I and III, the
// plain one for every other kernel and for unpacking (one in-place pass).
int set_layout(bml_sim *s, bool pair) {
  if (s->pair_layout == pair) return BML_OK;
  CUDA_TRY(launch_pair_layout(plane_L(s, s->cur), plane_T(s, s->cur), s->g, pair, s->st));
  s->pair_layout = pair;
  return BML_OK;
}

// Enqueue `k` steps with the configured model and kernel.  lr/tb point at
// the count slots of the first step, whose index is t0 (Model II tie-breaks).
int enqueue_steps(bml_sim *s, int64_t k, u64 *lr, u64 *tb, bool commit, int64_t t0 = 0) {
  const Geom &g = s->g;
  if (uses_planes(s->kernel)) {
    const bool pair = s->model != BML_MODEL_II && s->lane_words == 2 && s->band_rows != 0 &&
                      s->kernel != BML_KERNEL_BITPLANE;
    int rc = set_layout(s, pair);
    if (rc) return rc;
  }
  if (s->model == BML_MODEL_II) {
    int64_t done = 0;
    while (done < k) {
      int d = s->block_k;
      while (d > k - done) d >>= 1;
      const int a = s->cur, b = 1 - s->cur;
      if (s->lane_words == 2)
        CUDA_TRY(launch_stream2(plane_L(s, a), plane_T(s, a), plane_L(s, b), plane_T(s, b), g, d,
                                s->band_rows, lr + done, tb + done, s->st, 2, s->tie_seed,
                                (u64)(t0 + done)));
      else
        CUDA_TRY(launch_model2(plane_L(s, a), plane_T(s, a), plane_L(s, b), plane_T(s, b), g, d,
                               s->band_rows, s->tie_seed, (u64)(t0 + done), lr + done,
                               tb + done, s->st));
      if (commit) s->cur = b;
      done += d;
    }
    return BML_OK;
  }
  const bool m3 = s->model == BML_MODEL_III;
  if (m3 && (s->kernel == BML_KERNEL_BYTE || s->kernel == BML_KERNEL_BITPLANE ||
             s->lane_words == 0 || s->band_rows == 0))
    return fail(BML_ESTATE, "Model III runs on the streaming kernels only");
  if (s->kernel == BML_KERNEL_BYTE) {
    uint8_t *c0 = (uint8_t *)s->bytes[0].ptr, *c1 = (uint8_t *)s->bytes[1].ptr;
    for (int64_t t = 0; t < k; ++t) {
      CUDA_TRY(launch_byte_h(c0, c1, g, lr + t, s->st));
      CUDA_TRY(launch_byte_v(c1, c0, g, tb + t, s->st));
    }
    return BML_OK;
  }
  if (s->kernel == BML_KERNEL_BITPLANE) {
    for (int64_t t = 0; t < k; ++t) {
      const int a = s->cur, b = 1 - s->cur;
      CUDA_TRY(launch_plane_h(plane_L(s, a), plane_T(s, a), plane_L(s, b), g, lr + t, s->st));
      CUDA_TRY(launch_plane_v(plane_L(s, b), plane_T(s, a), plane_T(s, b), g, tb + t, s->st));
      if (commit) s->cur = b;
    }
    return BML_OK;
  }
  // lane_words == 0: the resident kernel, up to resident_max_steps() per launch
  if (s->lane_words == 0) {
    int64_t done = 0;
    while (done < k) {
      const int d = (int)std::min<int64_t>(k - done, resident_max_steps());
      const int a = s->cur, b = 1 - s->cur;
      CUDA_TRY(launch_resident(plane_L(s, a), plane_T(s, a), plane_L(s, b), plane_T(s, b), g, d,
                               s->band_rows, lr + done, tb + done, s->st));
      if (commit) s->cur = b;
      done += d;
    }
    return BML_OK;
  }
  // band_rows == 0: the direct one-pass fused kernel, one launch per step
  if (s->band_rows == 0) {
    for (int64_t t = 0; t < k; ++t) {
      const int a = s->cur, b = 1 - s->cur;
      CUDA_TRY(launch_fused_direct(plane_L(s, a), plane_T(s, a), plane_L(s, b), plane_T(s, b),
                                   g, lr + t, tb + t, s->st));
      if (commit) s->cur = b;
    }
    return BML_OK;
  }
  // streaming kernels: depth block_k, remainder by powers of two
  int64_t done = 0;
  while (done < k) {
    int d = s->block_k;
    while (d > k - done) d >>= 1;
    const int a = s->cur, b = 1 - s->cur;
    if (s->lane_words == 2)
      CUDA_TRY(launch_stream2(plane_L(s, a), plane_T(s, a), plane_L(s, b), plane_T(s, b), g, d,
                              s->band_rows, lr + done, tb + done, s->st, m3 ? 3 : 1));
    else
      CUDA_TRY(launch_stream(plane_L(s, a), plane_T(s, a), plane_L(s, b), plane_T(s, b), g, d,
                             s->band_rows, lr + done, tb + done, s->st, m3));
    if (commit) s->cur = b;
    done += d;
  }
  return BML_OK;
}

int64_t default_band(const Geom &g) { return g.M < 256 ? g.M : 256; }

// ------------------------------------------------------------ autotuner --
struct TuneKey {
  int64_t M, N;
  int dev;
  int model;
  bool operator<(const TuneKey &o) const {
    return std::tie(M, N, dev, model) < std::tie(o.M, o.N, o.dev, o.model);
  }
};
std::mutex g_tune_mu;
struct Tiling {
  int k;
  int64_t band;
  int lane_words;
};
std::map<TuneKey, Tiling> g_tune_cache;

int autotune(bml_sim *s) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  const TuneKey key{s->g.M, s->g.N, dev, s->model};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      s->block_k = it->second.k;
      s->band_rows = it->second.band;
      s->lane_words = it->second.lane_words;
      return BML_OK;
    }
  }
  // candidates: the direct fused kernel (depth 1, no bands), then the
  // streaming kernel at each depth with fixed band heights and with band
  // heights that make the tile count fill 1..4 whole waves of resident warps
  int sms = 148;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const bool m2 = s->model == BML_MODEL_II, m1 = s->model == BML_MODEL_I;
  std::vector<Tiling> cands;
  if (m1) cands.push_back({1, 0, 1});  // Models II and III have no one-pass kernel
  // the resident kernel, timed on 64-step launches (a call runs all its steps in one):
  // the lattice in one block, or split over a cluster of 2, 4 or 8 blocks (Model I)
  if (m1 && resident_applies(s->g)) {
    for (int64_t blocks : {1, 2, 4, 8}) {
      if (blocks > s->g.M) break;
      cands.push_back({kTuneSteps, (s->g.M + blocks - 1) / blocks, 0});
    }
  }
  for (int lw : {1, 2}) {
    if (lw == 2 && !stream2_applies(s->g)) continue;
    for (int k : {1, 2, 4, 8}) {
      std::vector<int64_t> bands;
      for (int64_t b : {16, 32, 64, 128, 256, 512, 1024}) bands.push_back(b);
      int wpb = 4;
      const int per_sm = lw == 2 ? stream2_occupancy(k, m2 ? 2 : 1)
                                 : (m2 ? model2_occupancy(s->g, k)
                                       : stream_occupancy(s->g, k, &wpb));
      const int64_t resident = (int64_t)sms * per_sm * wpb;
      const int64_t strips = lw == 2 ? 0 : make_strip_plan(s->g, k).n_strips;
      for (int waves = 1; waves <= 4; ++waves) {
        const int64_t nb = lw == 2 ? stream2_bands_for_tiles(s->g, k, resident * waves)
                                   : resident * waves / strips;
        if (nb >= 1) bands.push_back((s->g.M + nb - 1) / nb);
      }
      std::sort(bands.begin(), bands.end());
      bands.erase(std::unique(bands.begin(), bands.end()), bands.end());
      for (int64_t b : bands) {
        if (b < 2 * k && b < s->g.M) continue;  // halo work would dominate
        cands.push_back({k, b >= s->g.M ? s->g.M : b, lw});
        if (b >= s->g.M) break;
      }
    }
  }
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  const int saved_k = s->block_k;
  const int64_t saved_b = s->band_rows;
  const int saved_lw = s->lane_words;
  double best = 1e30;
  int best_k = 1, best_lw = 1;
  int64_t best_b = m1 ? 0 : default_band(s->g);
  const double cells = (double)s->g.M * (double)s->g.N;
  const int reps = cells > 1e8 ? 3 : (cells > 1e6 ? 10 : 20);
  int rc = BML_OK;
  // pass 1: every candidate, few repetitions; pass 2: the best four again
  // with more repetitions, so that near-ties are decided by a steadier time
  std::vector<std::pair<double, size_t>> scored;
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<size_t> which;
    if (pass == 0) {
      for (size_t i = 0; i < cands.size(); ++i) which.push_back(i);
    } else {
      std::sort(scored.begin(), scored.end());
      for (size_t i = 0; i < scored.size() && i < 4; ++i) which.push_back(scored[i].second);
      scored.clear();
    }
    const int r = pass == 0 ? reps : 3 * reps;
    for (size_t ci : which) {
      const Tiling &c = cands[ci];
      s->block_k = c.k;
      s->band_rows = c.band;
      s->lane_words = c.lane_words;
      if (c.k > kTuneSteps) {
        rc = fail(BML_EINVAL, "autotune: candidate depth %d exceeds the count scratch", c.k);
        goto done;
      }
      u64 *lr = (u64 *)s->scratch.ptr, *tb = lr + kTuneSteps;
      // warm-up (non-committing: reads cur, writes the other buffer)
      if ((rc = enqueue_steps(s, c.k, lr, tb, false))) goto done;
      cudaEventRecord(e0, s->st);
      for (int q = 0; q < r; ++q)
        if ((rc = enqueue_steps(s, c.k, lr, tb, false))) goto done;
      cudaEventRecord(e1, s->st);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = fail(BML_ECUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
        goto done;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      const double per_step = (double)ms / (r * c.k);
      scored.push_back({per_step, ci});
      if (pass == 1 && per_step < best) {
        best = per_step;
        best_k = c.k;
        best_b = c.band;
        best_lw = c.lane_words;
      }
    }
  }
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    s->block_k = saved_k;
    s->band_rows = saved_b;
    s->lane_words = saved_lw;
    return rc;
  }
  if (best_lw == 0) best_k = 0;  // resident: every step of a call in one launch
  s->block_k = best_k;
  s->band_rows = best_b;
  s->lane_words = best_lw;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = {best_k, best_b, best_lw};
  return BML_OK;
}

}  // namespace

// ------------------------------------------------------------- creation --
extern "C" int bml_create_ex(int64_t M, int64_t N, uint64_t seed, double p_lr, double p_tb,
                             int kernel, int block_k, void *stream, int64_t reserve_steps,
                             bml_sim **out) {
  if (!out) return fail(BML_EINVAL, "out is NULL");
  int rc = check_shape(M, N);
  if (rc) return rc;
  if (!(p_lr >= 0.0 && p_tb >= 0.0 && p_lr + p_tb <= 1.0))
    return fail(BML_EINVAL, "need p_lr >= 0, p_tb >= 0, p_lr + p_tb <= 1 (got %g, %g)", p_lr,
                p_tb);
  if (kernel < BML_KERNEL_AUTO || kernel > BML_KERNEL_RESIDENT)
    return fail(BML_EINVAL, "unknown kernel %d", kernel);
  if (kernel == BML_KERNEL_RESIDENT && !resident_applies(make_geom(M, N)))
    return fail(BML_EINVAL, "lattice %lld x %lld does not fit one block's shared memory",
                (long long)M, (long long)N);
  if (kernel == BML_KERNEL_TBLOCK) {
    if (block_k == 0) block_k = 4;
    if (block_k != 1 && block_k != 2 && block_k != 4 && block_k != 8)
      return fail(BML_EINVAL, "block_k must be 1, 2, 4 or 8 (got %d)", block_k);
  }
  if (reserve_steps < 0) return fail(BML_EINVAL, "reserve_steps < 0");

  bml_sim *s = new (std::nothrow) bml_sim;
  if (!s) return fail(BML_ENOMEM, "host allocation failed");
  s->g = make_geom(M, N);
  s->kernel = kernel;
  s->block_k = kernel == BML_KERNEL_TBLOCK ? block_k : (kernel == BML_KERNEL_RESIDENT ? 0 : 1);
  s->band_rows = kernel == BML_KERNEL_FUSED ? 0 : default_band(s->g);
  if (kernel == BML_KERNEL_RESIDENT) {
    s->band_rows = s->g.M;
    s->lane_words = 0;
  }
  s->st = (cudaStream_t)stream;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    s->alloc = g_alloc;
  }
  const Geom &g = s->g;
  const u64 t_lr = placement_threshold(p_lr), t_tb = placement_threshold(p_tb);
  if (uses_planes(kernel)) {
    for (int i = 0; i < 2; ++i)
      if ((rc = dev_alloc(s, s->planes[i], (size_t)(2 * g.M * g.P) * sizeof(u64)))) goto fail_;
    if (launch_init_planes(plane_L(s, 0), plane_T(s, 0), g, seed, t_lr, t_tb, s->st) !=
        cudaSuccess) {
      rc = fail(BML_ECUDA, "init kernel: %s", cudaGetErrorString(cudaGetLastError()));
      goto fail_;
    }
  } else {
    for (int i = 0; i < 2; ++i)
      if ((rc = dev_alloc(s, s->bytes[i], (size_t)(g.M * g.PB)))) goto fail_;
    if (launch_init_bytes((uint8_t *)s->bytes[0].ptr, g, seed, t_lr, t_tb, s->st) !=
        cudaSuccess) {
      rc = fail(BML_ECUDA, "init kernel: %s", cudaGetErrorString(cudaGetLastError()));
      goto fail_;
    }
  }
  if ((rc = dev_alloc(s, s->flag, 256))) goto fail_;
  if ((rc = dev_alloc(s, s->scratch, 2 * kTuneSteps * sizeof(u64)))) goto fail_;
  if ((rc = grow_counts(s, reserve_steps > 0 ? reserve_steps : 4096))) goto fail_;
  if (kernel == BML_KERNEL_AUTO) {
    if ((rc = autotune(s))) goto fail_;
  }
  if (cudaStreamSynchronize(s->st) != cudaSuccess) {
    rc = fail(BML_ECUDA, "create: %s", cudaGetErrorString(cudaGetLastError()));
    goto fail_;
  }
  *out = s;
  return BML_OK;
fail_:
  free_all(s);
  delete s;
  return rc;
}

extern "C" int bml_create(int64_t M, int64_t N, uint64_t seed, double density, bml_sim **out) {
  if (!(density >= 0.0 && density <= 1.0))
    return fail(BML_EINVAL, "density must be in [0, 1] (got %g)", density);
  return bml_create_ex(M, N, seed, density / 2, density / 2, BML_KERNEL_AUTO, 0, nullptr, 0,
                       out);
}

extern "C" void bml_destroy(bml_sim *s) {
  if (!s) return;
  free_all(s);
  delete s;
}

// ---------------------------------------------------------------- steps --
extern "C" int bml_reserve_steps(bml_sim *s, int64_t K) {
  if (!s) return fail(BML_EINVAL, "sim is NULL");
  if (K < 0) return fail(BML_EINVAL, "K < 0");
  return grow_counts(s, K);
}

extern "C" int bml_step(bml_sim *s, int64_t k) {
  if (!s) return fail(BML_EINVAL, "sim is NULL");
  if (k < 0) return fail(BML_EINVAL, "k < 0");
  if (k == 0) return BML_OK;
  int rc = grow_counts(s, s->steps_done + k);
  if (rc) return rc;
  rc = enqueue_steps(s, k, cnt_lr(s) + s->steps_done, cnt_tb(s) + s->steps_done, true,
                     s->steps_done);
  if (rc) return rc;
  s->steps_done += k;
  return BML_OK;
}

extern "C" int64_t bml_steps_done(const bml_sim *s) { return s ? s->steps_done : -1; }

extern "C" int bml_get_config(const bml_sim *s, int *kernel, int *block_k, int64_t *band_rows) {
  if (!s) return fail(BML_EINVAL, "sim is NULL");
  if (kernel) {
    *kernel = s->kernel;
    if (s->kernel == BML_KERNEL_AUTO)
      *kernel = s->lane_words == 0 ? BML_KERNEL_RESIDENT
                                   : (s->band_rows == 0 ? BML_KERNEL_FUSED : BML_KERNEL_TBLOCK);
  }
  if (block_k) *block_k = s->block_k;
  if (band_rows) *band_rows = s->band_rows;
  return BML_OK;
}

extern "C" int bml_set_tiling_ex(bml_sim *s, int block_k, int64_t band_rows, int lane_words) {
  if (!s) return fail(BML_EINVAL, "sim is NULL");
  if (lane_words != 1 && lane_words != 2) return fail(BML_EINVAL, "lane_words must be 1 or 2");
  if (lane_words == 2 && (!stream2_applies(s->g) || band_rows == 0))
    return fail(BML_EINVAL, "two words per lane need N %% 64 == 0, an even number of words "
                "per row, more than 32 of them, and band_rows >= 1");
  int rc = bml_set_tiling(s, block_k, band_rows);
  if (rc) return rc;
  s->lane_words = lane_words;
  return BML_OK;
}

extern "C" int bml_get_tiling(const bml_sim *s, int *block_k, int64_t *band_rows,
                              int *lane_words) {
  if (!s) return fail(BML_EINVAL, "sim is NULL");
  if (block_k) *block_k = s->block_k;
  if (band_rows) *band_rows = s->band_rows;
  if (lane_words) *lane_words = s->lane_words;
  return BML_OK;
}

extern "C" int bml_set_tiling(bml_sim *s, int block_k, int64_t band_rows) {
  if (!s) return fail(BML_EINVAL, "sim is NULL");
  if (!uses_planes(s->kernel) || s->kernel == BML_KERNEL_BITPLANE ||
      s->kernel == BML_KERNEL_RESIDENT)
    return fail(BML_EINVAL, "tiling applies to the streaming bitplane kernels only");
  if (block_k != 1 && block_k != 2 && block_k != 4 && block_k != 8)
    return fail(BML_EINVAL, "block_k must be 1, 2, 4 or 8 (got %d)", block_k);
  if (s->kernel == BML_KERNEL_FUSED && (block_k != 1 || band_rows != 0))
    return fail(BML_EINVAL, "the fused kernel runs one step per launch without bands");
  if (band_rows < 0 || band_rows > INT32_MAX || (band_rows == 0 && block_k != 1))
    return fail(BML_EINVAL, "bad band_rows (0 selects the direct one-pass kernel, depth 1)");
  if (band_rows == 0 && s->model != BML_MODEL_I)
    return fail(BML_EINVAL, "Models II and III have no one-pass kernel (band_rows >= 1)");
  s->block_k = block_k;
  s->band_rows = band_rows;
  s->lane_words = 1;
  return BML_OK;
}

extern "C" int bml_set_resident_blocks(bml_sim *s, int blocks) {
  if (!s) return fail(BML_EINVAL, "sim is NULL");
  if (s->lane_words != 0)
    return fail(BML_EINVAL, "the object does not run the resident kernel");
  if (blocks != 1 && blocks != 2 && blocks != 4 && blocks != 8)
    return fail(BML_EINVAL, "blocks must be 1, 2, 4 or 8 (got %d)", blocks);
  if (blocks > s->g.M)
    return fail(BML_EINVAL, "%d blocks need at least as many rows (M = %lld)", blocks,
                (long long)s->g.M);
  s->band_rows = (s->g.M + blocks - 1) / blocks;
  return BML_OK;
}

extern "C" int bml_set_model(bml_sim *s, int model, uint64_t tie_seed) {
  if (!s) return fail(BML_EINVAL, "sim is NULL");
  if (model != BML_MODEL_I && model != BML_MODEL_II && model != BML_MODEL_III)
    return fail(BML_EINVAL, "unknown model %d", model);
  if (model != BML_MODEL_I && s->kernel != BML_KERNEL_TBLOCK && s->kernel != BML_KERNEL_AUTO)
    return fail(BML_EINVAL, "Models II and III need an object created with BML_KERNEL_TBLOCK "
                "or AUTO");
  if (model != BML_MODEL_I && s->kernel == BML_KERNEL_TBLOCK && s->band_rows == 0)
    return fail(BML_EINVAL, "Models II and III have no one-pass kernel (band_rows >= 1)");
  if (s->model == BML_MODEL_III && model != BML_MODEL_III) {
    // Models I and II have no doubly occupied cells
    int *flag = (int *)s->flag.ptr;
    int h = 0;
    CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s->st));
    CUDA_TRY(launch_find_overlap(plane_L(s, s->cur), plane_T(s, s->cur), s->g, flag, s->st));
    CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    CUDA_TRY(cudaStreamSynchronize(s->st));
    if (h)
      return fail(BML_ESTATE, "the lattice holds doubly occupied cells (Model III only)");
  }
  const int old_model = s->model, old_k = s->block_k, old_lw = s->lane_words;
  const int64_t old_b = s->band_rows;
  const u64 old_seed = s->tie_seed;
  s->model = model;
  s->tie_seed = tie_seed;
  int rc = BML_OK;
  if (s->kernel == BML_KERNEL_AUTO) rc = autotune(s);  // TBLOCK keeps the caller's tiling
  if (!rc && cudaStreamSynchronize(s->st) != cudaSuccess)
    rc = fail(BML_ECUDA, "set_model: %s", cudaGetErrorString(cudaGetLastError()));
  if (rc) {
    s->model = old_model;
    s->tie_seed = old_seed;
    s->block_k = old_k;
    s->band_rows = old_b;
    s->lane_words = old_lw;
  }
  return rc;
}

extern "C" int bml_get_model(const bml_sim *s, int *model, uint64_t *tie_seed) {
  if (!s) return fail(BML_EINVAL, "sim is NULL");
  if (model) *model = s->model;
  if (tie_seed) *tie_seed = s->tie_seed;
  return BML_OK;
}

extern "C" int bml_synchronize(bml_sim *s) {
  if (!s) return fail(BML_EINVAL, "sim is NULL");
  CUDA_TRY(cudaStreamSynchronize(s->st));
  return BML_OK;
}

extern "C" int bml_moved_counts(bml_sim *s, int64_t first, int64_t n, int64_t *out_total,
                                int64_t *out_lr, int64_t *out_tb) {
  if (!s) return fail(BML_EINVAL, "sim is NULL");
  if (first < 0 || n < 0 || first + n > s->steps_done)
    return fail(BML_EINVAL, "count range [%lld, %lld) outside [0, %lld)", (long long)first,
                (long long)(first + n), (long long)s->steps_done);
  if (n == 0) return BML_OK;
  std::vector<int64_t> lr((size_t)n), tb((size_t)n);
  CUDA_TRY(cudaMemcpyAsync(lr.data(), cnt_lr(s) + first, (size_t)n * 8, cudaMemcpyDeviceToHost,
                           s->st));
  CUDA_TRY(cudaMemcpyAsync(tb.data(), cnt_tb(s) + first, (size_t)n * 8, cudaMemcpyDeviceToHost,
                           s->st));
  CUDA_TRY(cudaStreamSynchronize(s->st));
  for (int64_t t = 0; t < n; ++t) {
    if (out_lr) out_lr[t] = lr[(size_t)t];
    if (out_tb) out_tb[t] = tb[(size_t)t];
    if (out_total) out_total[t] = lr[(size_t)t] + tb[(size_t)t];
  }
  return BML_OK;
}

namespace {
// Device address of page-locked host memory that was allocated or registered
// on the current device and is mapped into its address space, else NULL
// (pageable memory, device memory, memory of another device's context).
int64_t *device_view(int64_t *host) {
  cudaPointerAttributes a;
  int dev = 0;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer || a.device != dev) return nullptr;
  return (int64_t *)a.devicePointer;
}
}  // namespace

extern "C" int bml_moved_counts_async(bml_sim *s, int64_t first, int64_t n, int64_t *out_lr,
                                      int64_t *out_tb) {
  if (!s) return fail(BML_EINVAL, "sim is NULL");
  if (first < 0 || n < 0 || first + n > s->steps_done)
    return fail(BML_EINVAL, "count range [%lld, %lld) outside [0, %lld)", (long long)first,
                (long long)(first + n), (long long)s->steps_done);
  if (n == 0) return BML_OK;
  // Page-locked host arrays that the device can address are written by a
  // small dependent kernel (no copy-engine round trip between two step
  // kernels); other host memory goes through cudaMemcpyAsync.
  int64_t *d_lr = nullptr, *d_tb = nullptr;
  const bool mapped = (!out_lr || (d_lr = device_view(out_lr))) &&
                      (!out_tb || (d_tb = device_view(out_tb)));
  if (mapped) {
    CUDA_TRY(launch_copy_counts(cnt_lr(s) + first, cnt_tb(s) + first, n, d_lr, d_tb, s->st));
    return BML_OK;
  }
  if (out_lr)
    CUDA_TRY(cudaMemcpyAsync(out_lr, cnt_lr(s) + first, (size_t)n * 8, cudaMemcpyDeviceToHost,
                             s->st));
  if (out_tb)
    CUDA_TRY(cudaMemcpyAsync(out_tb, cnt_tb(s) + first, (size_t)n * 8, cudaMemcpyDeviceToHost,
                             s->st));
  return BML_OK;
}

// -------------------------------------------------------- lattice I/O --
namespace {

// Enqueue: current state -> bytes with pitch PB in `dst` (device).
int state_to_pitched(bml_sim *s, uint8_t *dst) {
  if (uses_planes(s->kernel)) {
    int rc = set_layout(s, false);
    if (rc) return rc;
    CUDA_TRY(launch_unpack(plane_L(s, s->cur), plane_T(s, s->cur), dst, s->g, s->st));
  } else {
    CUDA_TRY(cudaMemcpyAsync(dst, s->bytes[0].ptr, (size_t)(s->g.M * s->g.PB),
                             cudaMemcpyDeviceToDevice, s->st));
  }
  return BML_OK;
}

int read_impl(bml_sim *s, uint8_t *out, cudaMemcpyKind kind) {
  const Geom &g = s->g;
  const uint8_t *src = nullptr;
  DevBuf stage;
  int rc;
  if (uses_planes(s->kernel)) {
    if ((rc = dev_alloc(s, stage, (size_t)(g.M * g.PB)))) return rc;
    if ((rc = state_to_pitched(s, (uint8_t *)stage.ptr))) {
      dev_free(s, stage);
      return rc;
    }
    src = (const uint8_t *)stage.ptr;
  } else {
    src = (const uint8_t *)s->bytes[0].ptr;
  }
  cudaError_t e = cudaMemcpy2DAsync(out, (size_t)g.N, src, (size_t)g.PB, (size_t)g.N,
                                    (size_t)g.M, kind, s->st);
  if (kind == cudaMemcpyDeviceToHost && e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  dev_free(s, stage);  // stream-ordered for allocator frees; cudaFree syncs
  if (e != cudaSuccess) return fail(BML_ECUDA, "read lattice: %s", cudaGetErrorString(e));
  return BML_OK;
}

int write_impl(bml_sim *s, const uint8_t *in, cudaMemcpyKind kind) {
  const Geom &g = s->g;
  int rc;
  DevBuf stage;
  uint8_t *dst;
  const int other = 1 - s->cur;
  if (uses_planes(s->kernel)) {
    if ((rc = dev_alloc(s, stage, (size_t)(g.M * g.PB)))) return rc;  // zeroed padding
    dst = (uint8_t *)stage.ptr;
  } else {
    dst = (uint8_t *)s->bytes[1].ptr;  // padding bytes of the byte buffers stay 0
  }
  int *bad = (int *)s->flag.ptr;
  int hbad = 0;
  cudaError_t e = cudaMemcpy2DAsync(dst, (size_t)g.PB, in, (size_t)g.N, (size_t)g.N,
                                    (size_t)g.M, kind, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s->st);
  if (e == cudaSuccess) {
    if (uses_planes(s->kernel))
      e = launch_pack(dst, plane_L(s, other), plane_T(s, other), g, bad, s->st,
                      s->model == BML_MODEL_III ? 3 : 2);
    else
      e = launch_check_bytes(dst, g, bad, s->st);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  dev_free(s, stage);
  if (e != cudaSuccess) return fail(BML_ECUDA, "write lattice: %s", cudaGetErrorString(e));
  if (hbad) {
    if (!uses_planes(s->kernel)) {
      // the rejected bytes sit in the scratch half of the byte state; the
      // lattice itself (bytes[0]) is untouched
    }
    return fail(BML_EINVAL, "lattice holds a value other than 0, 1, 2");
  }
  if (uses_planes(s->kernel)) {
    s->cur = other;
    s->pair_layout = false;  // packed in the plain layout
  } else {
    void *t = s->bytes[0].ptr;
    s->bytes[0].ptr = s->bytes[1].ptr;
    s->bytes[1].ptr = t;
  }
  // new trajectory: clear the count history
  CUDA_TRY(cudaMemsetAsync(s->counts.ptr, 0, s->counts.bytes, s->st));
  s->steps_done = 0;
  return BML_OK;
}

}  // namespace

extern "C" int bml_read_lattice(bml_sim *s, uint8_t *out) {
  if (!s || !out) return fail(BML_EINVAL, "NULL argument");
  return read_impl(s, out, cudaMemcpyDeviceToHost);
}

extern "C" int bml_read_lattice_device(bml_sim *s, uint8_t *d_out) {
  if (!s || !d_out) return fail(BML_EINVAL, "NULL argument");
  return read_impl(s, d_out, cudaMemcpyDeviceToDevice);
}

extern "C" int bml_write_lattice(bml_sim *s, const uint8_t *in) {
  if (!s || !in) return fail(BML_EINVAL, "NULL argument");
  return write_impl(s, in, cudaMemcpyHostToDevice);
}

extern "C" int bml_write_lattice_device(bml_sim *s, const uint8_t *d_in) {
  if (!s || !d_in) return fail(BML_EINVAL, "NULL argument");
  return write_impl(s, d_in, cudaMemcpyDeviceToDevice);
}
