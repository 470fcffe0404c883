// Lattice set-up and I/O kernels: seeded placement, byte <-> bitplane
// conversion, the copy of moved counts into host-mapped memory.
//
// Placement (Sec. 2 of the paper only says vehicles are placed at random):
// cell (i, j) draws u = SplitMix64 output n = i*N + j + 1 from state `seed`
// (Steele, Lea, Flood, OOPSLA 2014: state_n = seed + n * golden gamma, output
// = the variant-13 mix of state_n); LR if u < t_lr, TB if u - t_lr < t_tb,
// else EMPTY.
#include <cmath>

#include "device_common.cuh"

namespace bml {

Geom make_geom(int64_t M, int64_t N) {
  Geom g;
  g.M = M;
  g.N = N;
  g.W = (N + 63) / 64;
  g.P = (g.W + 1) & ~int64_t(1);
  g.PB = (N + 15) & ~int64_t(15);
  g.nb = (int32_t)(N - 64 * (g.W - 1));
  g.tail = g.nb == 64 ? ~0ull : ((1ull << g.nb) - 1ull);
  return g;
}

u64 placement_threshold(double p) {
  const double x = std::ldexp(p, 64);
  if (!(x > 0.0)) return 0;
  if (x >= 18446744073709551616.0) return ~0ull;
  return (u64)x;
}

// 0 EMPTY, 1 LR, 2 TB
__device__ __forceinline__ uint32_t place(u64 seed, u64 n, u64 t_lr, u64 t_tb) {
  const u64 u = splitmix64_at(seed, n);
  if (u < t_lr) return 1u;
  return (u - t_lr < t_tb) ? 2u : 0u;
}

// One thread per word of both planes.
__global__ void init_planes_kernel(u64 *__restrict__ L, u64 *__restrict__ T, Geom g, u64 seed,
                                   u64 t_lr, u64 t_tb) {
  const int64_t total = g.M * g.P;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / g.P, w = idx - i * g.P;
    u64 l = 0, t = 0;
    if (w < g.W) {
      const int nbits = w == g.W - 1 ? g.nb : 64;
      const u64 base = (u64)(i * g.N + 64 * w) + 1ull;
      for (int b = 0; b < nbits; ++b) {
        const uint32_t c = place(seed, base + (u64)b, t_lr, t_tb);
        l |= (u64)(c & 1u) << b;
        t |= (u64)(c >> 1) << b;
      }
    }
    L[idx] = l;
    T[idx] = t;
  }
}

// One thread per 16-byte chunk of the byte layout.
__global__ void init_bytes_kernel(uint8_t *__restrict__ c, Geom g, u64 seed, u64 t_lr,
                                  u64 t_tb) {
  const int64_t nq = g.PB / 16, total = g.M * nq;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / nq, q = idx - i * nq;
    uint32_t v[4] = {0, 0, 0, 0};
    for (int b = 0; b < 16; ++b) {
      const int64_t j = 16 * q + b;
      if (j < g.N) v[b >> 2] |= place(seed, (u64)(i * g.N + j) + 1ull, t_lr, t_tb) << (8 * (b & 3));
    }
    *reinterpret_cast<uint4 *>(c + i * g.PB + 16 * q) = make_uint4(v[0], v[1], v[2], v[3]);
  }
}

// bytes -> planes.  One thread per word; reads the word's 64 bytes as up to
// four 16-byte chunks that lie inside the row pitch.
__global__ void pack_kernel(const uint8_t *__restrict__ c, u64 *__restrict__ L,
                            u64 *__restrict__ T, Geom g, int *bad, uint32_t max_value) {
  const int64_t total = g.M * g.P;
  int badl = 0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / g.P, w = idx - i * g.P;
    u64 l = 0, t = 0;
    for (int q = 0; q < 4; ++q) {
      const int64_t off = 64 * w + 16 * q;
      if (off >= g.PB) break;
      const uint4 v = *reinterpret_cast<const uint4 *>(c + i * g.PB + off);
      const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
      for (int b = 0; b < 16; ++b) {
        const int64_t j = off + b;
        if (j >= g.N) break;
        const uint32_t x = (vv[b >> 2] >> (8 * (b & 3))) & 0xffu;
        badl |= x > max_value;
        l |= (u64)(x & 1u) << (16 * q + b);
        t |= (u64)((x >> 1) & 1u) << (16 * q + b);
      }
    }
    L[idx] = l;
    T[idx] = t;
  }
  if (badl) atomicOr(bad, 1);
}

// planes -> bytes.  One thread per 16-byte chunk.
__global__ void unpack_kernel(const u64 *__restrict__ L, const u64 *__restrict__ T,
                              uint8_t *__restrict__ c, Geom g) {
  const int64_t nq = g.PB / 16, total = g.M * nq;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / nq, q = idx - i * nq;
    const int64_t w = q >> 2;
    const int sh = 16 * (int)(q & 3);
    const uint32_t l = (uint32_t)(L[i * g.P + w] >> sh) & 0xffffu;
    const uint32_t t = (uint32_t)(T[i * g.P + w] >> sh) & 0xffffu;
    uint32_t v[4] = {0, 0, 0, 0};
    for (int b = 0; b < 16; ++b) {
      const uint32_t x = ((l >> b) & 1u) | (((t >> b) & 1u) << 1);
      v[b >> 2] |= x << (8 * (b & 3));
    }
    *reinterpret_cast<uint4 *>(c + i * g.PB + 16 * q) = make_uint4(v[0], v[1], v[2], v[3]);
  }
}

__global__ void check_bytes_kernel(const uint8_t *__restrict__ c, Geom g, int *bad) {
  const int64_t nq = g.PB / 16, total = g.M * nq;
  int badl = 0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / nq, q = idx - i * nq;
    const uint4 v = *reinterpret_cast<const uint4 *>(c + i * g.PB + 16 * q);
    const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
    for (int b = 0; b < 16; ++b) {
      if (16 * q + b >= g.N) break;
      badl |= ((vv[b >> 2] >> (8 * (b & 3))) & 0xffu) > 2u;
    }
  }
  if (badl) atomicOr(bad, 1);
}

static int grid_for(int64_t items, int threads) {
  int64_t blocks = (items + threads - 1) / threads;
  const int64_t cap = 148ll * 32;  // grid-stride loops cover the rest
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

cudaError_t launch_init_planes(u64 *L, u64 *T, const Geom &g, u64 seed, u64 t_lr, u64 t_tb,
                               cudaStream_t st) {
  init_planes_kernel<<<grid_for(g.M * g.P, 256), 256, 0, st>>>(L, T, g, seed, t_lr, t_tb);
  return cudaGetLastError();
}

cudaError_t launch_init_bytes(uint8_t *c, const Geom &g, u64 seed, u64 t_lr, u64 t_tb,
                              cudaStream_t st) {
  init_bytes_kernel<<<grid_for(g.M * (g.PB / 16), 256), 256, 0, st>>>(c, g, seed, t_lr, t_tb);
  return cudaGetLastError();
}

// any word with a cell set in both planes raises the flag
__global__ void find_overlap_kernel(const u64 *__restrict__ L, const u64 *__restrict__ T,
                                    int64_t words, int *flag) {
  int hit = 0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < words;
       q += (int64_t)gridDim.x * blockDim.x)
    hit |= (L[q] & T[q]) != 0ull;
  if (__any_sync(0xffffffffu, hit) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

cudaError_t launch_find_overlap(const u64 *L, const u64 *T, const Geom &g, int *flag,
                                cudaStream_t st) {
  find_overlap_kernel<<<grid_for(g.M * g.P, 256), 256, 0, st>>>(L, T, g.M * g.P, flag);
  return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t *c, u64 *L, u64 *T, const Geom &g, int *bad,
                        cudaStream_t st, int max_value) {
  pack_kernel<<<grid_for(g.M * g.P, 256), 256, 0, st>>>(c, L, T, g, bad, (uint32_t)max_value);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const u64 *L, const u64 *T, uint8_t *c, const Geom &g,
                          cudaStream_t st) {
  unpack_kernel<<<grid_for(g.M * (g.PB / 16), 256), 256, 0, st>>>(L, T, c, g);
  return cudaGetLastError();
}

cudaError_t launch_check_bytes(const uint8_t *c, const Geom &g, int *bad, cudaStream_t st) {
  check_bytes_kernel<<<grid_for(g.M * (g.PB / 16), 256), 256, 0, st>>>(c, g, bad);
  return cudaGetLastError();
}

namespace {

// Moved counts of n steps -> page-locked host arrays reached through their
// device mapping (PCIe writes from the kernel).  Launched as a dependent of
// the step kernels (waits for them to complete), so the next step kernel's
// launch still overlaps this one's.
__global__ void copy_counts_kernel(const u64 *__restrict__ lr, const u64 *__restrict__ tb,
                                   int64_t n, int64_t *dlr, int64_t *dtb) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (dlr) dlr[i] = (int64_t)lr[i];
    if (dtb) dtb[i] = (int64_t)tb[i];
  }
  pdl_release();
}

}  // namespace

cudaError_t launch_copy_counts(const u64 *lr, const u64 *tb, int64_t n, int64_t *dlr,
                               int64_t *dtb, cudaStream_t st) {
  const int64_t blocks64 = (n + 255) / 256;
  const unsigned blocks = (unsigned)(blocks64 < 1 ? 1 : (blocks64 > 148 ? 148 : blocks64));
  return launch_pdl(copy_counts_kernel, dim3(blocks), dim3(256), 0, st, lr, tb, n, dlr, dtb);
}

}  // namespace bml
