// A byte-per-cell step for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they want to step a
// lattice: code running inside a framework that owns every allocation
// through its own pool, code recorded into a pipeline where an allocation
// would synchronise the device, or embedded users with a fixed memory
// budget decided at start-up.  bml_step_bytes_noalloc serves them: the
// caller passes the lattice and the count arrays, and the one buffer the
// step needs besides them -- the lattice between the horizontal and the
// vertical phase -- is a fixed array compiled into this library.
//
// The array is a file-scope __device__ variable, so every GPU on which the
// library's device code is loaded holds its 16 MiB until the process exits.
// Host code cannot use the array's name as a device address (on the host it
// names a host-side shadow); the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on that device.
#include <mutex>

#include "../../include/bml.h"
#include "bml_internal.cuh"

namespace {

constexpr size_t kScratchBytes = BML_NOALLOC_MAX_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

int noalloc_fail(int code, const char *msg) {
  bml::set_last_error(msg);
  return code;
}

// Device address of the scratch array on the current device (set-up on the
// first call per device).
int scratch_address(uint8_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(BML_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(BML_EINVAL, "bml_step_bytes_noalloc: device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return noalloc_fail(BML_ECUDA, "bml_step_bytes_noalloc: cudaGetSymbolAddress failed");
    }
    g_noalloc_addr[dev] = p;
  }
  *out = (uint8_t *)g_noalloc_addr[dev];
  return BML_OK;
}

}  // namespace

extern "C" int bml_step_bytes_noalloc(uint8_t *d_cells, int64_t M, int64_t N, int64_t k,
                                      int64_t *d_moved_lr, int64_t *d_moved_tb, void *stream) {
  if (!d_cells || !d_moved_lr || !d_moved_tb)
    return noalloc_fail(BML_EINVAL, "bml_step_bytes_noalloc: NULL pointer");
  if (M < 1 || N < 1 || k < 0)
    return noalloc_fail(BML_EINVAL, "bml_step_bytes_noalloc: need M >= 1, N >= 1, k >= 0");
  if ((uintptr_t)d_cells % 16)
    return noalloc_fail(BML_EINVAL, "bml_step_bytes_noalloc: lattice not 16-byte aligned");
  const bml::Geom g = bml::make_geom(M, N);
  if (M > INT32_MAX || (double)M * (double)g.PB > (double)kScratchBytes)
    return noalloc_fail(BML_EINVAL,
                        "bml_step_bytes_noalloc: M * pitch exceeds the 16 MiB scratch "
                        "(BML_NOALLOC_MAX_BYTES); use bml_create_ex with BML_KERNEL_BYTE");
  uint8_t *scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  if (k == 0) return BML_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // the counts are accumulated with atomics: they must start at zero
  cudaError_t e = cudaMemsetAsync(d_moved_lr, 0, (size_t)k * sizeof(int64_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_moved_tb, 0, (size_t)k * sizeof(int64_t), st);
  for (int64_t t = 0; t < k && e == cudaSuccess; ++t) {
    // the horizontal phase overwrites every byte of the scratch rows it uses
    // before the vertical phase reads them, so nothing left there by an
    // earlier call is ever read
    e = bml::launch_byte_h(d_cells, scratch, g, (bml::u64 *)(d_moved_lr + t), st);
    if (e == cudaSuccess)
      e = bml::launch_byte_v(scratch, d_cells, g, (bml::u64 *)(d_moved_tb + t), st, true);
  }
  if (e != cudaSuccess) return noalloc_fail(BML_ECUDA, cudaGetErrorString(e));
  return BML_OK;
}
