"""Thin ctypes binding of libbml (include/bml.h): same names, argument
marshalling only.  Every step of the automaton runs in the CUDA library; if
the library is missing this module raises at import time -- there is no CPU
fallback.

PyTorch's role is limited to device memory and streams: `use_torch_allocator`
routes the library's device allocations through torch's caching allocator,
and `stream=` arguments take a torch.cuda.Stream (or a raw cudaStream_t).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbml.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libbml.so is not built (%s); run `python -m paper_1804_07981_b300.build`" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

BML_OK = 0
BML_EINVAL = -1
BML_ENOMEM = -2
BML_ECUDA = -3
BML_ETIMEOUT = -4
BML_ESTATE = -5

BML_KERNEL_AUTO = 0
BML_KERNEL_BYTE = 1
BML_KERNEL_BITPLANE = 2
BML_KERNEL_FUSED = 3
BML_KERNEL_TBLOCK = 4
BML_KERNEL_RESIDENT = 5

BML_MODEL_I = 1
BML_MODEL_II = 2
BML_MODEL_III = 3

KERNELS = {"auto": BML_KERNEL_AUTO, "byte": BML_KERNEL_BYTE, "bitplane": BML_KERNEL_BITPLANE,
           "fused": BML_KERNEL_FUSED, "tblock": BML_KERNEL_TBLOCK,
           "resident": BML_KERNEL_RESIDENT}

_i64, _u64, _dbl, _int, _vp = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                               ctypes.c_int, ctypes.c_void_p)
_i64p = ctypes.POINTER(ctypes.c_int64)


class BMLError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("bml error %d: %s" % (code, msg))
        self.code = code


def _sig(name, args, res=_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


ALLOC_FN = ctypes.CFUNCTYPE(_vp, ctypes.c_size_t, _vp, _vp)
FREE_FN = ctypes.CFUNCTYPE(None, _vp, ctypes.c_size_t, _vp, _vp)

_lib_set_allocator = _sig("bml_set_allocator", [ALLOC_FN, FREE_FN, _vp])
_lib_create = _sig("bml_create", [_i64, _i64, _u64, _dbl, ctypes.POINTER(_vp)])
_lib_create_ex = _sig("bml_create_ex", [_i64, _i64, _u64, _dbl, _dbl, _int, _int, _vp, _i64,
                                        ctypes.POINTER(_vp)])
_lib_reserve = _sig("bml_reserve_steps", [_vp, _i64])
_lib_step = _sig("bml_step", [_vp, _i64])
_lib_counts = _sig("bml_moved_counts", [_vp, _i64, _i64, _vp, _vp, _vp])
_lib_counts_async = _sig("bml_moved_counts_async", [_vp, _i64, _i64, _vp, _vp])
_lib_read = _sig("bml_read_lattice", [_vp, _vp])
_lib_write = _sig("bml_write_lattice", [_vp, _vp])
_lib_read_dev = _sig("bml_read_lattice_device", [_vp, _vp])
_lib_write_dev = _sig("bml_write_lattice_device", [_vp, _vp])
_lib_steps_done = _sig("bml_steps_done", [_vp], _i64)
_lib_get_config = _sig("bml_get_config", [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int), _i64p])
_lib_set_tiling = _sig("bml_set_tiling", [_vp, _int, _i64])
_lib_set_tiling_ex = _sig("bml_set_tiling_ex", [_vp, _int, _i64, _int])
_lib_get_tiling = _sig("bml_get_tiling", [_vp, ctypes.POINTER(_int), _i64p, ctypes.POINTER(_int)])
_lib_set_resident_blocks = _sig("bml_set_resident_blocks", [_vp, _int])
_lib_set_model = _sig("bml_set_model", [_vp, _int, _u64])
_lib_get_model = _sig("bml_get_model", [_vp, ctypes.POINTER(_int), ctypes.POINTER(_u64)])
_lib_sync = _sig("bml_synchronize", [_vp])
_lib_destroy = _sig("bml_destroy", [_vp], None)
_lib_last_error = _sig("bml_last_error", [], ctypes.c_char_p)


def bml_last_error() -> str:
    return (_lib_last_error() or b"").decode()


def _check(rc: int) -> None:
    if rc != BML_OK:
        raise BMLError(rc, bml_last_error())


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _host_ptr(a: np.ndarray):
    return a.ctypes.data_as(_vp)


# ---------------------------------------------------------------- allocator --
_torch_alloc_refs = None


def use_torch_allocator(enable: bool = True) -> None:
    """Route the library's device allocations through torch's caching
    allocator (objects created afterwards)."""
    global _torch_alloc_refs
    if not enable:
        _check(_lib_set_allocator(ALLOC_FN(), FREE_FN(), None))
        _torch_alloc_refs = None
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            dev = torch.cuda.current_device()
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
        except Exception:  # out of memory -> NULL -> BML_ENOMEM
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    refs = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(_lib_set_allocator(refs[0], refs[1], None))
    _torch_alloc_refs = refs  # keep the callbacks alive


# ---------------------------------------------------------------- functions --
def bml_create(M: int, N: int, seed: int, density: float) -> int:
    out = _vp()
    _check(_lib_create(M, N, seed, density, ctypes.byref(out)))
    return out.value


def bml_create_ex(M: int, N: int, seed: int, p_lr: float, p_tb: float, kernel: int = 0,
                  block_k: int = 0, stream=None, reserve_steps: int = 0) -> int:
    out = _vp()
    _check(_lib_create_ex(M, N, seed, p_lr, p_tb, kernel, block_k, _stream_handle(stream),
                          reserve_steps, ctypes.byref(out)))
    return out.value


def bml_reserve_steps(sim: int, K: int) -> None:
    _check(_lib_reserve(sim, K))


def bml_step(sim: int, k: int) -> None:
    _check(_lib_step(sim, k))


def bml_moved_counts(sim: int, first: int, n: int):
    """Returns (total, lr, tb), each int64[n]."""
    tot = np.zeros(n, dtype=np.int64)
    lr = np.zeros(n, dtype=np.int64)
    tb = np.zeros(n, dtype=np.int64)
    _check(_lib_counts(sim, first, n, _host_ptr(tot), _host_ptr(lr), _host_ptr(tb)))
    return tot, lr, tb


def bml_moved_counts_async(sim: int, first: int, n: int, out_lr: np.ndarray,
                           out_tb: np.ndarray) -> None:
    """Enqueue the LR / TB count copies of steps first+1..first+n into the
    given int64 host arrays (page-locked, e.g. from a pinned torch tensor);
    valid after the stream is synchronised."""
    for a in (out_lr, out_tb):
        if a is not None and (a.dtype != np.int64 or a.size < n or not a.flags.c_contiguous):
            raise ValueError("count arrays must be contiguous int64 with n entries")
    _check(_lib_counts_async(sim, first, n, None if out_lr is None else _host_ptr(out_lr),
                             None if out_tb is None else _host_ptr(out_tb)))


def bml_read_lattice(sim: int, M: int, N: int, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty((M, N), dtype=np.uint8)
    assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size == M * N
    _check(_lib_read(sim, _host_ptr(out)))
    return out


def bml_write_lattice(sim: int, lattice: np.ndarray) -> None:
    a = np.ascontiguousarray(lattice, dtype=np.uint8)
    _check(_lib_write(sim, _host_ptr(a)))


def bml_read_lattice_device(sim: int, d_out: int) -> None:
    _check(_lib_read_dev(sim, d_out))


def bml_write_lattice_device(sim: int, d_in: int) -> None:
    _check(_lib_write_dev(sim, d_in))


def bml_steps_done(sim: int) -> int:
    return int(_lib_steps_done(sim))


def bml_get_config(sim: int):
    k, bk, br = _int(), _int(), _i64()
    _check(_lib_get_config(sim, ctypes.byref(k), ctypes.byref(bk), ctypes.byref(br)))
    return k.value, bk.value, br.value


def bml_set_tiling(sim: int, block_k: int, band_rows: int) -> None:
    _check(_lib_set_tiling(sim, block_k, band_rows))


def bml_set_tiling_ex(sim: int, block_k: int, band_rows: int, lane_words: int) -> None:
    _check(_lib_set_tiling_ex(sim, block_k, band_rows, lane_words))


def bml_set_resident_blocks(sim: int, blocks: int) -> None:
    _check(_lib_set_resident_blocks(sim, blocks))


def bml_get_tiling(sim: int):
    k, lw = _int(), _int()
    b = _i64()
    _check(_lib_get_tiling(sim, ctypes.byref(k), ctypes.byref(b), ctypes.byref(lw)))
    return k.value, b.value, lw.value


def bml_set_model(sim: int, model: int, tie_seed: int = 0) -> None:
    _check(_lib_set_model(sim, model, tie_seed))


def bml_get_model(sim: int):
    m, seed = _int(), _u64()
    _check(_lib_get_model(sim, ctypes.byref(m), ctypes.byref(seed)))
    return m.value, seed.value


def bml_synchronize(sim: int) -> None:
    _check(_lib_sync(sim))


def bml_destroy(sim: int) -> None:
    _lib_destroy(sim)


# ----------------------------------------------------------- convenience --
class Lattice:
    """Owning wrapper of a bml_sim handle."""

    def __init__(self, M: int, N: int, seed: int = 1, density: float | None = None,
                 p_lr: float | None = None, p_tb: float | None = None, kernel="auto",
                 block_k: int = 0, stream=None, reserve_steps: int = 0):
        if density is not None:
            p_lr = p_tb = density / 2
        if p_lr is None or p_tb is None:
            raise ValueError("give density or both p_lr and p_tb")
        kid = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        self.M, self.N = M, N
        self._h = bml_create_ex(M, N, seed, p_lr, p_tb, kid, block_k, stream, reserve_steps)

    @property
    def handle(self) -> int:
        return self._h

    def step(self, k: int = 1) -> None:
        bml_step(self._h, k)

    def moved_counts(self, first: int = 0, n: int | None = None):
        if n is None:
            n = self.steps_done - first
        return bml_moved_counts(self._h, first, n)

    def read(self) -> np.ndarray:
        return bml_read_lattice(self._h, self.M, self.N)

    def write(self, lattice: np.ndarray) -> None:
        if lattice.shape != (self.M, self.N):
            raise ValueError("shape mismatch")
        bml_write_lattice(self._h, lattice)

    @property
    def steps_done(self) -> int:
        return bml_steps_done(self._h)

    @property
    def config(self):
        return bml_get_config(self._h)

    def set_tiling(self, block_k: int, band_rows: int, lane_words: int = 1) -> None:
        if lane_words == 1:
            bml_set_tiling(self._h, block_k, band_rows)
        else:
            bml_set_tiling_ex(self._h, block_k, band_rows, lane_words)

    def set_resident_blocks(self, blocks: int) -> None:
        bml_set_resident_blocks(self._h, blocks)

    @property
    def tiling(self):
        return bml_get_tiling(self._h)

    def set_model(self, model: int, tie_seed: int = 0) -> None:
        """BML_MODEL_I (default) or BML_MODEL_II (one synchronous phase,
        random tie-break seeded by tie_seed)."""
        bml_set_model(self._h, model, tie_seed)

    @property
    def model(self):
        return bml_get_model(self._h)

    def synchronize(self) -> None:
        bml_synchronize(self._h)

    def close(self) -> None:
        if self._h:
            bml_destroy(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------ surrogate network --
_lib_mlp_create = _sig("bml_mlp_create", [_vp, ctypes.POINTER(_vp)])
_lib_mlp_n = _sig("bml_mlp_num_params", [_vp], _i64)
_lib_mlp_set = _sig("bml_mlp_set_params", [_vp, _vp])
_lib_mlp_get = _sig("bml_mlp_get_params", [_vp, _vp])
_lib_mlp_fwd = _sig("bml_mlp_forward", [_vp, _vp, _i64, _vp])
_lib_mlp_train = _sig("bml_mlp_train_step", [_vp, _vp, _vp, _vp, _i64, ctypes.c_float,
                                              ctypes.c_float, _vp])
_lib_mlp_grads = _sig("bml_mlp_grads", [_vp, _vp, _vp, _vp, _i64, _vp, _vp])
_lib_mlp_fit = _sig("bml_mlp_train", [_vp, _vp, _vp, _vp, _i64, _i64, _i64, ctypes.c_float,
                                      ctypes.c_float, ctypes.c_uint64, _vp])
_lib_mlp_apply = _sig("bml_mlp_apply_grads", [_vp, _vp, ctypes.c_float, ctypes.c_float])
_lib_mlp_layer = _sig("bml_mlp_get_layer", [_vp, _int, _vp, _vp, _vp])
_lib_mlp_destroy = _sig("bml_mlp_destroy", [_vp], None)
_lib_gemm = _sig("bml_gemm_bf16", [_vp, _i64, _vp, _i64, _vp, _i64, _i64, _i64, _i64, _vp])
_lib_gemm_ex = _sig("bml_gemm_bf16_ex", [_vp, _i64, _vp, _i64, _vp, _i64, _i64, _i64, _i64,
                                         ctypes.c_uint, _vp])
BML_GEMM_TEST_STALL = 1


def bml_gemm_bf16(A: int, lda: int, B: int, ldb: int, C: int, ldc: int, M: int, N: int, K: int,
                  stream=None) -> None:
    _check(_lib_gemm(A, lda, B, ldb, C, ldc, M, N, K, _stream_handle(stream)))


def bml_gemm_bf16_ex(A: int, lda: int, B: int, ldb: int, C: int, ldc: int, M: int, N: int,
                     K: int, flags: int, stream=None) -> None:
    _check(_lib_gemm_ex(A, lda, B, ldb, C, ldc, M, N, K, flags, _stream_handle(stream)))


class MLP:
    """Owning wrapper of a bml_mlp handle.  Tensors passed to forward /
    train_step are torch CUDA float32 tensors (device memory)."""

    def __init__(self, stream=None):
        out = _vp()
        _check(_lib_mlp_create(_stream_handle(stream), ctypes.byref(out)))
        self._h = out.value
        self.n = int(_lib_mlp_n(self._h))

    def set_params(self, flat: np.ndarray) -> None:
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.n
        _check(_lib_mlp_set(self._h, _host_ptr(a)))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.n, dtype=np.float32)
        _check(_lib_mlp_get(self._h, _host_ptr(a)))
        return a

    def forward(self, x):
        import torch
        x = x.contiguous()
        out = torch.empty((x.shape[0], 2), dtype=torch.float32, device=x.device)
        _check(_lib_mlp_fwd(self._h, x.data_ptr(), x.shape[0], out.data_ptr()))
        return out

    def train_step(self, x, v, jam, lr: float, weight_decay: float = 0.0,
                   want_loss: bool = True):
        """One AdamW step; returns the batch loss before the update, or None
        when want_loss is False (then nothing waits for the device)."""
        loss = ctypes.c_float()
        _check(_lib_mlp_train(self._h, x.contiguous().data_ptr(), v.contiguous().data_ptr(),
                              jam.contiguous().data_ptr(), x.shape[0], lr, weight_decay,
                              ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def train(self, x, v, jam, steps: int, batch: int, lr: float, weight_decay: float = 0.0,
              seed: int = 0, want_losses: bool = True):
        """`steps` AdamW steps on mini-batches drawn on the device from the
        rows of (x, v, jam) (bml_mlp_train); returns every step's loss (numpy
        float32) or None."""
        n = x.shape[0]
        losses = np.empty(max(steps, 0), dtype=np.float32) if want_losses else None
        _check(_lib_mlp_fit(self._h, x.contiguous().data_ptr(), v.contiguous().data_ptr(),
                            jam.contiguous().data_ptr(), n, steps, batch, lr, weight_decay,
                            seed, _host_ptr(losses) if want_losses else None))
        return losses

    def grads(self, x, v, jam):
        g = np.empty(self.n, dtype=np.float32)
        loss = ctypes.c_float()
        _check(_lib_mlp_grads(self._h, x.contiguous().data_ptr(), v.contiguous().data_ptr(),
                              jam.contiguous().data_ptr(), x.shape[0], _host_ptr(g),
                              ctypes.byref(loss)))
        return g, loss.value

    def apply_grads(self, grads: np.ndarray, lr: float, weight_decay: float = 0.0) -> None:
        a = np.ascontiguousarray(grads, dtype=np.float32)
        _check(_lib_mlp_apply(self._h, _host_ptr(a), lr, weight_decay))

    # padded (rows, columns) of each layer's device weight buffers
    PADDED = ((128, 80), (128, 128), (128, 128), (16, 128))

    def layer(self, layer: int):
        """Padded device buffers of one layer (bml_mlp_get_layer): the BF16
        forward copy of W [out_pad][in_pad], its transposed copy and the last
        weight gradient [out_pad][in_pad], as float32 arrays."""
        r, c = self.PADDED[layer]
        W = np.empty((r, c), dtype=np.float32)
        WT = np.empty((c, r), dtype=np.float32)
        gW = np.empty((r, c), dtype=np.float32)
        _check(_lib_mlp_layer(self._h, layer, _host_ptr(W), _host_ptr(WT), _host_ptr(gW)))
        return W, WT, gW

    def close(self) -> None:
        if self._h:
            _lib_mlp_destroy(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------- allocation-free step --
BML_NOALLOC_MAX_BYTES = 16 * 1024 * 1024

_lib_noalloc = _sig("bml_step_bytes_noalloc", [_vp, _i64, _i64, _i64, _vp, _vp, _vp])


def bml_step_bytes_noalloc(d_cells: int, M: int, N: int, k: int, d_moved_lr: int,
                           d_moved_tb: int, stream=None) -> None:
    """Step a caller-owned device lattice (M rows of N rounded up to 16
    bytes) k times without any device allocation; see include/bml.h."""
    _check(_lib_noalloc(d_cells, M, N, k, d_moved_lr, d_moved_tb, _stream_handle(stream)))


# ----------------------------------------------------------------- ensemble --
BML_ENS_EARLY_EXIT = 1
BML_ENS_NO_GRAPH = 2
BML_ENS_TEST_STALL = 4

_lib_ens_create_ex = _sig("bml_ensemble_create_ex", [_i64, _vp, _vp, _vp, _vp, _vp, _int, _i64,
                                                      ctypes.c_uint, _vp, _i64,
                                                      ctypes.POINTER(_vp)])
_lib_ens_create = _sig("bml_ensemble_create", [_i64, _vp, _vp, _vp, _vp, _vp, _vp,
                                                ctypes.POINTER(_vp)])
_lib_ens_step = _sig("bml_ensemble_step", [_vp, _i64])
_lib_ens_counts = _sig("bml_ensemble_moved_counts", [_vp, _i64, _i64, _i64, _vp, _vp, _vp])
_lib_ens_traces = _sig("bml_ensemble_traces", [_vp, _i64, _i64, _vp, _vp])
_lib_ens_jam = _sig("bml_ensemble_jam_steps", [_vp, _vp])
_lib_ens_read1 = _sig("bml_ensemble_read_lattice", [_vp, _i64, _vp])
_lib_ens_read = _sig("bml_ensemble_read_lattices", [_vp, _vp])
_lib_ens_write = _sig("bml_ensemble_write_lattices", [_vp, _vp])
_lib_ens_steps = _sig("bml_ensemble_steps_done", [_vp], _i64)
_lib_ens_cfg = _sig("bml_ensemble_get_config", [_vp, ctypes.POINTER(_int), _i64p,
                                                 ctypes.POINTER(_int)])
_lib_ens_retire = _sig("bml_ensemble_retire", [_vp, _i64, _vp])
_lib_ens_plan = _sig("bml_ensemble_plan", [_i64, _vp, _vp, _i64, _int, _int, _i64p,
                                           ctypes.POINTER(ctypes.c_double), _vp])
_lib_ens_sync = _sig("bml_ensemble_synchronize", [_vp])
_lib_ens_cars = _sig("bml_ensemble_car_counts", [_vp, _vp])
_lib_ens_feat = _sig("bml_ensemble_features", [_vp, _i64, _i64, _int, _vp])
_lib_ens_lab = _sig("bml_ensemble_labels", [_vp, _i64, _vp, _vp])
_lib_ens_destroy = _sig("bml_ensemble_destroy", [_vp], None)


def _arr(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def bml_ensemble_create_ex(M, N, seed, p_lr, p_tb, block_k=0, band_rows=0, flags=0,
                           stream=None, reserve_steps=0) -> int:
    M, N = _arr(M, np.int64), _arr(N, np.int64)
    seed, p_lr, p_tb = _arr(seed, np.uint64), _arr(p_lr, np.float64), _arr(p_tb, np.float64)
    out = _vp()
    _check(_lib_ens_create_ex(len(M), _host_ptr(M), _host_ptr(N), _host_ptr(seed),
                              _host_ptr(p_lr), _host_ptr(p_tb), block_k, band_rows, flags,
                              _stream_handle(stream), reserve_steps, ctypes.byref(out)))
    return out.value


def bml_ensemble_create(M, N, seed, p_lr, p_tb, stream=None) -> int:
    M, N = _arr(M, np.int64), _arr(N, np.int64)
    seed, p_lr, p_tb = _arr(seed, np.uint64), _arr(p_lr, np.float64), _arr(p_tb, np.float64)
    out = _vp()
    _check(_lib_ens_create(len(M), _host_ptr(M), _host_ptr(N), _host_ptr(seed), _host_ptr(p_lr),
                           _host_ptr(p_tb), _stream_handle(stream), ctypes.byref(out)))
    return out.value


def bml_ensemble_step(ens: int, k: int) -> None:
    _check(_lib_ens_step(ens, k))


def bml_ensemble_moved_counts(ens: int, lattice: int, first: int, n: int):
    tot, lr, tb = (np.zeros(n, dtype=np.int64) for _ in range(3))
    _check(_lib_ens_counts(ens, lattice, first, n, _host_ptr(tot), _host_ptr(lr), _host_ptr(tb)))
    return tot, lr, tb


def bml_ensemble_traces(ens: int, count: int, first: int, n: int):
    lr = np.zeros((count, n), dtype=np.int64)
    tb = np.zeros((count, n), dtype=np.int64)
    _check(_lib_ens_traces(ens, first, n, _host_ptr(lr), _host_ptr(tb)))
    return lr, tb


def bml_ensemble_jam_steps(ens: int, count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.int64)
    _check(_lib_ens_jam(ens, _host_ptr(out)))
    return out


def bml_ensemble_read_lattice(ens: int, lattice: int, M: int, N: int) -> np.ndarray:
    out = np.empty((M, N), dtype=np.uint8)
    _check(_lib_ens_read1(ens, lattice, _host_ptr(out)))
    return out


def bml_ensemble_read_lattices(ens: int, total_cells: int) -> np.ndarray:
    out = np.empty(total_cells, dtype=np.uint8)
    _check(_lib_ens_read(ens, _host_ptr(out)))
    return out


def bml_ensemble_write_lattices(ens: int, concatenated: np.ndarray) -> None:
    a = np.ascontiguousarray(concatenated, dtype=np.uint8)
    _check(_lib_ens_write(ens, _host_ptr(a)))


def bml_ensemble_steps_done(ens: int) -> int:
    return int(_lib_ens_steps(ens))


def bml_ensemble_get_config(ens: int):
    k, g = _int(), _int()
    b = _i64()
    _check(_lib_ens_cfg(ens, ctypes.byref(k), ctypes.byref(b), ctypes.byref(g)))
    return k.value, b.value, bool(g.value)


def bml_ensemble_plan(M, N, band: int, depth: int, warps: int):
    """Host-side tile plan of an ensemble (no CUDA call): (tiles, score, rows
    covered per lattice)."""
    Ma = np.ascontiguousarray(M, dtype=np.int64)
    Na = np.ascontiguousarray(N, dtype=np.int64)
    tiles = _i64()
    score = ctypes.c_double()
    rows = np.zeros(Ma.size, dtype=np.int64)
    _check(_lib_ens_plan(Ma.size, _host_ptr(Ma), _host_ptr(Na), band, depth, warps,
                         ctypes.byref(tiles), ctypes.byref(score), _host_ptr(rows)))
    return tiles.value, score.value, rows


def bml_ensemble_synchronize(ens: int) -> None:
    _check(_lib_ens_sync(ens))


def bml_ensemble_destroy(ens: int) -> None:
    _lib_ens_destroy(ens)


class Ensemble:
    """Owning wrapper of a bml_ens handle."""

    def __init__(self, M, N, seed, p_lr, p_tb, block_k=0, band_rows=0, flags=0, stream=None,
                 reserve_steps=0):
        self.M = np.asarray(M, dtype=np.int64)
        self.N = np.asarray(N, dtype=np.int64)
        self.count = len(self.M)
        self.cells = self.M * self.N
        self.offsets = np.concatenate([[0], np.cumsum(self.cells)])
        self._h = bml_ensemble_create_ex(self.M, self.N, seed, p_lr, p_tb, block_k, band_rows,
                                         flags, stream, reserve_steps)

    @property
    def handle(self) -> int:
        return self._h

    def step(self, k: int) -> None:
        bml_ensemble_step(self._h, k)

    @property
    def steps_done(self) -> int:
        return bml_ensemble_steps_done(self._h)

    def traces(self, first: int = 0, n: int | None = None):
        if n is None:
            n = self.steps_done - first
        return bml_ensemble_traces(self._h, self.count, first, n)

    def moved_counts(self, lattice: int, first: int = 0, n: int | None = None):
        if n is None:
            n = self.steps_done - first
        return bml_ensemble_moved_counts(self._h, lattice, first, n)

    def jam_steps(self) -> np.ndarray:
        return bml_ensemble_jam_steps(self._h, self.count)

    def read_all(self) -> list:
        flat = bml_ensemble_read_lattices(self._h, int(self.offsets[-1]))
        return [flat[self.offsets[l]:self.offsets[l + 1]].reshape(self.M[l], self.N[l])
                for l in range(self.count)]

    def read(self, lattice: int) -> np.ndarray:
        return bml_ensemble_read_lattice(self._h, lattice, int(self.M[lattice]),
                                         int(self.N[lattice]))

    def write_all(self, lattices) -> None:
        flat = np.concatenate([np.ascontiguousarray(g, dtype=np.uint8).ravel() for g in lattices])
        bml_ensemble_write_lattices(self._h, flat)

    @property
    def config(self):
        return bml_ensemble_get_config(self._h)

    def retire(self, lattices) -> None:
        """Stop advancing the given lattices (bml_ensemble_retire)."""
        idx = np.ascontiguousarray(lattices, dtype=np.int64)
        _check(_lib_ens_retire(self._h, idx.size, _host_ptr(idx) if idx.size else None))

    def car_counts(self) -> np.ndarray:
        out = np.zeros(self.count, dtype=np.int64)
        _check(_lib_ens_cars(self._h, _host_ptr(out)))
        return out

    def features(self, first: int, n: int, points: int):
        """Device tensor (count, 3 + points) float32 of surrogate inputs."""
        import torch
        out = torch.empty((self.count, 3 + points), dtype=torch.float32, device="cuda")
        _check(_lib_ens_feat(self._h, first, n, points, out.data_ptr()))
        return out

    def labels(self, window: int):
        """Device tensors (v, jam), each (count,) float32."""
        import torch
        v = torch.empty(self.count, dtype=torch.float32, device="cuda")
        jam = torch.empty(self.count, dtype=torch.float32, device="cuda")
        _check(_lib_ens_lab(self._h, window, v.data_ptr(), jam.data_ptr()))
        return v, jam

    def synchronize(self) -> None:
        bml_ensemble_synchronize(self._h)

    def close(self) -> None:
        if self._h:
            bml_ensemble_destroy(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
