"""The C-ABI library loads on a machine without a GPU, exports every
function include/bml.h declares, and rejects invalid arguments before any
CUDA call (CPU only)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(bml_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["bml_create", "bml_create_ex", "bml_step", "bml_moved_counts",
                     "bml_read_lattice", "bml_write_lattice", "bml_destroy",
                     "bml_last_error", "bml_steps_done"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (bml_\w+)", out))
    assert set(declared_functions()) <= exported


@pytest.mark.parametrize("args", [
    (0, 10, 1, 0.1, 0.1), (10, 0, 1, 0.1, 0.1), (10, 10, 1, -0.1, 0.1),
    (10, 10, 1, 0.6, 0.5), (1 << 31, 10, 1, 0.1, 0.1), (1 << 20, 1 << 20, 1, 0.1, 0.1),
    (10, 10, 1, float("nan"), 0.1),
])
def test_create_rejects_bad_arguments(lib, args):
    with pytest.raises(lib.BMLError) as e:
        lib.bml_create_ex(*args)
    assert e.value.code == lib.BML_EINVAL
    assert lib.bml_last_error()


def test_create_rejects_bad_kernel_and_depth(lib):
    with pytest.raises(lib.BMLError) as e:
        lib.bml_create_ex(8, 8, 1, 0.1, 0.1, kernel=9)
    assert e.value.code == lib.BML_EINVAL
    with pytest.raises(lib.BMLError) as e:            # far too large for one block
        lib.bml_create_ex(4096, 4096, 1, 0.1, 0.1, kernel=lib.BML_KERNEL_RESIDENT, block_k=0)
    assert e.value.code == lib.BML_EINVAL
    with pytest.raises(lib.BMLError) as e:
        lib.bml_create_ex(8, 8, 1, 0.1, 0.1, kernel=lib.BML_KERNEL_TBLOCK, block_k=3)
    assert e.value.code == lib.BML_EINVAL
    with pytest.raises(lib.BMLError):
        lib.bml_create(8, 8, 1, 1.5)


def test_null_handles_are_rejected(lib):
    with pytest.raises(lib.BMLError):
        lib.bml_step(None, 1)
    with pytest.raises(lib.BMLError):
        lib.bml_moved_counts(None, 0, 1)
    assert lib.bml_steps_done(None) == -1
    with pytest.raises(lib.BMLError) as e:
        lib.bml_set_model(None, lib.BML_MODEL_II, 1)
    assert e.value.code == lib.BML_EINVAL
    with pytest.raises(lib.BMLError):
        lib.bml_get_model(None)
    lib.bml_destroy(None)


def test_allocation_failure_reports_enomem(lib):
    """An allocator that refuses memory makes creation fail with BML_ENOMEM
    (no CUDA call precedes the first allocation, so this runs on CPU)."""
    calls = []

    @lib.ALLOC_FN
    def refuse(nbytes, stream, ctx):
        calls.append(nbytes)
        return None

    @lib.FREE_FN
    def never(ptr, nbytes, stream, ctx):
        raise AssertionError("nothing was allocated")

    lib._check(lib._lib_set_allocator(refuse, never, None))
    try:
        with pytest.raises(lib.BMLError) as e:
            lib.bml_create_ex(64, 64, 1, 0.1, 0.1, kernel=lib.BML_KERNEL_FUSED)
        assert e.value.code == lib.BML_ENOMEM
        assert len(calls) == 1
    finally:
        lib.use_torch_allocator(False)


def test_set_allocator_needs_both_functions(lib):
    @lib.ALLOC_FN
    def a(nbytes, stream, ctx):
        return None
    with pytest.raises(lib.BMLError):
        lib._check(lib._lib_set_allocator(a, lib.FREE_FN(), None))


def test_mlp_train_rejects_bad_arguments_before_any_cuda_call(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    f = so.bml_mlp_train
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_float,
                  ctypes.c_float, ctypes.c_uint64, ctypes.c_void_p]
    assert f(None, 1, 1, 1, 10, 1, 8, 1e-3, 0.0, 1, None) == lib.BML_EINVAL
    assert f(1, None, 1, 1, 10, 1, 8, 1e-3, 0.0, 1, None) == lib.BML_EINVAL


def test_gemm_rejects_unknown_flags_before_any_cuda_call(lib):
    with pytest.raises(lib.BMLError) as e:
        lib.bml_gemm_bf16_ex(16, 64, 16, 64, 16, 32, 256, 32, 64, 1 << 7)
    assert e.value.code == lib.BML_EINVAL
