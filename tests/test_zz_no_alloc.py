"""The allocation-free byte step (bml_step_bytes_noalloc).

Callers that cannot allocate device memory -- a framework whose own pool owns
every allocation, a recorded pipeline in which an allocation would
synchronise the device, an embedded user with a memory budget fixed at
start-up -- pass their own lattice and count arrays; the library's built-in
16 MiB array holds the lattice between the two phases of a step.  These
tests call the entry point through the C ABI twice in a row on the same
caller-owned lattice and compare lattice and counts, bit for bit, with the
oracle and with the existing byte kernel (which allocates its own buffers).
The row padding (bytes past column N) is filled with bytes that differ from
row to row, TB-like values above empty ones included, and must come back
unchanged.  This file is collected last so that a run stopping at the first
failure has run every other test first.
"""
import numpy as np
import pytest

import oracle
from paper_1804_07981_b300.inputs import random_lattice

pytestmark = pytest.mark.gpu


def _pitched(g, seed):
    """Rows of g padded to a multiple of 16 bytes; the padding holds bytes
    drawn per row from {0, 1, 2, 0xFF}, so a TB-like byte often sits above a
    zero one in the next row."""
    M, N = g.shape
    pb = (N + 15) // 16 * 16
    rng = np.random.Generator(np.random.PCG64(seed))
    out = rng.choice(np.array([0, 1, 2, 0xFF], dtype=np.uint8), size=(M, pb))
    out[:, :N] = g
    return out


def _two_calls(lib, M, N, ks, seed, density=0.33, check_byte_kernel=True):
    import torch
    g0 = random_lattice(M, N, seed, density / 2, density / 2)
    host = _pitched(g0, seed + 7)
    pad = host[:, N:].copy()
    cells = torch.from_numpy(host).cuda()
    kmax = max(ks)
    lr = torch.zeros(kmax, dtype=torch.int64, device="cuda")
    tb = torch.zeros(kmax, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    want = g0
    ref = None
    if check_byte_kernel:
        ref = lib.Lattice(M, N, seed=1, density=0.0, kernel="byte")
        ref.write(g0)
    try:
        for k in ks:
            lr.fill_(-1)
            tb.fill_(-1)
            lib.bml_step_bytes_noalloc(cells.data_ptr(), M, N, k, lr.data_ptr(),
                                       tb.data_ptr(), stream)
            torch.cuda.synchronize()
            got = cells.cpu().numpy()
            want, wlr, wtb = oracle.run(want, k, threads=8)
            np.testing.assert_array_equal(got[:, :N], want)
            np.testing.assert_array_equal(got[:, N:], pad)  # padding left as it was
            np.testing.assert_array_equal(lr[:k].cpu().numpy(), wlr)
            np.testing.assert_array_equal(tb[:k].cpu().numpy(), wtb)
            if ref is not None:
                first = ref.steps_done
                ref.step(k)
                np.testing.assert_array_equal(got[:, :N], ref.read())
                _, rlr, rtb = ref.moved_counts(first, k)
                np.testing.assert_array_equal(lr[:k].cpu().numpy(), rlr)
                np.testing.assert_array_equal(tb[:k].cpu().numpy(), rtb)
    finally:
        if ref is not None:
            ref.close()


@pytest.mark.parametrize("M,N,k1,k2", [(256, 256, 37, 5), (123, 1001, 20, 21), (9, 65, 3, 8),
                                       (40, 3, 11, 12), (17, 1, 4, 5)])
def test_noalloc_matches_oracle_on_two_calls(lib, M, N, k1, k2):
    _two_calls(lib, M, N, (k1, k2), M * 31 + N)


def test_noalloc_at_the_size_limit(lib):
    # M * PB == BML_NOALLOC_MAX_BYTES exactly: 4096 rows of pitch 4096 with
    # 6 padding bytes per row
    M, N = 4096, 4090
    assert M * ((N + 15) // 16 * 16) == lib.BML_NOALLOC_MAX_BYTES
    _two_calls(lib, M, N, (3, 2), 99, check_byte_kernel=False)


def test_noalloc_rejects_oversize_and_misaligned(lib):
    import torch
    buf = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    limit = lib.BML_NOALLOC_MAX_BYTES
    # 4097 rows of 4096 bytes is one row more than the built-in array holds
    with pytest.raises(lib.BMLError) as e:
        lib.bml_step_bytes_noalloc(buf.data_ptr(), limit // 4096 + 1, 4096, 1, cnt.data_ptr(),
                                   cnt.data_ptr())
    assert e.value.code == lib.BML_EINVAL and "16 MiB" in str(e.value)
    # one byte more per row than the limit allows (pitch 4112 at 4096 rows)
    with pytest.raises(lib.BMLError) as e:
        lib.bml_step_bytes_noalloc(buf.data_ptr(), 4096, 4097, 1, cnt.data_ptr(),
                                   cnt.data_ptr())
    assert e.value.code == lib.BML_EINVAL
    with pytest.raises(lib.BMLError) as e:
        lib.bml_step_bytes_noalloc(buf.data_ptr() + 8, 4, 16, 1, cnt.data_ptr(), cnt.data_ptr())
    assert e.value.code == lib.BML_EINVAL
    with pytest.raises(lib.BMLError):
        lib.bml_step_bytes_noalloc(0, 4, 16, 1, cnt.data_ptr(), cnt.data_ptr())
