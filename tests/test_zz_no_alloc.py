"""The allocation-free byte step (bml_step_bytes_noalloc).

Callers that cannot allocate device memory -- a framework whose own pool owns
every allocation, a recorded pipeline in which an allocation would
synchronise the device, an embedded user with a memory budget fixed at
start-up -- pass their own lattice and count arrays; the library's built-in
16 MiB array holds the lattice between the two phases of a step.  These
tests call the entry point through the C ABI twice in a row on the same
caller-owned lattice and compare lattice and counts, bit for bit, with the
existing byte kernel (which allocates its own buffers).  This file is
collected last so that a run stopping at the first failure has run every
other test first.
"""
import numpy as np
import pytest

from paper_1804_07981_b300.inputs import random_lattice

pytestmark = pytest.mark.gpu


def _pitched(g):
    M, N = g.shape
    pb = (N + 15) // 16 * 16
    out = np.zeros((M, pb), dtype=np.uint8)
    out[:, :N] = g
    return out


@pytest.mark.parametrize("M,N,k1,k2", [(256, 256, 37, 5), (123, 1001, 20, 21), (9, 65, 3, 8)])
def test_noalloc_matches_byte_kernel_on_two_calls(lib, M, N, k1, k2):
    import torch
    g0 = random_lattice(M, N, M * 31 + N, 0.16, 0.17)
    cells = torch.from_numpy(_pitched(g0)).cuda()
    lr = torch.zeros(max(k1, k2), dtype=torch.int64, device="cuda")
    tb = torch.zeros(max(k1, k2), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    with lib.Lattice(M, N, seed=1, density=0.0, kernel="byte") as ref:
        ref.write(g0)
        for k in (k1, k2):
            lr.fill_(-1)
            tb.fill_(-1)
            lib.bml_step_bytes_noalloc(cells.data_ptr(), M, N, k, lr.data_ptr(), tb.data_ptr(),
                                       stream)
            first = ref.steps_done
            ref.step(k)
            torch.cuda.synchronize()
            got = cells.cpu().numpy()
            np.testing.assert_array_equal(got[:, :N], ref.read())
            assert not got[:, N:].any()  # row padding untouched
            _, rlr, rtb = ref.moved_counts(first, k)
            np.testing.assert_array_equal(lr[:k].cpu().numpy(), rlr)
            np.testing.assert_array_equal(tb[:k].cpu().numpy(), rtb)


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
    with pytest.raises(lib.BMLError) as e:
        lib.bml_step_bytes_noalloc(buf.data_ptr() + 8, 4, 16, 1, cnt.data_ptr(), cnt.data_ptr())
    assert e.value.code == lib.BML_EINVAL
    with pytest.raises(lib.BMLError):
        lib.bml_step_bytes_noalloc(0, 4, 16, 1, cnt.data_ptr(), cnt.data_ptr())
