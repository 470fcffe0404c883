"""GPU parity of the surrogate network (tcgen05 tensor-core GEMMs, BF16
operands, FP32 accumulation) against the fp64 oracle on the same
BF16-rounded weights and inputs."""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_1804_07981_b300.inputs import mlp_init_params

pytestmark = pytest.mark.gpu

IN = 67


@pytest.mark.parametrize("M,N,K", [(128, 128, 128), (1, 16, 16), (200, 48, 80), (384, 128, 640),
                                   (77, 16, 1024), (128, 80, 256)])
def test_gemm_matches_matmul(lib, M, N, K):
    import torch
    g = torch.Generator().manual_seed(M * 1000 + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    lib.bml_gemm_bf16(A.data_ptr(), K, B.data_ptr(), K, C.data_ptr(), N, M, N, K)
    want = A.double().cpu() @ B.double().cpu().T
    # fp32 accumulation of exact bf16 products
    assert torch.allclose(C.double().cpu(), want, rtol=1e-4, atol=1e-3 * np.sqrt(K))


def test_gemm_padded_leading_dims_and_many_tiles(lib):
    """Row strides above K (lda, ldb, ldc), a ragged last row tile and K
    not a multiple of the 64-element stage; then 1100 row tiles."""
    import torch
    for M, N, K, lda, ldb, ldc in [(300, 32, 96, 120, 104, 37), (140800, 128, 128, 128, 128, 128)]:
        g = torch.Generator().manual_seed(M + N + K)
        A = torch.randn(M, lda, generator=g).to(torch.bfloat16).cuda()
        B = torch.randn(N, ldb, generator=g).to(torch.bfloat16).cuda()
        C = torch.full((M, ldc), float("nan"), dtype=torch.float32, device="cuda")
        lib.bml_gemm_bf16(A.data_ptr(), lda, B.data_ptr(), ldb, C.data_ptr(), ldc, M, N, K)
        want = A[:, :K].double() @ B[:, :K].double().T
        got = C[:, :N].double()
        assert torch.allclose(got, want, rtol=1e-4, atol=1e-3 * np.sqrt(K))
        if ldc > N:
            assert torch.isnan(C[:, N:]).all()  # nothing written past column N


def _batch(B, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(0, 1, size=(B, IN))
    v = rng.uniform(0, 1, size=B)
    jam = (rng.uniform(size=B) < 0.4).astype(np.float64)
    return x, v, jam


def _rounded_params(seed):
    flat = mlp_init_params(IN, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    ps = ref.unflatten(flat, IN)
    for p in ps[1::2]:
        p += rng.normal(0, 0.05, size=p.shape)
    return ref.bf16_round(ref.flatten(ps))


@pytest.mark.parametrize("B", [1, 100, 128, 300])
def test_forward_matches_oracle(lib, B):
    import torch
    flat = _rounded_params(11)
    x, v, jam = _batch(B, 12)
    xr = ref.bf16_round(x)
    net = lib.MLP()
    net.set_params(flat.astype(np.float32))
    out = net.forward(torch.tensor(xr, dtype=torch.float32, device="cuda")).cpu().numpy()
    want, _ = ref.forward(ref.unflatten(flat, IN), xr)
    err = np.abs(out - want).max() / np.abs(want).max()
    assert err <= 1e-2, err
    # every element, not only the largest deviation (activations are BF16
    # between layers on the device, fp64 in the oracle)
    np.testing.assert_allclose(out, want, rtol=2e-2, atol=2e-2 * np.abs(want).max())
    net.close()


@pytest.mark.parametrize("B", [64, 256, 1000])
def test_gradients_match_oracle(lib, B):
    import torch
    flat = _rounded_params(21)
    x, v, jam = _batch(B, 22)
    xr = ref.bf16_round(x)
    net = lib.MLP()
    net.set_params(flat.astype(np.float32))
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    g, loss = net.grads(t(xr), t(v), t(jam))
    ps = ref.unflatten(flat, IN)
    want, want_loss = ref.backward(ps, xr, v, jam)
    assert abs(loss - want_loss) <= 1e-2 * abs(want_loss)
    gs = ref.unflatten(g.astype(np.float64), IN)
    for i, (a, w) in enumerate(zip(gs, want)):
        # every element of every tensor ...
        np.testing.assert_allclose(a, w, rtol=3e-2, atol=3e-2 * np.abs(w).max(),
                                   err_msg="tensor %d" % i)
        # ... and the tensor as a whole
        a, w = a.ravel(), w.ravel()
        cos = a @ w / (np.linalg.norm(a) * np.linalg.norm(w) + 1e-30)
        rel = np.linalg.norm(a - w) / (np.linalg.norm(w) + 1e-30)
        assert cos >= 0.999 and rel <= 2e-2, (i, cos, rel)
    # the padded device gradients hold the same values, and zeros in the
    # padding (input columns 67..79 of layer 0, output rows 2..15 of layer 3)
    for l in range(4):
        _, _, gW = net.layer(l)
        o, k = want[2 * l].shape
        np.testing.assert_array_equal(gW[:o, :k], gs[2 * l].astype(np.float32))
        assert not gW[o:, :].any() and not gW[:, k:].any(), l
    net.close()


def _check_padded_weights(net, flat):
    """The BF16 forward and transposed weight copies equal the master
    weights rounded to BF16, and every padding entry is exactly 0."""
    ps = ref.unflatten(flat.astype(np.float64), IN)
    for l in range(4):
        W, WT, _ = net.layer(l)
        o, k = ps[2 * l].shape
        np.testing.assert_array_equal(W[:o, :k], ref.bf16_round(ps[2 * l]).astype(np.float32))
        np.testing.assert_array_equal(WT, W.T)
        assert not W[o:, :].any() and not W[:, k:].any(), l


def test_padding_stays_zero_through_updates(lib):
    """After set_params, after AdamW steps with caller gradients and after
    on-device training, the padded weight copies hold BF16(master) in their
    [out][in] corner and 0 elsewhere."""
    import torch
    flat = _rounded_params(51)
    net = lib.MLP()
    net.set_params(flat.astype(np.float32))
    _check_padded_weights(net, net.get_params())
    rng = np.random.Generator(np.random.PCG64(52))
    for _ in range(3):
        net.apply_grads(rng.normal(0, 1e-2, size=flat.size).astype(np.float32), lr=1e-2,
                        weight_decay=0.01)
    _check_padded_weights(net, net.get_params())
    x, v, jam = _batch(300, 53)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    net.train(t(x), t(v), t(jam), 25, 128, lr=1e-2, weight_decay=1e-3, seed=7)
    _check_padded_weights(net, net.get_params())
    net.close()


def test_adamw_matches_oracle(lib):
    flat = _rounded_params(31)
    rng = np.random.Generator(np.random.PCG64(32))
    net = lib.MLP()
    net.set_params(flat.astype(np.float32))
    opt = ref.AdamW(flat.size)
    w = flat.astype(np.float32).astype(np.float64)
    for step in range(3):
        g = rng.normal(0, 1e-2, size=flat.size).astype(np.float32)
        net.apply_grads(g, lr=1e-3, weight_decay=0.01)
        w = opt.step(w, g.astype(np.float64), lr=1e-3, wd=0.01)
    got = net.get_params().astype(np.float64)
    assert np.max(np.abs(got - w)) <= 1e-6
    net.close()


def test_training_reduces_loss(lib):
    """A few hundred AdamW steps on a smooth synthetic target drive the loss
    well below its starting value (the update path works end to end)."""
    import torch
    rng = np.random.Generator(np.random.PCG64(41))
    B = 512
    x = rng.uniform(0, 1, size=(B, IN))
    v = 0.5 * x[:, 0] + 0.3 * x[:, 5] ** 2
    jam = (x[:, 1] + x[:, 2] > 1.0).astype(np.float64)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    net = lib.MLP()
    net.set_params(mlp_init_params(IN, 42).astype(np.float32))
    X, V, J = t(x), t(v), t(jam)
    first = net.train_step(X, V, J, lr=1e-3)
    for _ in range(300):
        last = net.train_step(X, V, J, lr=1e-3)
    assert last < 0.25 * first, (first, last)
    net.close()


def test_training_without_loss_readback_updates_identically(lib):
    """Steps that do not report their loss (nothing waits for the device)
    apply bit for bit the same updates as steps that do."""
    import torch
    rng = np.random.Generator(np.random.PCG64(43))
    B = 256
    x = rng.uniform(0, 1, size=(B, IN))
    v = 0.4 * x[:, 3]
    jam = (x[:, 4] > 0.5).astype(np.float64)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    X, V, J = t(x), t(v), t(jam)
    params = []
    for want in (True, False):
        net = lib.MLP()
        net.set_params(mlp_init_params(IN, 44).astype(np.float32))
        for _ in range(20):
            out = net.train_step(X, V, J, lr=1e-3, weight_decay=1e-4, want_loss=want)
            assert (out is None) == (not want)
        params.append(net.get_params())
        net.close()
    np.testing.assert_array_equal(params[0], params[1])


def test_training_is_reproducible(lib):
    """Two trainings from the same initial weights on the same data and draw
    seed end with bit-identical weights and per-step losses: every sum over
    the batch (loss, bias gradients, GEMM accumulations) is formed in a fixed
    order, whatever the order in which the blocks finish."""
    import torch
    n, B, steps = 3000, 1024, 200
    rng = np.random.Generator(np.random.PCG64(8))
    x = rng.uniform(0, 1, size=(n, IN))
    v = 0.6 * x[:, 2] - 0.1 * x[:, 9]
    jam = (x[:, 11] + x[:, 12] > 1.1).astype(np.float64)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    X, V, J = t(x), t(v), t(jam)
    p0 = mlp_init_params(IN, 12).astype(np.float32)
    runs = []
    for _ in range(2):
        net = lib.MLP()
        net.set_params(p0)
        losses = net.train(X, V, J, steps, B, lr=1e-3, weight_decay=1e-4, seed=5)
        runs.append((np.asarray(losses).copy(), net.get_params()))
        net.close()
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])


def _drawn_rows(seed, t, B, n):
    """Rows of training step t's mini-batch, restated from the documented
    draw: u = SplitMix64(seed, t * B + i + 1), row = floor(u * n / 2^64)."""
    M64 = (1 << 64) - 1
    rows = []
    for i in range(B):
        z = (seed + (t * B + i + 1) * 0x9E3779B97F4A7C15) & M64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        z ^= z >> 31
        rows.append((z * n) >> 64)
    return np.array(rows, dtype=np.int64)


def test_native_training_equals_train_steps_on_the_drawn_batches(lib):
    """bml_mlp_train (draw, gather and steps on the device) gives bit for
    bit the losses and weights of the same steps taken one by one on the
    batches the documented draw selects."""
    import torch
    n, B, steps, seed = 700, 128, 12, 99
    rng = np.random.Generator(np.random.PCG64(5))
    x = rng.uniform(0, 1, size=(n, IN))
    v = 0.3 * x[:, 0] + 0.2 * x[:, 5]
    jam = (x[:, 7] > 0.6).astype(np.float64)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    X, V, J = t(x), t(v), t(jam)
    p0 = mlp_init_params(IN, 3).astype(np.float32)
    a = lib.MLP()
    a.set_params(p0)
    losses = a.train(X, V, J, steps, B, lr=2e-3, weight_decay=1e-4, seed=seed)
    b = lib.MLP()
    b.set_params(p0)
    want = []
    for s in range(steps):
        idx = torch.tensor(_drawn_rows(seed, s, B, n), device="cuda")
        want.append(b.train_step(X[idx], V[idx], J[idx], lr=2e-3, weight_decay=1e-4))
    np.testing.assert_array_equal(losses, np.array(want, dtype=np.float32))
    np.testing.assert_array_equal(a.get_params(), b.get_params())
    # a second call continues the step index (new batches)
    more = a.train(X, V, J, 3, B, lr=2e-3, weight_decay=1e-4, seed=seed)
    for s in range(3):
        idx = torch.tensor(_drawn_rows(seed, steps + s, B, n), device="cuda")
        got = b.train_step(X[idx], V[idx], J[idx], lr=2e-3, weight_decay=1e-4)
        assert got == more[s]
    assert a.train(X, V, J, 0, B, lr=1e-3) is not None
    a.close()
    b.close()


def test_gemm_completion_wait_runs_out_and_reports_timeout(lib):
    """Test hook: no operand copy is issued, so the kernel's first
    completion wait gives up after its bound; the call returns BML_ETIMEOUT
    and the context stays usable (the next GEMM is exact)."""
    import torch
    g = torch.Generator().manual_seed(3)
    A = torch.randn(256, 64, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(32, 64, generator=g).to(torch.bfloat16).cuda()
    C = torch.zeros((256, 32), dtype=torch.float32, device="cuda")
    with pytest.raises(lib.BMLError) as e:
        lib.bml_gemm_bf16_ex(A.data_ptr(), 64, B.data_ptr(), 64, C.data_ptr(), 32, 256, 32, 64,
                             lib.BML_GEMM_TEST_STALL)
    assert e.value.code == lib.BML_ETIMEOUT
    lib.bml_gemm_bf16(A.data_ptr(), 64, B.data_ptr(), 64, C.data_ptr(), 32, 256, 32, 64)
    want = A.double().cpu() @ B.double().cpu().T
    assert torch.allclose(C.double().cpu(), want, rtol=1e-4, atol=1e-2)
