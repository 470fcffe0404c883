"""Pins of the fp64 surrogate-network oracle (CPU only): central finite
differences, closed forms, a special case that reduces to a matrix product,
the first AdamW step, and bfloat16 rounding against torch's conversion."""
import numpy as np
import pytest

from oracle import mlp
from paper_1804_07981_b300.inputs import mlp_init_params

IN = 67


def batch(B, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(0, 1, size=(B, IN))
    v = rng.uniform(0, 1, size=B)
    jam = (rng.uniform(0, 1, size=B) < 0.4).astype(np.float64)
    return x, v, jam


def test_shapes_and_count():
    assert mlp.num_params(IN) == 128 * 67 + 128 + 2 * (128 * 128 + 128) + 2 * 128 + 2
    assert mlp.num_params(IN) == 41986
    flat = mlp_init_params(IN, 1)
    assert flat.shape == (41986,)
    np.testing.assert_array_equal(mlp.flatten(mlp.unflatten(flat, IN)), flat)


def test_gradients_match_central_differences():
    ps = mlp.unflatten(mlp_init_params(IN, 3), IN)
    rng = np.random.Generator(np.random.PCG64(4))
    for p in ps[1::2]:
        p += rng.normal(0, 0.1, size=p.shape)  # non-zero biases
    x, v, jam = batch(16, 5)
    grads, _ = mlp.backward(ps, x, v, jam)
    flat, gflat = mlp.flatten(ps), mlp.flatten(grads)
    idx = rng.choice(flat.size, size=300, replace=False)
    idx = np.concatenate([idx, np.arange(flat.size - 258, flat.size)])  # all of layer 4
    h = 1e-6
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        num = (mlp.loss(mlp.unflatten(fp, IN), x, v, jam)
               - mlp.loss(mlp.unflatten(fm, IN), x, v, jam)) / (2 * h)
        assert abs(num - gflat[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, gflat[i])


def test_zero_weights_closed_form():
    ps = [np.zeros(s) for s in mlp.shapes(IN)]
    ps[-1][:] = [0.3, -0.7]
    x, v, jam = batch(10, 6)
    out, _ = mlp.forward(ps, x)
    np.testing.assert_allclose(out, np.tile([0.3, -0.7], (10, 1)))
    grads, L = mlp.backward(ps, x, v, jam)
    sig = 1 / (1 + np.exp(0.7))
    want_L = np.mean((0.3 - v) ** 2 + np.log1p(np.exp(-0.7)) + 0.7 * (1 - jam))
    assert abs(L - want_L) < 1e-12
    np.testing.assert_allclose(grads[-1], [2 * np.mean(0.3 - v), np.mean(sig - jam)], atol=1e-12)
    for g in grads[:-1]:
        assert not np.any(g)


def test_all_active_network_is_a_matrix_product():
    """With non-negative inputs and weights every ReLU passes its input, so
    the network is the affine map x -> x (W4 W3 W2 W1)^T + c."""
    rng = np.random.Generator(np.random.PCG64(7))
    ps = [rng.uniform(0, 0.05, size=s) for s in mlp.shapes(IN)]
    x = rng.uniform(0, 1, size=(9, IN))
    A = ps[6] @ ps[4] @ ps[2] @ ps[0]
    c = ps[6] @ (ps[4] @ (ps[2] @ ps[1] + ps[3]) + ps[5]) + ps[7]
    out, _ = mlp.forward(ps, x)
    np.testing.assert_allclose(out, x @ A.T + c, rtol=1e-12)


def test_bce_closed_forms():
    assert abs(mlp.bce_with_logits(np.array(0.0), 1.0) - np.log(2)) < 1e-15
    z = np.array([-30.0, -2.0, 0.5, 40.0])
    np.testing.assert_allclose(mlp.bce_with_logits(z, 0.0), np.log1p(np.exp(z)), rtol=1e-12)
    np.testing.assert_allclose(mlp.sigmoid(z), 1 / (1 + np.exp(-z)), rtol=1e-12)


def test_adamw_first_step_and_decay():
    rng = np.random.Generator(np.random.PCG64(8))
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    opt = mlp.AdamW(50)
    w1 = opt.step(w, g, lr=1e-2, wd=0.0)
    np.testing.assert_allclose(w1, w - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    opt = mlp.AdamW(50)
    w1 = opt.step(w, np.zeros(50), lr=1e-2, wd=0.1)
    np.testing.assert_allclose(w1, w * (1 - 1e-3), rtol=1e-12)


def test_bf16_rounding_matches_torch():
    import torch
    rng = np.random.Generator(np.random.PCG64(9))
    a = np.concatenate([rng.normal(scale=s, size=1000) for s in (1e-3, 1, 1e3)])
    a = np.concatenate([a, [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.3895313892515355e38]])
    want = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(a), want)
