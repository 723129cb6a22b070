"""Pins of the FP64 warm-start network reference: closed-form GELU values,
central finite differences of the loss against the backward pass (a dropped
term, a transposed product or a missing GELU' fails them), Adam on a scalar
quadratic, BF16 rounding on exactly representable and halfway values."""
import math

import numpy as np

from oracle import mlp


def test_gelu_closed_form():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(mlp.gelu(np.array([1.0])), [0.5 * (1 + math.erf(1 / math.sqrt(2)))], rtol=1e-15)
    np.testing.assert_allclose(mlp.gelu(np.array([30.0, -30.0])), [30.0, 0.0], atol=1e-12)
    np.testing.assert_allclose(mlp.gelu_grad(np.array([0.0])), [0.5], rtol=1e-15)
    z = np.linspace(-4, 4, 41)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-8)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    params = mlp.init_params(rng, [5, 7, 6, 4])
    params = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in params]
    X = rng.standard_normal((9, 5))
    T = rng.standard_normal((9, 4))
    mask = np.array([1.0, 1.0, 0.0, 1.0])
    loss, grads = mlp.loss_and_grads(params, X, T, mask)
    h = 1e-6
    for li in range(len(params)):
        for k in range(2):
            P = params[li][k]
            it = np.nditer(P, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                def shifted(d):
                    q = [list(p) for p in params]
                    arr = q[li][k].copy()
                    arr[idx] += d
                    q[li][k] = arr
                    return mlp.loss_and_grads([tuple(p) for p in q], X, T, mask)[0]
                fd = (shifted(h) - shifted(-h)) / (2 * h)
                assert abs(fd - grads[li][k][idx]) <= 1e-7 * max(1.0, abs(fd)), (li, k, idx)


def test_adam_scalar_quadratic():
    """f(w) = w^2 / 2: the first Adam step moves w by exactly lr (m^ / sqrt(v^)
    = g / |g| after bias correction), then keeps moving toward 0."""
    params = [(np.array([[3.0]]), np.array([0.0]))]
    st = {}
    p1 = mlp.adam(params, [(params[0][0], params[0][1])], st, lr=0.1, eps=0.0)
    assert abs(p1[0][0][0, 0] - 2.9) < 1e-15
    p = p1
    for _ in range(200):
        p = mlp.adam(p, [(p[0][0], p[0][1])], st, lr=0.1, eps=0.0)
    assert abs(p[0][0][0, 0]) < 0.5


def test_bf16_rounding():
    vals = np.array([1.0, -2.5, 3.140625, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8])
    got = mlp.bf16_round(vals)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    np.testing.assert_array_equal(got, [1.0, -2.5, 3.140625, 1.0, 1.0 + 2 ** -6])
