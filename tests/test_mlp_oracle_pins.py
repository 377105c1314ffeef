"""Pins of the FP64 surrogate-network oracle: the hand-written backward against
central finite differences of the forward, SiLU against scipy's logistic
function, one Adam step against its closed form, bf16 rounding against torch."""
import numpy as np
import pytest
from scipy import special

from oracle import mlp_oracle as M


def random_params(layers, seed=0, scale=0.5):
    rng = np.random.default_rng(seed)
    return [(rng.normal(0, scale / np.sqrt(a), (b, a)), rng.normal(0, 0.1, b)) for a, b in zip(layers, layers[1:])]


def test_silu_and_derivative():
    z = np.linspace(-30, 30, 2001)
    np.testing.assert_allclose(M.silu(z), z * special.expit(z), rtol=1e-14, atol=1e-300)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(M.dsilu(z), fd, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("layers", [(12, 16, 16, 16, 16, 2), M.LAYERS])
def test_backward_matches_finite_differences(layers):
    rng = np.random.default_rng(1)
    params = random_params(layers, seed=2)
    x = rng.uniform(-1, 1, (8, layers[0]))
    t = rng.normal(0, 1, (8, layers[-1]))
    _, grads = M.loss_and_grads(params, x, t)
    h = 1e-6
    for _ in range(24):
        li = int(rng.integers(len(params)))
        which = int(rng.integers(2))
        arr = params[li][which]
        idx = tuple(int(rng.integers(s)) for s in arr.shape)
        old = arr[idx]
        arr[idx] = old + h
        lp, _ = M.loss_and_grads(params, x, t)
        arr[idx] = old - h
        lm, _ = M.loss_and_grads(params, x, t)
        arr[idx] = old
        fd = (lp - lm) / (2 * h)
        an = grads[li][which][idx]
        assert an == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_adam_first_step_closed_form():
    params = random_params((3, 4, 2), seed=3)
    grads = random_params((3, 4, 2), seed=4)
    lr, eps = 1e-2, 1e-8
    new, m, v = M.adam_step(params, grads, M.zeros_like(params), M.zeros_like(params), 1, lr=lr, eps=eps)
    for (p, b), (g, gb), (q, qb) in zip(params, grads, new):
        # bias-corrected first step: m_hat = g, v_hat = g^2 -> update = -lr g / (|g| + eps)
        np.testing.assert_allclose(q, p - lr * g / (np.abs(g) + eps), rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(qb, b - lr * gb / (np.abs(gb) + eps), rtol=1e-13, atol=1e-15)


def test_flatten_round_trip_and_size():
    params = random_params(M.LAYERS, seed=5)
    vec = M.flatten(params)
    assert vec.size == 12 * 256 + 256 + 3 * (256 * 256 + 256) + 256 * 2 + 2
    back = M.unflatten(vec)
    for (W, b), (W2, b2) in zip(params, back):
        np.testing.assert_array_equal(W, W2)
        np.testing.assert_array_equal(b, b2)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(6).normal(0, 10, 100000)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.round_bf16(x), ref)
