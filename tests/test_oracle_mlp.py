"""Pins of the proposal network's reference: finite differences against the
analytic backward, bf16 rounding against its definition, closed forms."""
import numpy as np

from oracle import mlp


def test_bf16_round_definition():
    # values exactly between two bf16 numbers round to the even mantissa
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)
    assert mlp.bf16_round(one + ulp / 2) == one                  # tie -> even (1.0)
    assert mlp.bf16_round(one + 3 * ulp / 2) == one + 2 * ulp    # tie -> even (1 + 2 ulp)
    assert mlp.bf16_round(one + ulp / 2 + ulp / 8) == one + ulp  # above the midpoint
    assert mlp.bf16_round(np.float32(-2.5)) == np.float32(-2.5)  # exactly representable
    x = np.random.default_rng(0).normal(size=1000).astype(np.float32)
    r = mlp.bf16_round(x)
    assert (np.abs(r - x) <= np.abs(x) * 2.0 ** -8).all()


def test_closed_forms():
    rng = np.random.default_rng(1)
    p = mlp.Params.random(rng)
    p.W2[:] = 0.0
    x = rng.integers(0, 5, size=(10, mlp.IN)).astype(np.float32)
    y, _ = mlp.forward(p, x)
    assert np.allclose(y, np.maximum(p.b2, 0) @ p.w3 + p.b3)
    p = mlp.Params.random(rng)
    y0, _ = mlp.forward(p, np.zeros((1, mlp.IN), np.float32))
    h1 = mlp.bf16_round(np.maximum(p.b1, 0)).astype(np.float64)
    assert np.allclose(y0, np.maximum(h1 @ p.W2 + p.b2, 0) @ p.w3 + p.b3)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    p = mlp.Params.random(rng)
    n = 40
    x = rng.normal(size=(n, mlp.IN))
    label = (rng.random(n) < 0.4).astype(np.float64)
    weight = rng.random(n)

    def loss_of(pp):
        y, _ = mlp.forward(pp, x, round_h1=False)
        return mlp.logistic_loss(y, label, weight)[0]

    y, cache = mlp.forward(p, x, round_h1=False)
    _, dy = mlp.logistic_loss(y, label, weight)
    g = mlp.backward(p, cache, dy)
    eps = 1e-6
    for name, idx in [("W1", (3, 17)), ("W1", (31, 127)), ("W2", (5, 9)), ("W2", (100, 64)),
                      ("b1", (7,)), ("b2", (90,)), ("w3", (33,))]:
        arr = getattr(p, name)
        old = arr[idx]
        arr[idx] = old + eps
        lp = loss_of(p)
        arr[idx] = old - eps
        lm = loss_of(p)
        arr[idx] = old
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[name][idx]) <= 1e-6 * (1 + abs(fd)), (name, idx, fd, g[name][idx])
    old = p.b3
    p.b3 = old + eps
    lp = loss_of(p)
    p.b3 = old - eps
    lm = loss_of(p)
    p.b3 = old
    assert abs((lp - lm) / (2 * eps) - g["b3"]) <= 1e-6
