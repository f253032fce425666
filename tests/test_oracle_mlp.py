"""Pins of the FP64 MLP oracle of the learned proposal.  CPU only."""
import numpy as np

from oracle import mlp

RNG = np.random.default_rng(5)


def _theta():
    parts = [RNG.normal(size=s) * (0.4 if len(s) == 2 else 0.1) for s in mlp.SHAPES]
    return mlp.pack(parts)


def test_parameter_count():
    assert mlp.N_PARAMS == 24 * 64 + 64 + 64 * 64 + 64 + 64 * 64 + 64 == 9920


def test_gradient_matches_central_differences():
    theta = _theta()
    X = RNG.normal(size=(7, 24))
    y = RNG.integers(0, 64, size=7)
    _, g = mlp.loss_and_grad(theta, X, y)
    idx = RNG.choice(mlp.N_PARAMS, size=300, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, X, y) - mlp.loss(tm, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (i, fd, g[i])


def test_softmax_cross_entropy_closed_form():
    """With W = 0 the logits are the last bias: b3 = [0, ln 2, 0, ...] gives p_1 = 2/65, p_other = 1/65."""
    parts = [np.zeros(s) for s in mlp.SHAPES]
    parts[5][1] = np.log(2.0)
    theta = mlp.pack(parts)
    X = RNG.normal(size=(3, 24))
    assert np.isclose(mlp.loss(theta, X, [1, 1, 1]), -np.log(2 / 65))
    assert np.isclose(mlp.loss(theta, X, [0, 5, 9]), -np.log(1 / 65))
    L, g = mlp.loss_and_grad(theta, X, [1, 1, 1])
    db3 = mlp.unpack(g)[5]
    exp = np.full(64, 1 / 65)
    exp[1] = 2 / 65 - 1
    np.testing.assert_allclose(db3, exp, atol=1e-14)


def test_bf16_rounding():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, 1 + 2 ** -7, -2.5, 3.0e38], np.float32)
    r = mlp.bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                  # tie -> even
    assert r[2] == 1 + 2 ** -7          # above the tie -> up
    assert r[3] == 1 + 2 ** -7          # exact
    assert r[4] == -2.5
    assert np.isfinite(r[5])
