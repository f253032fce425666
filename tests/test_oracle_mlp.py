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


def test_relu_after_each_hidden_layer():
    """A hidden layer whose pre-activations are all negative passes nothing on: with b = -1 and the layer's
    incoming weights zero, every later logit is the last bias (uniform here, loss ln 64), whatever the
    other weights are."""
    X = RNG.normal(size=(5, 24))
    y = RNG.integers(0, 64, size=5)
    for layer in (0, 1):   # the first or the second hidden layer is switched off
        parts = [RNG.normal(size=s) for s in mlp.SHAPES]
        parts[2 * layer] = np.zeros(mlp.SHAPES[2 * layer])     # incoming weights of that layer
        parts[2 * layer + 1] = -np.ones(mlp.SHAPES[2 * layer + 1])
        if layer == 0:
            parts[3] = np.zeros(64)                           # the second layer then sees only zeros
        parts[5] = np.zeros(64)
        theta = mlp.pack(parts)
        z3, _ = mlp.forward(theta, X)
        np.testing.assert_array_equal(z3, 0.0)
        assert np.isclose(mlp.loss(theta, X, y), np.log(64.0))


def test_parameter_layout_rows_are_outputs():
    """W is stored row-major as [out, in]: a parameter vector with a single 1 at W1[o, i] and permutation
    matrices W2[p2, o] = 1, W3[p3, p2] = 1 routes input i to logit p3, after the two ReLUs (positive
    input)."""
    o, i, p2, p3 = 7, 19, 40, 3
    parts = [np.zeros(s) for s in mlp.SHAPES]
    parts[0][o, i] = 1.0
    perm2 = np.roll(np.arange(64), o - p2)          # perm2[o] = p2
    perm3 = np.roll(np.arange(64), p2 - p3)         # perm3[p2] = p3
    parts[2][perm2, np.arange(64)] = 1.0
    parts[4][perm3, np.arange(64)] = 1.0
    X = np.zeros((1, 24))
    X[0, i] = 2.5
    theta = mlp.pack(parts)
    z3, _ = mlp.forward(theta, X)
    want = np.zeros(64)
    want[p3] = 2.5
    np.testing.assert_array_equal(z3[0], want)
    assert theta[o * 24 + i] == 1.0 and theta[24 * 64 + 64 + p2 * 64 + o] == 1.0


def test_bf16_forward_equals_the_fp64_forward_on_representable_values():
    """With inputs and weights that bf16 holds exactly and sums that stay exact (one signed power of two
    per row after the first layer, multiples of 1/4 in the first), rounding to bf16 changes nothing: the
    inference-precision forward pass equals the FP64 one exactly.  A permuted, signed routing catches a
    transposed layer, a dropped ReLU or a misplaced bias."""
    rng = np.random.default_rng(11)
    for _ in range(5):
        parts = [np.zeros(s) for s in mlp.SHAPES]
        parts[0][np.arange(64), rng.integers(0, 24, 64)] = rng.integers(-8, 9, 64) / 4.0
        parts[1] = rng.integers(-16, 17, 64) / 16.0
        for w in (2, 4):
            parts[w][np.arange(64), rng.permutation(64)] = rng.choice([-2.0, -1.0, 0.5, 1.0, 2.0], 64)
        X = rng.integers(-8, 9, size=(6, 24)) / 4.0
        theta = mlp.pack(parts)
        z, _ = mlp.forward(theta, X)
        assert np.abs(z).max() > 0
        np.testing.assert_array_equal(mlp.forward_bf16(theta, X), z)


def test_bf16_forward_stays_within_the_rounding_bound():
    """General values: each of the three rounded layers adds at most a relative 2^-8 per factor, so the
    logits stay within a few percent of the magnitudes that produce them."""
    theta = _theta()
    X = RNG.normal(size=(9, 24))
    z, (X64, z1, h1, z2, h2) = mlp.forward(theta, X)
    W3 = mlp.unpack(theta)[4]
    scale = np.abs(h2) @ np.abs(W3).T + 1e-3
    assert np.all(np.abs(mlp.forward_bf16(theta, X) - z) <= 0.05 * scale)
