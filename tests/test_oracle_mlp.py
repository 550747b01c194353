"""Pins of the MLP oracle: a closed-form single-path network, linearity in the
output layer, and central finite differences of the loss for every parameter
group (a wrong transpose, a missing ReLU mask or a dropped 1/n fails them)."""
import numpy as np

from oracle import mlp


def test_single_path_closed_form():
    d = {name: np.zeros(shape) for name, shape in mlp.SIZES}
    d["W1"][3, 2] = 1.5
    d["b1"][3] = -0.25
    d["W2"][7, 3] = -2.0
    d["b2"][7] = 4.0
    d["w3"][7] = 0.5
    d["b3"][0] = 0.1
    p = mlp.pack(d)
    x = np.zeros((4, 6))
    x[:, 2] = [1.0, 0.0, 3.0, -1.0]
    y, _ = mlp.forward(p, x)
    # hand evaluation: h1_3 = relu(1.5 x2 - 0.25); h2_7 = relu(-2 h1_3 + 4); y = 0.5 h2_7 + 0.1
    h1 = np.maximum(1.5 * x[:, 2] - 0.25, 0)
    h2 = np.maximum(-2.0 * h1 + 4.0, 0)
    assert np.allclose(y, 0.5 * h2 + 0.1, rtol=0, atol=1e-15)
    assert y.tolist() == [0.5 * 1.5 + 0.1, 0.5 * 4 + 0.1, 0.1, 0.5 * 4 + 0.1]


def test_parameter_count_and_layout():
    assert mlp.NPARAM == 64 * 6 + 64 + 64 * 64 + 64 + 64 + 1 == 4673
    p = np.arange(mlp.NPARAM, dtype=np.float64)
    d = mlp.unpack(p)
    assert d["W1"][1, 0] == 6 and d["b1"][0] == 384 and d["W2"][0, 1] == 449 and d["b3"][0] == 4672
    assert np.array_equal(mlp.pack(d), p)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    p = rng.normal(0, 0.3, mlp.NPARAM)
    x = rng.normal(0, 1, (37, 6))
    t = rng.normal(0, 1, 37)
    loss, g = mlp.loss_and_grad(p, x, t)
    assert abs(loss - np.mean((mlp.forward(p, x)[0] - t) ** 2)) < 1e-15
    idx = np.concatenate([rng.choice(mlp.NPARAM, 300, replace=False), [0, 383, 384, 447, 448, 4543, 4544, 4672]])
    eps = 1e-6
    for k in idx:
        e = np.zeros(mlp.NPARAM)
        e[k] = eps
        fd = (mlp.loss_and_grad(p + e, x, t)[0] - mlp.loss_and_grad(p - e, x, t)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_output_layer_gradient_is_exact_linear_regression():
    """With h2 fixed (all pre-activations positive), dL/dw3 = (2/n) h2^T (y - t)."""
    rng = np.random.default_rng(6)
    d = {name: np.zeros(shape) for name, shape in mlp.SIZES}
    d["b1"][:] = 1.0
    d["b2"][:] = np.linspace(0.5, 2.0, 64)
    d["w3"][:] = rng.normal(size=64)
    p = mlp.pack(d)
    x = rng.normal(size=(10, 6))
    t = rng.normal(size=10)
    _, g = mlp.loss_and_grad(p, x, t)
    h2 = np.tile(d["b2"] + d["W2"].sum(axis=1), (10, 1))
    y = h2 @ d["w3"]
    gw3 = h2.T @ (2 * (y - t) / 10)
    assert np.allclose(mlp.unpack(g)["w3"], gw3, rtol=1e-13)
