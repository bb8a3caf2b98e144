"""Pin the FP64 reference of the warm-start network by central finite differences."""
import numpy as np

from oracle.neural import bf16_round, bilinear_map, loss_and_grad


def test_gradient_equals_finite_differences():
    rng = np.random.default_rng(0)
    dims = [3, 5, 4, 6 * 4]
    nparam = sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(len(dims) - 1))
    p = rng.standard_normal(nparam) * 0.5
    node_x = np.sort(rng.uniform(0, 2, 5))
    node_y = np.sort(rng.uniform(0, 1, 3))
    R = bilinear_map(6, 4, (0.0, 2.0, 0.0, 1.0), node_x, node_y)
    np.testing.assert_allclose(R.sum(axis=1), 1.0, atol=1e-14)      # partition of unity
    feat = rng.standard_normal((4, 3))
    tgt = rng.standard_normal((4, 15))
    mean, std = np.zeros(3), np.ones(3)
    _, g, _ = loss_and_grad(p, dims, mean, std, R, feat, tgt)
    h = 1e-6
    for i in rng.choice(nparam, 25, replace=False):
        e = np.zeros(nparam)
        e[i] = h
        lp = loss_and_grad(p + e, dims, mean, std, R, feat, tgt)[0]
        lm = loss_and_grad(p - e, dims, mean, std, R, feat, tgt)[0]
        assert abs((lp - lm) / (2 * h) - g[i]) < 1e-7 * max(1.0, abs(g[i]))


def test_bilinear_reproduces_linear_functions():
    node_x = np.linspace(0.05, 1.9, 7)
    node_y = np.linspace(0.0, 1.0, 5)
    R = bilinear_map(16, 9, (0.0, 2.0, 0.0, 1.0), node_x, node_y)
    gy = np.linspace(0.0, 1.0, 9)
    f = np.repeat(2.0 * gy - 1.0, 16)            # linear in y, constant in x
    np.testing.assert_allclose(R @ f, np.repeat(2.0 * node_y - 1.0, 7), atol=1e-14)


def test_bf16_rounding():
    assert bf16_round(np.array([1.0]))[0] == 1.0
    assert bf16_round(np.array([1.0 + 2 ** -8]))[0] == 1.0          # tie -> even
    assert bf16_round(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
