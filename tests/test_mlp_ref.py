"""The float64 reference of the dispatch MLP, pinned to the mathematics: its
hand-derived gradient equals central finite differences of its loss."""
import numpy as np

from oracle import mlp_ref


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.4, mlp_ref.n_params())
    x = rng.normal(0, 1, (23, mlp_ref.IN))
    t = rng.normal(0, 1, (23, mlp_ref.OUT))
    m = (rng.random((23, mlp_ref.OUT)) < 0.7).astype(float)
    loss, g = mlp_ref.loss_and_grad(p, x, t, m)
    assert abs(loss - mlp_ref.loss_only(p, x, t, m)) < 1e-12
    idx = rng.choice(p.size, 120, replace=False)
    eps = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += eps
        lp = mlp_ref.loss_only(q, x, t, m)
        q[i] -= 2 * eps
        lm = mlp_ref.loss_only(q, x, t, m)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_reference_layout_and_relu():
    p = np.zeros(mlp_ref.n_params())
    # only the output biases set: the prediction is the bias for every input
    p[-12:] = np.arange(12)
    y, _ = mlp_ref.forward(p, np.ones((3, 5)))
    assert np.array_equal(y, np.tile(np.arange(12.0), (3, 1)))
    assert mlp_ref.n_params() == 32 * 5 + 32 + 32 * 32 + 32 + 12 * 32 + 12
