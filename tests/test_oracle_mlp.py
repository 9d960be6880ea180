"""Oracle pin: the surrogate network's reference gradients against central finite differences
of the loss (an independent check of every chain-rule step)."""
import numpy as np

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    w = mlp.init(1)
    x = rng.uniform(-1, 1, (17, 3))
    t = rng.standard_normal((17, 3))
    m = (rng.uniform(size=(17, 3)) > 0.2).astype(float)
    g = mlp.grad(w, x, t, m)
    h = 1e-6
    for k in mlp.SHAPES:
        flat = w[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = mlp.loss(w, x, t, m)
            flat[i] = old - h
            lm = mlp.loss(w, x, t, m)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k].reshape(-1)[i] - fd) <= 1e-7 * max(1.0, abs(fd)), (k, i)


def test_silu_derivative():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.allclose(mlp.dsilu(z), fd, atol=1e-8)
