"""Pins of the float64 network reference: the analytic gradient against
central finite differences, bf16 rounding against its definition, and a
closed form (zero weights: the output is b3 and only b3 has a gradient)."""
import numpy as np

from oracle import mlp


def _params(seed, scale=0.3):
    return (np.random.default_rng(seed).standard_normal(mlp.N_PARAMS) * scale).astype(np.float32)


def test_bf16_round():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 3.14159], dtype=np.float32)
    r = mlp.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0          # tie -> even
    assert r[2] == 1.0 + 2 ** -7
    assert r[3] == 1.0 + 2 ** -6                # tie -> even (up)
    assert r[4] == -2.5
    assert abs(r[5] - 3.140625) < 1e-12


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    master = _params(2)
    # make the bf16 rounding exact so the finite differences see the same function
    master = mlp.bf16_round(master).astype(np.float32)
    x = rng.standard_normal((9, 8))
    t = rng.standard_normal((9, 2))
    loss, g = mlp.loss_and_grad(master, x, t)
    idx = np.concatenate([rng.choice(512, 6), 512 + rng.choice(4096, 6), 4608 + rng.choice(128, 4),
                          4736 + rng.choice(64, 3), 4800 + rng.choice(64, 3), [4864, 4865]])
    for i in idx:
        h = 2.0 ** -10  # exact in bf16 around these magnitudes only for biases; use float64 path
        p = mlp.unpack(master)
        def f(delta):
            mm = master.astype(np.float64).copy()
            mm[i] += delta
            # evaluate without re-rounding the perturbed weight
            o = 0
            q = {}
            for name, shape in mlp.SIZES:
                n = int(np.prod(shape))
                q[name] = mm[o:o + n].reshape(shape)
                o += n
            z1 = x @ q["W1"].T + q["b1"]
            h1 = np.maximum(z1, 0)
            z2 = h1 @ q["W2"].T + q["b2"]
            h2 = np.maximum(z2, 0)
            out = h2 @ q["W3"].T + q["b3"]
            return ((out - t) ** 2).sum() / x.shape[0]
        num = (f(h) - f(-h)) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 + 1e-4 * abs(num), (i, num, g[i])


def test_zero_weights_closed_form():
    master = np.zeros(mlp.N_PARAMS, dtype=np.float32)
    master[4864:4866] = [0.5, -1.0]
    x = np.random.default_rng(3).standard_normal((5, 8))
    t = np.array([[1.0, 1.0]] * 5)
    out, _ = mlp.forward(master, x)
    assert np.allclose(out, [[0.5, -1.0]] * 5)
    loss, g = mlp.loss_and_grad(master, x, t)
    assert np.isclose(loss, (0.25 + 4.0))
    assert np.allclose(g[4864:], [2 * (0.5 - 1.0), 2 * (-1.0 - 1.0)])
    assert not g[:4864].any()
