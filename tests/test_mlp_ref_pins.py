"""Pins of the FP64 reference MLP (gradients by central differences, Adam by hand)."""
import numpy as np

from oracle import mlp_ref as M


def _params(rng, dims):
    return [(rng.standard_normal((o, i)) / np.sqrt(i), rng.standard_normal(o) * 0.1)
            for i, o in zip(dims[:-1], dims[1:])]


def test_silu_and_derivative():
    z = np.linspace(-8, 8, 41)
    assert np.allclose(M.silu(z), z / (1 + np.exp(-z)), rtol=1e-15)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    assert np.allclose(M.silu_grad(z), fd, rtol=1e-8, atol=1e-10)


def test_gradients_central_differences():
    rng = np.random.default_rng(0)
    dims = [6, 16, 16, 16, 3]
    P = _params(rng, dims)
    x = rng.standard_normal((7, 6))
    t = rng.standard_normal((7, 3))
    loss, grads = M.loss_and_grads(P, x, t)
    for l in range(len(P)):
        for which in (0, 1):
            p = P[l][which]
            g = grads[l][which]
            for idx in [tuple(rng.integers(0, s) for s in p.shape) for _ in range(6)]:
                old = p[idx]
                p[idx] = old + 1e-6
                lp, _ = M.loss_and_grads(P, x, t)
                p[idx] = old - 1e-6
                lm, _ = M.loss_and_grads(P, x, t)
                p[idx] = old
                fd = (lp - lm) / 2e-6
                assert abs(g[idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (l, which, idx)


def test_adam_first_step_is_signed_lr():
    """At t = 1 the bias-corrected step is lr * g / (|g| + eps) ~ lr * sign(g)."""
    rng = np.random.default_rng(1)
    P = _params(rng, [4, 5, 2])
    G = [(rng.standard_normal(W.shape), rng.standard_normal(b.shape)) for W, b in P]
    st = {}
    new = M.adam_step(P, G, st, lr=1e-3)
    for (W, b), (Wn, bn), (gW, gb) in zip(P, new, G):
        assert np.allclose(W - Wn, 1e-3 * gW / (np.abs(gW) + 1e-8), rtol=1e-12)
        assert np.allclose(b - bn, 1e-3 * gb / (np.abs(gb) + 1e-8), rtol=1e-12)


def test_bf16_round():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159265, 1e-30, 65504.0])
    r = M.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0            # tie to even
    assert r[2] == 1.0 + 2 ** -7                  # rounds up
    assert abs(r[3] / v[3] - 1) < 2 ** -8
    assert np.all(np.abs(r / v - 1) <= 2 ** -8)
