"""Pins of the numpy reference network (tests/mlp_reference.py) used by the
GPU tests of the surrogate: its gradients against central finite
differences (BF16 rounding switched off so that small perturbations
count), its BF16 rounding against the bit pattern, its Adam step against the
closed form of the first step."""
import numpy as np

import mlp_reference as R


def test_gradients_match_finite_differences(monkeypatch):
    monkeypatch.setattr(R, "bf16", lambda a: np.asarray(a, dtype=np.float64))
    nf, w, d = 2, 8, 3
    n = sum(fo * fi + fo for fo, fi in R.layer_shapes(nf, w, d))
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.5, n)
    x = rng.uniform(0, 1, (20, 3))
    y = rng.normal(0, 1, (20, 4))
    mean, std = rng.normal(0, 1, 4), rng.uniform(0.5, 2, 4)
    _, g = R.grads(p, x, y, mean, std, nf, w, d)
    eps = 1e-6
    for k in rng.choice(n, 40, replace=False):
        q1, q2 = p.copy(), p.copy()
        q1[k] += eps
        q2[k] -= eps
        l1, _ = R.grads(q1, x, y, mean, std, nf, w, d)
        l2, _ = R.grads(q2, x, y, mean, std, nf, w, d)
        assert abs((l1 - l2) / (2 * eps) - g[k]) <= 1e-6 * max(1.0, abs(g[k]))


def test_bf16_rounding_bits():
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.14159265], dtype=np.float32)
    b = R.bf16(a)
    assert b[0] == 1.0
    assert b[1] == 1.0                       # tie: rounds to even
    assert b[2] == 1.0 + 2 ** -7             # above the tie: up
    assert b[3] == -2.5
    assert abs(b[4] - 3.140625) < 1e-7       # 8 significant bits
    assert np.all(b.view(np.uint32) & 0xFFFF == 0)


def test_first_adam_step_moves_each_weight_by_lr():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 4.0])
    q, m, v = R.adam_step(p, g, 0.0, 0.0, 1, 0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> step lr * sign(g)
    np.testing.assert_allclose(q, p - 0.01 * np.sign(g), rtol=0, atol=1e-6)   # eps = 1e-8 aside
