"""Pins of the FP64 reference network (oracle/mlp.py), CPU only: its gradient
against central differences of its own loss in the effective (BF16) weights,
GELU closed forms, BF16 rounding of known values, and invariances of the
features (a positive scale of one variable leaves them unchanged; a periodic
shift moves them with the mesh)."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1805_01443_gb300 import inputs


def test_gelu_closed_forms():
    x = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-15)
    assert mlp.gelu(0.0) == 0.0 and mlp.gelu_d(0.0) == 0.5
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_d(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)
    assert abs(mlp.gelu(10.0) - 10.0) < 1e-20


def test_bf16_round_to_nearest_even():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7, -2.5, 3.0e38],
                    dtype=np.float32)
    expect = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.5, 2.9969e38])
    r = mlp.bf16(vals)
    np.testing.assert_array_equal(r[:5], expect[:5])
    assert abs(r[5] / 3.0e38 - 1) < 2 ** -8


def test_gradient_matches_central_differences():
    """The loss as a function of the effective weights (already BF16, so the
    rounding is the identity on them) against the analytic gradient."""
    rng = np.random.default_rng(0)
    nin, B = 12, 40
    p = mlp.bf16(rng.normal(0, 0.4, size=mlp.nparams(nin)).astype(np.float32)).astype(np.float64)
    x = rng.normal(size=(B, nin))
    y = (rng.uniform(size=B) < 0.3).astype(float)
    loss, g = mlp.loss_and_grad(p, x, y, nin, pos_weight=3.0)

    def L(q):
        # evaluate in FP64 directly in the effective weights (no rounding)
        W1, b1, W2, b2, w3, b3 = (np.asarray(t, dtype=np.float64) for t in _split64(q, nin))
        h1 = mlp.gelu(x @ W1.T + b1)
        h2 = mlp.gelu(h1 @ W2.T + b2)
        z = h2 @ w3 + b3[0]
        w = np.where(y > 0.5, 3.0, 1.0)
        return float(np.mean(w * (np.logaddexp(0.0, z) - y * z)))

    assert L(p) == pytest.approx(loss, rel=1e-12)
    idx = rng.choice(p.size, size=60, replace=False)
    fd = np.array([(L(_bump(p, k, 1e-6)) - L(_bump(p, k, -1e-6))) / 2e-6 for k in idx])
    np.testing.assert_allclose(g[idx], fd, rtol=1e-5, atol=1e-9)


def _bump(p, k, h):
    q = p.copy()
    q[k] += h
    return q


def _split64(q, nin):
    H = mlp.H
    o = 0
    out = []
    for n, shape in [(H * nin, (H, nin)), (H, (H,)), (H * H, (H, H)), (H, (H,)), (H, (H,)), (1, (1,))]:
        out.append(q[o:o + n].reshape(shape))
        o += n
    return out


def test_features_scale_invariance_and_periodic_shift():
    cfg = inputs.density_wave(8, 2)
    o = oracle.Oracle(cfg)
    u = o.fetch() + inputs.modal_perturbation(o.shape, seed=4, amp=1e-2)
    o.set_state(u)
    f0 = mlp.features(o)
    u2 = u.copy()
    u2[1] *= 8.0  # a power of two: exact
    o.set_state(u2)
    np.testing.assert_array_equal(mlp.features(o), f0)
    o.set_state(np.roll(u, 1, axis=3))
    f1 = mlp.features(o)
    nx = 8
    for j in range(8):
        for i in range(8):
            np.testing.assert_array_equal(f1[j * nx + (i + 1) % nx], f0[j * nx + i])
    assert np.abs(f0).max() == 1.0
