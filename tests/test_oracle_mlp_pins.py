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


def _hand_net(nin):
    """A hand-set network whose logit is worked out below: only a few weights
    and biases are non-zero, and every pre-activation is either 0, 1, far
    above zero (GELU(x) = x to ~1e-40 for x >= 14) or far below it (GELU(x)
    ~ 0 for x <= -20)."""
    H = mlp.H
    W1 = np.zeros((H, nin), np.float32)
    b1 = np.zeros(H, np.float32)
    W2 = np.zeros((H, H), np.float32)
    b2 = np.zeros(H, np.float32)
    w3 = np.zeros(H, np.float32)
    W1[0, 0] = 1.0
    W1[1, 0] = 3.0
    W1[2, 1] = -1.0       # reads the second input only (catches a transposed W1)
    b1[0] = 2.0
    W2[0, 0] = 0.5 + 2.0 ** -12   # not a BF16 value: rounds to 0.5
    W2[0, 1] = 0.25
    W2[1, 0] = -2.0
    W2[2, 2] = 1.0
    b2[0] = 5.0
    b2[2] = 1.0
    w3[0] = -0.25
    w3[1] = 1.0
    w3[2] = 2.0
    b3 = np.array([0.5], np.float32)
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, b3])


def test_forward_of_a_hand_set_network():
    """Worked by hand.  x = (12, 0, ...):
         layer 1: a = (12 + 2, 36, 0, ...)            -> h1 = (14, 36, 0, ...)
         layer 2: a = (0.5*14 + 0.25*36 + 5, -2*14, 0 + 1) = (21, -28, 1)
                                                      -> h2 = (21, ~0, Phi(1))
         logit:   -0.25*21 + 1*~0 + 2*Phi(1) + 0.5
       (GELU(1) = Phi(1), the standard normal CDF at 1, a table value).
       x = (12, -14): unit 2 of layer 1 sees 14, so unit 2 of layer 2 sees
       14 + 1 = 15 and the logit is -5.25 + 2*15 + 0.5 = 25.25.
       x = (12, 20): unit 2 of layer 1 sees -20, GELU(-20) ~ -6e-88, and the
       logit is the first case's.
       A dropped bias, GELU on the logit, no GELU on a hidden layer, W1 or W2
       read transposed, or weights not rounded to BF16 (W2[0, 0] = 0.5 + 2^-12
       would add 14 * 2^-12 / 4 to the logit) each change one of the three."""
    nin = 5
    params = _hand_net(nin)
    x = np.zeros((3, nin))
    x[:, 0] = 12.0
    x[1, 1] = -14.0
    x[2, 1] = 20.0
    z = mlp.forward(params, x, nin)
    phi1 = 0.8413447460685429  # standard normal CDF at 1 (table value)
    z0 = -0.25 * 21.0 + 2.0 * phi1 + 0.5
    assert z[0] == pytest.approx(z0, rel=0, abs=1e-15)
    assert z[1] == pytest.approx(25.25, rel=0, abs=1e-14)
    assert z[2] == pytest.approx(z0, rel=0, abs=1e-15)
