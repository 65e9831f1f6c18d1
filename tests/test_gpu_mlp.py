"""The learned troubled-cell indicator's kernels against the FP64 reference
network (oracle/mlp.py).

Features (dg_features, the training inputs) are formed in FP64 and rounded
once on both sides: bit for bit.  Logits and gradients accumulate in FP32 on
the GPU (BF16 weights, the same on both sides): logits to 1e-4 absolute plus
1e-4 relative, the gradient to 1e-4 relative L2, the loss to 1e-5.  Fused
inference on the state, which forms its inputs on the fly in FP32 (within
2^-22 relative of the FP64-product features), against the reference network
on the oracle's features, at the same logit tolerance.  Training on the
GPU lowers the loss; limiter 2 without a network is the TVB limiter.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as ref
from paper_1805_01443_gb300 import dg, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def ring_state(n=24, p=3, steps=4, bc=1):
    cfg = inputs.shock_ring(n, p)
    cfg["mesh"]["bc"] = bc
    o = oracle.Oracle(cfg)
    o.step(steps)
    return cfg, o


@pytest.mark.parametrize("p,bc", [(3, 1), (2, 0), (1, 2), (4, 1)])
def test_features_bitwise(p, bc):
    cfg, o = ring_state(20, p, 3, bc)
    g = dg.Disc(cfg)
    try:
        g.set_state(o.fetch(), *o.get_time()[::2])
        ne = cfg["mesh"]["nx"] * cfg["mesh"]["ny"]
        elems = torch.arange(ne, dtype=torch.int32, device="cuda")
        fg = g.features(elems).cpu().numpy()
        fo = ref.features(o)
        if bc != 1:
            np.testing.assert_array_equal(fg, fo)
        else:
            # the fixed ghost elements are projected by each side on its own
            # (equal to round-off): bit for bit where the stencil is interior
            nx, ny = cfg["mesh"]["nx"], cfg["mesh"]["ny"]
            jj, ii = np.divmod(np.arange(ne), nx)
            inner = (ii > 0) & (ii < nx - 1) & (jj > 0) & (jj < ny - 1)
            np.testing.assert_array_equal(fg[inner], fo[inner])
            assert np.abs(fg - fo).max() <= 1e-13
    finally:
        g.close()


def batch(nin, B, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 0.5, size=(B, nin)).astype(np.float32)
    y = (rng.uniform(size=B) < 0.2).astype(np.float32)
    return x, y


def test_forward_and_gradient_match_reference():
    nin, B = 320, 1000
    net = dg.Mlp(nin, seed=5)
    try:
        p = net.get_params()
        x, y = batch(nin, B, 1)
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        z = net.forward(xd).cpu().numpy()
        zr = ref.forward(p, x, nin)
        assert np.abs(z - zr).max() <= 1e-4 + 1e-4 * np.abs(zr).max()
        g, loss = net.grad(xd, yd, pos_weight=4.0)
        lr, gr = ref.loss_and_grad(p, x, y, nin, pos_weight=4.0)
        assert loss == pytest.approx(lr, rel=1e-5)
        assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr)
    finally:
        net.close()


def test_training_lowers_the_loss_on_tvb_labels():
    """Labels from the TVB test on a shock-ring state, features of the same
    state: 300 Adam steps on the GPU cut the loss and fit the labels."""
    cfg, o = ring_state(48, 3, 6, 1)
    u = o.fetch()
    g = dg.Disc(cfg)
    net = dg.Mlp(5 * 4 * 16, seed=1)
    try:
        g.set_state(u, *o.get_time()[::2])
        y = g.indicator(5.0).ravel().astype(np.float32)
        assert 20 < y.sum() < y.size / 2
        ne = y.size
        x = g.features(torch.arange(ne, dtype=torch.int32, device="cuda"))
        yd = torch.from_numpy(y).cuda()
        pw = float((y.size - y.sum()) / y.sum())
        l0 = net.train_step(x, yd, pos_weight=pw, lr=3e-3)
        for _ in range(300):
            l1 = net.train_step(x, yd, pos_weight=pw, lr=3e-3)
        assert l1 < 0.3 * l0
        z = net.forward(x).cpu().numpy()
        acc = ((z > 0) == (y > 0.5)).mean()
        assert acc > 0.95
    finally:
        net.close()
        g.close()


@pytest.mark.parametrize("maker,p,bc,ny", [
    ("shock_ring", 3, 1, 40), ("shock_ring", 1, 1, 35), ("shock_ring", 2, 0, 40), ("shock_ring", 4, 2, 35),
    ("disc_small", 1, 1, 40), ("disc_small", 3, 3, 35), ("disc_small", 4, 0, 40)])
def test_fused_inference_matches_reference(maker, p, bc, ny):
    """The tensor-core pass (features on the fly, BF16 hi + lo activations
    against BF16 weights, FP32 accumulators) against the FP64 network on the
    oracle's features: 4 (adiabatic) and 3 (isothermal) variables, every
    degree, each boundary kind, a row count that leaves the last CTA's four
    tiles partly empty and ragged 32-element tiles (nx = 40)."""
    cfg = getattr(inputs, maker)(40, p)
    cfg["mesh"]["bc"] = bc
    cfg["mesh"]["ny"] = ny
    o = oracle.Oracle(cfg)
    o.step(3)
    nv = o.fetch().shape[0]
    nin = 5 * nv * (p + 1) ** 2
    g = dg.Disc(cfg)
    net = dg.Mlp(nin, seed=3)
    try:
        g.set_state(o.fetch(), *o.get_time()[::2])
        g.set_indicator(net, threshold=0.1)
        z, f = g.indicator_logits()
        zr = ref.forward(net.get_params(), ref.features(o), nin).reshape(z.shape)
        assert np.abs(z - zr).max() <= 1e-4 + 1e-4 * np.abs(zr).max()
        sure = np.abs(zr - 0.1) > 1e-3
        np.testing.assert_array_equal(f[sure], (zr[sure] > 0.1).astype(np.uint8))
    finally:
        net.close()
        g.close()


def test_limiter2_without_network_is_tvb_and_with_network_runs():
    cfg1 = inputs.shock_ring(32, 3)
    cfg2 = inputs.shock_ring(32, 3)
    cfg2["disc"]["limiter"] = 2
    a, b = dg.Disc(cfg1), dg.Disc(cfg2)
    net = dg.Mlp(320, seed=2)
    try:
        a.step(5)
        b.step(5)
        np.testing.assert_array_equal(a.fetch(), b.fetch())
        b.set_indicator(net, threshold=0.0)
        b.step(5)
        u = b.fetch()
        assert np.isfinite(u).all()
        # the flags the limiter used come from the network; the TVB flags of
        # the same stage value are still recorded beside them
        assert b.last_flags().shape == (32, 32)
    finally:
        net.close()
        a.close()
        b.close()


def test_network_calls_refuse_host_memory_and_bad_tensors():
    """dg_mlp_forward / grad / train_step and dg_features refuse host arrays
    with DG_ERR_ARG before any launch; the binding refuses tensors of the wrong
    dtype, shape or device before their pointers reach the library."""
    import ctypes
    L = dg.lib()
    nin, B = 320, 8
    net = dg.Mlp(nin, seed=4)
    g = dg.Disc(inputs.shock_ring(16, 3))
    try:
        x = np.zeros((B, nin), dtype=np.float32)
        y = np.zeros(B, dtype=np.float32)
        z = np.full(B, 7.0, dtype=np.float32)
        xp, yp, zp = (ctypes.c_void_p(a.ctypes.data) for a in (x, y, z))
        assert L.dg_mlp_forward(net.net, xp, B, zp, None) == dg.DG_ERR_ARG
        assert L.dg_mlp_grad(net.net, xp, yp, B, 1.0, None, None, None) == dg.DG_ERR_ARG
        assert L.dg_mlp_train_step(net.net, xp, yp, B, 1.0, 1e-3, None, None) == dg.DG_ERR_ARG
        assert np.all(z == 7.0)
        elems = np.arange(4, dtype=np.int32)
        out = np.zeros((4, nin), dtype=np.float32)
        assert L.dg_features(g.h, ctypes.c_void_p(elems.ctypes.data), 4,
                             ctypes.c_void_p(out.ctypes.data)) == dg.DG_ERR_ARG
        assert not out.any()
        xd = torch.zeros((B, nin), dtype=torch.float32, device="cuda")
        with pytest.raises(ValueError):
            net.forward(xd[:, :100])                       # too few inputs per row
        with pytest.raises(ValueError):
            net.forward(xd.double())                       # wrong dtype
        with pytest.raises(ValueError):
            net.forward(torch.zeros((B, nin)))             # host tensor
        with pytest.raises(ValueError):
            net.train_step(xd, torch.zeros(B - 1, device="cuda"))
        with pytest.raises(ValueError):
            g.features(torch.arange(4, dtype=torch.int64, device="cuda"))
        # the refusals left the handle and the network usable
        assert net.forward(xd).shape == (B,)
        assert g.features(torch.arange(4, dtype=torch.int32, device="cuda")).shape == (4, nin)
    finally:
        net.close()
        g.close()
