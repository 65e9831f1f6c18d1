"""Troubled-cell indicator and limiters of the FP64 form against the oracle.

The TVB flags are decided by the same FP64 operations on both sides (products
by sqrt(3), differences of means, M h^2 and comparisons, no fused multiply-add
in the decision), so they are compared bit for bit on the same state.  The
limited and positivity-limited states are compared element by element: the
point values inside the positivity limiter are sums of products whose rounding
order differs (<= 1e-13 of the largest coefficient).  Limited runs of the
shock-ring disc are compared after several steps element by element at 1e-12
of the largest coefficient, with the torque at the FP64 bar (1e-12 of the sum
of |terms|) and the TVB flags of the final state equal: no minmod decision
flips between the two sides on these runs (measured on the GB300: at most
1.2e-14 after 20 steps, torque within 7e-12 relative, no flag differs), so
the FP64 bar applies unchanged.
"""
import numpy as np
import pytest

import oracle
from paper_1805_01443_gb300 import dg, inputs

pytestmark = pytest.mark.gpu


def both(cfg, u=None, t=0.0):
    o = oracle.Oracle(cfg)
    g = dg.Disc(cfg)
    if u is not None:
        o.set_state(u, t)
        g.set_state(u, t)
    return o, g


def rough_state(cfg, seed, amp):
    """The initial data plus seeded noise on the non-mean modes (the means,
    and so the mean pressure of the cold disc centre, stay admissible)."""
    o = oracle.Oracle(cfg)
    d = inputs.modal_perturbation(o.shape, seed=seed, amp=amp)
    d[:, 0] = 0.0
    u = o.fetch() + d
    o.close()
    return u


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


STATES = [
    ("wave", lambda p: inputs.density_wave(16, p), 3e-2),
    ("ring", lambda p: inputs.shock_ring(40, p, limiter=1, positivity=0), 1e-2),
    ("disc-bc2", lambda p: dict(inputs.disc_small(36, p), mesh=dict(inputs.disc_small(36, p)["mesh"], bc=2,
                                                                         nx=37, ny=22)), 1e-3),
]


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("name,mk,amp", STATES, ids=[s[0] for s in STATES])
def test_tvb_flags_bitwise(name, mk, amp, p):
    cfg = mk(p)
    u = rough_state(cfg, seed=11 + p, amp=amp)
    o, g = both(cfg, u)
    try:
        for M in (0.0, 5.0, 50.0):
            fo, fg = o.indicator(M), g.indicator(M)
            np.testing.assert_array_equal(fg, fo)
            assert 0 < fo.sum() or M > 0
    finally:
        g.close()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_limit_matches_oracle(p):
    cfg = inputs.shock_ring(40, p, limiter=1, positivity=1)
    cfg["disc"]["tvb_m"] = 5.0
    u = rough_state(cfg, seed=3, amp=2e-2)
    o, g = both(cfg, u)
    try:
        flags = o.indicator(5.0)
        assert flags.sum() > 0
        o.limit()
        g.limit()
        assert relmax(g.fetch(), o.fetch()) <= 1e-13
        np.testing.assert_array_equal(g.last_flags(), flags)
    finally:
        g.close()


def test_limit_given_flags_matches_oracle():
    cfg = inputs.shock_ring(48, 3, limiter=1, positivity=0)
    u = rough_state(cfg, seed=5, amp=1e-2)
    o = oracle.Oracle(cfg)
    o.set_state(u)
    g = dg.Disc(dict(cfg, disc=dict(cfg["disc"], limiter=2)))
    g.set_state(u)
    try:
        flags = (np.random.default_rng(9).uniform(size=(48, 48)) < 0.2).astype(np.uint8)
        o.limit_flags(flags)
        g.limit_flags(flags)
        assert relmax(g.fetch(), o.fetch()) <= 1e-13
    finally:
        g.close()


@pytest.mark.parametrize("p", [1, 3, 4])
def test_positivity_matches_oracle(p):
    cfg = inputs.uniform_state(24, p, kind=1)
    cfg["disc"]["positivity"] = 1
    o = oracle.Oracle(cfg)
    u = o.fetch()
    rng = np.random.default_rng(p)
    u[:, 1:] = rng.uniform(-0.6, 0.6, size=u[:, 1:].shape) * (rng.uniform(size=(1, 1) + u.shape[2:]) < 0.3)
    u[3, 0] = 3.0
    o.set_state(u)
    g = dg.Disc(cfg)
    try:
        g.set_state(u)
        o.limit()
        g.limit()
        v = o.fetch()
        assert not np.array_equal(v, u)
        assert relmax(g.fetch(), v) <= 1e-13
    finally:
        g.close()


@pytest.mark.parametrize("p,n,steps", [(3, 32, 12), (2, 40, 12), (1, 40, 20), (4, 24, 8)])
def test_limited_shock_ring_run_matches_oracle(p, n, steps):
    """The config-5 disc (adiabatic, pressure ring x10, planet q = 1e-3,
    TVB-limited troubled cells, positivity) at small size: initial data and
    `steps` steps against the oracle, flags of the last stage value too."""
    cfg = inputs.shock_ring(n, p)
    o, g = both(cfg)
    try:
        assert relmax(g.fetch(), o.fetch()) <= 1e-13
        o.step(steps)
        g.step(steps)
        assert relmax(g.fetch(), o.fetch()) <= 1e-12
        assert g.get_time()[0] == pytest.approx(o.get_time()[0], rel=1e-12)
        gz, asum = o.torque()
        assert abs(g.torque() - gz) <= 1e-12 * asum
        M = cfg["disc"]["tvb_m"]
        np.testing.assert_array_equal(g.indicator(M), o.indicator(M))
    finally:
        g.close()


def test_limiters_rejected_outside_fp64_ssp3():
    cfg = inputs.shock_ring(16, 2)
    cfg["disc"]["rk"] = 2
    with pytest.raises(dg.DgError) as e:
        dg.Disc(cfg)
    assert e.value.code == dg.DG_ERR_UNSUPPORTED
