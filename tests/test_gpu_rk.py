"""The 5-stage SSP-RK(4,5) and 6-stage Cash-Karp tableaux of Appendix A on the
GPU (FP64 form) against the oracle's Butcher-form integrator: states, times
and torque series after several steps (1e-12), and the time order of the
methods on the density wave at a fixed small mesh (the error of halving dt)."""
import numpy as np
import pytest

import oracle
from paper_1805_01443_gb300 import dg, inputs

pytestmark = pytest.mark.gpu


def with_rk(cfg, rk):
    return dict(cfg, disc=dict(cfg["disc"], rk=rk))


@pytest.mark.parametrize("rk", [4, 5])
@pytest.mark.parametrize("mk", [lambda: inputs.density_wave(16, 3), lambda: inputs.disc_planet(32, 2, q=1e-4),
                                lambda: inputs.gresho_vortex(20, 4)], ids=["wave", "planet-disc", "gresho"])
def test_tableau_matches_oracle(mk, rk):
    cfg = with_rk(mk(), rk)
    o = oracle.Oracle(cfg)
    g = dg.Disc(cfg)
    try:
        for k in (1, 9):
            o.step(k)
            g.step(k)
        uo = o.fetch()
        assert np.abs(g.fetch() - uo).max() <= 1e-12 * np.abs(uo).max()
        assert g.get_time()[0] == pytest.approx(o.get_time()[0], rel=1e-13)
        if cfg["planet"]["enabled"]:
            assert g.torque() == pytest.approx(o.torque()[0], rel=1e-10)
    finally:
        g.close()


@pytest.mark.parametrize("rk,order", [(3, 3), (4, 4), (5, 5)])
def test_time_order_on_the_density_wave(rk, order):
    """P1 on 8^2 (spatial operator fixed, dt within its stability limit): the
    difference between runs with dt and dt/2 to the same time falls by about
    2^order when dt halves."""
    cfg = with_rk(inputs.density_wave(8, 1), rk)
    T = 0.2

    def run(dt):
        d = dg.Disc(cfg)
        try:
            d.step_dt(int(round(T / dt)), dt)
            return d.fetch()
        finally:
            d.close()

    u1, u2, u4 = run(0.01), run(0.005), run(0.0025)
    r = np.log2(np.abs(u1 - u2).max() / np.abs(u2 - u4).max())
    assert r >= order - 0.3, r
