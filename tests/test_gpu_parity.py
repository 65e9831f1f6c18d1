"""GPU parity of the FP64 CUDA path (through the C ABI) against the FP64 CPU oracle.

Both sides receive the same seeded inputs (the oracle's projected initial data,
plus seeded modal perturbations from paper_1805_01443_gb300.inputs) through
dg_set_state / ref_set_state.  Tolerances (FP64 path):
  * states: relative L2 per variable <= 1e-12, and element by element
    max |du| <= 1e-12 max |u| per variable;
  * operator L(u): ||dL|| <= 1e-12 ||L|| + 1e-15 ||u|| / dt_CFL per variable,
    and the same element by element in the max norm.  L is a near-cancelling
    sum of flux and source terms of size ~||u|| / dt_CFL (the stage update
    dt L relative to u), whose rounding differs between the two sides; the
    second term bounds that rounding (measured ~5e-17 of it on the GB300,
    with ||dL|| / ||L|| at most 4e-13);
  * torque: |dGamma| <= 1e-12 sum_n |Gamma_n| (the torque is a near-cancelling sum);
  * initial projection: relative L2 <= 1e-13.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1805_01443_gb300 import dg, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def rel_l2(a, b):
    return np.array([np.linalg.norm(a[v] - b[v]) / max(np.linalg.norm(b[v]), 1e-300)
                     for v in range(a.shape[0])])


def make_pair(cfg, perturb=0.0, seed=11):
    o = oracle.Oracle(cfg)
    g = dg.Disc(cfg)
    u0 = o.fetch()
    if perturb:
        u0 = u0 + inputs.modal_perturbation(o.shape, seed=seed, amp=perturb)
    o.set_state(u0)
    g.set_state(u0)
    return o, g, u0


def run_pair(o, g, nsteps):
    gz_o, ab_o = [], []
    for _ in range(nsteps):
        o.step(1)
        gz, ab = o.torque()
        gz_o.append(gz)
        ab_o.append(ab)
    g.step(nsteps)
    return np.array(gz_o), np.array(ab_o)


def max_rel(a, b):
    """Per variable: the largest element difference over the largest |element|."""
    return np.array([np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(a.shape[0])])


def assert_state_parity(o, g, tol=TOL):
    uo, ug = o.fetch(), g.fetch()
    err = rel_l2(ug, uo)
    assert np.all(err <= tol), err
    emax = max_rel(ug, uo)
    assert np.all(emax <= tol), emax
    to, dto, so = o.get_time()
    tg, dtg, sg = g.get_time()
    assert so == sg
    assert abs(tg - to) <= 1e-14 * max(abs(to), 1e-300) + 1e-300


# ----------------------------------------------------------------------------


@pytest.mark.parametrize("cfg", [
    inputs.disc_small(16, 2),
    inputs.disc_planet(24, 4),
    inputs.density_wave(12, 3),
    inputs.uniform_state(5, 1, kind=1, vx0=0.2),
    # odd nx and even ny: ragged tiles, and the origin (where Sigma ~ r^-1/2 is
    # singular) stays on an element edge, never on a quadrature node
    dict(inputs.disc_small(37, 3), mesh=dict(inputs.disc_small(37, 3)["mesh"], ny=22)),
], ids=["disc_p2", "planet_p4", "wave_p3", "uniform_p1", "ragged_37x22_p3"])
def test_initial_projection_parity(cfg):
    o = oracle.Oracle(cfg)
    with dg.Disc(cfg) as g:
        err = rel_l2(g.fetch(), o.fetch())
        assert np.all(err <= 1e-13), err
        # first CFL step from the element averages
        assert abs(g.get_time()[1] - o.cfl_dt()) <= 1e-14 * o.cfl_dt()


CASES = []
for p in [1, 2, 3, 4]:
    CASES.append(("disc", p, 37, 10))
    CASES.append(("wave", p, 12, 7))
    CASES.append(("transmissive", p, 10, 6))
CASES.append(("disc", 4, 64, 3))
CASES.append(("wave", 2, 1, 1))
CASES.append(("wave", 3, 33, 2))


def case_cfg(kind, p, nx, ny):
    if kind == "disc":
        cfg = inputs.disc_planet(nx, p)
        cfg["mesh"]["ny"] = ny
        cfg["mesh"]["y0"], cfg["mesh"]["y1"] = -0.6, 0.6
    elif kind == "wave":
        cfg = inputs.density_wave(nx, p)
        cfg["mesh"]["ny"] = ny
    else:
        cfg = inputs.uniform_state(nx, p, kind=2, vx0=0.3, vy0=-0.1, bc=2, h=0.5)
        cfg["mesh"]["ny"] = ny
    return cfg


@pytest.mark.parametrize("kind,p,nx,ny", CASES)
def test_operator_parity(kind, p, nx, ny):
    cfg = case_cfg(kind, p, nx, ny)
    o, g, u0 = make_pair(cfg, perturb=1e-3)
    Lo, Lg = o.rhs(), g.rhs()
    dt = o.cfl_dt()
    for v in range(u0.shape[0]):
        bound = TOL * np.linalg.norm(Lo[v]) + 1e-15 * np.linalg.norm(u0[v]) / dt
        assert np.linalg.norm(Lg[v] - Lo[v]) <= bound, (v, np.linalg.norm(Lg[v] - Lo[v]), bound)
        bmax = TOL * np.abs(Lo[v]).max() + 1e-15 * np.abs(u0[v]).max() / dt
        assert np.abs(Lg[v] - Lo[v]).max() <= bmax, (v, np.abs(Lg[v] - Lo[v]).max(), bmax)
    g.close()


@pytest.mark.parametrize("kind,p,nx,ny", CASES)
def test_step_parity_small(kind, p, nx, ny):
    cfg = case_cfg(kind, p, nx, ny)
    o, g, _ = make_pair(cfg, perturb=1e-3)
    gz_o, ab_o = run_pair(o, g, 3)
    assert_state_parity(o, g)
    gz_g = g.torque_series()
    assert len(gz_g) == 3
    assert np.all(np.abs(gz_g - gz_o) <= TOL * ab_o)
    g.close()


def test_disc_p2_64_fifty_steps():
    """Locally isothermal disc, P2 on 64x64, no planet: 1 step and 50 steps."""
    cfg = inputs.disc_small(64, 2)
    o, g, _ = make_pair(cfg)
    run_pair(o, g, 1)
    assert_state_parity(o, g)
    gz_o, ab_o = run_pair(o, g, 49)
    assert_state_parity(o, g)
    gz_g = g.torque_series()
    assert len(gz_g) == 50
    assert np.all(np.abs(gz_g[1:] - gz_o) <= TOL * ab_o)
    g.close()


def test_planet_disc_p4_256_two_hundred_steps():
    """Planet-disc P4 on 256x256, q = 1e-5, damping zones: 200 steps, state and
    every step's torque."""
    cfg = inputs.disc_planet(256, 4)
    o, g, _ = make_pair(cfg)
    gz_o, ab_o = run_pair(o, g, 200)
    assert_state_parity(o, g)
    gz_g = g.torque_series()
    assert len(gz_g) == 200
    err = np.abs(gz_g - gz_o) / ab_o
    assert np.all(err <= TOL), err.max()
    g.close()


def test_planet_disc_p4_512_full_size_step():
    """The P4 512x512 workload at full size, in the benchmark's launch
    configuration: one step, state and torque."""
    cfg = inputs.disc_planet_512()
    o, g, _ = make_pair(cfg)
    gz_o, ab_o = run_pair(o, g, 1)
    assert_state_parity(o, g)
    assert abs(g.torque() - gz_o[0]) <= TOL * ab_o[0]
    g.close()


def test_ssp22_and_fixed_dt_parity():
    cfg = inputs.disc_planet(24, 3)
    cfg["disc"]["rk"] = 2
    o, g, _ = make_pair(cfg, perturb=1e-4)
    o.step_dt(4, 2e-3)
    g.step_dt(4, 2e-3)
    assert_state_parity(o, g)
    g.close()


def test_conservation_on_gpu():
    cfg = inputs.density_wave(16, 3)
    o, g, u0 = make_pair(cfg, perturb=1e-2)
    c0 = g.conserved()
    tot = u0[:, 0].sum(axis=(1, 2)) / 256.0
    np.testing.assert_allclose(c0, tot, rtol=1e-13, atol=1e-15)
    g.step(25)
    np.testing.assert_allclose(g.conserved(), c0, rtol=0, atol=1e-13 * np.abs(c0).max())
    g.close()


def test_set_fetch_roundtrip_and_resume_bit_identical():
    cfg = inputs.disc_planet(40, 2)
    u0 = oracle.Oracle(cfg).fetch() + inputs.modal_perturbation((3, 9, 40, 40), seed=5, amp=1e-4)
    with dg.Disc(cfg) as a, dg.Disc(cfg, torch_memory=False) as b:
        a.set_state(u0, t=0.25, step=7)
        assert np.array_equal(a.fetch(), u0)
        a.step(10)
        b.set_state(u0, t=0.25, step=7)
        b.step(4)
        mid = b.fetch()
        t, _, st = b.get_time()
        b.set_state(mid, t=t, step=st)
        b.step(6)
        assert np.array_equal(a.fetch(), b.fetch())
        assert a.get_time() == b.get_time()


def test_numeric_failure_is_reported_and_state_kept():
    cfg = inputs.uniform_state(8, 2, kind=1, vx0=0.5)
    with dg.Disc(cfg) as g:
        u = g.fetch()
        bad = u.copy()
        bad[0, 0, 3, 4] = float("nan")
        with pytest.raises(dg.DgError) as e:
            g.set_state(bad)
        assert e.value.code == dg.DG_ERR_NUMERIC
        bad = u.copy()
        bad[0, 0, 2, 2] = -1.0
        with pytest.raises(dg.DgError) as e:
            g.set_state(bad)
        assert e.value.code == dg.DG_ERR_NUMERIC
        # a good state clears the status; a step far beyond the CFL limit fails and
        # leaves the state at the last good step
        pert = u + inputs.modal_perturbation(u.shape, seed=2, amp=0.3)
        g.set_state(pert)
        g.step(1)
        good = g.fetch()
        g.step_dt(3, 50.0)
        with pytest.raises(dg.DgError) as e:
            g.sync()
        assert e.value.code == dg.DG_ERR_NUMERIC
        with pytest.raises(dg.DgError):
            g.fetch()
        out = np.empty_like(good)
        rc = dg.lib().dg_fetch(g.h, dg._ptr(out))
        assert rc == dg.DG_ERR_NUMERIC
        assert np.array_equal(out, good)


def test_torch_stream_and_workspace():
    import torch
    cfg = inputs.disc_planet(32, 3)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = dg.Disc(cfg)
    b = dg.Disc(cfg, torch_memory=False)
    a.step(5)
    b.step(5)
    assert np.array_equal(a.fetch(), b.fetch())
    a.close()
    b.close()
