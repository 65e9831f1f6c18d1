"""Pins of the oracle's troubled-cell indicator and limiters (CPU only).

Each check rests on something other than the oracle's own formulas: special
cases with a known answer (a linear field is never troubled; a large TVB
constant flags nothing), invariants the method guarantees (means are kept;
the limited state passes its own test; positivity holds at every check point;
mass is conserved by a limited run), the closed form of the positivity time
step (Sec. 2.4), and the limited Shu-Osher driver against the pinned Butcher
form of SSP(3,3) when no limiter acts.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1805_01443_gb300 import inputs


def np_basis(p, x):
    V = np.polynomial.legendre.legvander(np.asarray(x, dtype=float), p)
    return V * np.sqrt(2 * np.arange(p + 1) + 1.0)


def nodal_values(u, p, pts):
    """Point values of every element at the tensor points pts x pts (numpy basis)."""
    B = np_basis(p, pts)
    m = p + 1
    c = u.reshape(u.shape[0], m, m, *u.shape[2:])
    return np.einsum("vabji,qa,rb->vqrji", c, B, B)


def linear_field(p, kind=1):
    """rho = 2 + 0.3 x + 0.2 y (exact in every degree), uniform p on a
    transmissive box."""
    cfg = inputs.uniform_state(12, p, kind=kind)
    cfg["mesh"]["bc"] = 2
    o = oracle.Oracle(cfg)
    u = o.fetch()
    u[:, 1:] = 0.0  # exact constants in the other variables (projection leaves round-off)
    m = p + 1
    dx = 1.0 / 12
    xs = (np.arange(12) + 0.5) * dx
    u[0, 0] = 2.0 + 0.3 * xs[None, :] + 0.2 * xs[:, None]
    u[0, m] = 0.3 * dx / 2 / math.sqrt(3.0)   # mode (1, 0): slope * dx/2 / sqrt(3)
    u[0, 1] = 0.2 * dx / 2 / math.sqrt(3.0)   # mode (0, 1)
    o.set_state(u)
    return o, u


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_linear_field_is_never_troubled_inside(p):
    o, _ = linear_field(p)
    f = o.indicator(0.0)  # plain minmod, the strictest test
    assert f[1:-1, 1:-1].sum() == 0
    # transmissive edges see a zero difference on their outer side
    assert f[:, 0].all() and f[0, :].all()


def wave_state(p, n=16):
    cfg = inputs.density_wave(n, p)
    o = oracle.Oracle(cfg)
    u = o.fetch() + inputs.modal_perturbation(o.shape, seed=7, amp=3e-2)
    o.set_state(u)
    return o, u


@pytest.mark.parametrize("p", [1, 3])
def test_flags_shrink_with_the_tvb_constant(p):
    o, _ = wave_state(p)
    counts = [int(o.indicator(M).sum()) for M in (0.0, 1.0, 10.0, 100.0, 1e9)]
    assert counts[0] > 0
    assert all(a >= b for a, b in zip(counts, counts[1:]))
    assert counts[-1] == 0


@pytest.mark.parametrize("p", [1, 2, 4])
def test_limiter_keeps_means_and_passes_its_own_test(p):
    o, u = wave_state(p)
    cfg = dict(o.cfg)
    cfg["disc"] = dict(cfg["disc"], limiter=1, tvb_m=0.0)
    lim = oracle.Oracle(cfg)
    lim.set_state(u)
    before = lim.indicator(0.0)
    assert before.sum() > 0
    lim.limit()
    v = lim.fetch()
    m = p + 1
    np.testing.assert_array_equal(v[:, 0], u[:, 0])
    # troubled elements hold only the mean and the two linear modes
    keep = np.zeros((m * m,), bool)
    keep[[0, 1, m]] = True
    assert np.all(v[:, ~keep][..., before.astype(bool)] == 0.0)
    # untouched elements are unchanged
    np.testing.assert_array_equal(v[..., ~before.astype(bool)], u[..., ~before.astype(bool)])
    # the limited state passes its own test: limiting again moves it by at
    # most rounding (sqrt(3) (s / sqrt(3)) can exceed s by an ulp, which the
    # plain minmod then clips back)
    lim.limit()
    v2 = lim.fetch()
    assert np.abs(v2 - v).max() <= 4e-16 * np.abs(v).max()


def test_limit_flags_equals_limit_on_the_same_flags():
    o, u = wave_state(2)
    cfg = dict(o.cfg)
    cfg["disc"] = dict(cfg["disc"], limiter=1, tvb_m=5.0)
    a, b = oracle.Oracle(cfg), oracle.Oracle(cfg)
    a.set_state(u)
    b.set_state(u)
    flags = a.indicator(5.0)
    a.limit()
    b.limit_flags(flags)
    np.testing.assert_array_equal(a.fetch(), b.fetch())


@pytest.mark.parametrize("p", [1, 3, 4])
def test_positivity_limiter_restores_positive_points(p):
    cfg = inputs.uniform_state(8, p, kind=1)
    cfg["disc"]["positivity"] = 1
    o = oracle.Oracle(cfg)
    u = o.fetch()
    m = p + 1
    rng = np.random.default_rng(3)
    # large random high modes: negative density and pressure at many points
    u[:, 1:] = rng.uniform(-0.8, 0.8, size=u[:, 1:].shape)
    u[3, 0] = 3.0
    o.set_state(u)
    o.limit()
    v = o.fetch()
    np.testing.assert_array_equal(v[:, 0], u[:, 0])
    xg, _ = np.polynomial.legendre.leggauss(m)
    pts_vol = nodal_values(v, p, xg)
    faces = np.concatenate([nodal_values(v, p, np.array([s]))[:, :, 0] for s in (-1.0, 1.0)], axis=1)
    rho = pts_vol[0]
    assert rho.min() >= 1e-13 * (1 - 1e-9) - 1e-15
    E, mx, my = pts_vol[3], pts_vol[1], pts_vol[2]
    pres = 0.4 * (E - 0.5 * (mx ** 2 + my ** 2) / rho)
    assert pres.min() >= -1e-12
    assert np.isfinite(faces).all()
    # a state that is already positive everywhere is left alone
    w = oracle.Oracle(cfg)
    u2 = w.fetch()
    u2[:, 1:] = 1e-3 * rng.uniform(-1, 1, size=u2[:, 1:].shape)
    w.set_state(u2)
    w.limit()
    np.testing.assert_array_equal(w.fetch(), u2)


@pytest.mark.parametrize("p,expect", [(1, 1 / 4), (2, 1 / 12), (3, 1 / 12), (4, 1 / 24)])
def test_positivity_time_step_closed_form(p, expect):
    """Sec. 2.4: C min(1/(2p+1), w_1/2), w_1 the endpoint weight of the
    N-point Gauss-Lobatto rule (N = 2, 3, 3, 4 for p = 1..4: weights 1/2,
    1/6, 1/6, 1/12 normalised to sum 1)."""
    cfg = inputs.uniform_state(10, p, kind=1, vx0=0.3, vy0=-0.2)
    plain = oracle.Oracle(cfg).cfl_dt()
    cfg["disc"]["positivity"] = 1
    pos = oracle.Oracle(cfg).cfl_dt()
    assert pos / plain == pytest.approx(min(1 / (2 * p + 1), expect) * (2 * p + 1), rel=1e-14)


def test_shu_osher_driver_equals_butcher_form_without_limiting():
    cfg = inputs.density_wave(12, 3)
    a, b = oracle.Oracle(cfg), oracle.Oracle(cfg)
    u = a.fetch() + inputs.modal_perturbation(a.shape, seed=2, amp=1e-2)
    a.set_state(u)
    b.set_state(u)
    a.step(4)
    b.step_so(4)
    ua, ub = a.fetch(), b.fetch()
    assert np.abs(ua - ub).max() <= 1e-13 * np.abs(ua).max()
    assert a.get_time() == pytest.approx(b.get_time(), rel=1e-14)


def test_limited_run_conserves_mass_periodic():
    cfg = inputs.density_wave(16, 2, amp=0.6)
    cfg["disc"].update({"limiter": 1, "tvb_m": 0.0, "positivity": 1})
    o = oracle.Oracle(cfg)
    m0 = o.fetch()[:, 0].sum(axis=(1, 2))
    o.step(20)
    m1 = o.fetch()[:, 0].sum(axis=(1, 2))
    np.testing.assert_allclose(m1, m0, rtol=1e-13, atol=1e-13)


def test_shock_ring_pressure_step():
    """ic 3: the disc of ic 0 with pressure x10 inside r < 1.5.  Inside the
    ring only the energy differs, by 9 p/(gamma - 1) with p = h^2 v_K^2 Sigma
    of the disc (Sec. 5.1): compared with a numpy projection of that p."""
    ring = inputs.shock_ring(32, 2, limiter=0, positivity=0)
    ring["disc"]["noise_amp"] = 0.0
    disc = inputs.shock_ring(32, 2, limiter=0, positivity=0)
    disc["disc"].update({"noise_amp": 0.0, "ic": 0})
    ur, ud = oracle.Oracle(ring).fetch(), oracle.Oracle(disc).fetch()
    np.testing.assert_array_equal(ur[:3], ud[:3])
    n, dx = 32, 5.0 / 32
    xc = -2.5 + (np.arange(n) + 0.5) * dx
    R = np.hypot(xc[None, :], xc[:, None])
    xg, wg = np.polynomial.legendre.leggauss(10)
    checked = 0
    for j in range(n):
        for i in range(n):
            if 0.5 < R[j, i] < 1.5 - dx:
                X = xc[i] + 0.5 * dx * xg[:, None]
                Y = xc[j] + 0.5 * dx * xg[None, :]
                r = np.hypot(X, Y)
                pmean = 0.25 * np.einsum("q,r,qr->", wg, wg, 0.05 ** 2 * r ** -1.5)
                assert (ur[3, 0, j, i] - ud[3, 0, j, i]) * 0.4 / 9.0 == pytest.approx(pmean, rel=1e-5)
                checked += 1
            elif R[j, i] > 1.5 + dx:
                assert np.array_equal(ur[3, :, j, i], ud[3, :, j, i])
    assert checked > 50


# ---- worked cases: the values the limiters produce, computed by hand ----------
#
# A periodic 3 x 3 mesh of elements dx = 0.5 by dy = 0.25 (box [0, 1.5] x
# [0, 0.75]).  Element means rho(i, j) = a_i + b_j with a = (1.0, 1.5, 1.7) and
# b = (0.0, 0.4, 0.5), so the centre element (1, 1) sees
#   x: forward difference 1.7 - 1.5 = 0.2, backward 1.5 - 1.0 = 0.5
#   y: forward difference 0.5 - 0.4 = 0.1, backward 0.4 - 0.0 = 0.4
# Its face increments (the linear mode times phi_1(+1) = sqrt(3)) are 0.35 in x
# and -0.3 in y; every other element has no linear mode and is never troubled.
# Plain minmod (M = 0) gives minmod(0.35, 0.2, 0.5) = 0.2 in x and
# minmod(-0.3, 0.1, 0.4) = 0 in y.  The TVB bound M h^2 keeps the x increment
# for M >= 0.35 / 0.5^2 = 1.4 and the y increment for M >= 0.3 / 0.25^2 = 4.8.

SQ3 = math.sqrt(3.0)


def tvb_worked_case(p, tvb_m):
    cfg = inputs.uniform_state(3, p, kind=1)
    cfg["mesh"].update({"x1": 1.5, "y1": 0.75, "bc": 0})
    cfg["disc"].update({"limiter": 1, "tvb_m": tvb_m, "positivity": 0})
    o = oracle.Oracle(cfg)
    m = p + 1
    rng = np.random.default_rng(11)
    u = np.zeros(o.shape)
    u[:, 1:] = rng.uniform(-0.05, 0.05, size=u[:, 1:].shape)  # higher modes everywhere
    u[:, m] = 0.0   # no linear modes ...
    u[:, 1] = 0.0
    a, b = np.array([1.0, 1.5, 1.7]), np.array([0.0, 0.4, 0.5])
    u[0, 0] = a[None, :] + b[:, None]
    u[1:, 0] = np.array([0.1, -0.2, 3.0])[:, None, None]
    u[0, m, 1, 1] = 0.35 / SQ3   # ... except the centre element's density
    u[0, 1, 1, 1] = -0.3 / SQ3
    o.set_state(u)
    return o, u


@pytest.mark.parametrize("tvb_m,flag", [(0.0, 1), (1.39, 1), (1.41, 1), (4.79, 1), (4.81, 0), (50.0, 0)])
def test_tvb_flag_flips_at_m_h_squared(tvb_m, flag):
    o, _ = tvb_worked_case(2, tvb_m)
    f = o.indicator(tvb_m)
    expect = np.zeros((3, 3), np.uint8)
    expect[1, 1] = flag
    np.testing.assert_array_equal(f, expect)


@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("tvb_m,sx,sy", [(0.0, 0.2, 0.0), (1.39, 0.2, 0.0), (3.0, 0.35, 0.0)])
def test_tvb_limited_linear_modes_worked_case(p, tvb_m, sx, sy):
    """The troubled centre element becomes its means plus the limited face
    increments divided by sqrt(3); all its other modes vanish, in every
    variable; the other elements are untouched."""
    o, u = tvb_worked_case(p, tvb_m)
    o.limit()
    v = o.fetch()
    m = p + 1
    c = v[:, :, 1, 1]
    np.testing.assert_array_equal(c[:, 0], u[:, 0, 1, 1])
    assert c[0, m] == pytest.approx(sx / SQ3, rel=1e-15, abs=1e-17)
    assert c[0, 1] == pytest.approx(sy / SQ3, abs=1e-17)
    rest = np.ones(m * m, bool)
    rest[[0, 1, m]] = False
    assert np.all(c[:, rest] == 0.0)
    assert np.all(c[1:, [1, m]] == 0.0)
    others = np.ones((3, 3), bool)
    others[1, 1] = False
    np.testing.assert_array_equal(v[..., others], u[..., others])


# A single P1 element (periodic 1 x 1 mesh, so it is its own neighbour) with
# mean density 1 and face increment sqrt(3) u_10 = 1.5 in x: the density is
# negative at the face x = -1 (a check point) but positive at the volume
# nodes xi = +-1/sqrt(3).  Zhang & Shu's scaling (Sec. 2.4) with eps = 1e-13
# is theta = (1 - eps) / (1 - rho_min), applied to every non-mean mode of the
# density.  Then the pressure: uniform density 1, no momentum,
# energy mean 1 and energy increment 2 give p = 0.4 (1 + 2 xi), -0.4 at
# x = -1 against a mean pressure 0.4: theta = (0.4 - eps) / (0.4 + 0.4) on
# the non-mean modes of every variable.

def positivity_element_case():
    cfg = inputs.uniform_state(1, 1, kind=1)
    cfg["disc"].update({"positivity": 1, "limiter": 0})
    o = oracle.Oracle(cfg)
    return o


def test_positivity_theta_for_the_density_closed_form():
    o = positivity_element_case()
    u = np.zeros(o.shape)
    u[0, 0] = 1.0
    u[0, 2] = 1.5 / SQ3          # mode (1, 0) of the density
    u[0, 1] = 0.01               # mode (0, 1): +-0.01 sqrt(3) at the face points
    u[3, 0] = 5.0                # plenty of energy: the pressure stays positive
    o.set_state(u)
    o.limit()
    v = o.fetch()
    # rho = 1 + 1.5 xi + 0.01 sqrt(3) eta; its smallest check-point value is at
    # the face x = -1, eta = -1/sqrt(3): 1 - 1.5 - 0.01 = -0.51 (the face
    # y = -1 gives 1 - 1.5/sqrt(3) - 0.01 sqrt(3) > 0, the volume nodes more)
    theta = (1.0 - 1e-13) / (1.0 + 0.51)
    assert theta == pytest.approx(0.66225165563, rel=1e-10)
    np.testing.assert_allclose(v[0, 1:], theta * u[0, 1:], rtol=1e-14, atol=0)
    assert v[0, 0] == 1.0
    np.testing.assert_array_equal(v[1:], u[1:])


def test_positivity_theta_for_the_pressure_closed_form():
    o = positivity_element_case()
    u = np.zeros(o.shape)
    u[0, 0] = 1.0
    u[3, 0] = 1.0
    u[3, 2] = 2.0 / SQ3          # energy increment 2 in x
    u[3, 1] = 0.1                # and a y mode that the scaling shrinks too
    u[1, 3] = 0.02               # a momentum mode (1, 1), small enough to keep rho v^2 tiny
    o.set_state(u)
    o.limit()
    v = o.fetch()
    # at the check point x = -1, eta = -1/sqrt(3): E = 1 - 2 - 0.1 = -1.1 and
    # the kinetic term 0.5 (0.02 * sqrt(3) * (-1) * (-1))^2 = 0.0006, so
    # p = 0.4 (-1.1 - 0.0006); the mean pressure is 0.4
    pmin = 0.4 * (-1.1 - 0.5 * (0.02 * 3.0 * (-1.0 / SQ3) * (-1.0)) ** 2)
    theta = (0.4 - 1e-13) / (0.4 - pmin)
    assert theta == pytest.approx(0.4 / (0.4 + 0.44024), rel=1e-10)
    np.testing.assert_allclose(v[:, 1:], theta * u[:, 1:], rtol=1e-13, atol=0)
    np.testing.assert_array_equal(v[:, 0], u[:, 0])
