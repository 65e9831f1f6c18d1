"""Precision form (dg_disc.prec = 1) against the FP64 oracle and the FP64 GPU path.

The precision form evaluates the operator in FP32 on the perturbation about the
projected equilibrium (FP64 background residual, FP64 torque reduction and
sums).  Stated bounds, per result:
  * operator L(u): ||dL|| <= 1e-6 ||L|| per variable (FP32 rounding of the
    perturbation terms is ~1e-7);
  * states: relative L2 on Sigma <= 1e-5 and on momentum <= 1e-5;
  * torque: relative L2 of the per-step torque series <= 1e-6; on the same
    state, the precision-form torque (float-float terms) matches the FP64
    oracle to <= 1e-7 relative and <= 1e-11 of the sum of |terms|;
  * the perturbation itself, Sigma - Sigma_bg, the honest measure of the
    form's error: relative L2 <= 3e-5 after 200 steps at 128^2 (measured
    3.8e-6 on the GB300), <= 1e-4 after 1000 steps at 512^2 (3.1e-5), and the
    change of Sigma over one full-size 512^2 step <= 2e-5 (1.6e-6).
"""
import numpy as np
import pytest

import oracle
from paper_1805_01443_gb300 import dg, inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def prec_cfg(cfg):
    c = {k: (dict(v) if isinstance(v, dict) else v) for k, v in cfg.items()}
    c["disc"]["prec"] = 1
    return c


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def background_sigma(cfg):
    bg = {k: (dict(v) if isinstance(v, dict) else v) for k, v in cfg.items()}
    bg["disc"]["noise_amp"] = 0.0
    return oracle.Oracle(bg).fetch()[0]


@pytest.mark.parametrize("n,p,bc", [(64, 4, 1), (48, 3, 1), (40, 2, 1), (33, 1, 1), (40, 3, 0), (36, 4, 2),
                                    (40, 2, 3), (34, 4, 0)])
def test_precision_operator(n, p, bc):
    """L(u) of the precision form against the oracle for every boundary kind:
    background ghosts (1), the periodic wrap (0: the neighbour's background
    is the far edge's), mirrored traces (2) and copied boundary elements (3:
    the copy's background is at the element's opposite face)."""
    cfg = inputs.disc_planet(n, p)
    cfg["mesh"]["bc"] = bc
    o = oracle.Oracle(cfg)
    with dg.Disc(prec_cfg(cfg)) as g:
        u0 = o.fetch() + inputs.modal_perturbation(o.shape, seed=4, amp=1e-4)
        o.set_state(u0)
        g.set_state(u0)
        # the state round trip u_b + (float)(u - u_b) keeps the FP64 background
        assert rel(g.fetch()[0], u0[0]) < 1e-10
        Lo, Lg = o.rhs(), g.rhs()
        for v in range(3):
            assert np.linalg.norm(Lg[v] - Lo[v]) <= 1e-6 * np.linalg.norm(Lo[v]), v


def test_precision_planet_disc_p4_128_vs_oracle():
    """P4 128x128 planet disc, q = 3e-5, 200 steps against the FP64 oracle."""
    cfg = inputs.disc_planet(128, 4, q=3e-5)
    o = oracle.Oracle(cfg)
    with dg.Disc(prec_cfg(cfg)) as g:
        u0 = o.fetch()
        g.set_state(u0)
        tq = []
        for _ in range(200):
            o.step(1)
            tq.append(o.torque()[0])
        g.step(200)
        uo, ug = o.fetch(), g.fetch()
        tg = g.torque_series()
        sb = background_sigma(cfg)
        assert rel(ug[0], uo[0]) <= 1e-5
        assert max(rel(ug[1], uo[1]), rel(ug[2], uo[2])) <= 1e-5
        assert rel(ug[0] - sb, uo[0] - sb) <= 3e-5
        assert np.abs(ug[0] - uo[0]).max() <= 3e-5 * np.abs(uo[0] - sb).max()
        assert rel(tg, np.array(tq)) <= 1e-6
        assert g.get_time()[2] == 200


def strip(p, nx, ny, yc):
    """The planet disc on a strip of square elements centred at height yc."""
    cfg = inputs.disc_planet(nx, p, q=3e-5)
    cfg["mesh"]["ny"] = ny
    h = 0.5 * 5.0 * ny / nx
    cfg["mesh"]["y0"], cfg["mesh"]["y1"] = yc - h, yc + h
    return cfg


@pytest.mark.parametrize("p,nx,ny,yc", [(3, 38, 10, 0.0), (4, 70, 6, 0.0), (2, 34, 1, 1.3), (1, 66, 2, -1.0)])
def test_precision_steps_ragged_meshes(p, nx, ny, yc):
    """Strips with ragged 32-element tiles (tails of 6, 6, 2 and 2 elements),
    one or a few rows, damping zones and the planet: 20 steps against the FP64
    oracle (the last stage's zone-first CTA order, the tail tiles' torque
    partials and boundary rows that are both bottom and top all take part).
    Even element counts, as in every configuration of the method: an odd
    count in both directions centres an element on the star, whose
    r^-1/2 density cusp then blows the solution up (in the oracle too)."""
    cfg = strip(p, nx, ny, yc)
    o = oracle.Oracle(cfg)
    with dg.Disc(prec_cfg(cfg)) as g:
        g.set_state(o.fetch())
        tq = []
        for _ in range(20):
            o.step(1)
            tq.append(o.torque()[0])
        g.step(20)
        uo, ug = o.fetch(), g.fetch()
        assert rel(ug[0], uo[0]) <= 1e-5
        assert max(rel(ug[1], uo[1]), rel(ug[2], uo[2])) <= 1e-5
        assert rel(g.torque_series(), np.array(tq)) <= 1e-6
        assert g.get_time()[2] == 20


@pytest.mark.parametrize("prec", [0, 1])
def test_zero_wave_speed_element_is_no_cfl_constraint(prec):
    """An element centred on the star (odd counts in both directions) has no
    sound speed at its centre and no mean velocity: its CFL bound is +inf,
    which the step minimum ignores, as in the oracle; the time step matches."""
    cfg = strip(3, 37, 9, 0.0)
    o = oracle.Oracle(cfg)
    u = o.fetch()
    u[1:3, 0, 4, 18] = 0.0  # the element at the origin: no mean momentum (and c_s = 0 at its centre)
    o.set_state(u)
    with dg.Disc(dict(cfg, disc=dict(cfg["disc"], prec=prec))) as g:
        g.set_state(u)
        dt = g.get_time()[1]
        assert np.isfinite(dt) and dt > 0.0
        assert dt == pytest.approx(o.cfl_dt(), rel=1e-12)


def test_precision_planet_disc_p4_512_thousand_steps():
    """The precision-form workload at full size: P4 512x512, q = 3e-5, 1000 steps,
    against the FP64 GPU path (itself matched to the oracle to 1e-12)."""
    cfg = inputs.disc_planet_512()
    with dg.Disc(cfg) as a, dg.Disc(prec_cfg(cfg)) as p:
        a.step(1000)
        p.step(1000)
        ua, up = a.fetch(), p.fetch()
        ta, tp = a.torque_series(), p.torque_series()
        sb = a.fetch()[0] * 0
    with dg.Disc(dict(cfg, disc=dict(cfg["disc"], noise_amp=0.0))) as b:
        sb = b.fetch()[0]
    e_sig = rel(up[0], ua[0])
    e_pert = rel(up[0] - sb, ua[0] - sb)
    e_tq = rel(tp, ta)
    print("P4 512^2, 1000 steps: rel L2 Sigma %.2e, Sigma - Sigma_bg %.2e, torque %.2e"
          % (e_sig, e_pert, e_tq))
    assert e_sig <= 1e-5
    assert max(rel(up[1], ua[1]), rel(up[2], ua[2])) <= 1e-5
    assert e_pert <= 1e-4
    assert e_tq <= 1e-6


def test_precision_planet_disc_p4_512_full_size_step_vs_oracle():
    """The benchmark's workload and launch configuration (P4 512x512, q = 3e-5,
    precision form), one SSP(3,3) step at the oracle's CFL step, against the
    oracle directly: the whole state within the form's bounds, element by
    element within 1e-9 of each variable's largest coefficient, every
    element's density mean within 1e-10 of the largest one, the change of
    Sigma over the step within 2e-5, and the torque within 1e-6 (measured on
    the GB300: 1.3e-11, 7.4e-13, 1.6e-6 and 3.5e-8)."""
    cfg = inputs.disc_planet_512()
    o = oracle.Oracle(cfg)
    dt = o.cfl_dt()
    with dg.Disc(prec_cfg(cfg)) as g:
        u0 = o.fetch()
        g.set_state(u0)
        o.step_dt(1, dt)
        g.step_dt(1, dt)
        uo, ug = o.fetch(), g.fetch()
        tg = g.torque()
    to = o.torque()[0]
    assert rel(ug[0], uo[0]) <= 1e-5
    assert max(rel(ug[1], uo[1]), rel(ug[2], uo[2])) <= 1e-5
    for v in range(3):
        assert np.abs(ug[v] - uo[v]).max() <= 1e-9 * np.abs(uo[v]).max(), v
    assert rel(ug[0] - u0[0], uo[0] - u0[0]) <= 2e-5
    assert np.abs(ug[0, 0] - uo[0, 0]).max() <= 1e-10 * np.abs(uo[0, 0]).max()
    assert abs(tg - to) <= 1e-6 * abs(to)


@pytest.mark.parametrize("n,p,q", [(128, 4, 3e-5), (96, 3, 1e-4), (64, 2, 1e-3), (40, 1, 1e-3)])
def test_precision_torque_same_state(n, p, q):
    """The torque kernel alone: the precision form's torque of its own state
    against the FP64 oracle's torque of that same state (fetched as
    u_b + delta in FP64), at several steps."""
    cfg = prec_cfg(inputs.disc_planet(n, p, q=q))
    o = oracle.Oracle(inputs.disc_planet(n, p, q=q))
    with dg.Disc(cfg) as g:
        for k in (1, 7, 20):
            g.step(k)
            tg = g.torque_series()[-1]
            t, _, st = g.get_time()
            o.set_state(g.fetch(), t, st)
            gz, asum = o.torque_now(t)
            assert abs(tg - gz) <= 1e-7 * abs(gz), (k, tg, gz)
            assert abs(tg - gz) <= 1e-11 * asum, (k, tg, gz, asum)


def test_precision_conserved_sums_in_fp64():
    cfg = inputs.disc_small(64, 2)
    with dg.Disc(cfg) as a, dg.Disc(prec_cfg(cfg)) as p:
        c0 = a.conserved()
        np.testing.assert_allclose(p.conserved(), c0, rtol=0, atol=1e-12 * abs(c0[0]))
        a.step(20)
        p.step(20)
        # FP32 stepping of the perturbation: totals agree to ~1e-8 of the mass
        np.testing.assert_allclose(p.conserved(), a.conserved(), rtol=0, atol=1e-8 * abs(c0[0]))


def test_precision_form_rejects_other_eos():
    cfg = prec_cfg(inputs.density_wave(8, 2))
    with pytest.raises(dg.DgError) as e:
        dg.Disc(cfg)
    assert e.value.code == dg.DG_ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", [0, 1])
def test_set_state_from_pinned_memory_reads_in_place(prec):
    """A page-locked host buffer is read in place by the conversion kernel,
    ordinary host memory is staged by a copy: both give the same state, bit
    for bit, and the same steps after it (ragged 32-element tiles: nx = 40)."""
    cfg = inputs.disc_planet(40, 3)
    cfg["mesh"]["ny"] = 36
    cfg["disc"]["prec"] = prec
    a, b = dg.Disc(cfg), dg.Disc(cfg)
    try:
        a.step(2)
        u = a.fetch()
        t, _, st = a.get_time()
        pinned_t = torch.empty(u.shape, dtype=torch.float64, pin_memory=True)
        pinned = pinned_t.numpy()
        pinned[...] = u + 1e-9 * np.sin(np.arange(u.size)).reshape(u.shape)
        plain = pinned.copy()
        a.set_state(pinned, t, st)
        b.set_state(plain, t, st)
        np.testing.assert_array_equal(a.fetch(), b.fetch())
        assert a.get_time() == b.get_time()
        a.step(3)
        b.step(3)
        np.testing.assert_array_equal(a.fetch(), b.fetch())
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_stage_timing_counts_every_stage_launch(prec):
    """dg_set_timing / dg_timing: the records cover every stage launch (three
    per SSP(3,3) step in both forms) and the kernel time is a part of the
    step time."""
    cfg = inputs.disc_planet(64, 3)
    cfg["disc"]["prec"] = prec
    with dg.Disc(cfg) as g:
        g.step(1)
        g.sync()
        g.set_timing(True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        g.step(5)
        b.record()
        b.synchronize()
        ms, n = g.timing()
        g.set_timing(False)
        assert n == 15
        assert 0.0 < ms <= a.elapsed_time(b)
        assert g.timing() == (0.0, 0)


@pytest.mark.parametrize("prec", [0, 1])
def test_async_upload_pipeline_matches_synchronous_calls(prec):
    """dg_set_state_async / dg_torque_async in a pipelined loop (the upload of
    step k+1 queued while step k runs, each step's torque read without
    waiting) give the same torques, state and time as dg_set_state, dg_step
    and dg_torque called in turn, bit for bit; ordinary host memory is
    refused."""
    cfg = inputs.disc_planet(64, 3)
    cfg["disc"]["prec"] = prec
    with dg.Disc(cfg) as a, dg.Disc(cfg) as b:
        a.step(2)
        u = a.fetch()
        t, _, st = a.get_time()
        ups = []
        for k in range(3):
            pin = torch.empty(u.shape, dtype=torch.float64, pin_memory=True).numpy()
            pin[...] = u + 1e-8 * k * np.cos(np.arange(u.size)).reshape(u.shape)
            ups.append(pin)
        tq = torch.empty(3, dtype=torch.float64, pin_memory=True).numpy()
        a.set_state_async(ups[0], t, st)
        for k in range(3):
            a.step(1)
            a.torque_async(tq, k)
            if k + 1 < 3:
                a.set_state_async(ups[k + 1], t, st)
        a.sync()
        ref = []
        for k in range(3):
            b.set_state(ups[k].copy(), t, st)
            b.step(1)
            ref.append(b.torque())
        np.testing.assert_array_equal(tq, np.array(ref))
        np.testing.assert_array_equal(a.fetch(), b.fetch())
        assert a.get_time() == b.get_time()
        with pytest.raises(dg.DgError):
            a.set_state_async(np.zeros(u.shape), t, st)


def test_background_residual_kept_only_where_it_matters():
    """R_b = L(u_b) is kept only in tiles holding a coefficient above 1e-10 of
    its maximum (the singular centre, the softened core, the box edge); the
    precision form's operator on the noise-free background then equals the
    oracle's L(u_b) element by element within the FP32 rounding of R_b, the
    dropped part and the FP64 rounding of the operator's cancelling terms.
    R_b is stored as FP32 values at the nodes: a rounding error e_qr <=
    2^-24 |R_b(q, r)| moves mode ab by sum_qr (w_q/2)(w_r/2) phi_a phi_b e_qr,
    which by Cauchy-Schwarz and the basis' discrete orthonormality is at most
    max|phi_a phi_b| 2^-24 ||R_b||_2 over the element's modes of the variable
    (max|phi_a phi_b| at the nodes: 2.7 at P4), so the bound carries
    1.7e-7 x that element norm."""
    cfg = inputs.disc_planet(128, 4)
    cfg["disc"]["noise_amp"] = 0.0
    cfg["planet"]["enabled"] = 0
    o = oracle.Oracle(cfg)
    with dg.Disc(prec_cfg(cfg)) as g:
        n, r, z = g.prec_tiles()
        assert n == 128 * 4 and 0 < r < n and 0 < z < n
        u = o.fetch()
        g.set_state(u)
        Lo, Lg = o.rhs(), g.rhs()
        dt = o.cfl_dt()
    rmax = np.abs(Lo).max()
    enorm = np.sqrt((Lo ** 2).sum(axis=1, keepdims=True))
    bound = 1.2e-7 * np.abs(Lo) + 1.7e-7 * enorm + 1.01e-10 * rmax + 1e-15 * np.abs(u).max() / dt
    ratio = np.abs(Lg - Lo) / bound
    w = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    assert np.all(ratio <= 1.0), (float(ratio[w]), w, float(Lg[w]), float(Lo[w]), float(enorm[w[0], 0, w[2], w[3]]),
                                 float(rmax))


def test_delta_upload_matches_the_fp64_upload():
    """dg_set_delta_async (the FP32 perturbation, half the bytes) gives the
    steps of dg_set_state_async of u_b + delta, and dg_fetch_delta returns the
    delta the steps leave.  The FP64 upload recovers delta as
    (float)((u_b + delta) - u_b), which can move a coefficient far smaller
    than u_b by a few of its own FP32 units: the results agree to FP32
    rounding of delta."""
    cfg = prec_cfg(inputs.disc_planet(64, 4, q=3e-5))
    with dg.Disc(cfg) as a, dg.Disc(cfg) as b:
        a.step(3)
        delta = torch.from_numpy(a.fetch_delta()).pin_memory().numpy()
        full = torch.from_numpy(a.fetch()).pin_memory().numpy()
        t, _, st = a.get_time()
        a.set_delta_async(delta, t, st)
        b.set_state_async(full, t, st)
        a.step(4)
        b.step(4)
        a.sync()
        b.sync()
        da, db = a.fetch_delta(), b.fetch_delta()
        for v in range(3):
            assert np.abs(da[v] - db[v]).max() <= 1e-6 * np.abs(db[v]).max(), v
        assert a.get_time()[0] == pytest.approx(b.get_time()[0], rel=1e-12)
        assert a.get_time()[2] == b.get_time()[2]
        assert rel(a.torque_series(), b.torque_series()) <= 1e-7
        assert rel(a.fetch()[0], b.fetch()[0]) <= 1e-10
        # the fetched delta is the state the handle steps from
        full = a.fetch()
        c = torch.from_numpy(a.fetch_delta()).pin_memory().numpy()
        t, _, st = a.get_time()
        b.set_delta_async(c, t, st)
        b.sync()
        np.testing.assert_array_equal(b.fetch(), full)
    with dg.Disc(inputs.disc_small(16, 2)) as f64:
        with pytest.raises(dg.DgError) as e:
            f64.fetch_delta()
        assert e.value.code == dg.DG_ERR_UNSUPPORTED


def test_pipelined_delta_uploads_match_in_place_conversion():
    """dg_set_delta_async converts each upload on its own stream into a spare
    state buffer, which trades places with the current one, so that the
    conversion overlaps the steps queued before it.  A loop of uploads, steps
    and torque reads queued without waiting, with two steps between some
    uploads and an FP64 upload among them, gives the torques, state and time
    of the in-place conversion on the handle's stream (the path of a handle
    held by a batch) bit for bit."""
    cfg = prec_cfg(inputs.disc_planet(64, 4, q=3e-5))
    with dg.Disc(cfg) as a, dg.Disc(cfg) as b, dg.Disc(cfg) as src:
        src.step(3)
        d0 = src.fetch_delta()
        t, _, st = src.get_time()
        pins = []
        for k in range(5):
            pin = torch.empty(d0.shape, dtype=torch.float32, pin_memory=True).numpy()
            pin[...] = d0 * np.float32(1.0 + 1e-3 * k)
            pins.append(pin)
        full = torch.empty(src.shape, dtype=torch.float64, pin_memory=True).numpy()
        full[...] = src.fetch()
        nsteps = [1, 2, 1, 1, 2]
        tq = torch.empty(8, dtype=torch.float64, pin_memory=True).numpy()
        tr = torch.empty(8, dtype=torch.float64, pin_memory=True).numpy()
        held = dg.Batch([b])  # b's uploads now convert in place
        try:
            for d, rec in ((a, tq), (b, tr)):
                i = 0
                for k in range(5):
                    if k == 3:
                        d.set_state_async(full, t, st)
                        d.step(1)
                        d.torque_async(rec, i)
                        i += 1
                    d.set_delta_async(pins[k], t + k, st + k)
                    for _ in range(nsteps[k]):
                        d.step(1)
                        d.torque_async(rec, i)
                        i += 1
                    if d is b:
                        d.sync()  # nothing of b overlaps
                d.sync()
            np.testing.assert_array_equal(tq, tr)
            np.testing.assert_array_equal(a.fetch_delta(), b.fetch_delta())
            assert a.get_time() == b.get_time()
        finally:
            held.close()
        # out of the batch, b's next upload takes the pipelined path as well
        a.set_delta_async(pins[0], t, st)
        b.set_delta_async(pins[0], t, st)
        a.step(2)
        b.step(2)
        np.testing.assert_array_equal(a.fetch_delta(), b.fetch_delta())
        assert a.get_time() == b.get_time()


def test_delta_exchange_is_the_node_values():
    """dg_fetch_delta returns delta = u - u_b as its values at the m x m
    Gauss-Legendre nodes of each element (index q*m + r), the documented
    exchange format of the precision form: the fetched FP64 modes minus the
    noise-free background (the oracle's projection), mapped to the nodes with
    the basis values sqrt(2a+1) P_a(xi_q) sqrt(2b+1) P_b(xi_r), give the same
    numbers to the FP32 rounding of delta."""
    from numpy.polynomial import legendre
    p = 3
    m = p + 1
    cfg = inputs.disc_planet(40, p)
    bg = {k: (dict(v) if isinstance(v, dict) else v) for k, v in cfg.items()}
    bg["disc"]["noise_amp"] = 0.0
    ob = oracle.Oracle(bg)
    try:
        ub = ob.fetch()
    finally:
        ob.close()
    with dg.Disc(prec_cfg(cfg)) as g:
        g.step(3)
        u = g.fetch()
        d = g.fetch_delta()
    xi, _ = legendre.leggauss(m)
    phi = np.array([[np.sqrt(2 * a + 1) * legendre.legval(x, [0] * a + [1]) for a in range(m)] for x in xi])
    V = np.einsum("qa,rb->qrab", phi, phi).reshape(m * m, m * m)
    dn = np.einsum("nk,vkji->vnji", V, u - ub)
    for v in range(3):
        scale = np.abs(dn[v]).max()
        # FP32 rounding of delta (2^-24 of a value) and the FP64 rounding of u_b
        assert np.abs(d[v] - dn[v]).max() <= 2e-7 * scale + 1e-13 * np.abs(u[v]).max(), v
