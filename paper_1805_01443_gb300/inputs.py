"""Seeded synthetic workloads: parameter sets and random perturbations.

This module holds no arithmetic of the method.  It names the workloads by what
they are (disc, order, mesh) with the parameters of the paper's planet-disc
runs (Sec. 5.1: G = M_* = 1, planet on a fixed circular orbit at r_p = 1 with
Omega_p = 1, smoothing eps = 0.6 H with H = h r_p, h = 0.05) and supplies seeded
random modal perturbations that the tests feed to both the CUDA path and the
oracle.  Both sides read these dicts; neither side's arithmetic lives here.
"""
import copy

import numpy as np

H_ASPECT = 0.05


def _disc_base(n, order, seed, planet_q=None, damping=False, bc=1):
    cfg = {
        "order": order,
        "mesh": {"nx": n, "ny": n, "x0": -2.5, "x1": 2.5, "y0": -2.5, "y1": 2.5, "bc": bc},
        "eos": {"kind": 0, "gamma": 1.4, "h": H_ASPECT},
        "planet": {"q": 0.0, "r_p": 1.0, "eps": 0.6 * H_ASPECT * 1.0, "omega_p": 1.0,
                   "phi0": 0.0, "enabled": 0},
        "disc": {"ic": 0, "star": 1, "r_soft": 0.2, "sigma_slope": -0.5, "sigma_floor": 1e-4,
                 "noise_amp": 1e-4, "seed": seed, "rdamp_in": 0.0, "rdamp_out": 0.0,
                 "cfl": 0.1, "rk": 3, "prec": 0, "amp": 0.0, "vx0": 0.0, "vy0": 0.0,
                 "limiter": 0, "tvb_m": 50.0, "positivity": 0, "ring_r": 0.0, "ring_p": 1.0},
    }
    if planet_q is not None:
        cfg["planet"]["q"] = planet_q
        cfg["planet"]["enabled"] = 1
    if damping:
        cfg["disc"]["rdamp_in"] = 0.4
        cfg["disc"]["rdamp_out"] = 2.1
    return cfg


def disc_small(n=64, order=2, seed=1):
    """Locally isothermal Keplerian disc, P2 on 64x64, no planet, 50 steps."""
    return _disc_base(n, order, seed)


def disc_planet(n=256, order=4, seed=2, q=1e-5):
    """Planet-disc, P4 on 256x256, q = 1e-5, damping zones r < 0.4 and r > 2.1, 200 steps."""
    return _disc_base(n, order, seed, planet_q=q, damping=True)


def disc_planet_512(n=512, order=4, seed=3, q=3e-5):
    """Planet-disc, P4 on 512x512, q = 3e-5, damping zones, 1000 steps (precision form)."""
    return _disc_base(n, order, seed, planet_q=q, damping=True)


def density_wave(n=32, order=2, amp=0.2):
    """Adiabatic density wave rho = 1 + amp sin(2 pi (x + y)), v = (1, 1), p = 1 on the
    periodic unit square: an exact translating solution of Eq. 1 without gravity."""
    return {
        "order": order,
        "mesh": {"nx": n, "ny": n, "x0": 0.0, "x1": 1.0, "y0": 0.0, "y1": 1.0, "bc": 0},
        "eos": {"kind": 1, "gamma": 1.4, "h": 0.0},
        "planet": {"q": 0.0, "r_p": 1.0, "eps": 0.03, "omega_p": 1.0, "phi0": 0.0, "enabled": 0},
        "disc": {"ic": 1, "star": 0, "r_soft": 0.2, "sigma_slope": -0.5, "sigma_floor": 1e-4,
                 "noise_amp": 0.0, "seed": 0, "rdamp_in": 0.0, "rdamp_out": 0.0, "cfl": 0.1,
                 "rk": 3, "prec": 0, "amp": amp, "vx0": 1.0, "vy0": 1.0, "limiter": 0,
                 "tvb_m": 50.0, "positivity": 0, "ring_r": 0.0, "ring_p": 1.0},
    }


def uniform_state(n=8, order=2, kind=1, vx0=0.0, vy0=0.0, bc=0, h=0.0):
    """Uniform state rho = 1, v = (vx0, vy0), p = 1 on the unit square."""
    cfg = density_wave(n, order, amp=0.0)
    cfg["disc"]["ic"] = 2
    cfg["disc"]["vx0"] = vx0
    cfg["disc"]["vy0"] = vy0
    cfg["eos"]["kind"] = kind
    cfg["eos"]["h"] = h
    cfg["mesh"]["bc"] = bc
    return cfg


def shock_ring(n=1024, order=3, seed=5, q=1e-3, limiter=1, positivity=1):
    """Adiabatic (gamma = 1.4) planet disc with an imposed shock ring: the disc
    of Sec. 5.1 with pressure x10 inside r < 1.5, gap-opening planet q = 1e-3,
    damping zones, seeded noise; TVB-limited troubled cells and the
    positivity limiter."""
    cfg = _disc_base(n, order, seed, planet_q=q, damping=True)
    cfg["eos"]["kind"] = 1
    cfg["eos"]["gamma"] = 1.4
    cfg["disc"].update({"ic": 3, "ring_r": 1.5, "ring_p": 10.0, "limiter": limiter,
                        "positivity": positivity})
    return cfg


def isentropic_vortex(n=32, order=3, beta=5.0, cfl=0.1):
    """Sec. 4.1: the isentropic vortex on the periodic box [0, 10]^2, gamma 1.4,
    free stream rho = p = 1, v = (1, 1); it returns to its start at T = 10."""
    cfg = density_wave(n, order)
    cfg["mesh"].update({"x1": 10.0, "y1": 10.0})
    cfg["disc"].update({"ic": 4, "amp": beta, "vx0": 1.0, "vy0": 1.0, "cfl": cfl})
    return cfg


def gresho_vortex(n=40, order=3, cfl=0.1):
    """Sec. 4.2: the Gresho vortex on [0, 1]^2 with gradient-free boundaries
    (zero-gradient ghost elements), gamma 1.4; a steady solution."""
    cfg = density_wave(n, order)
    cfg["mesh"]["bc"] = 3
    cfg["disc"].update({"ic": 5, "amp": 0.0, "vx0": 0.0, "vy0": 0.0, "cfl": cfl})
    return cfg


def paper_disc(n=128, order=4, q=6e-5, positivity=1):
    """The paper's own planet disc (Sec. 5.1): box [-2.25, 2.25]^2, adiabatic
    gamma = 1.4, uniform Sigma_0 = 1 and p_0 = h^2 = 2.5e-3 tapered beyond
    r_ex = 1.75, solid-body rotation inside r_in = 0.4 (the star's core
    radius), planet q = 6e-5 on the fixed orbit r_p = 1 with eps = 0.03,
    damping radii r_in 1.15^(3/2) and r_ex 1.15^(-3/2), the positivity
    limiter on; no seeded noise (the disc starts smooth)."""
    cfg = _disc_base(n, order, 0, planet_q=q, damping=True)
    cfg["mesh"].update({"x0": -2.25, "x1": 2.25, "y0": -2.25, "y1": 2.25})
    cfg["eos"].update({"kind": 1, "gamma": 1.4})
    cfg["disc"].update({"ic": 6, "r_soft": 0.4, "noise_amp": 0.0, "rdamp_in": 0.4 * 1.15 ** 1.5,
                        "rdamp_out": 1.75 * 1.15 ** -1.5, "positivity": positivity})
    return cfg


def batch_discs(n=48, seed0=100, prec=1):
    """Batched workload: n independent planet discs (damping zones as above),
    instance k with seed seed0 + k, mesh {128, 256, 384, 512}^2 cycling with k,
    degree {2, 3, 4} cycling with k, and planet mass q = 10^U(-6, -4) drawn
    from the instance's seed."""
    sizes, orders = (128, 256, 384, 512), (2, 3, 4)
    out = []
    for k in range(n):
        seed = seed0 + k
        q = 10.0 ** np.random.Generator(np.random.PCG64(seed)).uniform(-6.0, -4.0)
        cfg = _disc_base(sizes[k % 4], orders[k % 3], seed, planet_q=float(q), damping=True)
        cfg["disc"]["prec"] = prec
        out.append(cfg)
    return out


def batch_small(prec=1):
    """Small mixed batch for parity tests: degrees 1-4, square and rectangular
    meshes, tile rows with a ragged last tile."""
    shapes = [(40, 24, 1, 1e-5), (48, 48, 2, 3e-5), (64, 32, 3, 1e-4), (72, 40, 4, 3e-5),
              (32, 32, 4, 1e-6), (96, 64, 2, 1e-4)]
    out = []
    for k, (nx, ny, p, q) in enumerate(shapes):
        cfg = _disc_base(nx, p, 200 + k, planet_q=q, damping=True)
        cfg["mesh"]["ny"] = ny
        cfg["disc"]["prec"] = prec
        out.append(cfg)
    return out


WORKLOADS = {
    "disc_p2_64": disc_small,
    "disc_p4_256": disc_planet,
    "disc_p4_512": disc_planet_512,
}


def workload(name, **kw):
    return copy.deepcopy(WORKLOADS[name](**kw))


def modal_perturbation(shape, seed, amp=1e-3, decay=0.5):
    """Seeded uniform random modal coefficients of shape (nv, m*m, ny, nx) with
    amplitude amp * decay**(a + b) for mode (a, b): a rough but resolved field."""
    nv, M, ny, nx = shape
    m = int(round(M ** 0.5))
    rng = np.random.Generator(np.random.PCG64(seed))
    out = rng.uniform(-1.0, 1.0, size=shape)
    scale = np.array([amp * decay ** (k // m + k % m) for k in range(M)])
    return out * scale[None, :, None, None]
