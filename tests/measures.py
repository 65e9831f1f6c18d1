"""Error measures of the validation problems (Sec. 4), from canonical
coefficient arrays, in numpy: test infrastructure.

L1 is the Sec. 4.1 quadrature: sum over elements of (1/4) sum_ij |e(x_i, y_j)|
w_i w_j dx dy at the (p+1)^2 Gauss-Legendre nodes."""
import numpy as np


def _basis(p, x):
    V = np.polynomial.legendre.legvander(x, p) * np.sqrt(2 * np.arange(p + 1) + 1.0)
    dV = np.zeros_like(V)
    for a in range(p + 1):
        c = np.zeros(a + 1)
        c[a] = 1.0
        dV[:, a] = np.polynomial.legendre.legval(x, np.polynomial.legendre.legder(c)) * np.sqrt(2 * a + 1.0)
    return V, dV


def nodal(u, p, deriv=None):
    """Values (or d/dxi, d/deta) of every variable at the GL nodes, [v][q][r][j][i]."""
    m = p + 1
    xg, _ = np.polynomial.legendre.leggauss(m)
    B, dB = _basis(p, xg)
    c = u.reshape(u.shape[0], m, m, *u.shape[2:])
    A = dB if deriv == "x" else B
    Bb = dB if deriv == "y" else B
    return np.einsum("vabji,qa,rb->vqrji", c, A, Bb)


def node_coords(cfg):
    mesh, p = cfg["mesh"], cfg["order"]
    nx, ny = mesh["nx"], mesh["ny"]
    dx = (mesh["x1"] - mesh["x0"]) / nx
    dy = (mesh["y1"] - mesh["y0"]) / ny
    xg, wg = np.polynomial.legendre.leggauss(p + 1)
    xc = mesh["x0"] + (np.arange(nx) + 0.5) * dx
    yc = mesh["y0"] + (np.arange(ny) + 0.5) * dy
    X = xc[None, None, None, :] + 0.5 * dx * xg[:, None, None, None]
    Y = yc[None, None, :, None] + 0.5 * dy * xg[None, :, None, None]
    X, Y = np.broadcast_arrays(X, Y)
    W = 0.25 * wg[:, None, None, None] * wg[None, :, None, None] * dx * dy
    return X, Y, W, dx, dy


def l1(err, W):
    return float(np.sum(np.abs(err) * W))


def isentropic_vortex_density(X, Y, t, beta=5.0, gamma=1.4, L=10.0):
    xc, yc = 0.5 * L + t, 0.5 * L + t
    dx = (X - xc + 0.5 * L) % L - 0.5 * L
    dy = (Y - yc + 0.5 * L) % L - 0.5 * L
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - dx * dx - dy * dy)
    return T ** (1.0 / (gamma - 1.0))


def vortex_l1_density(u, cfg, t):
    X, Y, W, _, _ = node_coords(cfg)
    rho = nodal(u, cfg["order"])[0]
    return l1(rho - isentropic_vortex_density(X, Y, t, cfg["disc"]["amp"]), W)


def gresho_errors(u, cfg):
    """Relative L1 errors (%) of the vorticity and of the density against the
    steady Gresho vortex (Sec. 4.2)."""
    p = cfg["order"]
    X, Y, W, dx, dy = node_coords(cfg)
    val = nodal(u, p)
    ddx = nodal(u, p, "x") * (2.0 / dx)
    ddy = nodal(u, p, "y") * (2.0 / dy)
    rho, mx, my = val[0], val[1], val[2]
    vx, vy = mx / rho, my / rho
    dvy_dx = (ddx[2] - vy * ddx[0]) / rho
    dvx_dy = (ddy[1] - vx * ddy[0]) / rho
    w_h = dvy_dx - dvx_dy
    r = np.hypot(X - 0.5, Y - 0.5)
    w = np.where(r < 0.2, 10.0, np.where(r < 0.4, 2.0 / np.maximum(r, 1e-300) - 10.0, 0.0))
    e_w = 100.0 * l1(w_h - w, W) / l1(w, W)
    e_r = 100.0 * l1(rho - 1.0, W) / l1(np.ones_like(rho), W)
    return e_w, e_r
