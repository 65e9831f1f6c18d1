"""FP64 CPU reference of the learned troubled-cell indicator (numpy).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the library's feature,
forward and gradient kernels; never imported by the product library.  It
shares no code with the CUDA path.

Network: x (nin) -> GELU(W1 x + b1) (64) -> GELU(W2 h1 + b2) (64) -> w3.h2 + b3,
with the weights rounded to BF16 (round to nearest even of the FP32 master
copy) and every product and sum in FP64.  Loss: mean over the batch of
w_y (softplus(z) - y z), w_1 = pos_weight, w_0 = 1; its gradient with respect
to the master copy treats the BF16 rounding as the identity.  GELU is the
exact form x Phi(x) = x (1 + erf(x / sqrt 2)) / 2.

Features of element (i, j): stencil s = 0 the element, 1 left, 2 right,
3 below, 4 above (outside elements: periodic wrap, the fixed ghost element,
or the element itself for the transmissive boundary); for each variable v
the modes divided by S_v = max |mode| of v over the stencil (1 if all
vanish): x = c * (1 / S_v), the reciprocal and the product in FP64, the product
rounded once to FP32.
"""
import numpy as np
from scipy.special import erf

H = 64


def bf16(a):
    """Round FP32 values to BF16, round to nearest even (returned as float64)."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def gelu(a):
    return 0.5 * a * (1.0 + erf(a / np.sqrt(2.0)))


def gelu_d(a):
    return 0.5 * (1.0 + erf(a / np.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / np.sqrt(2.0 * np.pi)


def split(params, nin):
    p = np.asarray(params, dtype=np.float32)
    o = 0
    W1 = p[o:o + H * nin].reshape(H, nin); o += H * nin
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o:o + 1]; o += 1
    assert o == p.size
    return W1, b1, W2, b2, w3, b3


def nparams(nin):
    return H * nin + H + H * H + H + H + 1


def forward(params, x, nin, keep=False):
    W1, b1, W2, b2, w3, b3 = (bf16(t) for t in split(params, nin))
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ W1.T + b1
    h1 = gelu(a1)
    a2 = h1 @ W2.T + b2
    h2 = gelu(a2)
    z = h2 @ w3 + b3[0]
    if keep:
        return z, (x, a1, h1, a2, h2, W2, w3)
    return z


def loss_and_grad(params, x, y, nin, pos_weight=1.0):
    z, (x, a1, h1, a2, h2, W2, w3) = forward(params, x, nin, keep=True)
    y = np.asarray(y, dtype=np.float64)
    B = z.size
    w = np.where(y > 0.5, pos_weight, 1.0)
    sp = np.logaddexp(0.0, z)
    loss = float(np.mean(w * (sp - y * z)))
    dz = w * (1.0 / (1.0 + np.exp(-z)) - y) / B
    g_w3 = h2.T @ dz
    g_b3 = np.array([dz.sum()])
    d2 = np.outer(dz, w3) * gelu_d(a2)
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * gelu_d(a1)
    g_W1 = d1.T @ x
    g_b1 = d1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, g_b3])
    return loss, g


def features(o, elems=None):
    """FP32 features [n, 5 nv M] of an oracle.Oracle's current state."""
    u = o.fetch()
    nv, M, ny, nx = u.shape
    bc = o.mesh.bc
    gl, gr, gb, gt = o.ghosts() if bc == 1 else (None,) * 4
    if elems is None:
        elems = np.arange(nx * ny)

    def elem(i, j, ci, cj):
        if 0 <= i < nx and 0 <= j < ny:
            return u[:, :, j, i]
        if bc == 0:
            return u[:, :, j % ny, i % nx]
        if bc == 1:
            if i < 0:
                return gl[:, :, j]
            if i >= nx:
                return gr[:, :, j]
            return gb[:, :, i] if j < 0 else gt[:, :, i]
        return u[:, :, cj, ci]

    out = np.zeros((len(elems), 5 * nv * M), dtype=np.float32)
    for t, e in enumerate(elems):
        i, j = int(e) % nx, int(e) // nx
        st = np.stack([elem(i, j, i, j), elem(i - 1, j, i, j), elem(i + 1, j, i, j),
                       elem(i, j - 1, i, j), elem(i, j + 1, i, j)])  # [5][nv][M]
        S = np.abs(st).max(axis=(0, 2))
        S = np.where(S > 0.0, S, 1.0)
        out[t] = (st * (1.0 / S)[None, :, None]).astype(np.float32).ravel()
    return out
