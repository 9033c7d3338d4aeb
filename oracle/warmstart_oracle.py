"""Plain numpy (FP64) reference of the learned initial-guess network -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the bench's CPU baseline may import this module; the product
path never calls it.

The paper's solver starts SQMR (Alg. 4) from a given x0.  The learned warm start predicts that x0
from the right-hand side b with a small 3D convolutional network, trained on solutions the method
itself produces; SQMR with the unchanged symmetric V-cycle preconditioner then runs from it, so the
tolerance reached is never affected by the network.  The paper has no such network: this file
defines it, written out plainly.

Data layout: a cell field is an array (nz, ny, nx, C) -- channels last, x fastest among the
spatial axes.  Packed MAC vectors are [u (nx+1) ny nz | v nx (ny+1) nz | w nx ny (nz+1) | p nx ny nz].

Network (four levels, 16 channels, no bias terms, leaky ReLU with slope 0.1 -- so the map b -> x0
is positively homogeneous: x0(a b) = a x0(b) for a > 0):

    X0 = cells(b) / rms(b)                         4 channels: face-averaged velocity parts, pressure part
    a0 = act(conv(X0, W0))      s0 = act(conv(a0, W1))                    level 0, n^3
    a1 = act(conv(pool(s0), W2)) s1 = act(conv(a1, W3))                   level 1, (n/2)^3
    a2 = act(conv(pool(s1), W4)) s2 = act(conv(a2, W5))                   level 2
    a3 = act(conv(pool(s2), W6)) b3 = act(conv(a3, W7))                   level 3, (n/8)^3
    c2 = act(conv(up(b3) + s2, W8))
    c1 = act(conv(up(c2) + s1, W9))
    c0 = act(conv(up(c1) + s0, W10))
    P  = c0 W11                                    1 x 1 x 1 convolution, 16 -> 4 channels
    x0 = scale * rms(b) * faces(P)

conv: 3 x 3 x 3, zero padding, weights W[t, ci, co] with tap t = 9 (dz+1) + 3 (dy+1) + (dx+1);
pool: mean over 2 x 2 x 2 blocks; up: nearest-neighbour doubling; cells(b): the velocity component
of a cell is the mean of its two faces along that axis, the pressure is b's pressure entry;
faces(P): an interior face takes the mean of its two cells, a wall face 0, the pressure is P's.
Loss, with x* a solution the method produced for b:  ||x0 - x*||^2 / ||x*||^2 (error form), or
with the operator L of the problem ||L (x0 - x*)||^2 / ||b||^2 (residual form: the quantity SQMR's
stopping test measures, since L x* = b up to the solve's tolerance).
"""
import numpy as np

SLOPE = 0.1
CH = 16
TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
# (rows, cin, cout) of every weight tensor in the flat parameter vector, in order
SHAPES = [(27, 4, CH)] + [(27, CH, CH)] * 10 + [(1, CH, 4)]


def num_weights():
    return int(sum(a * b * c for a, b, c in SHAPES))


def split_weights(w):
    out, o = [], 0
    for s in SHAPES:
        m = s[0] * s[1] * s[2]
        out.append(np.asarray(w[o:o + m], dtype=np.float64).reshape(s))
        o += m
    return out


# ---------------------------------------------------------------------------------- packed <-> cells

def _split(x, n):
    nu, nv, nw = (n + 1) * n * n, n * (n + 1) * n, n * n * (n + 1)
    u = x[:nu].reshape(n, n, n + 1)
    v = x[nu:nu + nv].reshape(n, n + 1, n)
    w = x[nu + nv:nu + nv + nw].reshape(n + 1, n, n)
    p = x[nu + nv + nw:].reshape(n, n, n)
    return u, v, w, p


def cells(b, n):
    u, v, w, p = _split(b, n)
    return np.stack([0.5 * (u[:, :, :-1] + u[:, :, 1:]), 0.5 * (v[:, :-1, :] + v[:, 1:, :]),
                     0.5 * (w[:-1] + w[1:]), p], axis=-1)


def faces(P, n):
    u = np.zeros((n, n, n + 1))
    v = np.zeros((n, n + 1, n))
    w = np.zeros((n + 1, n, n))
    u[:, :, 1:-1] = 0.5 * (P[:, :, :-1, 0] + P[:, :, 1:, 0])
    v[:, 1:-1, :] = 0.5 * (P[:, :-1, :, 1] + P[:, 1:, :, 1])
    w[1:-1] = 0.5 * (P[:-1, :, :, 2] + P[1:, :, :, 2])
    return np.concatenate([u.ravel(), v.ravel(), w.ravel(), P[..., 3].ravel()])


def faces_T(y, n):
    """Adjoint of faces(): <faces(P), y> = <P, faces_T(y)>."""
    u, v, w, p = _split(y, n)
    G = np.zeros((n, n, n, 4))
    G[:, :, :-1, 0] += 0.5 * u[:, :, 1:-1]
    G[:, :, 1:, 0] += 0.5 * u[:, :, 1:-1]
    G[:, :-1, :, 1] += 0.5 * v[:, 1:-1, :]
    G[:, 1:, :, 1] += 0.5 * v[:, 1:-1, :]
    G[:-1, :, :, 2] += 0.5 * w[1:-1]
    G[1:, :, :, 2] += 0.5 * w[1:-1]
    G[..., 3] = p
    return G


def rms(b):
    return float(np.sqrt(np.mean(np.asarray(b, dtype=np.float64) ** 2)))


# ---------------------------------------------------------------------------------- layers

def conv(x, W):
    """3x3x3 convolution (cross-correlation), zero padding: y[v] = sum_t x[v + off_t] W[t]."""
    nz, ny, nx, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((nz, ny, nx, W.shape[2]))
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += xp[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx] @ W[t]
    return y


def conv_bwd_data(g, W):
    """dx[v] = sum_t g[v - off_t] W[t]^T."""
    nz, ny, nx, _ = g.shape
    gp = np.pad(g, ((1, 1), (1, 1), (1, 1), (0, 0)))
    dx = np.zeros((nz, ny, nx, W.shape[1]))
    for t, (dz, dy, dx_) in enumerate(TAPS):
        dx += gp[1 - dz:1 - dz + nz, 1 - dy:1 - dy + ny, 1 - dx_:1 - dx_ + nx] @ W[t].T
    return dx


def conv_bwd_weight(x, g):
    """dW[t] = sum_v x[v + off_t]^T g[v]."""
    nz, ny, nx, ci = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    gf = g.reshape(-1, g.shape[-1])
    dW = np.zeros((27, ci, g.shape[-1]))
    for t, (dz, dy, dx) in enumerate(TAPS):
        dW[t] = xp[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx].reshape(-1, ci).T @ gf
    return dW


def act(z):
    return np.where(z > 0, z, SLOPE * z)


def act_bwd(g, y):
    """Gradient through act given its output y (same sign as its input)."""
    return np.where(y > 0, g, SLOPE * g)


def pool(x):
    nz, ny, nx, c = x.shape
    return x.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).mean(axis=(1, 3, 5))


def up(x):
    return x.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)


def up_T(g):
    """Adjoint of up(): sum over the 8 children."""
    nz, ny, nx, c = g.shape
    return g.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).sum(axis=(1, 3, 5))


def pool_T(g):
    """Adjoint of pool(): every child receives its parent's value / 8."""
    return up(g) / 8.0


# ---------------------------------------------------------------------------------- network

def forward(b, w, n, scale):
    W = split_weights(w)
    r = rms(b)
    c = {"rms": r, "X0": cells(b, n) / r}
    c["a0"] = act(conv(c["X0"], W[0]))
    c["s0"] = act(conv(c["a0"], W[1]))
    c["p1"] = pool(c["s0"])
    c["a1"] = act(conv(c["p1"], W[2]))
    c["s1"] = act(conv(c["a1"], W[3]))
    c["p2"] = pool(c["s1"])
    c["a2"] = act(conv(c["p2"], W[4]))
    c["s2"] = act(conv(c["a2"], W[5]))
    c["p3"] = pool(c["s2"])
    c["a3"] = act(conv(c["p3"], W[6]))
    c["b3"] = act(conv(c["a3"], W[7]))
    c["u2"] = up(c["b3"]) + c["s2"]
    c["c2"] = act(conv(c["u2"], W[8]))
    c["u1"] = up(c["c2"]) + c["s1"]
    c["c1"] = act(conv(c["u1"], W[9]))
    c["u0"] = up(c["c1"]) + c["s0"]
    c["c0"] = act(conv(c["u0"], W[10]))
    c["P"] = c["c0"] @ W[11][0]
    x0 = scale * r * faces(c["P"], n)
    return x0, c


def predict(b, w, n, scale):
    return forward(b, w, n, scale)[0]


def loss(b, xstar, w, n, scale, apply=None):
    x0, _ = forward(b, w, n, scale)
    if apply is None:
        return float(np.sum((x0 - xstar) ** 2) / np.sum(xstar ** 2))
    return float(np.sum(apply(x0 - xstar) ** 2) / np.sum(np.asarray(b) ** 2))


def loss_and_grad(b, xstar, w, n, scale, apply=None):
    """Loss and its gradient with respect to the flat weight vector (reverse mode, by hand).
    apply: None for the error form, else a function x -> L x (L symmetric) for the residual form."""
    W = split_weights(w)
    x0, c = forward(b, w, n, scale)
    diff = x0 - xstar
    if apply is None:
        den = float(np.sum(xstar ** 2))
        L = float(np.sum(diff ** 2) / den)
        dx0 = 2.0 * diff / den
    else:
        den = float(np.sum(np.asarray(b) ** 2))
        r = apply(diff)
        L = float(np.sum(r ** 2) / den)
        dx0 = 2.0 * apply(r) / den
    dP = scale * c["rms"] * faces_T(dx0, n)
    g = [None] * 12
    g[11] = (c["c0"].reshape(-1, CH).T @ dP.reshape(-1, 4))[None]
    dz = act_bwd(dP @ W[11][0].T, c["c0"])
    g[10] = conv_bwd_weight(c["u0"], dz)
    du0 = conv_bwd_data(dz, W[10])
    dz = act_bwd(up_T(du0), c["c1"])
    g[9] = conv_bwd_weight(c["u1"], dz)
    du1 = conv_bwd_data(dz, W[9])
    dz = act_bwd(up_T(du1), c["c2"])
    g[8] = conv_bwd_weight(c["u2"], dz)
    du2 = conv_bwd_data(dz, W[8])
    dz = act_bwd(up_T(du2), c["b3"])
    g[7] = conv_bwd_weight(c["a3"], dz)
    dz = act_bwd(conv_bwd_data(dz, W[7]), c["a3"])
    g[6] = conv_bwd_weight(c["p3"], dz)
    ds2 = du2 + pool_T(conv_bwd_data(dz, W[6]))
    dz = act_bwd(ds2, c["s2"])
    g[5] = conv_bwd_weight(c["a2"], dz)
    dz = act_bwd(conv_bwd_data(dz, W[5]), c["a2"])
    g[4] = conv_bwd_weight(c["p2"], dz)
    ds1 = du1 + pool_T(conv_bwd_data(dz, W[4]))
    dz = act_bwd(ds1, c["s1"])
    g[3] = conv_bwd_weight(c["a1"], dz)
    dz = act_bwd(conv_bwd_data(dz, W[3]), c["a1"])
    g[2] = conv_bwd_weight(c["p1"], dz)
    ds0 = du0 + pool_T(conv_bwd_data(dz, W[2]))
    dz = act_bwd(ds0, c["s0"])
    g[1] = conv_bwd_weight(c["a0"], dz)
    dz = act_bwd(conv_bwd_data(dz, W[1]), c["a0"])
    g[0] = conv_bwd_weight(c["X0"], dz)
    return L, np.concatenate([a.ravel() for a in g])


def adam(w, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) in place; step counts from 1."""
    m *= beta1
    m += (1 - beta1) * grad
    v *= beta2
    v += (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    w -= lr * mh / (np.sqrt(vh) + eps)
    return w
