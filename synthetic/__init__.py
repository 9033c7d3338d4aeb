"""Seeded synthetic inputs for the MAC Stokes solver: the one module that both the CUDA path's
tests/bench and the CPU oracle draw their inputs from.

It holds no arithmetic of the solver itself.  It only evaluates given fields at MAC face centres
and lays them out:

* packed unknown layout (x fastest):  [u (nz, ny, nx+1) | v (nz, ny+1, nx) | w (nz+1, ny, nx) | p (nz, ny, nx)]
  u sits at x = i h, y = (j+1/2) h, z = (k+1/2) h, and analogously for v, w; p at cell centres.
* ghost-extended Dirichlet layout:     [u (nz+2, ny+2, nx+1) | v (nz+2, ny+1, nx+2) | w (nz+1, ny+2, nx+2)]
  i.e. one extra face row on each side of every tangential axis (index -1 .. n).

Workloads:
* ``mms``: the manufactured divergence-free velocity u = curl(phi, phi, phi) with
  phi = sin^2(pi x) sin^2(pi y) sin^2(pi z) and pressure cos(pi x) cos(pi y) cos(pi z); the forcing
  f = -eta Lap(u) + grad(p) is evaluated analytically at face centres.
* ``bumps``: forcing = sum of K random Gaussian bumps per velocity component, centres uniform in the
  unit cube, widths uniform in [0.02, 0.1], amplitudes N(0, 1); zero continuity source; no-slip walls.
* ``lid``: lid-driven cavity, u = 1 on the top wall (z = 1), no-slip elsewhere, zero forcing.
* ``porous_labels`` / ``cylinder_labels``: cell labels (ghost-extended cell grid, x fastest; 0 interior,
  1 Dirichlet, 2 exterior) of a box holding random spherical obstacles (optionally some of them
  exterior), or a z-aligned cylinder in a channel;
  interior cells cut off from the largest 6-connected interior region are made Dirichlet.
  ``plug_flow`` gives the channel's Dirichlet data: u = 1 on the open inflow side (x = 0), the same flux
  out of the open outflow side (x = 1), no-slip on the other walls and on the obstacles.
* ``channel_labels`` / ``channel_inflow``: a channel along x whose last columns of cells are exterior
  (an open outflow, Sec. 7 cylinder examples), optionally with a z-aligned cylinder of Dirichlet cells,
  and its inflow data: the fully developed duct profile on the x = 0 side, nothing at the outlet.

Random numbers come from numpy's PCG64 seeded per problem; evaluation runs in torch float64 on
whatever device is asked for (CPU for the oracle, CUDA to build large inputs quickly).
"""
import math

import numpy as np
import torch

PI = math.pi


def packed_sizes(nx, ny, nz):
    nu, nv, nw, np_ = (nx + 1) * ny * nz, nx * (ny + 1) * nz, nx * ny * (nz + 1), nx * ny * nz
    return nu, nv, nw, np_


def packed_len(nx, ny=None, nz=None):
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return sum(packed_sizes(nx, ny, nz))


def ghost_len(nx, ny=None, nz=None):
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return (nx + 1) * (ny + 2) * (nz + 2) + (nx + 2) * (ny + 1) * (nz + 2) + (nx + 2) * (ny + 2) * (nz + 1)


def unpack(x, nx, ny=None, nz=None):
    """Views (u, v, w, p) of a packed vector, shaped (z, y, x)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    nu, nv, nw, np_ = packed_sizes(nx, ny, nz)
    u = x[:nu].reshape(nz, ny, nx + 1)
    v = x[nu:nu + nv].reshape(nz, ny + 1, nx)
    w = x[nu + nv:nu + nv + nw].reshape(nz + 1, ny, nx)
    p = x[nu + nv + nw:].reshape(nz, ny, nx)
    return u, v, w, p


def _axes(n, h, staggered, ghost, device):
    """Coordinates along one axis: face positions i*h (staggered) or centres (i+1/2)h, optionally with
    one ghost entry on each side (centres only)."""
    if staggered:
        return torch.arange(n + 1, device=device, dtype=torch.float64) * h
    lo = -1 if ghost else 0
    hi = n + 1 if ghost else n
    return (torch.arange(lo, hi, device=device, dtype=torch.float64) + 0.5) * h


def face_coords(comp, nx, ny, nz, h, ghost=False, device="cpu"):
    """1D coordinate vectors (x, y, z) of the faces of component comp (0 u, 1 v, 2 w, 3 cell centres)."""
    n = (nx, ny, nz)
    return tuple(_axes(n[d], h, comp == d, ghost and comp != 3, device) for d in range(3))


def _grid(fn, xs, ys, zs):
    Z, Y, X = torch.meshgrid(zs, ys, xs, indexing="ij")
    return fn(X, Y, Z)


# ---------------------------------------------------------------------------------------------
# manufactured solution

def _S(t):
    return torch.sin(PI * t) ** 2


def _S1(t):
    return PI * torch.sin(2 * PI * t)


def _S2(t):
    return 2 * PI ** 2 * torch.cos(2 * PI * t)


def _S3(t):
    return -4 * PI ** 3 * torch.sin(2 * PI * t)


def _vel(a, b, c):
    # component along axis a of curl(phi, phi, phi); b, c are the next two axes cyclically
    return _S(a) * (_S1(b) * _S(c) - _S(b) * _S1(c))


def _lap_vel(a, b, c):
    return (_S2(a) * (_S1(b) * _S(c) - _S(b) * _S1(c))
            + _S(a) * (_S3(b) * _S(c) - _S2(b) * _S1(c) + _S1(b) * _S2(c) - _S(b) * _S3(c)))


def mms_velocity(comp, X, Y, Z):
    return [_vel(X, Y, Z), _vel(Y, Z, X), _vel(Z, X, Y)][comp]


def mms_pressure(X, Y, Z):
    return torch.cos(PI * X) * torch.cos(PI * Y) * torch.cos(PI * Z)


def mms_forcing(comp, X, Y, Z, eta):
    lap = [_lap_vel(X, Y, Z), _lap_vel(Y, Z, X), _lap_vel(Z, X, Y)][comp]
    sx, sy, sz = torch.sin(PI * X), torch.sin(PI * Y), torch.sin(PI * Z)
    cx, cy, cz = torch.cos(PI * X), torch.cos(PI * Y), torch.cos(PI * Z)
    grad = [-PI * sx * cy * cz, -PI * cx * sy * cz, -PI * cx * cy * sz][comp]
    return -eta * lap + grad


def mms(n, eta=1.0, device="cpu"):
    """Manufactured problem on an n^3 unit-cube grid.  Returns dict with packed forcing ``f``,
    ghost-extended Dirichlet data ``g`` and the packed exact solution ``exact`` (float64 tensors)."""
    h = 1.0 / n
    f_parts, x_parts, g_parts = [], [], []
    for c in range(3):
        xs, ys, zs = face_coords(c, n, n, n, h, device=device)
        f_parts.append(_grid(lambda X, Y, Z: mms_forcing(c, X, Y, Z, eta), xs, ys, zs).reshape(-1))
        x_parts.append(_grid(lambda X, Y, Z: mms_velocity(c, X, Y, Z), xs, ys, zs).reshape(-1))
        gx, gy, gz = face_coords(c, n, n, n, h, ghost=True, device=device)
        g_parts.append(_grid(lambda X, Y, Z: mms_velocity(c, X, Y, Z), gx, gy, gz).reshape(-1))
    xs, ys, zs = face_coords(3, n, n, n, h, device=device)
    p = _grid(mms_pressure, xs, ys, zs).reshape(-1)
    f_parts.append(torch.zeros_like(p))
    x_parts.append(p)
    return {"f": torch.cat(f_parts), "g": torch.cat(g_parts), "exact": torch.cat(x_parts), "h": h, "n": n}


# ---------------------------------------------------------------------------------------------
# Gaussian bumps

def bump_params(seed, nbumps=16):
    """Centres U[0,1]^3, widths U[0.02, 0.1], amplitudes N(0,1) per velocity component."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(0.0, 1.0, size=(nbumps, 3))
    widths = rng.uniform(0.02, 0.1, size=nbumps)
    amps = rng.standard_normal(size=(nbumps, 3))
    return centres, widths, amps


def bumps(n, seed, nbumps=16, device="cpu", dtype=torch.float64):
    """Gaussian-bump forcing on an n^3 unit-cube grid with no-slip walls.  Returns dict with packed
    ``f`` (zero continuity source) and ``g`` = None (homogeneous Dirichlet data)."""
    h = 1.0 / n
    centres, widths, amps = bump_params(seed, nbumps)
    parts = []
    for c in range(3):
        xs, ys, zs = face_coords(c, n, n, n, h, device=device)
        acc = torch.zeros(len(zs), len(ys), len(xs), dtype=torch.float64, device=device)
        for b in range(nbumps):
            s = 2.0 * widths[b] ** 2
            gx = torch.exp(-(xs - centres[b, 0]) ** 2 / s)
            gy = torch.exp(-(ys - centres[b, 1]) ** 2 / s)
            gz = torch.exp(-(zs - centres[b, 2]) ** 2 / s)
            acc.add_(float(amps[b, c]) * gz[:, None, None] * gy[None, :, None] * gx[None, None, :])
        parts.append(acc.reshape(-1))
    parts.append(torch.zeros(n ** 3, dtype=torch.float64, device=device))
    return {"f": torch.cat(parts).to(dtype), "g": None, "h": h, "n": n}


# ---------------------------------------------------------------------------------------------
# lid-driven cavity (Sec. 6, 3D driven cavity): u = 1 on the top side, zero elsewhere

def lid(n, device="cpu"):
    h = 1.0 / n
    g_parts = []
    for c in range(3):
        gx, gy, gz = face_coords(c, n, n, n, h, ghost=True, device=device)
        val = torch.zeros(len(gz), len(gy), len(gx), dtype=torch.float64, device=device)
        if c == 0:
            val[-1, :, :] = 1.0  # ghost u faces above the top wall carry the lid speed
        g_parts.append(val.reshape(-1))
    f = torch.zeros(packed_len(n), dtype=torch.float64, device=device)
    return {"f": f, "g": torch.cat(g_parts), "h": h, "n": n}


def random_vector(n, seed, nx=None, device="cpu"):
    """Seeded N(0,1) packed vector (entries outside the unknown set are not zeroed here)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = packed_len(n) if nx is None else packed_len(*nx)
    return torch.from_numpy(rng.standard_normal(m)).to(device)


# ---------------------------------------------------------------------------------------------
# initial weights of the learned initial-guess network: He-style N(0, 2 / fan_in), seeded (PCG64).
# Tensor shapes (taps, in channels, out channels) in the order of the flat weight vector.
NET_SHAPES = [(27, 4, 16)] + [(27, 16, 16)] * 10 + [(1, 16, 4)]


def net_weights(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.concatenate([rng.standard_normal(a * b * c) * np.sqrt(2.0 / (a * b)) for a, b, c in NET_SHAPES])


# ---------------------------------------------------------------------------------------------
# domains given by cell labels: obstacles inside the box (Sec. 5, Sec. 6 porous / cylinder examples)

def _connected(lab):
    """Interior cells outside the largest 6-connected interior region become Dirichlet."""
    from scipy import ndimage
    comp, ncomp = ndimage.label(lab == 0)
    if ncomp > 1:
        sizes = np.bincount(comp.reshape(-1))[1:]
        keep = 1 + int(np.argmax(sizes))
        lab[(comp != keep) & (lab == 0)] = 1
    return lab


def _shell(nx, ny, nz):
    lab = np.ones((nz + 2, ny + 2, nx + 2), np.uint8)
    lab[1:-1, 1:-1, 1:-1] = 0
    return lab


def porous_labels(nx, ny=None, nz=None, seed=0, nspheres=12, rmin=0.05, rmax=0.12, exterior_every=0):
    """Box with nspheres random spheres of Dirichlet cells (centres U[0,1]^3 scaled to the box, radii
    U[rmin, rmax] times the smallest side); with exterior_every = m > 0 every m-th sphere (0, m, 2m, ...)
    is made of exterior cells (label 2) instead.  Returns uint8 (nz+2, ny+2, nx+2)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.Generator(np.random.PCG64(seed))
    lab = _shell(nx, ny, nz)
    zc, yc, xc = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    m = min(nx, ny, nz)
    for s_idx in range(nspheres):
        c = rng.uniform(0.0, 1.0, 3) * np.array([nx, ny, nz])
        r = rng.uniform(rmin, rmax) * m
        inside = (xc - c[0]) ** 2 + (yc - c[1]) ** 2 + (zc - c[2]) ** 2 <= r * r
        lab[1:-1, 1:-1, 1:-1][inside] = 2 if exterior_every and s_idx % exterior_every == 0 else 1
    return _connected(lab)


def cylinder_labels(nx, ny=None, nz=None, centre=(0.25, 0.5), radius=0.1):
    """Channel along x with a z-aligned cylinder of Dirichlet cells; centre as fractions of (nx, ny),
    radius as a fraction of ny.  Returns uint8 (nz+2, ny+2, nx+2)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    lab = _shell(nx, ny, nz)
    yc, xc = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    inside = (xc - centre[0] * nx) ** 2 + (yc - centre[1] * ny) ** 2 <= (radius * ny) ** 2
    lab[1:-1, 1:-1, 1:-1][:, inside] = 1
    return _connected(lab)


def plug_flow(nx, ny=None, nz=None, labels=None, device="cpu"):
    """Ghost-extended Dirichlet data of a channel along x: u = 1 on the open part of the x = 0 side (faces
    of interior cells), a uniform outflow on the open part of the x = 1 side carrying the same flux, zero
    on every other face (walls and obstacles), so the continuity equation is solvable."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    if labels is None:
        open_in = open_out = torch.ones(nz, ny, dtype=torch.float64, device=device)
    else:
        lab = torch.as_tensor(np.asarray(labels).reshape(nz + 2, ny + 2, nx + 2))
        open_in = (lab[1:-1, 1:-1, 1] == 0).to(torch.float64).to(device)
        open_out = (lab[1:-1, 1:-1, nx] == 0).to(torch.float64).to(device)
    u = torch.zeros(nz + 2, ny + 2, nx + 1, dtype=torch.float64, device=device)
    u[1:-1, 1:-1, 0] = open_in
    u[1:-1, 1:-1, nx] = open_out * (open_in.sum() / open_out.sum())
    v = torch.zeros((nz + 2) * (ny + 1) * (nx + 2), dtype=torch.float64, device=device)
    w = torch.zeros((nz + 1) * (ny + 2) * (nx + 2), dtype=torch.float64, device=device)
    return torch.cat([u.reshape(-1), v, w])


def channel_labels(nx, ny=None, nz=None, outlet=1, cylinder=None):
    """Channel along x with an open outflow: the last `outlet` columns of cells (i >= nx - outlet) are
    exterior (label 2), the ghost shell is Dirichlet, and an optional z-aligned cylinder of Dirichlet
    cells -- cylinder = (cx, cy, r) in cells; a cell is inside when its centre lies strictly inside the
    circle -- stands in the flow.  Returns uint8 (nz+2, ny+2, nx+2)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    lab = _shell(nx, ny, nz)
    if cylinder is not None:
        cx, cy, r = cylinder
        yc, xc = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
        inside = (xc - cx) ** 2 + (yc - cy) ** 2 < r * r
        lab[1:-1, 1:-1, 1:-1][:, inside] = 1
    lab[1:-1, 1:-1, 1 + nx - outlet:1 + nx] = 2
    return _connected(lab)


def channel_inflow(nx, ny=None, nz=None, labels=None, mean=1.0, device="cpu"):
    """Ghost-extended Dirichlet data of a channel along x with an open (exterior) outlet: on the x = 0
    side the fully developed duct profile u = 16 U y z (1 - y)(1 - z) in units of the side lengths
    (mean-velocity scale U = mean), on faces of interior cells only; zero on every other face (no-slip
    walls and obstacles).  Nothing is prescribed at the outlet."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    yc = (torch.arange(ny, dtype=torch.float64, device=device) + 0.5) / ny
    zc = (torch.arange(nz, dtype=torch.float64, device=device) + 0.5) / nz
    prof = 16.0 * mean * (zc * (1 - zc))[:, None] * (yc * (1 - yc))[None, :]
    if labels is not None:
        lab = torch.as_tensor(np.asarray(labels).reshape(nz + 2, ny + 2, nx + 2))
        prof = prof * (lab[1:-1, 1:-1, 1] == 0).to(torch.float64).to(device)
    u = torch.zeros(nz + 2, ny + 2, nx + 1, dtype=torch.float64, device=device)
    u[1:-1, 1:-1, 0] = prof
    v = torch.zeros((nz + 2) * (ny + 1) * (nx + 2), dtype=torch.float64, device=device)
    w = torch.zeros((nz + 1) * (ny + 2) * (nx + 2), dtype=torch.float64, device=device)
    return torch.cat([u.reshape(-1), v, w])
