"""Pins of the CPU oracle on domains given by cell labels (Sec. 5): obstacles of Dirichlet cells
inside the box.  Runs without a GPU.

The label path is pinned against the box path (itself pinned against dense matrices) through two
facts that hold for a MAC grid whose Dirichlet cells carry their face values as data:
* on the unknowns, the labelled operator is the box operator applied to a vector that vanishes off
  the labelled unknowns (the stencil of a face or cell does not change, only which neighbours are
  unknowns);
* a box of m^3 cells framed by two layers of Dirichlet cells on an (m+4)^3 grid is the m^3 box
  problem shifted by two cells in each direction: unknowns, V1 set (Sec. 5), right-hand side and the
  one-level smoothers (Sec. 3.1, 3.2, whose orders depend on cell parities only) agree entry by
  entry.
"""
import numpy as np
import pytest

import oracle
import synthetic


def _rand(n, seed):
    return np.random.default_rng(seed).standard_normal(n)


def _sizes(n):
    return [(n, n, n + 1), (n, n + 1, n), (n + 1, n, n), (n, n, n)]


def _ghost_sizes(n):
    return [(n + 2, n + 2, n + 1), (n + 2, n + 1, n + 2), (n + 1, n + 2, n + 2)]


def _split(v, shapes):
    out, o = [], 0
    for s in shapes:
        m = int(np.prod(s))
        out.append(v[o:o + m].reshape(s))
        o += m
    return out


def _shrink(v, n, m, shapes_n, shapes_m, off):
    """Entries of the m-grid's layout read out of the n-grid's layout, shifted by off cells."""
    parts = _split(v, shapes_n)
    out = []
    for P, s in zip(parts, shapes_m):
        out.append(P[off:off + s[0], off:off + s[1], off:off + s[2]].reshape(-1))
    return np.concatenate(out)


def _embed(v, n, m, shapes_n, shapes_m, off, fill):
    parts = _split(fill.copy(), shapes_n)
    for P, Q in zip(parts, _split(v, shapes_m)):
        P[off:off + Q.shape[0], off:off + Q.shape[1], off:off + Q.shape[2]] = Q
    return np.concatenate([P.reshape(-1) for P in parts])


def _frame_labels(n, layers=2):
    lab = np.ones((n + 2, n + 2, n + 2), np.uint8)
    a, b = 1 + layers, n + 1 - layers
    lab[a:b, a:b, a:b] = 0
    return lab


# ----------------------------------------------------------------------------------------------
# Sec. 5: classification and the operator of a labelled domain


@pytest.mark.parametrize("seed", [0, 1])
def test_labelled_apply_is_masked_box_apply(seed):
    n = 12
    lab = synthetic.porous_labels(n, seed=seed, nspheres=6, rmin=0.12, rmax=0.25)
    assert (lab[1:-1, 1:-1, 1:-1] == 1).any()
    ol = oracle.Oracle(n, eta=0.7, gamma=0.01, levels=2, coarsest_max=6, labels=lab)
    ob = oracle.Oracle(n, eta=0.7, gamma=0.01, levels=2, coarsest_max=6)
    act, _ = ol.masks()
    actb, _ = ob.masks()
    assert act.sum() < actb.sum() and not (act & ~actb).any()
    x = _rand(ol.n(), seed + 5) * act
    for pen in (False, True):
        y = ol.apply(x, penalised=pen)
        ref = ob.apply(x, penalised=pen) * act
        assert np.max(np.abs(y - ref)) <= 1e-13 * np.max(np.abs(ref))
        assert not y[~act.astype(bool)].any()


def test_labelled_classification_by_brute_force():
    # Sec. 5, written out cell by cell: a face is Dirichlet if either cell beside it is Dirichlet, else an
    # unknown if either cell is interior (between two interior cells, or a Neumann face next to an exterior
    # cell), else inactive; pressures of interior cells are unknowns.  V1: every unknown of an interior
    # cell with a Dirichlet cell among its 26 neighbours or an exterior cell within two cells
    n = 6
    lab = _frame_labels(n, 0)
    lab[3, 3, 3] = lab[2, 4, 3] = 1  # two obstacle cells, (i, j, k) = (2, 2, 2) and (2, 3, 1)
    lab[1 + 5, 1 + 1, 1 + 4] = lab[1 + 5, 1 + 1, 1 + 5] = 2  # two exterior cells, (4, 1, 5) and (5, 1, 5)
    o = oracle.Oracle(n, levels=1, coarsest_max=n, labels=lab)
    act, v1 = o.masks()
    L = lambda i, j, k: lab[k + 1, j + 1, i + 1] if min(i, j, k) >= -1 and max(i, j, k) <= n else 1
    shapes = _sizes(n)
    ea, ev = [], []
    cellv1 = np.zeros((n, n, n), bool)
    for k in range(n):
        for j in range(n):
            for i in range(n):
                if L(i, j, k) != 0:
                    continue
                near = [L(i + a, j + b, k + c) for a in range(-2, 3) for b in range(-2, 3) for c in range(-2, 3)]
                near1 = [L(i + a, j + b, k + c) for a in range(-1, 2) for b in range(-1, 2) for c in range(-1, 2)]
                cellv1[k, j, i] = 1 in near1 or 2 in near
    for c, s in enumerate(shapes):
        A = np.zeros(s, np.uint8)
        V = np.zeros(s, np.uint8)
        for k in range(s[0]):
            for j in range(s[1]):
                for i in range(s[2]):
                    if c == 3:
                        A[k, j, i] = L(i, j, k) == 0
                        V[k, j, i] = A[k, j, i] and cellv1[k, j, i]
                        continue
                    e = [(1, 0, 0), (0, 1, 0), (0, 0, 1)][c]
                    mi, mj, mk = i - e[0], j - e[1], k - e[2]
                    pair = (L(i, j, k), L(mi, mj, mk))
                    A[k, j, i] = 1 not in pair and 0 in pair
                    if A[k, j, i]:
                        V[k, j, i] = (k < n and j < n and i < n and cellv1[k, j, i]) or \
                            (min(mi, mj, mk) >= 0 and cellv1[mk, mj, mi])
        ea.append(A.reshape(-1))
        ev.append(V.reshape(-1))
    assert np.array_equal(act, np.concatenate(ea))
    assert np.array_equal(v1, np.concatenate(ev))
    # the Neumann faces of the two exterior cells are unknowns
    assert o.has_neumann()


def test_coarse_label_is_dirichlet_if_any_child_is():
    # Sec. 5: a coarse cell is Dirichlet as soon as one of its 8 children is
    n = 8
    lab = _frame_labels(n, 0)
    lab[1 + 5, 1 + 2, 1 + 3] = 1  # fine cell (3, 2, 5) -> coarse cell (1, 1, 2)
    o = oracle.Oracle(n, levels=2, coarsest_max=4, labels=lab)
    act1, _ = o.masks(1)
    m = 4
    p = act1[-m ** 3:].reshape(m, m, m)
    expect = np.ones((m, m, m), bool)
    expect[2, 1, 1] = False
    assert np.array_equal(p.astype(bool), expect)


# ----------------------------------------------------------------------------------------------
# a framed box is the smaller box, shifted


@pytest.mark.parametrize("kb", [1, 2])
def test_framed_box_equals_smaller_box(kb):
    m, off = 6, 2
    n = m + 2 * off
    h, eta = 1.0 / m, 0.9
    ol = oracle.Oracle(n, h=h, eta=eta, levels=1, coarsest_max=n, kb=kb, labels=_frame_labels(n, off))
    ob = oracle.Oracle(m, h=h, eta=eta, levels=1, coarsest_max=m, kb=kb)
    Sn, Sm = _sizes(n), _sizes(m)
    shrink = lambda v: _shrink(v, n, m, Sn, Sm, off)
    act_l, v1_l = ol.masks()
    act_b, v1_b = ob.masks()
    assert act_l.sum() == act_b.sum()
    assert np.array_equal(shrink(act_l), act_b) and np.array_equal(shrink(v1_l), v1_b)

    # right-hand side: forcing and Dirichlet data of the small box, garbage where no unknown reads it
    f_b = _rand(ob.n(), 1)
    g_b = _rand(sum(int(np.prod(s)) for s in _ghost_sizes(m)), 2)
    f_l = _embed(f_b, n, m, Sn, Sm, off, _rand(ol.n(), 3))
    g_l = _embed(g_b, n, m, _ghost_sizes(n), _ghost_sizes(m), off,
                 _rand(sum(int(np.prod(s)) for s in _ghost_sizes(n)), 4))
    # the ghost layer of the small box sits one cell outside it: shift the ghost layouts by off too
    assert np.allclose(shrink(ol.rhs(f_l, g_l)), ob.rhs(f_b, g_b), rtol=0, atol=1e-12 * np.abs(ob.rhs(f_b, g_b)).max())

    x_b = _rand(ob.n(), 5) * act_b
    b_b = _rand(ob.n(), 6) * act_b
    emb = lambda v: _embed(v, n, m, Sn, Sm, off, np.zeros(ol.n()))
    for name, fl, fb in (("apply", lambda: ol.apply(emb(x_b)), lambda: ob.apply(x_b)),
                         ("dgs", lambda: ol.dgs(emb(x_b), emb(b_b)), lambda: ob.dgs(x_b, b_b)),
                         ("vanka", lambda: ol.vanka(emb(x_b), emb(b_b)), lambda: ob.vanka(x_b, b_b)),
                         ("smooth", lambda: ol.smooth(emb(x_b), emb(b_b)), lambda: ob.smooth(x_b, b_b))):
        yl, yb = fl(), fb()
        assert np.max(np.abs(shrink(yl) - yb)) <= 1e-12 * np.max(np.abs(yb)), name
        assert np.abs(yl).sum() == pytest.approx(np.abs(shrink(yl)).sum(), rel=1e-14), name


# ----------------------------------------------------------------------------------------------
# V-cycle and SQMR on obstacle domains


def _assemble(fn, n, active):
    cols = np.nonzero(active)[0]
    C = np.zeros((len(cols), len(cols)))
    for a, q in enumerate(cols):
        e = np.zeros(n)
        e[q] = 1.0
        C[:, a] = fn(e)[cols]
    return C


@pytest.mark.parametrize("variant", ["", "additive", "dwj", "kb2", "wcycle"])
def test_labelled_vcycle_symmetric(variant):
    n = 8
    lab = synthetic.porous_labels(n, seed=3, nspheres=4, rmin=0.15, rmax=0.3)
    o = oracle.Oracle(n, eta=1e-3, levels=3 if variant == "wcycle" else 2, coarsest_max=2, labels=lab,
                      kb=2 if variant == "kb2" else 1, additive=variant == "additive", dwj=variant == "dwj",
                      cycle=2 if variant == "wcycle" else 1)
    act, _ = o.masks()
    W = _assemble(o.vcycle, o.n(), act)
    assert np.max(np.abs(W)) > 0
    assert np.max(np.abs(W - W.T)) <= 1e-11 * np.max(np.abs(W))


@pytest.mark.parametrize("eta", [1.0, 1e-3])
def test_labelled_sqmr_matches_direct_solve(eta):
    n = 8
    lab = synthetic.porous_labels(n, seed=4, nspheres=4, rmin=0.15, rmax=0.3)
    o = oracle.Oracle(n, eta=eta, levels=2, coarsest_max=4, labels=lab)
    act, _ = o.masks()
    act = act.astype(bool)
    npc = n ** 3
    pact = act[-npc:]
    b = _rand(o.n(), 13) * act
    b[-npc:][pact] -= b[-npc:][pact].mean()
    x, rc, it, rr, _ = o.sqmr(b, tol=1e-13, maxit=300)
    assert rc == 0 and rr < 1e-13
    cols = np.nonzero(act)[0]
    A = _assemble(o.apply, o.n(), act)
    ref = np.linalg.lstsq(A, b[cols], rcond=None)[0]
    npa = int(pact.sum())
    ref[-npa:] -= ref[-npa:].mean()
    assert np.max(np.abs(x[cols] - ref)) <= 1e-9 * np.max(np.abs(ref))
    assert not x[~act].any()


def test_labelled_iterations_stay_flat():
    # Sec. 7: the iteration count of the MG-preconditioned solver barely grows under refinement,
    # with obstacles as in the box
    its = []
    for n in (16, 32):
        lab = synthetic.porous_labels(n, seed=7, nspheres=6, rmin=0.1, rmax=0.2)
        o = oracle.Oracle(n, eta=1.0, labels=lab, coarsest_max=4)
        act, _ = o.masks()
        b = _rand(o.n(), 9) * act
        pact = act[-n ** 3:].astype(bool)
        b[-n ** 3:][pact] -= b[-n ** 3:][pact].mean()
        x, rc, it, rr, _ = o.sqmr(b, tol=1e-8, maxit=200)
        assert rc == 0
        its.append(it)
    assert its[1] <= its[0] + 6, its


# ----------------------------------------------------------------------------------------------
# exterior cells (Sec. 5): Neumann faces as do-nothing outflow unknowns, inactive faces, coarsening


def _mixed(n, seed):
    return synthetic.porous_labels(n, seed=seed, nspheres=8, rmin=0.12, rmax=0.25, exterior_every=2)


def test_exterior_and_dirichlet_labellings_differ_on_the_finest_level():
    # reading of Sec. 5: a face between an interior and an exterior cell is an unknown carrying the
    # homogeneous Neumann (do-nothing) condition, so exterior cells are not Dirichlet cells with zero
    # data: the unknown set grows by the Neumann faces and the operator rows next to them change
    n = 12
    lab = _mixed(n, 1)
    assert (lab == 2).any() and (lab[1:-1, 1:-1, 1:-1] == 1).any()
    dl = np.where(lab == 2, 1, lab).astype(np.uint8)
    oe = oracle.Oracle(n, eta=0.7, gamma=0.01, levels=2, coarsest_max=6, labels=lab)
    od = oracle.Oracle(n, eta=0.7, gamma=0.01, levels=2, coarsest_max=6, labels=dl)
    ae, ve = oe.masks()
    ad, vd = od.masks()
    assert not (ad & ~ae).any() and (ae & ~ad).sum() > 0  # Neumann faces: unknowns with exterior cells only
    assert oe.has_neumann() and not od.has_neumann()
    x = _rand(oe.n(), 2) * ad
    ye, yd = oe.apply(x), od.apply(x)
    diff = np.abs(ye - yd)[ad]
    assert diff.max() > 1e-3 * np.abs(yd).max()
    # away from exterior cells (V2 rows of the Dirichlet labelling) the rows agree
    v2 = ad & ~vd
    assert np.max(np.abs(ye - yd)[v2]) <= 1e-13 * np.abs(yd).max()


@pytest.mark.parametrize("gamma", [0.0, 0.01])
def test_exterior_operator_symmetric(gamma):
    # the dropped viscous terms at Neumann faces are symmetric pairs and B^T stays the transpose of B
    n = 8
    lab = synthetic.porous_labels(n, seed=3, nspheres=4, rmin=0.15, rmax=0.3, exterior_every=2)
    o = oracle.Oracle(n, eta=0.7, gamma=gamma, levels=1, coarsest_max=n, labels=lab)
    act = o.masks()[0]
    A = _assemble(lambda e: o.apply(e, penalised=gamma > 0), o.n(), act)
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    # the pressure has no null space once a Neumann face exists
    assert o.has_neumann()
    s = np.linalg.svd(A, compute_uv=False)
    assert s[-1] > 1e-8 * s[0]


def test_exterior_rhs_reads_dirichlet_faces_only():
    # the data g is read on faces of Dirichlet cells only, and not across an exterior cell (a dropped term)
    n = 12
    lab = _mixed(n, 1)
    oe = oracle.Oracle(n, levels=2, coarsest_max=6, labels=lab)
    f = _rand(oe.n(), 3)
    g = _rand(synthetic.ghost_len(n), 4)
    L = lambda i, j, k: lab[k + 1, j + 1, i + 1]
    gz, o = g.copy(), 0
    for c, (sz, sy, sx) in enumerate(_ghost_sizes(n)):
        for kk in range(sz):
            for jj in range(sy):
                for ii in range(sx):
                    i, j, k = ii - (c != 0), jj - (c != 1), kk - (c != 2)
                    e = [(1, 0, 0), (0, 1, 0), (0, 0, 1)][c]
                    if L(i, j, k) != 1 and L(i - e[0], j - e[1], k - e[2]) != 1:
                        gz[o] = 0.0
                    o += 1
    assert not np.array_equal(gz, g)
    be = oe.rhs(f, g)
    assert np.max(np.abs(be - oe.rhs(f, gz))) <= 1e-13 * np.max(np.abs(be))
    assert np.max(np.abs(be - oe.rhs(f, np.zeros_like(g)))) > 1e-3 * np.max(np.abs(be))  # the data does enter


def _plane_poiseuille(nx, ny, outlet, U, eta):
    """Labels, Dirichlet data and the exact discrete solution of plane Poiseuille flow in a channel
    along x, walls at y = 0 and y = ny h, two cell layers in z whose ghost faces carry the exact
    velocity (so the flow is z-independent) and `outlet` exterior columns at the end.  The velocity
    u(y) = 4 U y (H - y) / H^2 is quadratic, so the MAC second difference is exact; the pressure
    p = G (x_e - x), G = 8 U eta / H^2, is linear and zero at x_e, the centre of the first exterior
    cell (the do-nothing condition sets the exterior pressure to 0)."""
    nz = 2
    h = 1.0 / ny
    H = ny * h
    lab = synthetic.channel_labels(nx, ny, nz, outlet=outlet)
    prof = lambda y: 4.0 * U * y * (H - y) / H ** 2
    # ghost-extended u data: every u face (walls, ghosts in y and z) carries the exact profile
    yg = (np.arange(-1, ny + 1) + 0.5) * h
    ug = np.broadcast_to(prof(yg)[None, :, None], (nz + 2, ny + 2, nx + 1)).copy()
    ug[:, :, 1 + nx - outlet:] = 0.0  # beyond the outflow face nothing is prescribed
    g = np.concatenate([ug.reshape(-1), np.zeros((nz + 2) * (ny + 1) * (nx + 2)),
                        np.zeros((nz + 1) * (ny + 2) * (nx + 2))])
    xe = (nx - outlet + 0.5) * h
    G = 8.0 * U * eta / H ** 2
    yc = (np.arange(ny) + 0.5) * h
    ue = np.zeros((nz, ny, nx + 1))
    ue[:, :, 1:nx - outlet + 1] = prof(yc)[None, :, None]  # unknown faces up to the outflow face
    pe = np.zeros((nz, ny, nx))
    xc = (np.arange(nx) + 0.5) * h
    pe[:, :, :nx - outlet] = G * (xe - xc[:nx - outlet])[None, None, :]
    exact = np.concatenate([ue.reshape(-1), np.zeros(nx * (ny + 1) * nz), np.zeros(nx * ny * (nz + 1)),
                            pe.reshape(-1)])
    return lab, g, exact, h


@pytest.mark.parametrize("eta", [1.0, 1e-3])
def test_plane_poiseuille_through_an_exterior_outlet_is_exact(eta):
    # Sec. 7 channel flows: a homogeneous Neumann condition on the outflow lets the fully developed
    # profile leave the domain unchanged; the discrete solution is the exact Poiseuille flow (quadratic
    # velocity, linear pressure), with no data at the outlet
    nx, ny, outlet = 16, 8, 2
    lab, g, exact, h = _plane_poiseuille(nx, ny, outlet, U=1.0, eta=eta)
    o = oracle.Oracle(nx, ny, 2, h=h, eta=eta, levels=2, coarsest_max=8, labels=lab)
    assert o.has_neumann()
    act = o.masks()[0]
    b = o.rhs(None, g)
    x, rc, it, rr, _ = o.sqmr(b, tol=1e-13, maxit=200)
    assert rc == 0 and rr < 1e-13, (rc, it, rr)
    assert np.max(np.abs((x - exact)[act])) <= 1e-9 * np.max(np.abs(exact))
    # flux balance: what enters at x = 0 leaves through the Neumann faces of the outflow
    u = x[:(nx + 1) * ny * 2].reshape(2, ny, nx + 1)
    inflow = g[:(nx + 1) * (ny + 2) * 4].reshape(4, ny + 2, nx + 1)[1:-1, 1:-1, 0].sum()
    assert abs(u[:, :, nx - outlet].sum() - inflow) <= 1e-10 * inflow


def test_exterior_outlet_differs_from_a_closed_end():
    # the same channel with Dirichlet (closed) cells at the end cannot carry the inflow: its solve has
    # no solution with nonzero net inflow (continuity), while the exterior outlet carries all of it
    nx, ny, outlet = 16, 8, 2
    lab, g, exact, h = _plane_poiseuille(nx, ny, outlet, U=1.0, eta=1.0)
    closed = np.where(lab == 2, 1, lab).astype(np.uint8)
    oc = oracle.Oracle(nx, ny, 2, h=h, levels=2, coarsest_max=8, labels=closed)
    gc = g.copy()
    gu = gc[:(nx + 1) * (ny + 2) * 4].reshape(4, ny + 2, nx + 1)
    gu[:, :, nx - outlet:] = 0.0  # no-slip data on the closed end
    bc = oc.rhs(None, gc)
    act = oc.masks()[0]
    npc = nx * ny * 2
    # sum of the continuity right-hand side = net inflow / h: nonzero, so L x = b is inconsistent
    assert abs(bc[-npc:][act[-npc:]].sum()) > 1.0


def test_duct_outflow_converges_with_flux_balance_and_symmetry():
    # 3D stand-in of the Sec. 7 cylinder example: a square duct with a z-aligned cylinder, the duct
    # inflow profile at x = 0 and an exterior outlet; MG-SQMR converges, the outflow carries the
    # inflow's flux, and the flow is mirror-symmetric in z (the geometry and data are)
    nx, ny, nz = 32, 16, 16
    lab = synthetic.channel_labels(nx, ny, nz, outlet=4, cylinder=(8.0, 8.0, 2.5))
    g = synthetic.channel_inflow(nx, ny, nz, labels=lab).numpy()
    o = oracle.Oracle(nx, ny, nz, h=1.0 / ny, eta=1e-3, gamma=1e-3, kb=2, coarsest_max=4, labels=lab)
    b = o.rhs(None, g)
    x, rc, it, rr, _ = o.sqmr(b, tol=1e-10, maxit=200)
    assert rc == 0 and rr < 1e-10, (rc, it, rr)
    u, v, w, p = synthetic.unpack(x, nx, ny, nz)
    gu = g[:(nx + 1) * (ny + 2) * (nz + 2)].reshape(nz + 2, ny + 2, nx + 1)
    inflow = gu[1:-1, 1:-1, 0].sum()
    assert abs(u[:, :, nx - 4].sum() - inflow) <= 1e-8 * inflow
    assert np.max(np.abs(u - u[::-1])) <= 1e-7 * np.max(np.abs(u))
    assert np.max(np.abs(w + w[::-1])) <= 1e-7 * np.max(np.abs(u))
    assert it <= 40, it


def test_table1_cylinder_rows():
    # Table 1 cylinder rows: with the Sec. 7 geometry, the exterior outflow column and the V1 reading,
    # the labelled classification gives the printed total (and, in 3D, boundary) DOF counts
    import os
    golden = os.path.join(os.path.dirname(__file__), "golden", "table1_cylinder.txt")
    rows = [l for l in open(golden) if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    for row in rows:
        parts = [p.strip() for p in row.split(",")]
        nx, ny, nz = map(int, parts[1:4])
        h, cx, cy, r = map(float, parts[4:8])
        total, boundary = int(parts[8]), int(parts[9])
        # nx interior columns plus one exterior column beyond the outflow face
        lab = synthetic.channel_labels(nx + 1, ny, nz, outlet=1, cylinder=(cx / h, cy / h, r / h))
        na, nv = oracle.count_dofs(nx + 1, ny, nz, lab)
        assert na == total, (parts[0], na, total)
        if boundary >= 0:
            assert nv == boundary, (parts[0], nv, boundary)


@pytest.mark.parametrize("kind,coarse_p_active", [(2, True), (1, False)])
def test_exterior_children_do_not_make_a_coarse_cell_dirichlet(kind, coarse_p_active):
    # Sec. 5: Dirichlet if any child is Dirichlet, else interior if any child is interior, else
    # exterior.  A 2^3 block of exterior (Dirichlet) fine cells becomes one exterior (Dirichlet) cell
    # on level 1, whose level-2 parent is interior (Dirichlet)
    n = 16
    lab = _frame_labels(n, 0)
    lab[1 + 4:1 + 6, 1 + 4:1 + 6, 1 + 4:1 + 6] = kind  # fine cells 4..5 -> level-1 cell 2 -> level-2 cell 1
    o = oracle.Oracle(n, levels=3, coarsest_max=4, labels=lab)
    p1 = o.masks(1)[0][-8 ** 3:].reshape(8, 8, 8)
    assert not p1[2, 2, 2] and p1.sum() == 8 ** 3 - 1
    p2 = o.masks(2)[0][-4 ** 3:].reshape(4, 4, 4)
    assert bool(p2[1, 1, 1]) == coarse_p_active and p2.sum() == 4 ** 3 - (0 if coarse_p_active else 1)


@pytest.mark.parametrize("variant", ["", "dwj"])
def test_exterior_vcycle_symmetric(variant):
    n = 8
    lab = synthetic.porous_labels(n, seed=3, nspheres=4, rmin=0.15, rmax=0.3, exterior_every=2)
    assert (lab == 2).any()
    o = oracle.Oracle(n, eta=1e-3, levels=2, coarsest_max=4, labels=lab, dwj=variant == "dwj")
    act, _ = o.masks()
    W = _assemble(o.vcycle, o.n(), act)
    assert np.max(np.abs(W - W.T)) <= 1e-11 * np.max(np.abs(W))


def test_exterior_sqmr_matches_direct_solve():
    n = 8
    lab = synthetic.porous_labels(n, seed=4, nspheres=4, rmin=0.15, rmax=0.3, exterior_every=2)
    o = oracle.Oracle(n, levels=2, coarsest_max=4, labels=lab)
    act = o.masks()[0].astype(bool)
    pact = act[-n ** 3:]
    assert o.has_neumann()  # Neumann faces fix the pressure level: L is nonsingular, no mean to remove
    b = _rand(o.n(), 13) * act
    x, rc, it, rr, _ = o.sqmr(b, tol=1e-13, maxit=300)
    assert rc == 0 and rr < 1e-13
    cols = np.nonzero(act)[0]
    ref = np.linalg.solve(_assemble(o.apply, o.n(), act), b[cols])
    assert np.max(np.abs(x[cols] - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_explicit_box_labels_reproduce_table1():
    # Table 1 (3D 128^3 driven cavity): the box written out as labels, through the labelled
    # classification, gives the printed total and boundary DOF counts
    import os
    golden = os.path.join(os.path.dirname(__file__), "golden", "table1_box.txt")
    rows = [l for l in open(golden) if l.strip() and not l.startswith("#")]
    for row in rows:
        parts = [p.strip() for p in row.split(",")]
        nx, ny, nz, total, boundary = map(int, parts[1:])
        lab = np.ones((nz + 2, ny + 2, nx + 2), np.uint8)
        lab[1:-1, 1:-1, 1:-1] = 0
        assert oracle.count_dofs(nx, ny, nz, lab) == (total, boundary)


def test_labelled_restriction_is_scaled_transpose_of_prolongation():
    # Sec. 2: R = P^T / 8 also where obstacles and exterior cells remove fine and coarse unknowns; P
    # reaches no fine DOF that is not an unknown, R reads none
    n = 8
    lab = synthetic.porous_labels(n, seed=2, nspheres=4, rmin=0.15, rmax=0.3, exterior_every=2)
    o = oracle.Oracle(n, levels=2, coarsest_max=4, labels=lab)
    act0 = o.masks(0)[0].astype(bool)
    act1 = o.masks(1)[0].astype(bool)
    n0, n1 = o.n(0), o.n(1)
    P = np.zeros((n0, n1))
    for c in np.nonzero(act1)[0]:
        e = np.zeros(n1)
        e[c] = 1.0
        P[:, c] = o.prolong_add(e, np.zeros(n0))
    R = np.zeros((n1, n0))
    for f in np.nonzero(act0)[0]:
        e = np.zeros(n0)
        e[f] = 1.0
        R[:, f] = o.restrict(e)
    assert np.max(np.abs(P)) > 0
    assert np.max(np.abs(8.0 * R - P.T)) < 1e-15
    assert np.max(np.abs(P[~act0])) == 0.0 and np.max(np.abs(R[~act1])) == 0.0


def test_labelled_coarse_solve_is_the_inverse_of_the_coarse_operator():
    # Alg. 1: the coarsest level is solved exactly with L~ of that level (labels coarsened per Sec. 5)
    n = 8
    lab = synthetic.porous_labels(n, seed=6, nspheres=4, rmin=0.15, rmax=0.3, exterior_every=2)
    o = oracle.Oracle(n, levels=2, coarsest_max=4, labels=lab)
    lc = o.nlevels - 1
    act = o.masks(lc)[0].astype(bool)
    cols = np.nonzero(act)[0]
    A = _assemble(lambda e: o.apply(e, level=lc, penalised=True), o.n(lc), act)
    b = _rand(o.n(lc), 21) * act
    x = o.coarse_solve(b)
    ref = np.linalg.solve(A, b[cols])
    assert np.max(np.abs(x[cols] - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert not x[~act].any()
