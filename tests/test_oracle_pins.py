"""Pins of the CPU oracle against things other than itself (runs without a GPU).

Each test names the passage of Tao & Sifakis (arXiv 2312.10615) that fixes the checked fact.
"""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla


import oracle
import synthetic
from tests.dense_stokes import DenseBox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(n, seed):
    return np.random.default_rng(seed).standard_normal(n)


def _masked(v, mask):
    v = v.copy()
    v[~mask] = 0.0
    return v


# ----------------------------------------------------------------------------------------------
# Sec. 5 / Table 1: DOF classification

def test_table1_box_row():
    rows = [l for l in open(os.path.join(GOLDEN, "table1_box.txt")) if l.strip() and not l.startswith("#")]
    for row in rows:
        parts = [p.strip() for p in row.split(",")]
        nx, ny, nz, total, boundary = map(int, parts[1:])
        assert oracle.count_dofs(nx, ny, nz) == (total, boundary)


@pytest.mark.parametrize("n", [2, 4, 6])
def test_classification_matches_dense(n):
    o = oracle.Oracle(n, coarsest_max=n, levels=1)
    D = DenseBox(n)
    act, v1 = o.masks()
    assert np.array_equal(act, D.active)
    assert np.array_equal(v1, D.v1)
    assert np.array_equal(o.dgs_order(), D.dgs_order())


# ----------------------------------------------------------------------------------------------
# Eq. 2 and Sec. 4: operator

@pytest.mark.parametrize("dims", [(4, 4, 4), (6, 4, 5), (5, 7, 3)])
def test_apply_matches_dense(dims):
    nx, ny, nz = dims
    o = oracle.Oracle(nx, ny, nz, h=0.37, eta=0.7, gamma=0.01, levels=1, coarsest_max=8)
    D = DenseBox(nx, ny, nz, h=0.37, eta=0.7, gamma=0.01)
    x = _masked(_rand(D.n, 1), D.active)
    for pen, M in ((False, D.L), (True, D.Lt)):
        y = o.apply(x, penalised=pen)
        ref = M @ x
        assert np.max(np.abs(y - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_operator_symmetric_and_nullspace():
    o = oracle.Oracle(8, levels=1)
    act, _ = o.masks()
    x, y = _masked(_rand(o.n(), 2), act), _masked(_rand(o.n(), 3), act)
    for pen in (False, True):
        a, b = x @ o.apply(y, penalised=pen), y @ o.apply(x, penalised=pen)
        assert abs(a - b) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(o.apply(y, penalised=pen))
    p = np.zeros(o.n())
    p[o.n() - 8 ** 3:] = 1.0
    assert np.max(np.abs(o.apply(p))) < 1e-12  # constant pressure lies in ker L (Sec. 4)


def test_LM_top_right_block_vanishes_in_interior():
    # Eq. (disc): in the interior LM = [[-eta Lap, 0], [-div, Lap]]
    D = DenseBox(8, eta=1.3)
    LM = (D.L @ D.M).toarray()
    nf = D.offsets[3]
    deep = np.zeros(D.n, bool)
    # velocity rows at least two cells away from every wall
    for c in range(3):
        dims = [(9, 8, 8), (8, 9, 8), (8, 8, 9)][c]
        k, j, i = np.meshgrid(*[np.arange(m) for m in dims[::-1]], indexing="ij")
        idx = [i, j, k]
        ok = np.ones_like(i, bool)
        for d in range(3):
            lo, hi = (2, dims[d] - 3) if d == c else (2, dims[d] - 3)
            ok &= (idx[d] >= lo) & (idx[d] <= hi)
        deep[D.offsets[c]:D.offsets[c + 1]] = ok.reshape(-1)
    block = LM[np.ix_(deep[:nf].nonzero()[0], np.arange(nf, D.n))]
    assert np.max(np.abs(block)) < 1e-9 * np.max(np.abs(LM))


# ----------------------------------------------------------------------------------------------
# Alg. 2 and App. A, Eq. (SDGS): distributive Gauss-Seidel on V2

def _dgs_dense(D, x, b, forward):
    # DGS relaxes the V2 rows; the distribution uses the full columns M_{:,j}, j in V2 (Alg. 2)
    order = D.dgs_order()
    Lt = D.Lt.toarray()
    Mc = D.M.toarray()[:, order]
    G = np.tril(Lt[order, :] @ Mc)  # lower triangle of (L~M) on the V2 rows/columns, traversal order
    r = b - Lt @ x
    out = x.copy()
    if forward:
        out += Mc @ np.linalg.solve(G, r[order])  # x + M G~^{-1} (b - L~x)
    else:
        out[order] += np.linalg.solve(G.T, Mc.T @ r)  # x + G~^{-T} M^T (b - L~x)
    return out


@pytest.mark.parametrize("n", [5, 6])
def test_dgs_equals_matrix_form(n):
    o = oracle.Oracle(n, eta=0.8, gamma=0.05, levels=1)
    D = DenseBox(n, eta=0.8, gamma=0.05)
    x = _masked(_rand(D.n, 4), D.active)
    b = _masked(_rand(D.n, 5), D.active)
    for direction, fwd in ((1, True), (-1, False)):
        got = o.dgs(x, b, direction=direction)
        ref = _dgs_dense(D, x, b, fwd)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_dgs_diagonal_is_row_times_column():
    # Alg. 2: d_j = L~_{j,} . M_{,j}
    D = DenseBox(6, eta=0.9, gamma=0.02)
    o = oracle.Oracle(6, eta=0.9, gamma=0.02, levels=1)
    order = D.dgs_order()
    LM = (D.Lt.toarray()[order, :] @ D.M.toarray()[:, order])
    d = o.dgs_diag()
    assert np.allclose(d[order], np.diag(LM), rtol=1e-13, atol=0)


# ----------------------------------------------------------------------------------------------
# Smoother symmetry: Thm 1 (DGS), Thm 3 (symmetric multiplicative Vanka), Thm 4 (Alg. 3)

def _assemble(fn, n, active):
    cols = np.nonzero(active)[0]
    C = np.zeros((len(cols), len(cols)))
    for a, q in enumerate(cols):
        e = np.zeros(n)
        e[q] = 1.0
        C[:, a] = fn(e)[cols]
    return C


# eta = 1e-3 is the paper's viscosity (Sec. 7); there the local saddle-point matrices need row pivoting
@pytest.mark.parametrize("variant", ["", "additive", "dwj"])
@pytest.mark.parametrize("eta", [1.0, 1e-3])
@pytest.mark.parametrize("which", ["dgs", "vanka", "smooth"])
def test_smoother_C_symmetric(which, eta, variant):
    if (which == "dgs" and variant == "additive") or (which == "vanka" and variant == "dwj"):
        pytest.skip("this piece does not depend on the variant")
    o = oracle.Oracle(6, eta=eta, gamma=1e-3, levels=1, kb=1, additive=variant == "additive", dwj=variant == "dwj")
    act, _ = o.masks()
    z = np.zeros(o.n())
    fn = {"dgs": lambda e: o.dgs(z, e, direction=0),
          "vanka": lambda e: o.vanka(z, e, colour=-1),
          "smooth": lambda e: o.smooth(z, e)}[which]
    C = _assemble(fn, o.n(), act)
    assert np.max(np.abs(C)) > 0
    assert np.max(np.abs(C - C.T)) <= 1e-11 * np.max(np.abs(C))


def test_forward_dgs_alone_is_not_symmetric():
    # the reason for the backward sweep (Sec. 3.1): the plain right-preconditioned sweep is not symmetric
    o = oracle.Oracle(6, levels=1)
    act, _ = o.masks()
    z = np.zeros(o.n())
    C = _assemble(lambda e: o.dgs(z, e, direction=1), o.n(), act)
    assert np.max(np.abs(C - C.T)) > 1e-3 * np.max(np.abs(C))


@pytest.mark.parametrize("eta", [1.0, 1e-3])
def test_vanka_single_patch_is_exact_local_solve(eta):
    # Sec. 3.2: on a 2^3 grid every colour holds one cell, so after that colour the residual of
    # L~ vanishes on the cell's patch (exact local saddle-point solve).
    o = oracle.Oracle(2, eta=eta, levels=1, coarsest_max=2)
    D = DenseBox(2, eta=eta)
    x = _masked(_rand(D.n, 6), D.active)
    b = _masked(_rand(D.n, 7), D.active)
    for col in range(8):
        x = o.vanka(x, b, colour=col)
        i, j, k = col & 1, (col >> 1) & 1, (col >> 2) & 1
        r = b - D.Lt @ x
        patch = []
        # faces of cell (i,j,k) and its pressure, packed indices
        nx = 2
        patch += [i + s + (nx + 1) * (j + nx * k) for s in (0, 1)]
        patch += [D.offsets[1] + i + nx * (j + s + (nx + 1) * k) for s in (0, 1)]
        patch += [D.offsets[2] + i + nx * (j + nx * (k + s)) for s in (0, 1)]
        patch += [D.offsets[3] + i + nx * (j + nx * k)]
        patch = [q for q in patch if D.active[q]]
        assert np.max(np.abs(r[patch])) < 1e-12 * np.max(np.abs(b))


def test_additive_vanka_is_damped_sum_of_local_solves():
    # Eq. (av): x + (1/2) sum_i C_i^T (C_i L~ C_i^T)^{-1} C_i (b - L~ x), every V1 patch from the same state
    n = 4
    o = oracle.Oracle(n, levels=1, coarsest_max=2, additive=True)
    D = DenseBox(n)
    Lt = D.Lt.toarray()
    x = _masked(_rand(D.n, 40), D.active)
    b = _masked(_rand(D.n, 41), D.active)
    r = b - Lt @ x
    ref = x.copy()
    nx = n
    for k in range(n):
        for j in range(n):
            for i in range(n):
                if 0 < i < n - 1 and 0 < j < n - 1 and 0 < k < n - 1:
                    continue  # interior cells are V2
                patch = [i + s + (nx + 1) * (j + nx * k) for s in (0, 1)]
                patch += [D.offsets[1] + i + nx * (j + s + (nx + 1) * k) for s in (0, 1)]
                patch += [D.offsets[2] + i + nx * (j + nx * (k + s)) for s in (0, 1)]
                patch += [D.offsets[3] + i + nx * (j + nx * k)]
                patch = [q for q in patch if D.active[q]]
                K = Lt[np.ix_(patch, patch)]
                ref[patch] += 0.5 * np.linalg.solve(K, r[patch])
    got = o.vanka(x, b, colour=-1)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_dwj_is_block_sequential_weighted_jacobi():
    # Sec. 3.1 DWJ, symmetric: velocity then pressure Jacobi steps on L~M (right-preconditioned), then
    # pressure then velocity steps on M^T L~ (left-preconditioned), weight 6/7, V2 rows only
    n = 6
    o = oracle.Oracle(n, levels=1, coarsest_max=2, dwj=True)
    D = DenseBox(n)
    Lt = D.Lt.toarray()
    M = D.M.toarray()
    d = np.diag(Lt @ M)
    v2 = D.active & ~D.v1
    vel = v2.copy()
    vel[D.offsets[3]:] = False
    pre = v2 & ~vel
    w = 6.0 / 7.0
    x = _masked(_rand(D.n, 43), D.active)
    b = _masked(_rand(D.n, 44), D.active)
    y = x.copy()
    r = b - Lt @ y
    y[vel] += w * r[vel] / d[vel]
    r = b - Lt @ y
    y += w * M[:, pre] @ (r[pre] / d[pre])
    r = b - Lt @ y
    y[pre] += w * (M[:, pre].T @ r) / d[pre]
    r = b - Lt @ y
    y[vel] += w * r[vel] / d[vel]
    got = o.dgs(x, b, direction=0)
    assert np.max(np.abs(got - y)) < 1e-12 * np.max(np.abs(y))


def test_wcycle_two_levels_equals_vcycle():
    # with an exact coarsest solve the second coarse visit of a two-level W-cycle corrects nothing
    ov = oracle.Oracle(8, levels=2, coarsest_max=4)
    ow = oracle.Oracle(8, levels=2, coarsest_max=4, cycle=2)
    act, _ = ov.masks()
    s = _masked(_rand(ov.n(), 42), act)
    tv, tw = ov.vcycle(s), ow.vcycle(s)
    assert np.max(np.abs(tv - tw)) < 1e-11 * np.max(np.abs(tv))


def test_wcycle_symmetric_and_at_least_as_fast():
    o = oracle.Oracle(8, levels=3, coarsest_max=2, cycle=2)
    act, _ = o.masks()
    W = _assemble(o.vcycle, o.n(), act)
    assert np.max(np.abs(W - W.T)) <= 1e-11 * np.max(np.abs(W))
    # Sec. 8.2: the W-cycle converges at least as fast per iteration as the V-cycle
    prob = synthetic.bumps(16, seed=0)
    its = []
    for cyc in (1, 2):
        oc = oracle.Oracle(16, coarsest_max=4, cycle=cyc)
        b = oc.rhs(prob["f"].numpy(), None)
        its.append(oc.sqmr(b, tol=1e-8, maxit=100)[2])
    assert its[1] <= its[0]


# ----------------------------------------------------------------------------------------------
# Sec. 2: transfers  P = 8 R^T, trilinear velocity, constant pressure

def test_restriction_is_scaled_transpose_of_prolongation():
    o = oracle.Oracle(8, levels=2, coarsest_max=4)
    act0, _ = o.masks(0)
    act1, _ = o.masks(1)
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
    assert np.max(np.abs(8.0 * R - P.T)) < 1e-15
    assert np.max(np.abs(P[~act0])) == 0.0


def test_prolongation_reproduces_linear_fields():
    # trilinear interpolation reproduces linear velocity fields on faces away from the walls
    n = 16
    o = oracle.Oracle(n, levels=2, coarsest_max=8)
    act0, _ = o.masks(0)
    h0, h1 = 1.0 / n, 2.0 / n
    coef = np.array([0.3, -1.1, 0.7, 2.0])

    def lin(X, Y, Z):
        return coef[0] + coef[1] * X + coef[2] * Y + coef[3] * Z

    def sample(nn, h):
        parts = []
        for c in range(3):
            xs, ys, zs = synthetic.face_coords(c, nn, nn, nn, h)
            Z, Y, X = np.meshgrid(zs.numpy(), ys.numpy(), xs.numpy(), indexing="ij")
            parts.append(lin(X, Y, Z).reshape(-1))
        xs, ys, zs = synthetic.face_coords(3, nn, nn, nn, h)
        Z, Y, X = np.meshgrid(zs.numpy(), ys.numpy(), xs.numpy(), indexing="ij")
        parts.append(np.full(nn ** 3, 0.0))
        return np.concatenate(parts)

    act1, _ = o.masks(1)
    ec = _masked(sample(n // 2, h1), act1)
    fine = o.prolong_add(ec, np.zeros(o.n(0)))
    ref = sample(n, h0)
    # faces whose interpolation stencil stays two fine cells away from every wall
    ok = np.zeros(o.n(0), bool)
    for c in range(3):
        dims = [(n + 1, n, n), (n, n + 1, n), (n, n, n + 1)][c]
        k, j, i = np.meshgrid(*[np.arange(m) for m in dims[::-1]], indexing="ij")
        idx = [i, j, k]
        good = np.ones_like(i, bool)
        for d in range(3):
            good &= (idx[d] >= 3) & (idx[d] <= n - 3)
        offs = [0, (n + 1) * n * n, 2 * (n + 1) * n * n][c]
        ok[offs:offs + good.size] = good.reshape(-1)
    assert ok.sum() > 100
    assert np.max(np.abs(fine[ok] - ref[ok])) < 1e-12


def test_pressure_restriction_is_mean_of_children():
    o = oracle.Oracle(8, levels=2, coarsest_max=4)
    r = np.zeros(o.n(0))
    p = _rand(512, 8)
    r[o.n(0) - 512:] = p
    bc = o.restrict(r)
    ref = p.reshape(4, 2, 4, 2, 4, 2).mean(axis=(1, 3, 5)).reshape(-1)
    assert np.max(np.abs(bc[o.n(1) - 64:] - ref)) < 1e-15


# ----------------------------------------------------------------------------------------------
# Alg. 1: coarse solve, V-cycle linearity/symmetry (Sec. 3, conditions for a symmetric W^dagger)

@pytest.mark.parametrize("eta", [1.0, 1e-3])
def test_one_level_vcycle_is_exact_inverse(eta):
    o = oracle.Oracle(4, eta=eta, levels=1, gamma=1e-2)
    D = DenseBox(4, eta=eta, gamma=1e-2)
    s = _masked(_rand(D.n, 9), D.active)
    t = o.vcycle(s)
    assert np.max(np.abs(D.Lt @ t - s)) < 1e-10 * np.max(np.abs(s))


@pytest.mark.parametrize("eta", [1.0, 1e-3])
def test_vcycle_dense_symmetric(eta):
    o = oracle.Oracle(8, eta=eta, levels=2, coarsest_max=4)
    act, _ = o.masks()
    W = _assemble(o.vcycle, o.n(), act)
    assert np.max(np.abs(W - W.T)) <= 1e-11 * np.max(np.abs(W))


def test_vcycle_random_symmetric_3_levels():
    o = oracle.Oracle(16, levels=3, coarsest_max=4)
    act, _ = o.masks()
    x, y = _masked(_rand(o.n(), 10), act), _masked(_rand(o.n(), 11), act)
    a, b = x @ o.vcycle(y), y @ o.vcycle(x)
    assert abs(a - b) <= 1e-12 * max(abs(a), 1e-300) + 1e-12 * np.linalg.norm(x) * np.linalg.norm(o.vcycle(y))


# ----------------------------------------------------------------------------------------------
# Alg. 4: SQMR

def test_unpreconditioned_sqmr_equals_minres():
    # With no preconditioner SQMR on a symmetric matrix is the quasi-minimal-residual smoothing of
    # a Lanczos process with orthogonal residuals, i.e. MINRES (exact arithmetic).
    D = DenseBox(4)
    o = oracle.Oracle(4, levels=1)
    b = _masked(_rand(D.n, 12), D.active)
    b[D.offsets[3]:] -= b[D.offsets[3]:].mean()  # consistent right-hand side (constant p in ker L)
    act = np.nonzero(D.active)[0]
    A = D.L[act][:, act]
    iters = []
    spla.minres(A, b[act], rtol=1e-30, maxiter=8, callback=lambda xk: iters.append(xk.copy()))
    for j in range(1, 7):
        x, rc, it, rr, _ = o.sqmr(b, precond=False, fixed_iters=j, maxit=j)
        xj = x[act]
        ref = iters[j - 1].copy()
        # compare modulo a constant pressure (the oracle removes the pressure mean on exit)
        npr = D.sizes[3]
        ref[-npr:] -= ref[-npr:].mean()
        assert np.max(np.abs(xj - ref)) <= 1e-8 * np.max(np.abs(ref)), j


@pytest.mark.parametrize("eta", [1.0, 1e-3])
def test_mg_sqmr_matches_direct_solve(eta):
    n = 8
    o = oracle.Oracle(n, eta=eta, levels=2, coarsest_max=4)
    D = DenseBox(n, eta=eta)
    b = _masked(_rand(D.n, 13), D.active)
    b[D.offsets[3]:] -= b[D.offsets[3]:].mean()
    x, rc, it, rr, _ = o.sqmr(b, tol=1e-13, maxit=200)
    assert rc == 0 and rr < 1e-13
    act = np.nonzero(D.active)[0]
    ref = np.linalg.lstsq(D.L[act][:, act].toarray(), b[act], rcond=None)[0]
    ref[-n ** 3:] -= ref[-n ** 3:].mean()
    assert np.max(np.abs(x[act] - ref)) <= 1e-10 * np.max(np.abs(ref))


def _mms_error(n):
    prob = synthetic.mms(n)
    o = oracle.Oracle(n, coarsest_max=8)
    b = o.rhs(prob["f"].numpy(), prob["g"].numpy())
    x, rc, it, rr, _ = o.sqmr(b, tol=1e-12, maxit=100)
    act, _ = o.masks()
    assert rc == 0
    ex = prob["exact"].numpy()
    nf = o.n() - n ** 3
    ev = np.max(np.abs((x - ex)[:nf][act[:nf]]))
    ep = np.max(np.abs((x - ex)[nf:]))
    return ev, ep, it


def test_mms_second_order_convergence():
    # Sec. 2 MAC scheme with Dirichlet ghosts at the exact values: second-order accurate
    e8, p8, _ = _mms_error(8)
    e16, p16, _ = _mms_error(16)
    e32, p32, _ = _mms_error(32)
    assert e8 / e16 > 3.3 and e16 / e32 > 3.6, (e8, e16, e32)
    assert p8 / p16 > 3.0 and p16 / p32 > 3.3, (p8, p16, p32)


def test_lm_block_triangular_on_v2_rows():
    # with full distribution columns the top-right block of L~M vanishes on every V2 velocity row
    # (V1 is one cell thick, so every V2 stencil sees only regular cells) -- Eq. (disc)
    D = DenseBox(8, eta=1.1, gamma=0.0)
    LM = (D.L @ D.M).toarray()
    nf = D.offsets[3]
    rows = np.nonzero(D.v2[:nf])[0]
    assert np.max(np.abs(LM[np.ix_(rows, np.arange(nf, D.n))])) < 1e-9 * np.max(np.abs(LM))


def test_dgs_is_stable_iteration():
    # repeated symmetric DGS must not amplify any error component (V1 frozen apart from the
    # distribution): its growth factor per sweep stays at most ~1
    o = oracle.Oracle(16, levels=2, coarsest_max=8)
    act, _ = o.masks()
    e = _masked(_rand(o.n(), 14), act)
    z = np.zeros(o.n())
    for _ in range(30):
        e2 = o.dgs(e, z)
        g = np.linalg.norm(e2) / np.linalg.norm(e)
        e = e2 / np.linalg.norm(e2)
    assert g < 1.02, g


def test_iteration_counts_flat_under_refinement():
    # Sec. 7.1: consistent convergence under refinement (16^3 -> 64^3, Gaussian bumps, tol 1e-8)
    its = []
    for n in (16, 32, 64):
        prob = synthetic.bumps(n, seed=0)
        o = oracle.Oracle(n, coarsest_max=8)
        b = o.rhs(prob["f"].numpy(), None)
        x, rc, it, rr, _ = o.sqmr(b, tol=1e-8, maxit=100)
        assert rc == 0 and rr < 1e-8
        its.append(it)
    assert max(its) <= min(its) + 4, its


# ----------------------------------------------------------------------------------------------
# Alg. 1 iterated as a solver on L~ (Sec. 3; the pure multigrid of the paper's comparisons, Sec. 6)

@pytest.mark.parametrize("variant", ["", "additive", "dwj", "kb2"])
def test_vcycle_from_initial_guess_is_residual_correction(variant):
    # every smoother is a linear stationary iteration and the coarse correction is linear, so a cycle
    # started at x0 equals x0 + W^+ (b - L~ x0): the pure-multigrid iterate can be formed either way
    o = oracle.Oracle(16, eta=1e-3, levels=3, coarsest_max=4, kb=2 if variant == "kb2" else 1,
                      additive=variant == "additive", dwj=variant == "dwj")
    act, _ = o.masks()
    b, x0 = _masked(_rand(o.n(), 30), act), _masked(_rand(o.n(), 31), act)
    lit = o.vcycle_x0(b, x0)
    rc = x0 + o.vcycle(b - o.apply(x0, penalised=True))
    assert np.max(np.abs(lit - rc)) <= 1e-12 * np.max(np.abs(lit))


@pytest.mark.parametrize("eta", [1.0, 1e-3])
def test_one_level_pure_multigrid_is_a_direct_solve(eta):
    # with one level the cycle is the exact coarsest solve of L~: one cycle solves L~ x = b
    D = DenseBox(4, eta=eta)
    o = oracle.Oracle(4, eta=eta, levels=1, coarsest_max=4)
    b = _masked(_rand(D.n, 32), D.active)
    x, rc, it, rr, hist = o.mg_solve(b, tol=1e-10, maxit=5)  # rounding floor of the solve: ~1e-12
    assert rc == 0 and it == 1 and hist[0] == pytest.approx(1.0)
    act = np.nonzero(D.active)[0]
    ref = np.linalg.solve(D.Lt[act][:, act].toarray(), b[act])
    assert np.max(np.abs(x[act] - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_pure_multigrid_converges_to_the_penalised_solution():
    # the fixed point of x <- V-cycle(L~, b, x) is L~^{-1} b (not the Stokes solution, which differs by
    # O(gamma)); on the unit-viscosity box each cycle reduces the residual by a fixed factor
    n = 8
    D = DenseBox(n, gamma=1e-3)
    o = oracle.Oracle(n, levels=2, coarsest_max=4)
    b = _masked(_rand(D.n, 33), D.active)
    x, rc, it, rr, hist = o.mg_solve(b, tol=1e-12, maxit=100)
    assert rc == 0 and rr < 1e-12
    act = np.nonzero(D.active)[0]
    ref = np.linalg.solve(D.Lt[act][:, act].toarray(), b[act])
    assert np.max(np.abs(x[act] - ref)) <= 1e-9 * np.max(np.abs(ref))
    rates = hist[1:] / hist[:-1]
    assert np.all(rates < 0.5), rates


# ----------------------------------------------------------------------------------------------
# the threaded oracle (order-free loops on several OpenMP threads) is the sequential one, bit for bit


@pytest.mark.parametrize("variant", ["", "additive", "dwj"])
@pytest.mark.parametrize("domain", ["box", "mixed"])
def test_threaded_oracle_is_bit_identical(domain, variant):
    import synthetic
    n = 16
    lab = None if domain == "box" else synthetic.porous_labels(n, seed=2, nspheres=5, rmin=0.1, rmax=0.2,
                                                                exterior_every=2)
    o = oracle.Oracle(n, eta=1e-3, coarsest_max=8, labels=lab, additive=variant == "additive",
                      dwj=variant == "dwj")
    act = o.masks()[0]
    b = np.random.default_rng(3).standard_normal(o.n()) * act
    outs = []
    try:
        for th in (1, 4):
            oracle.set_threads(th)
            x, rc, it, rr, _ = o.sqmr(b, tol=1e-30, maxit=3, fixed_iters=3)
            outs.append((o.vcycle(b), o.smooth(np.zeros(o.n()), b), o.apply(b), x))
    finally:
        oracle.set_threads(1)
    for a, c in zip(*outs):
        assert np.array_equal(a, c)
