"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element on the same
seeded inputs, plus full-size properties and edge cases.  Needs a GB300 (sm_103a).

Tolerances (relative to the max-norm of the oracle result):
* FP64 path: every kernel does the oracle's arithmetic in a different order, so single pieces agree to
  ~1e-15 per operation; 1e-12 covers a smoother sweep / transfer, 1e-11 a V-cycle (about 200 dependent
  updates), 1e-10 an SQMR iterate (the FP64 bound the solver states).
* FP32 V-cycle: unit round-off 6e-8 times ~200 dependent updates on O(1) data -> 1e-4 for a V-cycle.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

smg = pytest.importorskip("paper_2312_10615_gb300")
DEV = torch.device("cuda:0")


def rel_err(got, ref):
    got = got.cpu().numpy() if isinstance(got, torch.Tensor) else got
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def rand_masked(o, seed, level=0):
    act, _ = o.masks(level)
    v = np.random.default_rng(seed).standard_normal(o.n(level))
    v[~act] = 0.0
    return v


def cuda(v):
    return torch.from_numpy(np.ascontiguousarray(v)).to(DEV)


_cache = {}


def pair(dims, precision=smg.PREC_FP64, **kw):
    """(oracle, GPU handle) for a box, cached per module run."""
    key = (dims, precision, tuple(sorted(kw.items())))
    if key not in _cache:
        nx, ny, nz = dims
        o = oracle.Oracle(nx, ny, nz, coarsest_max=8, **kw)
        skw = {("kb_vanka" if k == "kb" else k): v for k, v in kw.items()}
        S = smg.Stokes(nx, ny, nz, precision=precision, **skw)
        assert S.levels == o.nlevels
        _cache[key] = (o, S)
    return _cache[key]


# ---------------------------------------------------------------------------------------------- a1

@pytest.mark.parametrize("dims", [(32, 32, 32), (24, 16, 20), (9, 7, 5), (2, 2, 2)])
def test_apply_parity(dims):
    o, S = pair(dims)
    x = rand_masked(o, 1)
    y = S.apply(cuda(x))
    assert rel_err(y, o.apply(x)) < 1e-13


def test_apply_ignores_entries_off_the_unknowns():
    o, S = pair((24, 16, 20))
    x = np.random.default_rng(2).standard_normal(o.n())  # garbage on walls too
    act, _ = o.masks()
    y = S.apply(cuda(x)).cpu().numpy()
    assert rel_err(y, o.apply(np.where(act, x, 0.0))) < 1e-13
    assert np.all(y[~act] == 0.0)


def test_rhs_parity_mms():
    o, S = pair((24, 24, 24))
    prob = synthetic.mms(24)
    b = S.rhs(prob["f"].to(DEV), prob["g"].to(DEV))
    assert rel_err(b, o.rhs(prob["f"].numpy(), prob["g"].numpy())) < 1e-13


def test_rhs_parity_lid_and_host_pointers():
    o, S = pair((24, 24, 24))
    prob = synthetic.lid(24)
    ref = o.rhs(prob["f"].numpy(), prob["g"].numpy())
    b = np.zeros(o.n())
    smg.stokes_rhs(S.h, prob["f"].numpy().copy(), prob["g"].numpy().copy(), b)  # host in, host out
    assert rel_err(b, ref) < 1e-13


# ---------------------------------------------------------------------------------------------- a4-a6

SMOOTH_CASES = [(3, "dgs_fwd"), (4, "dgs_bwd"), (1, "dgs_sym"), (2, "vanka_sym"), (0, "alg3")] + \
    [(10 + c, f"vanka_colour{c}") for c in range(8)]


@pytest.mark.parametrize("level", [0, 1])
@pytest.mark.parametrize("which,name", SMOOTH_CASES)
def test_smoother_piece_parity(which, name, level):
    o, S = pair((32, 32, 32))
    x = rand_masked(o, 3, level)
    b = rand_masked(o, 4, level)
    got = cuda(x)
    smg.stokes_smooth(S.h, level, which, got, cuda(b))
    if which == 0:
        ref = o.smooth(x, b, level=level)
    elif which in (1, 3, 4):
        ref = o.dgs(x, b, level=level, direction={1: 0, 3: 1, 4: -1}[which])
    elif which == 2:
        ref = o.vanka(x, b, level=level, colour=-1)
    else:
        ref = o.vanka(x, b, level=level, colour=which - 10)
    assert rel_err(got, ref) < 1e-12, name


def test_smoother_non_cubic():
    o, S = pair((24, 16, 32))
    x, b = rand_masked(o, 5), rand_masked(o, 6)
    got = cuda(x)
    smg.stokes_smooth(S.h, 0, 0, got, cuda(b))
    assert rel_err(got, o.smooth(x, b)) < 1e-12


# ---------------------------------------------------------------------------------------------- a2, a3, a7

@pytest.mark.parametrize("level", [0, 1])
def test_restrict_parity(level):
    o, S = pair((32, 32, 32))
    r = rand_masked(o, 7, level)
    bc = torch.zeros(o.n(level + 1), dtype=torch.float64, device=DEV)
    smg.stokes_restrict(S.h, level, cuda(r), bc)
    assert rel_err(bc, o.restrict(r, level=level)) < 1e-13


@pytest.mark.parametrize("level", [0, 1])
def test_prolong_parity(level):
    o, S = pair((32, 32, 32))
    e = rand_masked(o, 8, level + 1)
    x = rand_masked(o, 9, level)
    got = cuda(x)
    smg.stokes_prolong_add(S.h, level, cuda(e), got)
    assert rel_err(got, o.prolong_add(e, x, level=level)) < 1e-13


@pytest.mark.parametrize("dims", [(32, 32, 32), (48, 48, 48)])
def test_coarse_solve_parity(dims):
    o, S = pair(dims)
    lc = o.nlevels - 1
    b = rand_masked(o, 10, lc)
    x = torch.zeros(o.n(lc), dtype=torch.float64, device=DEV)
    smg.stokes_coarse_solve(S.h, cuda(b), x)
    assert rel_err(x, o.coarse_solve(b)) < 1e-10


# ---------------------------------------------------------------------------------------------- a8

@pytest.mark.parametrize("dims", [(32, 32, 32), (48, 48, 48), (24, 16, 32), (16, 16, 16)])
def test_vcycle_parity(dims):
    o, S = pair(dims)
    s = rand_masked(o, 11)
    t = S.precondition(cuda(s))
    assert rel_err(t, o.vcycle(s)) < 1e-11


def test_vcycle_parity_kb2():
    o, S = pair((32, 32, 32), kb=2)
    s = rand_masked(o, 12)
    assert rel_err(S.precondition(cuda(s)), o.vcycle(s)) < 1e-11


def test_vcycle_is_linear_and_symmetric_fp64():
    o, S = pair((32, 32, 32))
    x, y = cuda(rand_masked(o, 13)), cuda(rand_masked(o, 14))
    Mx, My = S.precondition(x), S.precondition(y)
    a, b = float(x @ My), float(y @ Mx)
    assert abs(a - b) <= 1e-12 * float(torch.linalg.norm(x) * torch.linalg.norm(My))
    Mxy = S.precondition(2.0 * x + y)
    assert float(torch.max(torch.abs(Mxy - 2.0 * Mx - My))) <= 1e-12 * float(torch.max(torch.abs(Mxy)))


def test_vcycle_fp32_parity_and_symmetry():
    o, S = pair((32, 32, 32), precision=smg.PREC_FP32)
    s = rand_masked(o, 15)
    assert rel_err(S.precondition(cuda(s)), o.vcycle(s)) < 1e-4
    x, y = cuda(rand_masked(o, 16)), cuda(rand_masked(o, 17))
    a, b = float(x @ S.precondition(y)), float(y @ S.precondition(x))
    assert abs(a - b) <= 1e-5 * float(torch.linalg.norm(x) * torch.linalg.norm(S.precondition(y)))


def test_persistent_vanka_matches_per_colour_launches():
    # one cooperative launch per symmetric sweep (grid barriers) vs two launches per colour
    o, _ = pair((32, 32, 32))
    Sp = smg.Stokes(32, autotune=False)
    Sc = smg.Stokes(32, vanka_persistent=True)
    for l in range(Sp.levels - 1):
        assert smg.stokes_level_schedule(Sp.h, l)[0] == 0 and smg.stokes_level_schedule(Sc.h, l)[0] == 1
    s = cuda(rand_masked(o, 26))
    assert float(torch.max(torch.abs(Sp.precondition(s) - Sc.precondition(s)))) == 0.0
    Sp.close()
    Sc.close()


@pytest.mark.parametrize("cluster", [4, 8, 16])
def test_cluster_vanka_sweep_matches_per_colour_launches(cluster):
    # every level's symmetric Vanka sweep in one thread-block cluster with hardware barriers
    Sp = smg.Stokes(48, precision=smg.PREC_FP32, autotune=False)
    Sc = smg.Stokes(48, precision=smg.PREC_FP32, autotune=False)
    for l in range(Sc.levels - 1):
        smg.stokes_set_level_schedule(Sc.h, l, 2, cluster)
        assert smg.stokes_level_schedule(Sc.h, l)[:2] == (2, cluster)
    s = cuda(np.random.default_rng(28).standard_normal(Sc.n))
    assert float(torch.max(torch.abs(Sp.precondition(s) - Sc.precondition(s)))) == 0.0
    Sp.close()
    Sc.close()


def test_shared_memory_vanka_sweep_matches_per_colour_launches():
    # small levels: the whole symmetric sweep in one block on a shared-memory copy of the level
    Sp = smg.Stokes(32, precision=smg.PREC_FP32, autotune=False)
    Sm = smg.Stokes(32, precision=smg.PREC_FP32, autotune=False)
    smg.stokes_set_level_schedule(Sm.h, 1, 3)  # the 16^3 level fits
    assert smg.stokes_level_schedule(Sm.h, 1)[:2] == (3, 1)
    with pytest.raises(smg.StokesError):
        smg.stokes_set_level_schedule(Sm.h, 0, 3)  # 32^3 in FP32 does not fit in 227 KB
    s = cuda(np.random.default_rng(29).standard_normal(Sm.n))
    assert float(torch.max(torch.abs(Sp.precondition(s) - Sm.precondition(s)))) == 0.0
    b = Sm.rhs(synthetic.bumps(32, seed=5, device=DEV)["f"], None)
    xp, ip = Sp.solve(b, tol=1e-8)
    xm, im = Sm.solve(b, tol=1e-8)
    assert ip.iterations == im.iterations and float(torch.max(torch.abs(xp - xm))) == 0.0
    Sp.close()
    Sm.close()


@pytest.mark.parametrize("kb", [1, 2])
@pytest.mark.parametrize("precision", [smg.PREC_FP64, smg.PREC_FP32, smg.PREC_MIXED_BF16])
def test_one_launch_per_colour_step_matches_per_colour_launches(precision, kb):
    # two copies of the Vanka state, one launch per colour step: bit-identical V-cycles and solves
    n = 48
    Sp = smg.Stokes(n, precision=precision, kb_vanka=kb, autotune=False)
    Sg = smg.Stokes(n, precision=precision, kb_vanka=kb, autotune=False)
    for l in range(Sg.levels - 1):
        smg.stokes_set_level_schedule(Sg.h, l, 4, 0)
        assert smg.stokes_level_schedule(Sg.h, l)[:2] == (4, 0)
    s = cuda(np.random.default_rng(30).standard_normal(Sg.n))
    assert torch.equal(Sp.precondition(s), Sg.precondition(s))
    b = Sg.rhs(synthetic.bumps(n, seed=6, device=DEV)["f"], None)
    xp, ip = Sp.solve(b, tol=1e-8)
    xg, ig = Sg.solve(b, tol=1e-8)
    assert ip.iterations == ig.iterations and torch.equal(xp, xg)
    Sp.close()
    Sg.close()


@pytest.mark.parametrize("dims", [(64, 64, 64), (48, 24, 16)])
@pytest.mark.parametrize("precision", [smg.PREC_FP64, smg.PREC_FP32, smg.PREC_MIXED_BF16])
def test_fused_velocity_dgs_matches_in_place_launches(precision, dims):
    # both velocity parities of a DGS stage in one out-of-place pass: the same bits as the two
    # in-place launches, for the V-cycle, one symmetric DGS sweep and a whole solve
    nx, ny, nz = dims
    Sp = smg.Stokes(nx, ny, nz, precision=precision, autotune=False)
    Sf = smg.Stokes(nx, ny, nz, precision=precision, autotune=False)
    for l in range(Sf.levels - 1):
        assert smg.stokes_level_dgs(Sp.h, l)[0] == 0
        smg.stokes_set_level_dgs(Sf.h, l, 1)
        assert smg.stokes_level_dgs(Sf.h, l)[0] == 1
    s = cuda(np.random.default_rng(31).standard_normal(Sf.n))
    assert torch.equal(Sp.precondition(s), Sf.precondition(s))
    xs, bs = cuda(np.random.default_rng(32).standard_normal(Sf.n)), cuda(np.random.default_rng(33).standard_normal(Sf.n))
    a, c = xs.clone(), xs.clone()
    smg.stokes_smooth(Sp.h, 0, 1, a, bs)
    smg.stokes_smooth(Sf.h, 0, 1, c, bs)
    assert torch.equal(a, c)
    if nx == ny == nz:
        b = Sf.rhs(synthetic.bumps(nx, seed=7, device=DEV)["f"], None)
        xp, ip = Sp.solve(b, tol=1e-8)
        xf, i_f = Sf.solve(b, tol=1e-8)
        assert ip.iterations == i_f.iterations and torch.equal(xp, xf)
    Sp.close()
    Sf.close()


@pytest.mark.parametrize("precision", [smg.PREC_FP64, smg.PREC_FP32, smg.PREC_MIXED_BF16])
def test_autotuned_schedule_is_bit_identical(precision):
    # the autotuner only picks how the Vanka sweeps are launched, never what they compute
    Sa = smg.Stokes(64, precision=precision)
    Sp = smg.Stokes(64, precision=precision, autotune=False)
    for l in range(Sa.levels - 1):
        mode, blocks, ms = smg.stokes_level_schedule(Sa.h, l)
        assert mode in (0, 1, 2, 3, 4) and ms > 0 and (mode in (0, 4) or blocks >= 1)
    s = cuda(np.random.default_rng(27).standard_normal(Sa.n))
    assert float(torch.max(torch.abs(Sa.precondition(s) - Sp.precondition(s)))) == 0.0
    b = Sa.rhs(synthetic.bumps(64, seed=4, device=DEV)["f"], None)
    xa, ia = Sa.solve(b, tol=1e-8)
    xp, ip = Sp.solve(b, tol=1e-8)
    assert ia.iterations == ip.iterations and float(torch.max(torch.abs(xa - xp))) == 0.0
    Sa.close()
    Sp.close()


def test_graph_and_eager_paths_agree():
    o, Sg = pair((32, 32, 32))
    Se = smg.Stokes(32, use_graphs=False)
    s = cuda(rand_masked(o, 18))
    assert float(torch.max(torch.abs(Sg.precondition(s) - Se.precondition(s)))) == 0.0
    Se.close()


@pytest.mark.parametrize("precision", [smg.PREC_FP32, smg.PREC_FP64])
def test_device_loop_equals_host_loop(precision):
    # the SQMR loop as one graph (while node, stopping test on the device) against the host-driven eager
    # loop: same iteration counts, statuses and bits -- converged, cut off by max_iter, restarted after
    # an explicit residual that did not confirm, and unpreconditioned
    n = 32
    Sg = smg.Stokes(n, precision=precision)
    Se = smg.Stokes(n, precision=precision, use_graphs=False)
    b = Sg.rhs(synthetic.bumps(n, seed=8, device=DEV)["f"], None)
    for tol, maxit in ((1e-8, 200), (1e-30, 7), (1e-13, 60)):
        xg, xe = torch.zeros_like(b), torch.zeros_like(b)
        ig = smg.sqmr_solve(Sg.h, b, xg, tol, maxit, check=False)
        ie = smg.sqmr_solve(Se.h, b, xe, tol, maxit, check=False)
        assert (ig.status, ig.iterations, ig.rel_residual) == (ie.status, ie.iterations, ie.rel_residual)
        assert float(torch.max(torch.abs(xg - xe))) == 0.0
    xg, xe = torch.zeros_like(b), torch.zeros_like(b)
    ig = smg.sqmr_solve_unpreconditioned(Sg.h, b, xg, 1e-6, 400, check=False)
    ie = smg.sqmr_solve_unpreconditioned(Se.h, b, xe, 1e-6, 400, check=False)
    assert (ig.status, ig.iterations) == (ie.status, ie.iterations)
    assert float(torch.max(torch.abs(xg - xe))) == 0.0
    assert smg.stokes_device_loop(Sg.h) and not smg.stokes_device_loop(Se.h)
    Sg.close()
    Se.close()


# ---------------------------------------------------------------------------------------------- a9, a10

def test_sqmr_manufactured_32_parity():
    # 32^3, unit viscosity, manufactured solution, x0 = 0, tol 1e-10 (the parity workload)
    o, S = pair((32, 32, 32))
    prob = synthetic.mms(32)
    b_ref = o.rhs(prob["f"].numpy(), prob["g"].numpy())
    x_ref, rc, it_ref, rr_ref, _ = o.sqmr(b_ref, tol=1e-10, maxit=100)
    assert rc == 0 and rr_ref < 1e-10
    b = S.rhs(prob["f"].to(DEV), prob["g"].to(DEV))
    # equal iteration count: compare the iterates
    x = torch.zeros_like(b)
    info = smg.sqmr_solve(S.h, b, x, tol=1e-30, max_iter=it_ref, check=False)
    assert info.iterations == it_ref
    assert rel_err(x, x_ref) < 1e-10
    # on its own the GPU solve meets the tolerance, within one iteration of the oracle
    x2, info2 = S.solve(b, tol=1e-10, max_iter=100)
    assert info2.status == 0 and info2.rel_residual < 1e-10
    assert abs(info2.iterations - it_ref) <= 1
    assert rel_err(x2, x_ref) < 1e-9


def test_sqmr_bumps_48_parity():
    o, S = pair((48, 48, 48))
    prob = synthetic.bumps(48, seed=3)
    b_ref = o.rhs(prob["f"].numpy(), None)
    x_ref, rc, it_ref, _, _ = o.sqmr(b_ref, tol=1e-8, maxit=100, fixed_iters=8)
    b = S.rhs(prob["f"].to(DEV), None)
    x = torch.zeros_like(b)
    info = smg.sqmr_solve(S.h, b, x, tol=1e-30, max_iter=8, check=False)
    assert info.iterations == 8
    assert rel_err(x, x_ref) < 1e-10


def test_sqmr_fp32_vcycle_accuracy():
    # FP32 V-cycle, FP64 SQMR: the same tolerance is met; the solution agrees with the FP64 oracle
    o, S = pair((32, 32, 32), precision=smg.PREC_FP32)
    prob = synthetic.bumps(32, seed=1)
    b_ref = o.rhs(prob["f"].numpy(), None)
    x_ref, rc, it_ref, _, _ = o.sqmr(b_ref, tol=1e-12, maxit=200)
    b = S.rhs(prob["f"].to(DEV), None)
    x, info = S.solve(b, tol=1e-10, max_iter=200)
    assert info.status == 0 and info.rel_residual < 1e-10
    assert rel_err(x, x_ref) < 1e-7


# ---------------------------------------------------------------------------------------------- variants

VARIANTS = [dict(kb=2), dict(kb=3), dict(cycle=2), dict(additive=True), dict(additive=True, kb=3), dict(dwj=True)]


@pytest.mark.parametrize("kw", VARIANTS, ids=lambda kw: "-".join(f"{k}{v}" for k, v in kw.items()))
def test_variant_parity(kw):
    # k_b sweeps (Sec. 7), the W-cycle (Sec. 8.2) and additive Vanka (Eq. av): a smoothing step, a
    # V/W-cycle and six SQMR iterations against the oracle with the same variant
    o = oracle.Oracle(32, coarsest_max=8, **kw)
    S = smg.Stokes(32, **{("kb_vanka" if k == "kb" else k): v for k, v in kw.items()})
    x, b = rand_masked(o, 51), rand_masked(o, 52)
    got = cuda(x)
    smg.stokes_smooth(S.h, 0, 0, got, cuda(b))
    assert rel_err(got, o.smooth(x, b)) < 1e-12
    s = rand_masked(o, 50)
    assert rel_err(S.precondition(cuda(s)), o.vcycle(s)) < 1e-11
    prob = synthetic.bumps(32, seed=6)
    b_ref = o.rhs(prob["f"].numpy(), None)
    x_ref, _, _, _, _ = o.sqmr(b_ref, tol=1e-30, maxit=6, fixed_iters=6)
    bb = S.rhs(prob["f"].to(DEV), None)
    xx = torch.zeros_like(bb)
    info = smg.sqmr_solve(S.h, bb, xx, tol=1e-30, max_iter=6, check=False)
    assert info.iterations == 6 and rel_err(xx, x_ref) < 1e-10
    _, info8 = S.solve(bb, tol=1e-8)
    assert info8.status == 0
    S.close()


def test_variants_non_cubic():
    # the variant kernels on a box whose axes differ (strides, V2 ranges, colour counts per axis)
    for kw in (dict(dwj=True), dict(additive=True), dict(cycle=2)):
        o = oracle.Oracle(24, 16, 32, coarsest_max=8, **kw)
        S = smg.Stokes(24, 16, 32, **kw)
        x, b = rand_masked(o, 53), rand_masked(o, 54)
        got = cuda(x)
        smg.stokes_smooth(S.h, 0, 0, got, cuda(b))
        assert rel_err(got, o.smooth(x, b)) < 1e-12, kw
        s = rand_masked(o, 55)
        assert rel_err(S.precondition(cuda(s)), o.vcycle(s)) < 1e-11, kw
        S.close()


# ---------------------------------------------------------------------------------------------- BF16 levels

def test_mixed_bf16_pieces_close_to_oracle():
    # the two finest levels store b and r as BF16 (8 significant bits): a V-cycle, a smoothing step
    # and a restriction agree with the FP64 oracle to the BF16 rounding of their operands
    o, S = pair((32, 32, 32), precision=smg.PREC_MIXED_BF16)
    s = rand_masked(o, 31)
    assert rel_err(S.precondition(cuda(s)), o.vcycle(s)) < 3e-2
    for level in (0, 1):  # the BF16 levels (level 2 is the coarsest)
        x, b = rand_masked(o, 32, level), rand_masked(o, 33, level)
        got = cuda(x)
        smg.stokes_smooth(S.h, level, 0, got, cuda(b))
        assert rel_err(got, o.smooth(x, b, level=level)) < 3e-2, level
    r = rand_masked(o, 34, 0)
    bc = torch.zeros(S.length(1), dtype=torch.float64, device=DEV)
    smg.stokes_restrict(S.h, 0, cuda(r), bc)
    assert rel_err(bc, o.restrict(r, level=0)) < 1e-2


def test_sqmr_mixed_bf16_accuracy():
    # BF16 operand storage changes the preconditioner, not the tolerance: the solution matches the
    # FP64 oracle's as closely as the FP32 V-cycle's does
    o, S = pair((32, 32, 32), precision=smg.PREC_MIXED_BF16)
    prob = synthetic.bumps(32, seed=1)
    b_ref = o.rhs(prob["f"].numpy(), None)
    x_ref, rc, it_ref, _, _ = o.sqmr(b_ref, tol=1e-12, maxit=200)
    b = S.rhs(prob["f"].to(DEV), None)
    x, info = S.solve(b, tol=1e-10, max_iter=200)
    assert info.status == 0 and info.rel_residual < 1e-10
    assert rel_err(x, x_ref) < 1e-7
    _, info8 = S.solve(b, tol=1e-8, max_iter=200)
    _, o8, it8, _, _ = o.sqmr(b_ref, tol=1e-8, maxit=200)
    assert info8.iterations <= it8 + 2


# ---------------------------------------------------------------------------------------------- F1

def test_lid_cavity_32_parity():
    # 3D lid-driven cavity (Sec. 7): eta = gamma = 1e-3, lid u = 1 on the top ghost row; the GPU
    # iterates equal the oracle's at the same iteration count
    o = oracle.Oracle(32, 32, 32, eta=1e-3, gamma=1e-3, coarsest_max=8)
    S = smg.Stokes(32, viscosity=1e-3, gamma=1e-3)
    prob = synthetic.lid(32)
    b_ref = o.rhs(prob["f"].numpy(), prob["g"].numpy())
    x_ref, rc, it_ref, _, _ = o.sqmr(b_ref, tol=1e-8, maxit=100, fixed_iters=8)
    b = S.rhs(prob["f"].to(DEV), prob["g"].to(DEV))
    assert rel_err(b, b_ref) < 1e-13
    x = torch.zeros_like(b)
    info = smg.sqmr_solve(S.h, b, x, tol=1e-30, max_iter=8, check=False)
    assert info.iterations == 8
    assert rel_err(x, x_ref) < 1e-10
    S.close()


def test_lid_cavity_128():
    # the paper's 3D cavity at 128^3, 5 levels: FP64 and FP32 V-cycles reach 1e-8; the flow is mirror
    # symmetric about y = 1/2 (u, w, p even, v odd); the two solutions agree
    n = 128
    prob = synthetic.lid(n, device=DEV)
    out = {}
    for prec in (smg.PREC_FP64, smg.PREC_FP32):
        S = smg.Stokes(n, viscosity=1e-3, gamma=1e-3, precision=prec)
        assert S.levels == 5
        b = S.rhs(prob["f"], prob["g"])
        x, info = S.solve(b, tol=1e-10, max_iter=200)
        assert info.status == 0 and info.rel_residual < 1e-10
        assert S.residual_norm(b, x) / float(torch.linalg.norm(b)) < 1e-10
        out[prec] = (x, info.iterations)
        S.close()
    x64, it64 = out[smg.PREC_FP64]
    x32, it32 = out[smg.PREC_FP32]
    assert abs(it64 - it32) <= 2
    assert float(torch.max(torch.abs(x32 - x64)) / torch.max(torch.abs(x64))) < 1e-7
    u, v, w, p = synthetic.unpack(x64.cpu(), n)
    scale = float(torch.max(torch.abs(x64[: 3 * (n + 1) * n * n])))
    # the colour orders of the smoothers are not mirror symmetric, so the mirror image agrees to the
    # solve's accuracy only
    assert float(torch.max(torch.abs(u - u.flip(1)))) < 1e-7 * scale
    assert float(torch.max(torch.abs(v + v.flip(1)))) < 1e-7 * scale
    assert float(torch.max(torch.abs(w - w.flip(1)))) < 1e-7 * scale
    assert abs(float(p.mean())) < 1e-12 * float(torch.max(torch.abs(p)))
    # the lid drags the top layer forward (u > 0 just under the lid) and the return flow runs below
    assert float(u[-1, n // 2, n // 2]) > 0.1 and float(u[n // 2, n // 2, n // 2]) < 0.0


def test_sqmr_host_pointers_match_device():
    o, S = pair((32, 32, 32))
    prob = synthetic.bumps(32, seed=2)
    b = S.rhs(prob["f"].to(DEV), None)
    xd, info_d = S.solve(b, tol=1e-8)
    bh = b.cpu().numpy().copy()
    xh = np.zeros_like(bh)
    info_h = smg.sqmr_solve(S.h, bh, xh, tol=1e-8)
    assert info_h.iterations == info_d.iterations
    assert rel_err(xh, xd.cpu().numpy()) == 0.0


def test_batch_solve_matches_single_solves():
    # independent problems of uneven sizes solved concurrently give the same bits as one by one
    sizes, handles, rhs, xs, ref = [16, 24, 32, 48], [], [], [], []
    for k, n in enumerate(sizes):
        S = smg.Stokes(n, precision=smg.PREC_FP32)
        b = S.rhs(synthetic.bumps(n, seed=k, device=DEV)["f"], None)
        x1, info1 = S.solve(b, tol=1e-8)
        handles.append(S)
        rhs.append(b)
        xs.append(torch.zeros_like(b))
        ref.append((x1, info1.iterations))
    infos, done = smg.sqmr_solve_batch([S.h for S in handles], rhs, xs, tol=1e-8, nstreams=3)
    for (x1, it1), x2, info in zip(ref, xs, infos):
        assert info.status == 0 and info.iterations == it1
        assert float(torch.max(torch.abs(x1 - x2))) == 0.0
    assert all(d > 0 for d in done)
    for S in handles:
        S.close()


def test_batch_on_fresh_handles():
    # the first solve of a handle allocates its SQMR vectors; solved on the batch's own non-blocking
    # streams, their zero fill must be complete before the solve's kernels run
    sizes = [24, 32, 16, 48, 32, 24, 40, 16, 32, 24, 48, 16]
    for rep in range(2):
        handles, rhs, xs = [], [], []
        for k, n in enumerate(sizes):
            S = smg.Stokes(n, precision=smg.PREC_FP32)
            handles.append(S)
            rhs.append(S.rhs(synthetic.bumps(n, seed=50 + k + rep, device=DEV)["f"], None))
            xs.append(torch.zeros_like(rhs[-1]))
        infos, _ = smg.sqmr_solve_batch([S.h for S in handles], rhs, xs, tol=1e-8, nstreams=6)
        for S, b, x2, info in zip(handles, rhs, xs, infos):
            x1, info1 = S.solve(b, tol=1e-8)
            assert info.status == 0 and info.iterations == info1.iterations
            assert float(torch.max(torch.abs(x1 - x2))) == 0.0
        for S in handles:
            S.close()


def test_residual_norm_entry():
    o, S = pair((24, 16, 20))
    b, x = rand_masked(o, 19), rand_masked(o, 20)
    ref = np.linalg.norm(b - o.apply(x))
    assert abs(smg.stokes_residual_norm(S.h, cuda(b), cuda(x)) - ref) <= 1e-12 * ref


# ---------------------------------------------------------------------------------------------- edges

def test_zero_rhs_gives_zero_solution():
    o, S = pair((16, 16, 16))
    b = torch.zeros(o.n(), dtype=torch.float64, device=DEV)
    x0 = cuda(rand_masked(o, 21))
    x, info = S.solve(b, x0=x0)
    assert info.status == 0 and float(torch.max(torch.abs(x))) == 0.0


def test_max_iter_zero_and_nan():
    o, S = pair((16, 16, 16))
    b = cuda(rand_masked(o, 22))
    x = torch.zeros_like(b)
    info = smg.sqmr_solve(S.h, b, x, tol=1e-8, max_iter=0, check=False)
    assert info.status == smg.ERR_NOT_CONVERGED
    b[5] = float("nan")
    info = smg.sqmr_solve(S.h, b, x, tol=1e-8, max_iter=5, check=False)
    assert info.status == smg.ERR_NAN


def test_invalid_arguments():
    with pytest.raises(smg.StokesError) as e:
        smg.Stokes(1, 4, 4)
    assert e.value.code == smg.ERR_INVALID_ARG
    with pytest.raises(smg.StokesError):
        smg.Stokes(8, viscosity=0.0)
    with pytest.raises(smg.StokesError):
        smg.Stokes(9, 9, 9, levels=2)  # odd dimensions cannot be coarsened
    with pytest.raises(smg.StokesError) as e:
        smg.Stokes(64, levels=1)  # dense coarsest solve of a 64^3 grid is refused
    assert e.value.code == smg.ERR_INVALID_ARG


def test_smallest_grid_solve():
    o, S = pair((2, 2, 2))
    b = rand_masked(o, 23)
    b[o.n() - 8:] -= b[o.n() - 8:].mean()
    x_ref, rc, it, _, _ = o.sqmr(b, tol=1e-12, maxit=50)
    x, info = S.solve(cuda(b), tol=1e-12, max_iter=50)
    assert info.status == 0 and rel_err(x, x_ref) < 1e-10


# ---------------------------------------------------------------------------------------------- full size

@pytest.fixture(scope="module")
def big():
    n = 256
    o = oracle.Oracle(n, coarsest_max=8)
    S = smg.Stokes(n)
    return n, o, S


def test_full_size_apply_parity(big):
    n, o, S = big
    x = rand_masked(o, 24)
    assert rel_err(S.apply(cuda(x)), o.apply(x)) < 1e-13


def test_full_size_vcycle_parity(big):
    # one V-cycle at 256^3 in the bench's launch configuration (CUDA graph), against the oracle
    n, o, S = big
    s = rand_masked(o, 25)
    assert rel_err(S.precondition(cuda(s)), o.vcycle(s)) < 1e-11


def test_full_size_solve_properties(big):
    n, o, S = big
    prob = synthetic.bumps(n, seed=0, device=DEV)
    b = S.rhs(prob["f"], None)
    x, info = S.solve(b, tol=1e-8, max_iter=100)
    assert info.status == 0 and info.rel_residual < 1e-8
    r = torch.zeros_like(b)
    smg.stokes_apply(S.h, x, r)
    assert float(torch.linalg.norm(b - r) / torch.linalg.norm(b)) < 1e-8
    nf = S.n - n ** 3
    assert abs(float(x[nf:].mean())) < 1e-12 * float(torch.max(torch.abs(x[nf:])))


def test_apply_on_unaligned_buffers_matches_aligned():
    # the four-entries-per-thread residual path needs 16-byte aligned arrays; views that start one
    # element into an allocation take the one-entry path and give the same result
    o, S = pair((32, 32, 32))
    x = rand_masked(o, 60)
    ya = S.apply(cuda(x))
    xs = torch.zeros(o.n() + 1, dtype=torch.float64, device=DEV)
    xs[1:] = cuda(x)
    ys = torch.zeros(o.n() + 1, dtype=torch.float64, device=DEV)
    smg.stokes_apply(S.h, xs[1:], ys[1:])
    assert rel_err(ys[1:], ya.cpu().numpy()) < 1e-15
    assert rel_err(ya, o.apply(x)) < 1e-13


@pytest.mark.parametrize("precision", [smg.PREC_FP64, smg.PREC_FP32])
def test_reported_residual_matches_recomputed(precision):
    # the converged solve reports the residual of its confirmation step; the returned x (pressure mean
    # removed afterwards) has the same residual up to rounding
    o, S = pair((32, 32, 32), precision=precision)
    b = o.rhs(synthetic.bumps(32, seed=9)["f"].numpy(), None)
    x, info = S.solve(cuda(b), tol=1e-9)
    assert info.status == 0
    ref = smg.stokes_residual_norm(S.h, cuda(b), x) / np.linalg.norm(b)
    assert ref < 1e-9
    assert info.rel_residual == pytest.approx(ref, rel=1e-6, abs=1e-15)
