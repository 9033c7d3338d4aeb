"""The solvers the paper compares MG-preconditioned SQMR against, on the GPU, against the oracle:
Alg. 1 iterated outright on L~ (pure multigrid, Sec. 3 / Sec. 6) and Alg. 4 without preconditioner.
Needs a GB300.

Tolerances (relative to the max-norm of the oracle result): a pure-multigrid iterate after a few
cycles 1e-10 (the GPU forms x + V(b - L~x), the oracle runs the cycle from x; both equal in exact
arithmetic, each cycle adds ~1e-13); plain-SQMR iterates 1e-10 (FP64 recurrences, as in the box).
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


def cuda(v):
    return torch.from_numpy(np.ascontiguousarray(v)).to(DEV)


def bumps_rhs(o, n, seed):
    return o.rhs(synthetic.bumps(n, seed=seed)["f"].numpy(), None)


VARIANTS = [dict(), dict(kb=2), dict(cycle=2), dict(additive=True), dict(dwj=True)]


@pytest.mark.parametrize("kw", VARIANTS, ids=lambda kw: "-".join(f"{k}{v}" for k, v in kw.items()) or "base")
def test_pure_multigrid_iterates_match_oracle(kw):
    n = 32
    o = oracle.Oracle(n, coarsest_max=8, **kw)
    S = smg.Stokes(n, **{("kb_vanka" if k == "kb" else k): v for k, v in kw.items()})
    b = bumps_rhs(o, n, 40)
    x_ref, rc, it, rr, hist = o.mg_solve(b, tol=1e-30, maxit=4)
    assert it == 4
    x = torch.zeros(o.n(), dtype=torch.float64, device=DEV)
    info = smg.mg_solve(S.h, cuda(b), x, tol=1e-30, max_iter=4, check=False)
    assert info.status == smg.ERR_NOT_CONVERGED and info.iterations == 4 and info.vcycles == 4
    assert rel_err(x, x_ref) < 1e-10
    assert info.rel_residual == pytest.approx(rr, rel=1e-6)
    S.close()


def test_pure_multigrid_converges_like_the_oracle():
    n = 32
    o = oracle.Oracle(n, coarsest_max=8)
    S = smg.Stokes(n)
    b = bumps_rhs(o, n, 41)
    x_ref, rc, it, rr, _ = o.mg_solve(b, tol=1e-8, maxit=200)
    assert rc == 0
    x, info = torch.zeros(o.n(), dtype=torch.float64, device=DEV), None
    info = smg.mg_solve(S.h, cuda(b), x, tol=1e-8, max_iter=200)
    assert info.status == 0 and abs(info.iterations - it) <= 1 and info.rel_residual < 1e-8
    assert rel_err(x, x_ref) < 1e-7
    # the limit is the penalised solution: its L~ residual vanishes, its Stokes residual is O(gamma)
    r_pen = b - o.apply(x.cpu().numpy(), penalised=True)
    assert np.linalg.norm(r_pen) < 1e-8 * np.linalg.norm(b)


def test_pure_multigrid_fp32_cycle_reaches_fp64_accuracy():
    # FP64 residual, FP32 cycle: the iteration is mixed-precision iterative refinement and still
    # reaches an L~ residual far below FP32 round-off
    n = 32
    o = oracle.Oracle(n, coarsest_max=8)
    S = smg.Stokes(n, precision=smg.PREC_FP32)
    b = bumps_rhs(o, n, 42)
    x, info = torch.zeros(o.n(), dtype=torch.float64, device=DEV), None
    info = smg.mg_solve(S.h, cuda(b), x, tol=1e-11, max_iter=200)
    assert info.status == 0
    x_ref, rc, _, _, _ = o.mg_solve(b, tol=1e-12, maxit=200)
    assert rel_err(x, x_ref) < 1e-9


def test_pure_multigrid_on_labelled_domain():
    n = 32
    lab = synthetic.porous_labels(n, seed=0, nspheres=10, rmin=0.08, rmax=0.18)
    o = oracle.Oracle(n, coarsest_max=8, labels=lab)
    S = smg.Stokes(n, labels=lab)
    act, _ = o.masks()
    f = np.random.default_rng(43).standard_normal(o.n()) * act
    f[-n ** 3:] = 0.0
    b = o.rhs(f, synthetic.plug_flow(n, labels=lab).numpy())
    x_ref, _, _, rr, _ = o.mg_solve(b, tol=1e-30, maxit=3)
    x = torch.zeros(o.n(), dtype=torch.float64, device=DEV)
    info = smg.mg_solve(S.h, cuda(b), x, tol=1e-30, max_iter=3, check=False)
    assert info.iterations == 3 and rel_err(x, x_ref) < 1e-10


def test_pure_multigrid_edge_cases_and_host_pointers():
    n = 16
    o = oracle.Oracle(n, coarsest_max=8)
    S = smg.Stokes(n)
    b = bumps_rhs(o, n, 44)
    xh = np.zeros(o.n())
    info = smg.mg_solve(S.h, b.copy(), xh, tol=1e-8, max_iter=100)  # host in, host out
    x_ref, rc, it, _, _ = o.mg_solve(b, tol=1e-8, maxit=100)
    assert info.status == 0 and abs(info.iterations - it) <= 1 and rel_err(xh, x_ref) < 1e-7
    x = torch.zeros(o.n(), dtype=torch.float64, device=DEV)
    info = smg.mg_solve(S.h, cuda(b), x, tol=1e-8, max_iter=0, check=False)
    assert info.status == smg.ERR_NOT_CONVERGED and info.iterations == 0 and info.rel_residual == pytest.approx(1.0)
    z = torch.zeros(o.n(), dtype=torch.float64, device=DEV)
    x.fill_(1.0)
    info = smg.mg_solve(S.h, z, x, tol=1e-8, max_iter=5)
    assert info.status == 0 and float(x.abs().max()) == 0.0
    bn = b.copy()
    bn[7] = np.nan
    info = smg.mg_solve(S.h, cuda(bn), x, tol=1e-8, max_iter=5, check=False)
    assert info.status == smg.ERR_NAN


@pytest.mark.parametrize("name", ["box", "porous"])
def test_plain_sqmr_iterates_match_oracle(name):
    n = 32
    lab = None if name == "box" else synthetic.porous_labels(n, seed=0, nspheres=10, rmin=0.08, rmax=0.18)
    o = oracle.Oracle(n, coarsest_max=8, labels=lab)
    S = smg.Stokes(n, labels=lab)
    act, _ = o.masks()
    f = np.random.default_rng(45).standard_normal(o.n()) * act
    f[-n ** 3:] = 0.0
    b = o.rhs(f, None)
    x_ref, _, _, _, _ = o.sqmr(b, tol=1e-30, maxit=12, precond=False, fixed_iters=12)
    x = torch.zeros(o.n(), dtype=torch.float64, device=DEV)
    info = smg.sqmr_solve_unpreconditioned(S.h, cuda(b), x, tol=1e-30, max_iter=12, check=False)
    assert info.iterations == 12 and info.vcycles == 0
    assert rel_err(x, x_ref) < 1e-10


def test_plain_sqmr_converges_on_a_small_box():
    n = 8
    o = oracle.Oracle(n, coarsest_max=8)
    S = smg.Stokes(n)
    b = bumps_rhs(o, n, 46)
    x_ref, rc, it, _, _ = o.sqmr(b, tol=1e-8, maxit=3000, precond=False)
    assert rc == 0
    x = torch.zeros(o.n(), dtype=torch.float64, device=DEV)
    info = smg.sqmr_solve_unpreconditioned(S.h, cuda(b), x, tol=1e-8, max_iter=3000)
    assert info.status == 0 and info.rel_residual < 1e-8
    assert abs(info.iterations - it) <= max(3, it // 20)
    assert rel_err(x, x_ref) < 1e-6
    # the preconditioned solver needs far fewer iterations (the point of the paper)
    _, info_mg = S.solve(cuda(b), tol=1e-8)
    assert info_mg.iterations * 3 < info.iterations
