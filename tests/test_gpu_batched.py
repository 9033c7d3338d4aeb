"""Batched handles (stokes_create_batch / sqmr_solve_batched): one launch per V-cycle and SQMR step for
all problems of a grid.  Every problem's result must carry the bits, iteration count and status of
the same problem solved alone (stokes_create + sqmr_solve), whatever the schedule either handle runs.
Needs a GB300 (sm_103a)."""
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu

smg = pytest.importorskip("paper_2312_10615_gb300")
DEV = torch.device("cuda:0")


def _rhs(S, n, seed):
    return S.rhs(synthetic.bumps(n, seed=seed, device=DEV)["f"], None)


def _compare(B, S, rhs, starts, tol, max_iter):
    xs = [x.clone() for x in starts]
    infos = smg.sqmr_solve_batched(B.h, rhs, xs, tol, max_iter, check=False)
    for b, x0, x2, info in zip(rhs, starts, xs, infos):
        x1 = x0.clone()
        info1 = smg.sqmr_solve(S.h, b, x1, tol, max_iter, check=False)
        assert (info.status, info.iterations, info.vcycles) == (info1.status, info1.iterations, info1.vcycles)
        assert info.rel_residual == info1.rel_residual
        assert float(torch.max(torch.abs(x1 - x2))) == 0.0
    return infos


def _check_against_single(n, nb, seeds, precision, tol=1e-8, max_iter=200, labels=None, kw=None):
    kw = dict(kw or {})
    B = smg.Stokes(n, precision=precision, labels=labels, batch=nb, **kw)
    assert smg.stokes_batch_size(B.h) == nb
    S = smg.Stokes(n, precision=precision, labels=labels, **kw)
    rhs = [_rhs(S, n, sd) for sd in seeds]
    infos = _compare(B, S, rhs, [torch.zeros_like(b) for b in rhs], tol, max_iter)
    B.close()
    S.close()
    return infos


@pytest.mark.parametrize("precision", [smg.PREC_FP32, smg.PREC_FP64, smg.PREC_MIXED_BF16])
def test_batched_equals_single_solves(precision):
    infos = _check_against_single(24, 4, [11, 12, 13, 14], precision)
    assert all(i.status == 0 for i in infos)


def test_batched_problems_stop_at_their_own_iteration():
    # a zero right-hand side (done before the first iteration), a warm-started one and ordinary ones:
    # the problems stop at different iterations and each keeps its single-solve bits
    n = 32
    B = smg.Stokes(n, precision=smg.PREC_FP32, batch=4)
    S = smg.Stokes(n, precision=smg.PREC_FP32)
    rhs = [_rhs(S, n, 21), torch.zeros(S.n, dtype=torch.float64, device=DEV), _rhs(S, n, 22), _rhs(S, n, 23)]
    starts = [torch.zeros_like(b) for b in rhs]
    starts[3] = S.solve(rhs[3], tol=1e-4)[0]
    infos = _compare(B, S, rhs, starts, 1e-8, 200)
    its = [i.iterations for i in infos]
    assert all(i.status == 0 for i in infos) and its[1] == 0 and len(set(its)) > 2
    B.close()
    S.close()


def test_batched_not_converged_keeps_the_single_solve_bits():
    infos = _check_against_single(16, 3, [31, 32, 33], smg.PREC_FP32, tol=1e-30, max_iter=5)
    assert all(i.status == smg.ERR_NOT_CONVERGED and i.iterations == 5 for i in infos)


def test_batched_labelled_domain_and_variants():
    n = 24
    lab = synthetic.porous_labels(n, seed=3, nspheres=3, rmin=0.15, rmax=0.25, exterior_every=2)
    _check_against_single(n, 3, [41, 42, 43], smg.PREC_FP32, labels=lab)
    _check_against_single(n, 2, [44, 45], smg.PREC_FP32, kw=dict(kb_vanka=2, cycle=2))
    _check_against_single(n, 2, [46, 47], smg.PREC_FP32, kw=dict(additive=True))


def test_batched_non_cubic_grid():
    B = smg.Stokes(32, 16, 24, precision=smg.PREC_FP32, batch=3)
    S = smg.Stokes(32, 16, 24, precision=smg.PREC_FP32)
    g = torch.Generator().manual_seed(5)
    rhs = []
    for _ in range(3):
        v = torch.randn(S.n, generator=g, dtype=torch.float64).to(DEV)
        y = torch.zeros_like(v)
        smg.stokes_apply(S.h, v, y)  # a right-hand side with 0 off the unknowns
        rhs.append(y)
    _compare(B, S, rhs, [torch.zeros_like(b) for b in rhs], 1e-8, 200)
    B.close()
    S.close()


def test_single_problem_calls_refuse_a_batched_handle():
    B = smg.Stokes(16, precision=smg.PREC_FP32, batch=2)
    v = torch.zeros(B.n, dtype=torch.float64, device=DEV)
    with pytest.raises(smg.StokesError):
        smg.sqmr_solve(B.h, v, v.clone())
    with pytest.raises(smg.StokesError):
        smg.stokes_apply(B.h, v, v.clone())
    with pytest.raises(smg.StokesError):
        smg.mg_precondition(B.h, v, v.clone())
    B.close()
    with pytest.raises(smg.StokesError):
        smg.Stokes(16, precision=smg.PREC_FP32, batch=2, dwj=True)
