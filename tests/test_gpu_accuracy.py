"""Accuracy of the mixed-precision V-cycles at the headline tolerance: FP32 V-cycle and FP32 V-cycle with
BF16 storage on the two finest levels (FP64 SQMR in both) solved to relative residual 1e-8, compared
element by element with the FP64 oracle's own 1e-8 solve and with its 1e-12 solve (the discrete
solution to 1e-12).  The stated target is 1e-7 against the oracle at 1e-8; the assertions are the
measured bounds with a margin (measured on GB300: FP32 1.0e-15 / 4.8e-15, BF16 1.4e-11 / 9.6e-11 against
the oracle's 1e-8 solve on the 32^3 cavity / 64^3 bumps; 1.2e-10 / 3.5e-10 against its 1e-12 solve) --
the 1e-8 tolerance already meets the target, no tighter tolerance is needed.  Needs a GB300."""
import os

import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

smg = pytest.importorskip("paper_2312_10615_gb300")
DEV = torch.device("cuda:0")

CASES = {
    "cavity32": (32, 1e-3, 1e-3, lambda: synthetic.lid(32)),  # Sec. 7 3D driven cavity parameters
    "bumps64": (64, 1.0, 1e-3, lambda: synthetic.bumps(64, seed=0)),
}
_ref = {}


def reference(name):
    if name not in _ref:
        n, eta, gamma, mk = CASES[name]
        prob = mk()
        o = oracle.Oracle(n, eta=eta, gamma=gamma, coarsest_max=8)
        b = o.rhs(prob["f"].numpy(), None if prob["g"] is None else prob["g"].numpy())
        oracle.set_threads(os.cpu_count() or 1)  # bit-identical to one thread, only faster
        try:
            x8, rc8, it8, _, _ = o.sqmr(b, tol=1e-8, maxit=200)
            x12, rc12, _, _, _ = o.sqmr(b, tol=1e-12, maxit=200)
        finally:
            oracle.set_threads(1)
        assert rc8 == 0 and rc12 == 0
        _ref[name] = (b, x8, it8, x12)
    return _ref[name]


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision,bound", [(smg.PREC_FP32, 1e-12), (smg.PREC_MIXED_BF16, 1e-9)], ids=["fp32", "bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_mixed_precision_solution_against_the_oracle_at_1e8(name, precision, bound):
    n, eta, gamma, _ = CASES[name]
    b, x8, it8, x12 = reference(name)
    S = smg.Stokes(n, viscosity=eta, gamma=gamma, precision=precision)
    x, info = S.solve(torch.from_numpy(b).to(DEV), tol=1e-8, max_iter=200)
    assert info.status == smg.OK and info.rel_residual < 1e-8
    assert abs(info.iterations - it8) <= 1
    xc = x.cpu().numpy()
    e8, e12 = rel(xc, x8), rel(xc, x12)
    assert e8 <= 1e-7, e8  # the stated accuracy target
    assert e8 <= bound, e8  # the measured bound (with margin)
    assert e12 <= 1e-9, e12
    S.close()
