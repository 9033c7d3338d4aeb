"""Failure detection without a GPU fault: the bounded grid-barrier wait of the persistent Vanka
schedule runs out when the barrier waits for blocks the launch does not have, the call returns
STOKES_ERR_TIMEOUT, and the context stays usable.  Needs a GB300."""
import time

import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu

smg = pytest.importorskip("paper_2312_10615_gb300")


@pytest.mark.parametrize("precision", [smg.PREC_FP32, smg.PREC_FP64])
def test_grid_barrier_wait_runs_out_and_reports_timeout(precision):
    n = 32
    S = smg.Stokes(n, precision=precision, autotune=False)
    t0 = time.time()
    rc = smg.stokes_test_grid_barrier(S.h, 0, 1, 4096)
    assert rc == smg.ERR_TIMEOUT, smg.stokes_strerror(rc)
    assert time.time() - t0 < 30.0
    # the same sweep with the barrier waiting for the launch's own blocks completes
    assert smg.stokes_test_grid_barrier(S.h, 0, 0, 1 << 22) == smg.OK
    # the context and the handle stay usable: a solve afterwards converges
    prob = synthetic.bumps(n, seed=1, device="cuda")
    b = S.rhs(prob["f"], None)
    x, info = S.solve(b, tol=1e-8)
    assert info.status == smg.OK and info.rel_residual < 1e-8
    torch.cuda.synchronize()
    S.close()


def test_grid_barrier_arguments():
    S = smg.Stokes(16, autotune=False)
    for args in ((S.levels - 1, 1, 100), (0, -1, 100), (0, 1, 0), (0, 1, (1 << 22) + 1)):
        assert smg.stokes_test_grid_barrier(S.h, *args) == smg.ERR_INVALID_ARG
    S.close()
