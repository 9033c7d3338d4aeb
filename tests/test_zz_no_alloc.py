"""The allocation-free residual norm entry point (for callers that cannot allocate device memory)
against the handle-based stokes_residual_norm, through the C ABI, on two calls in a row.

Collected last on purpose (file name), so a run that stops at the first failure has run every
other test first; it also passes alone in a fresh process."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

smg = pytest.importorskip("paper_2312_10615_gb300")


def _vec(n, seed, dev):
    return torch.from_numpy(np.random.default_rng(seed).standard_normal(n)).to(dev)


@pytest.mark.parametrize("dims,own_stream,h_arg", [((24, 16, 20), False, None), ((64, 64, 64), False, None),
                                                   ((24, 16, 20), True, 0.0)])
def test_noalloc_residual_norm_matches_handle_entry(dims, own_stream, h_arg):
    dev = torch.device("cuda:0")
    nx, ny, nz = dims
    S = smg.Stokes(nx, ny, nz)
    n = S.n
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    # h = 0 selects the documented default 1/nx; a caller-created stream orders the two kernels itself
    h = 1.0 / nx if h_arg is None else h_arg
    stream = torch.cuda.Stream(device=dev) if own_stream else None
    for call, seed in enumerate((1, 2)):  # two calls in a row share the library's scratch array
        b, x = _vec(n, 10 * seed, dev), _vec(n, 10 * seed + 1, dev)
        ref = smg.stokes_residual_norm(S.h, b, x)
        torch.cuda.synchronize()
        if stream is not None:
            smg.stokes_residual_norm_noalloc(nx, ny, nz, h, 1.0, b, x, out, stream=stream.cuda_stream)
            stream.synchronize()
        else:
            smg.stokes_residual_norm_noalloc(nx, ny, nz, h, 1.0, b, x, out)
            torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * ref, (call, got, ref)
    S.close()


def test_noalloc_rejects_bad_arguments():
    dev = torch.device("cuda:0")
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    # undersized vectors never reach the library: the binding checks the packed length first
    small = torch.zeros(10, dtype=torch.float64, device=dev)
    with pytest.raises(smg.StokesError) as e:
        smg.stokes_residual_norm_noalloc(4, 4, 4, 0.25, 1.0, small, small, out)
    assert e.value.code == smg.ERR_INVALID_ARG
    # grids needing more partial sums than the fixed scratch holds; vectors of the full length
    nx = 512
    n = 4 * nx ** 3 + 3 * nx ** 2
    big = torch.zeros(n, dtype=torch.float64, device=dev)
    with pytest.raises(smg.StokesError) as e:
        smg.stokes_residual_norm_noalloc(nx, nx, nx, 1.0 / nx, 1.0, big, big, out)
    assert e.value.code == smg.ERR_INVALID_ARG
    del big
    n4 = 4 * 4 ** 3 + 3 * 4 ** 2
    b4 = torch.zeros(n4, dtype=torch.float64, device=dev)
    # non-finite cell size or viscosity, and host pointers
    for h, eta in ((float("inf"), 1.0), (0.25, float("inf")), (0.25, float("nan")), (0.25, 0.0)):
        with pytest.raises(smg.StokesError) as e:
            smg.stokes_residual_norm_noalloc(4, 4, 4, h, eta, b4, b4, out)
        assert e.value.code == smg.ERR_INVALID_ARG
    host = np.zeros(n4)
    with pytest.raises(smg.StokesError) as e:
        smg.stokes_residual_norm_noalloc(4, 4, 4, 0.25, 1.0, host, host, out)
    assert e.value.code == smg.ERR_INVALID_ARG
