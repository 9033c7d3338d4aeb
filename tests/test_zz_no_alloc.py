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


@pytest.mark.parametrize("dims", [(24, 16, 20), (64, 64, 64)])
def test_noalloc_residual_norm_matches_handle_entry(dims):
    dev = torch.device("cuda:0")
    nx, ny, nz = dims
    S = smg.Stokes(nx, ny, nz)
    n = S.n
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    for call, seed in enumerate((1, 2)):  # two calls in a row share the library's scratch array
        b, x = _vec(n, 10 * seed, dev), _vec(n, 10 * seed + 1, dev)
        ref = smg.stokes_residual_norm(S.h, b, x)
        smg.stokes_residual_norm_noalloc(nx, ny, nz, 1.0 / nx, 1.0, b, x, out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * ref, (call, got, ref)
    S.close()


def test_noalloc_rejects_oversized_grid_and_host_pointers():
    dev = torch.device("cuda:0")
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    small = torch.zeros(10, dtype=torch.float64, device=dev)
    with pytest.raises(smg.StokesError) as e:
        smg.stokes_residual_norm_noalloc(512, 512, 512, 1.0 / 512, 1.0, small, small, out)  # > 16384 partials
    assert e.value.code == smg.ERR_INVALID_ARG
    host = np.zeros(10)
    with pytest.raises(smg.StokesError):
        smg.stokes_residual_norm_noalloc(4, 4, 4, 0.25, 1.0, host, host, out)
