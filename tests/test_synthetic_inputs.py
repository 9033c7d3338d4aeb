"""The seeded input generators hold no solver arithmetic; these checks make sure the inputs have the
structure the tests and the bench rely on (runs without a GPU)."""
import numpy as np
import pytest
from scipy import ndimage

import synthetic


@pytest.mark.parametrize("exterior_every", [0, 2])
def test_porous_labels_shape_shell_and_connectivity(exterior_every):
    n = 24
    lab = synthetic.porous_labels(n, seed=3, nspheres=10, rmin=0.1, rmax=0.2, exterior_every=exterior_every)
    assert lab.shape == (n + 2, n + 2, n + 2) and lab.dtype == np.uint8
    shell = np.ones_like(lab, bool)
    shell[1:-1, 1:-1, 1:-1] = False
    assert np.all(lab[shell] == 1)  # the ghost shell is Dirichlet
    inner = lab[1:-1, 1:-1, 1:-1]
    assert (inner == 0).any() and (inner != 0).any()
    assert set(np.unique(lab)) <= ({0, 1, 2} if exterior_every else {0, 1})
    # every interior cell belongs to one 6-connected region (no pocket adds a pressure null vector)
    _, ncomp = ndimage.label(lab == 0)
    assert ncomp == 1
    # the same seed gives the same labels
    assert np.array_equal(lab, synthetic.porous_labels(n, seed=3, nspheres=10, rmin=0.1, rmax=0.2,
                                                       exterior_every=exterior_every))


def test_cylinder_labels_block_the_channel_partly():
    lab = synthetic.cylinder_labels(48, 24, 16, radius=0.2)
    inner = lab[1:-1, 1:-1, 1:-1]
    assert inner.shape == (16, 24, 48)
    blocked = inner[0] != 0  # one z-plane (the cylinder is z-aligned)
    assert all(np.array_equal(blocked, inner[k] != 0) for k in range(16))
    assert 0 < blocked.mean() < 0.2


@pytest.mark.parametrize("with_labels", [False, True])
def test_plug_flow_balances_the_flux(with_labels):
    nx, ny, nz = 20, 12, 10
    lab = synthetic.porous_labels(nx, ny, nz, seed=1, nspheres=6, rmin=0.2, rmax=0.3) if with_labels else None
    g = synthetic.plug_flow(nx, ny, nz, labels=lab).numpy()
    assert g.size == synthetic.ghost_len(nx, ny, nz)
    u = g[:(nz + 2) * (ny + 2) * (nx + 1)].reshape(nz + 2, ny + 2, nx + 1)
    rest = g[(nz + 2) * (ny + 2) * (nx + 1):]
    assert not rest.any()  # v and w carry no data
    inflow, outflow = u[1:-1, 1:-1, 0], u[1:-1, 1:-1, nx]
    assert inflow.sum() == pytest.approx(outflow.sum(), rel=1e-14)
    assert not u[:, :, 1:nx].any()  # nothing on inner faces
    if with_labels:
        # no flow into or out of a non-interior cell next to the inflow / outflow sides
        assert not inflow[lab[1:-1, 1:-1, 1] != 0].any()
        assert not outflow[lab[1:-1, 1:-1, nx] != 0].any()


def test_bumps_are_seeded_and_velocity_only():
    a = synthetic.bumps(12, seed=5)["f"].numpy()
    b = synthetic.bumps(12, seed=5)["f"].numpy()
    c = synthetic.bumps(12, seed=6)["f"].numpy()
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.size == synthetic.packed_len(12)
    assert not a[-12 ** 3:].any()  # zero continuity source
