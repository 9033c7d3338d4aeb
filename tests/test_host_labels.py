"""The library's host-side classification of labelled domains (Sec. 5) against the oracle, without a
GPU: per level, the unknowns, the Vanka set V1 and, for every face next to exterior cells, the viscous
terms its row drops (the do-nothing outflow reading) -- the flags every labelled kernel reads."""
import numpy as np
import pytest

import oracle
import synthetic

smg = pytest.importorskip("paper_2312_10615_gb300")

DOMAINS = {
    "porous16": ((16, 16, 16), lambda: synthetic.porous_labels(16, seed=0, nspheres=6, rmin=0.1, rmax=0.2)),
    "mixed16": ((16, 16, 16), lambda: synthetic.porous_labels(16, seed=1, nspheres=6, rmin=0.1, rmax=0.2,
                                                                exterior_every=2)),
    "outlet32x16x16": ((32, 16, 16), lambda: synthetic.channel_labels(32, 16, 16, outlet=4, cylinder=(8.0, 8.0, 2.5))),
}


@pytest.mark.parametrize("name", list(DOMAINS))
def test_host_flags_match_the_oracle_classification(name):
    (nx, ny, nz), mk = DOMAINS[name]
    lab = mk()
    o = oracle.Oracle(nx, ny, nz, coarsest_max=4, labels=lab)
    for level in range(o.nlevels):
        f = smg.stokes_label_flags(lab, nx, ny, nz, level=level)
        act, v1 = o.masks(level)
        assert np.array_equal((f & 1).astype(bool), act), (name, level)
        assert np.array_equal(((f & 1) != 0) & ((f & 2) == 0), v1), (name, level)


@pytest.mark.parametrize("name", ["mixed16", "outlet32x16x16"])
def test_host_drop_counts_match_the_oracle_operator(name):
    # the diagonal of a face row is (6 - dropped terms) eta/h^2, and a dropped normal neighbour has no
    # coupling, in the oracle's operator (entries read off L applied to unit vectors)
    (nx, ny, nz), mk = DOMAINS[name]
    lab = mk()
    o = oracle.Oracle(nx, ny, nz, h=1.0, eta=1.0, coarsest_max=4, labels=lab)  # small coarsest LU
    f = smg.stokes_label_flags(lab, nx, ny, nz, level=0)
    act = o.masks()[0]
    npc = nx * ny * nz
    faces = np.nonzero(act[:-npc] & ((f[:-npc] >> 3) != 0))[0]
    assert faces.size > 0
    sizes = [(nx + 1) * ny * nz, nx * (ny + 1) * nz, nx * ny * (nz + 1)]
    offs = np.cumsum([0] + sizes)
    strides = [[1, nx + 1, (nx + 1) * ny], [1, nx, nx * (ny + 1)], [1, nx, nx * ny]]
    rng = np.random.default_rng(0)
    sample = np.concatenate([faces, rng.choice(np.nonzero(act[:-npc])[0], 50, replace=False)])
    for q in sample:
        e = np.zeros(o.n())
        e[q] = 1.0
        col = o.apply(e)
        m = (int(f[q]) >> 3) & 7
        assert col[q] == pytest.approx(6.0 - m, abs=1e-12), q
        c = int(np.searchsorted(offs, q, side="right") - 1)
        sn = strides[c][c]
        for bit, nb in ((64, q - sn), (128, q + sn)):
            if offs[c] <= nb < offs[c + 1] and act[nb]:
                assert col[nb] == pytest.approx(0.0 if f[q] & bit else -1.0, abs=1e-12), (q, bit)
