"""The transfer tiles (thread-block shape and z-planes per thread of the restriction and the
prolongation) are a schedule choice only: every tile, the autotuner's pick included, gives a V-cycle
bit-identical to the default tile.  Needs a GB300."""
import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu

smg = pytest.importorskip("paper_2312_10615_gb300")
DEV = torch.device("cuda:0")

TILES = [(32, 8, 8), (32, 8, 4), (32, 8, 2), (32, 8, 1), (32, 4, 1), (16, 8, 1), (8, 8, 1), (8, 4, 1), (64, 4, 3)]


@pytest.mark.parametrize("precision", [smg.PREC_FP32, smg.PREC_FP64, smg.PREC_MIXED_BF16])
def test_every_transfer_tile_gives_the_same_vcycle(precision):
    n = 64
    S0 = smg.Stokes(n, precision=precision, autotune=False)
    St = smg.Stokes(n, precision=precision, autotune=False)
    s = torch.from_numpy(np.random.default_rng(3).standard_normal(synthetic.packed_len(n))).to(DEV)
    ref = S0.precondition(s)
    for l in range(S0.levels - 1):
        assert smg.stokes_level_tiles(S0.h, l)[0] == (32, 8, 8)
    for rt in TILES:
        for pt in (rt, TILES[(TILES.index(rt) + 3) % len(TILES)]):
            for l in range(St.levels - 1):
                smg.stokes_set_level_tiles(St.h, l, rt, pt)
            assert torch.equal(St.precondition(s), ref), (rt, pt)
    S0.close()
    St.close()


def test_autotuned_tiles_bit_identical_and_reported():
    n = 64
    S0 = smg.Stokes(n, precision=smg.PREC_FP32, autotune=False)
    Sa = smg.Stokes(n, precision=smg.PREC_FP32, autotune=True)
    s = torch.from_numpy(np.random.default_rng(4).standard_normal(synthetic.packed_len(n))).to(DEV)
    assert torch.equal(Sa.precondition(s), S0.precondition(s))
    for l in range(Sa.levels - 1):
        rt, pt, ms = smg.stokes_level_tiles(Sa.h, l)
        assert rt in TILES and pt in TILES and ms[0] > 0 and ms[1] > 0
    with pytest.raises(smg.StokesError):
        smg.stokes_set_level_tiles(Sa.h, 0, (7, 3, 1), (32, 8, 1))
    S0.close()
    Sa.close()
