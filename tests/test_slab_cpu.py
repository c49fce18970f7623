"""Host logic of the slab decomposition (paper_2510_04197_gb300.slab): band
heights, neighbour ranks and the boundary kinds of each band."""
import pytest

from paper_2510_04197_gb300 import dvbm as D
from paper_2510_04197_gb300 import slab


@pytest.mark.parametrize("Ny,parts", [(64, 2), (64, 3), (100, 3), (4096, 8), (24, 3), (17, 4), (8, 2)])
def test_split_rows(Ny, parts):
    h = slab.split_rows(Ny, parts)
    assert len(h) == parts and sum(h) == Ny and min(h) >= 4
    if Ny % (8 * parts) == 0:  # tile-aligned bands when the rows allow it
        assert all(v % 8 == 0 for v in h)


def test_split_rows_refuses_too_few_rows():
    with pytest.raises(ValueError):
        slab.split_rows(7, 2)


def test_neighbours_ring_and_chain():
    assert [slab.neighbours(r, 1, True) for r in range(1)] == [(0, 0)]
    assert [slab.neighbours(r, 2, True) for r in range(2)] == [(1, 1), (0, 0)]
    assert [slab.neighbours(r, 3, True) for r in range(3)] == [(2, 1), (0, 2), (1, 0)]
    assert [slab.neighbours(r, 3, False) for r in range(3)] == [(None, 1), (0, 2), (1, None)]
    # every send has a matching receive: band r's upper is band u iff u's lower is r
    for world in (2, 3, 5):
        for periodic in (True, False):
            for r in range(world):
                lo, up = slab.neighbours(r, world, periodic)
                if up is not None:
                    assert slab.neighbours(up, world, periodic)[0] == r


def test_band_boundaries():
    walls = [D.ZEROGRAD, D.ZEROGRAD, (D.WALL, (0.0, 0.0), 1.0), (D.WALL, (0.5, 0.0), 1.2)]
    assert slab.band_bcs(None, 0, 2) == ([0, 0, D.EXTERNAL, D.EXTERNAL], True)
    assert slab.band_bcs(walls, 0, 3) == ([1, 1, walls[2], D.EXTERNAL], False)
    assert slab.band_bcs(walls, 1, 3) == ([1, 1, D.EXTERNAL, D.EXTERNAL], False)
    assert slab.band_bcs(walls, 2, 3) == ([1, 1, D.EXTERNAL, walls[3]], False)
    assert slab.band_bcs(walls, 0, 1) == ([1, 1, walls[2], walls[3]], False)
