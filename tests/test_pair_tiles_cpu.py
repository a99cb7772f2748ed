"""Host logic of the pair contraction's output tiles (no GPU): the tiles of a
batch of hole pairs cover every element the pass needs exactly once, list no
tile without a needed element, and follow the banded order."""
import numpy as np
import pytest

import paper_2312_07008_gb300 as pkg

BM = 128


def needed_mask(nc, na, nv, pairs, energy_only):
    nh, np_ = nc + na, na + nv
    need = np.zeros((nh * np_, nh * np_), dtype=bool)
    for i, j in pairs:
        blk = np.ones((np_, np_), dtype=bool)
        blk[:na, :na] = False
        if energy_only:
            blk[:na, :] = False
            blk[:, :na] = False
        need[i * np_:(i + 1) * np_, j * np_:(j + 1) * np_] |= blk
    return need


@pytest.mark.parametrize("ks,bn", [(5, 48), (3, 64), (4, 64)])
@pytest.mark.parametrize("nc,na,nv", [(3, 0, 40), (4, 2, 61), (2, 5, 130), (5, 3, 7)])
@pytest.mark.parametrize("energy_only", [False, True])
def test_tiles_cover_each_needed_element_once(ks, bn, nc, na, nv, energy_only):
    nh, np_ = nc + na, na + nv
    rng = np.random.default_rng(nc * 100 + na * 10 + nv)
    allp = [(i, j) for i in range(nh) for j in range(i, nh)]
    pick = rng.choice(len(allp), size=max(1, len(allp) // 2), replace=False)
    pairs = [allp[k] for k in sorted(pick)]
    tiles = pkg.dsrg_fno_debug_pair_tiles(ks, nc, na, nv, pairs, energy_only)
    assert len(set(tiles)) == len(tiles)
    need = needed_mask(nc, na, nv, pairs, energy_only)
    cover = np.zeros_like(need, dtype=np.int32)
    R = nh * np_
    for mt, nt in tiles:
        assert 0 <= mt * BM < R and 0 <= nt * bn < R
        sub = need[mt * BM:(mt + 1) * BM, nt * bn:(nt + 1) * bn]
        assert sub.any(), (mt, nt)            # no tile without a needed element
        cover[mt * BM:(mt + 1) * BM, nt * bn:(nt + 1) * bn] += 1
    assert np.all(cover[need] == 1)
    # banded order: row tiles in bands of 8, column tiles ascending inside a band
    band = [mt // 8 for mt, _ in tiles]
    assert band == sorted(band)
    for b in set(band):
        cols = [nt for (mt, nt) in tiles if mt // 8 == b]
        assert cols == sorted(cols)


def test_tiles_of_a_whole_workload_waste_little():
    """nvir 1200, CAS(10,10), 60 core: the listed tiles hold the needed
    elements of all pairs with under 2 % padding (per-pair tiling: 10 %)."""
    nc, na, nv = 60, 10, 1200
    nh, np_ = nc + na, na + nv
    pairs = [(i, j) for i in range(nh) for j in range(i, nh)]
    tiles = pkg.dsrg_fno_debug_pair_tiles(5, nc, na, nv, pairs, False)
    needed = len(pairs) * (np_ * np_ - na * na)
    assert len(tiles) * 128 * 48 <= 1.02 * needed
