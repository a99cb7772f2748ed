"""The stacked-B issue schedule of the digit-plane MMAs (host logic, no GPU):
every digit product of a k step is computed exactly once, into the right
level accumulator, with shapes tcgen05.mma accepts."""
import pytest

EXACT = 3                       # levels kept exact per chunk
TILE_N = {3: 64, 4: 64, 5: 48, 6: 32}


@pytest.fixture(scope="module")
def pkg():
    from paper_2312_07008_gb300 import build as b
    b.build()
    import paper_2312_07008_gb300 as p
    return p


@pytest.mark.parametrize("ks,count", [(3, 3), (4, 7), (5, 8), (6, 9)])
def test_every_product_once_in_its_level(pkg, ks, count):
    sched = pkg.binding.dsrg_fno_debug_mma_schedule(ks)
    assert len(sched) == count
    seen = []
    for a, b0, nb, level, ncols in sched:
        assert 0 <= a < ks and nb >= 1 and level == a + b0
        levels = range(level, level + nb)
        # one accumulator set per MMA: all exact or all tail levels
        assert all(L < EXACT for L in levels) or all(L >= EXACT for L in levels)
        assert level + nb - 1 <= ks - 1
        # tcgen05.mma kind::f16, M = 128: N a multiple of 16 in [16, 256]
        assert ncols == nb * TILE_N[ks] and ncols % 16 == 0 and 16 <= ncols <= 256
        seen += [(a, b0 + t) for t in range(nb)]
    want = [(a, b) for a in range(ks) for b in range(ks) if a + b <= ks - 1]
    assert sorted(seen) == sorted(want)
    assert len(seen) == len(set(seen)) == ks * (ks + 1) // 2


@pytest.mark.parametrize("ks", [3, 4, 5, 6])
def test_first_mma_of_each_set_starts_every_level(pkg, ks):
    """The accumulate flag is 0 only for the A-plane-0 MMA of a set, so that
    MMA must come first among the set's MMAs and write every level of it."""
    sched = pkg.binding.dsrg_fno_debug_mma_schedule(ks)
    for tail in (False, True):
        mine = [m for m in sched if (m[3] >= EXACT) == tail]
        if not mine:
            assert tail and ks <= EXACT
            continue
        a, b0, nb, level, _ = mine[0]
        assert a == 0
        top = min(ks, EXACT)
        assert (level, nb) == ((EXACT, ks - EXACT) if tail else (0, top))


def test_fewer_mma_issues_and_a_plane_reads(pkg):
    """Per k step: MMAs issued (= A-plane reads from shared memory) against
    one MMA per digit product; B rows read stay the same."""
    for ks in (3, 4, 5, 6):
        sched = pkg.binding.dsrg_fno_debug_mma_schedule(ks)
        products = ks * (ks + 1) // 2
        assert len(sched) < products
        assert sum(m[2] for m in sched) == products


def test_bad_arguments(pkg):
    with pytest.raises(pkg.DsrgFnoError):
        pkg.binding.dsrg_fno_debug_mma_schedule(7)
