"""Host logic of the forest entry points (no GPU): the neighbour links the
library builds agree with a brute-force search over the finest-level cells,
and invalid forests are refused before any device call."""
import numpy as np
import pytest

import paper_2210_06438_gb300 as hydro
import synth
from paper_2210_06438_gb300 import _build


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return hydro.load()


def _owner(lv, nb0):
    lmax = int(lv[:, 0].max())
    M = nb0 << lmax
    own = np.full((M, M, M), -1, dtype=np.int64)
    for s, (L, bx, by, bz) in enumerate(lv):
        w = 1 << (lmax - int(L))
        own[bz * w:(bz + 1) * w, by * w:(by + 1) * w, bx * w:(bx + 1) * w] = s
    return own, lmax, M


@pytest.mark.parametrize("nb0,seed,prob", [(2, 7, 0.25), (1, 3, 0.6), (3, 5, 0.15)])
def test_links_match_brute_force(lib, nb0, seed, prob):
    lv = synth.forest_leaves(nb0, 2, synth.random_refine(seed, prob), seed=seed)
    kind, nbr = hydro.forest_links(lv, nb0, 8)
    own, lmax, M = _owner(lv, nb0)
    assert (own >= 0).all()
    seen = {-1: 0, 0: 0, 1: 0}
    for s, (L, bx, by, bz) in enumerate(lv):
        w = 1 << (lmax - int(L))
        lo = [bx * w, by * w, bz * w]
        for face in range(6):
            d, side = face >> 1, face & 1
            c = list(lo)
            c[d] = (lo[d] - 1) % M if side == 0 else (lo[d] + w) % M
            t = own[c[2], c[1], c[0]]
            assert kind[s][face] == int(lv[t, 0]) - int(L), (s, face)
            assert nbr[s][face] == t, (s, face)
            seen[kind[s][face]] += 1
    if nb0 != 1:
        assert min(seen.values()) > 0, seen


def _leaves_uniform(nb0, L=0):
    m = nb0 << L
    return np.array([(L, x, y, z) for z in range(m) for y in range(m) for x in range(m)], dtype=np.int32)


def test_one_level_links_are_periodic_neighbours(lib):
    lv = _leaves_uniform(3)
    kind, nbr = hydro.forest_links(lv, 3, 8)
    for s, (_, x, y, z) in enumerate(lv):
        assert kind[s] == [0] * 6
        want = [((x - 1) % 3, y, z), ((x + 1) % 3, y, z), (x, (y - 1) % 3, z), (x, (y + 1) % 3, z),
                (x, y, (z - 1) % 3), (x, y, (z + 1) % 3)]
        assert [tuple(lv[t, 1:]) for t in nbr[s]] == want


def _bad(lv, nb0=2, N=8):
    with pytest.raises(hydro.HydroError) as ei:
        hydro.forest_links(lv, nb0, N)
    assert ei.value.code == hydro.HYDRO_EINVAL


def test_invalid_forests_refused(lib):
    good = _leaves_uniform(2)
    hydro.forest_links(good, 2, 8)
    _bad(good[:-1])                                     # a gap
    _bad(np.concatenate([good, good[:1]]))              # a duplicate
    ch = np.array([(1, 0, 0, 0)], dtype=np.int32)
    _bad(np.concatenate([good, ch]))                    # overlap: a child of a leaf
    _bad(np.concatenate([good[:-1], [(0, 2, 1, 1)]]))   # coordinate out of range
    _bad(np.concatenate([good[:-1], [(-1, 1, 1, 1)]]))  # negative level
    _bad(good, N=7)                                     # odd N
    _bad(good, N=4)                                     # a 3-cell slab would span two finer leaves
    _bad(good, N=258)
    _bad(good, nb0=0)
    # level 2 next to level 0 (periodic wrap): not 2:1 balanced
    lv = [tuple(r) for r in good if tuple(r[1:]) != (0, 0, 0)]
    lv += [(1, i, j, k) for k in (0, 1) for j in (0, 1) for i in (0, 1) if (i, j, k) != (0, 0, 0)]
    lv += [(2, i, j, k) for k in (0, 1) for j in (0, 1) for i in (0, 1)]
    _bad(np.array(lv, dtype=np.int32))
    # deepest level allowed, and one beyond it
    deep = _leaves_uniform(1, 0)
    deep[0, 0] = hydro.FOREST_MAX_LEVEL + 1
    _bad(deep, nb0=1)


def test_create_checks_fields_before_the_device(lib):
    with pytest.raises(hydro.HydroError) as ei:
        hydro.Forest(_leaves_uniform(2), 2, 8, 5)
    assert ei.value.code == hydro.HYDRO_EINVAL
    with pytest.raises(hydro.HydroError) as ei:
        hydro.Forest(_leaves_uniform(2)[:-1], 2, 8, 6)
    assert ei.value.code == hydro.HYDRO_EINVAL
