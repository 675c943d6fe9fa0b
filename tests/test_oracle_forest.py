"""Pins of the forest oracle (multi-level ghost cells and flux correction)
against facts that do not depend on it: a one-level forest is the periodic
domain of Sec. V-A's ghost exchange, constants stay exact, linear data gives
closed-form ghost values, the corrected RHS conserves every field to
rounding (Sec. III: conservation to machine precision), and a mirrored
forest gives the mirrored result.  Also the generator's invariants
(exact cover, 2:1 face balance) checked by brute force."""
import numpy as np
import pytest

import oracle
import synth
from oracle import forest as of

NB0, N = 2, 8


def _forest(seed=7, prob=0.25, max_level=2, nb0=NB0):
    return synth.forest_leaves(nb0, max_level, synth.random_refine(seed, prob), seed=seed)


def _boxes(leaves, nb0, lmax):
    """Leaf boxes in units of level-lmax blocks: [n][3] lo and the width."""
    lv = leaves[:, 0].astype(np.int64)
    w = np.left_shift(1, lmax - lv)
    return leaves[:, 1:].astype(np.int64) * w[:, None], w


def test_generator_exact_cover_and_balance():
    for seed, prob in ((7, 0.25), (11, 0.4), (5, 0.1)):
        lv = _forest(seed, prob)
        assert len({tuple(l) for l in lv}) == len(lv)
        lmax = int(lv[:, 0].max())
        lo, w = _boxes(lv, NB0, lmax)
        M = NB0 << lmax
        # exact cover: volumes add up and no two boxes overlap
        assert int((w ** 3).sum()) == M ** 3
        occ = np.zeros((M, M, M), dtype=np.int32)
        for (x, y, z), ww in zip(lo, w):
            occ[z:z + ww, y:y + ww, x:x + ww] += 1
        assert np.all(occ == 1)
        # 2:1 across every shared face, periodic, by brute force over pairs
        owner = np.zeros((M, M, M), dtype=np.int64)
        for s, ((x, y, z), ww) in enumerate(zip(lo, w)):
            owner[z:z + ww, y:y + ww, x:x + ww] = s
        for ax in range(3):
            a = owner
            b = np.roll(owner, -1, axis=2 - ax)
            diff = np.abs(lv[a, 0] - lv[b, 0])
            assert diff.max() <= 1


def test_one_level_forest_is_the_periodic_domain():
    """All leaves at level 0: ghost values are plain periodic copies, so the
    result equals the single-block oracle on gather_blocks of the global
    array, bit for bit (leaves given in shuffled order)."""
    nb0 = 3
    lv = synth.forest_leaves(nb0, 0, lambda *a: False, seed=4)
    assert np.all(lv[:, 0] == 0) and len(lv) == 27
    glob = synth.plain_domain(seed=9, n=nb0 * N, nf=7)
    blocks = synth.gather_blocks(glob, N, blocks=[tuple(l[1:]) for l in lv])
    U = [b[:, 3:-3, 3:-3, 3:-3] for b in blocks]
    dx0 = 1.0 / (nb0 * N)
    for mode in (0, oracle.MODE_MIXED, oracle.FLUX_KNP):
        got, gam = of.rhs(lv, nb0, U, dx0, mode=mode)
        for s in range(len(lv)):
            ref, ra, fl = oracle.rhs_block(blocks[s], 3, 5.0 / 3.0, dx0, mode)
            assert np.array_equal(got[s], ref)
            assert gam[s] == ra


def test_uniform_state_is_exact_zero():
    lv = _forest(4, 0.25)
    assert len(set(lv[:, 0])) == 3
    n = len(lv)
    shp = (n, N, N, N)
    X = np.full((3,) + shp, 1.0 / 3.0)
    Uc = synth.conserved_from_states(np.full(shp, 1.3), np.full(shp, 0.2), np.full(shp, -0.1),
                                     np.full(shp, 0.05), np.full(shp, 0.9), X)
    U = list(np.moveaxis(Uc, 0, 1))
    got, gam = of.rhs(lv, NB0, U, 1.0 / 16)
    for o in got:
        assert np.all(o == 0.0)
    c = np.sqrt(5.0 / 3.0 * 0.9 / 1.3)
    assert np.all(gam == pytest.approx(0.2 + c, rel=1e-15))


def _contains(lv, nb0, x):
    """Index of the leaf whose box contains point x (unit cube), brute force."""
    for s, (L, bx, by, bz) in enumerate(lv):
        w = 1.0 / (nb0 << int(L))
        if all(b * w <= xi < (b + 1) * w for b, xi in zip((bx, by, bz), x)):
            return s
    raise AssertionError("point not covered")


def test_linear_field_ghost_values():
    """Ghosts of a field linear in space (periodic coordinates wrapped into
    the cube): a same-level or coarser source gives the field at the centre
    of the source cell; finer sources give their mean, which is the field at
    the ghost cell's own centre."""
    lv = _forest(4, 0.25)
    nb0 = NB0
    coef = np.array([0.7, -1.3, 2.1])
    xyz = synth.forest_cell_centres(lv, nb0, N)
    U = [np.stack([1.0 + np.tensordot(coef, xyz[s], axes=1)] * 6) for s in range(len(lv))]
    fo = of.Forest(lv, nb0, N)
    checked = {"same": 0, "coarse": 0, "fine": 0}
    for s in range(0, len(lv), 3):
        L, b = int(lv[s, 0]), lv[s, 1:]
        gb = of.ghosted_block(fo, U, s)
        w = 1.0 / ((nb0 << L) * N)
        for d in range(3):
            for side in (0, 1):
                for depth in (1, 2, 3):
                    cd = -depth if side == 0 else N - 1 + depth
                    for ja in range(0, N, 3):
                        for jb in range(0, N, 5):
                            c = [0, 0, 0]
                            ta, tb = ((1, 2), (0, 2), (0, 1))[d]
                            c[d], c[ta], c[tb] = cd, ja, jb
                            centre = [((b[e] * N + c[e] + 0.5) * w) % 1.0 for e in range(3)]
                            src = _contains(lv, nb0, centre)
                            Ls = int(lv[src, 0])
                            if Ls <= L:
                                ws = 1.0 / ((nb0 << Ls) * N)
                                at = [(np.floor(x / ws) + 0.5) * ws for x in centre]
                                checked["same" if Ls == L else "coarse"] += 1
                            else:
                                at = centre
                                checked["fine"] += 1
                            want = 1.0 + coef @ np.array(at)
                            got = gb[0, c[2] + 3, c[1] + 3, c[0] + 3]
                            assert got == pytest.approx(want, rel=0, abs=1e-14)
    assert min(checked.values()) > 50, checked


@pytest.mark.parametrize("mode", [0, oracle.MODE_MIXED, oracle.FLUX_KNP])
def test_conservation_to_rounding_and_correction_is_needed(mode):
    lv = _forest(7, 0.25)
    U, dx0 = synth.smooth_forest_state(lv, NB0, N, nf=8, seed=21)
    got, _ = of.rhs(lv, NB0, list(U), dx0, mode=mode)
    vol = (dx0 / (1 << lv[:, 0].astype(np.int64))) ** 3
    tot = sum(got[s].sum(axis=(1, 2, 3)) * vol[s] for s in range(len(lv)))
    mag = sum(np.abs(got[s]).sum(axis=(1, 2, 3)) * vol[s] for s in range(len(lv)))
    assert np.all(np.abs(tot) <= 1e-14 * mag)
    # without the correction the levels exchange different fluxes
    fo = of.Forest(lv, NB0, N)
    raw = sum(oracle.rhs_block(of.ghosted_block(fo, list(U), s), 3, 5.0 / 3.0, dx0 / (1 << int(lv[s, 0])),
                               mode)[0].sum(axis=(1, 2, 3)) * vol[s] for s in range(len(lv)))
    assert np.all(np.abs(raw[:5]) > 1e3 * np.abs(tot[:5]) + 1e-12 * mag[:5])


def test_mirror_symmetry():
    """x -> 1 - x: leaves and cells mirrored, s_x negated; dU/dt mirrors
    with the s_x rate negated (normwise 1e-13: rounding order differs)."""
    lv = _forest(7, 0.25)
    U, dx0 = synth.smooth_forest_state(lv, NB0, N, nf=6, seed=22)
    got, gam = of.rhs(lv, NB0, list(U), dx0)
    mv = lv.copy()
    mv[:, 1] = (NB0 << lv[:, 0]) - 1 - lv[:, 1]
    MU = U[:, :, :, :, ::-1].copy()
    MU[:, 1] *= -1
    mg, mgam = of.rhs(mv, NB0, list(MU), dx0)
    for s in range(len(lv)):
        back = mg[s][:, :, :, ::-1].copy()
        back[1] *= -1
        scale = np.abs(got[s]).max(axis=(1, 2, 3), keepdims=True)
        assert np.all(np.abs(back - got[s]) <= 1e-13 * scale)
    assert np.allclose(mgam, gam, rtol=1e-14, atol=0)


def test_unbalanced_forest_is_refused():
    # a level-2 block next to level-0 blocks
    lv = [(0, 1, 0, 0), (0, 0, 1, 0), (0, 1, 1, 0), (0, 0, 0, 1), (0, 1, 0, 1), (0, 0, 1, 1), (0, 1, 1, 1)]
    lv += [(1, i, j, k) for k in (0, 1) for j in (0, 1) for i in (0, 1) if (i, j, k) != (0, 0, 0)]
    lv += [(2, i, j, k) for k in (0, 1) for j in (0, 1) for i in (0, 1)]
    lv = np.array(lv, dtype=np.int32)
    U, dx0 = synth.smooth_forest_state(lv, 2, N, nf=6)
    with pytest.raises(ValueError, match="2:1"):
        of.rhs(lv, 2, list(U), dx0)


# ----------------------------------------------------- 26-point variant --
def _full_forest():
    """Three levels, 2:1 balanced across faces, edges and corners (the
    26-point variant reads edge and corner ghosts): 90 leaves."""
    lv = synth.forest_leaves(3, 2, synth.random_refine(1, 0.1), seed=1, balance="full")
    assert np.bincount(lv[:, 0]).tolist() == [19, 63, 8]
    return lv


def test_quad26_one_level_forest_is_the_periodic_domain():
    nb0 = 2
    lv = synth.forest_leaves(nb0, 0, lambda *a: False, seed=5)
    glob = synth.plain_domain(seed=19, n=nb0 * N, nf=6)
    blocks = synth.gather_blocks(glob, N, blocks=[tuple(l[1:]) for l in lv])
    U = [b[:, 3:-3, 3:-3, 3:-3] for b in blocks]
    dx0 = 1.0 / (nb0 * N)
    got, gam = of.rhs(lv, nb0, U, dx0, mode=oracle.QUAD26)
    for s in range(len(lv)):
        ref, ra, _ = oracle.rhs_block(blocks[s], 3, 5.0 / 3.0, dx0, oracle.QUAD26)
        assert np.array_equal(got[s], ref) and gam[s] == ra


def test_quad26_constant_state_and_conservation():
    lv = _full_forest()
    n = len(lv)
    shp = (n, N, N, N)
    Uc = synth.conserved_from_states(np.full(shp, 1.1), np.full(shp, 0.3), np.full(shp, 0.1),
                                     np.full(shp, -0.2), np.full(shp, 0.7), None)
    got, _ = of.rhs(lv, 3, list(np.moveaxis(Uc, 0, 1)), 1.0 / 24, mode=oracle.QUAD26)
    for o in got:
        assert np.all(o == 0.0)
    U, dx0 = synth.smooth_forest_state(lv, 3, N, nf=7, seed=23)
    for mode in (oracle.QUAD26, oracle.QUAD26 | oracle.MODE_MIXED):
        got, _ = of.rhs(lv, 3, list(U), dx0, mode=mode)
        vol = (dx0 / (1 << lv[:, 0].astype(np.int64))) ** 3
        tot = sum(got[s].sum(axis=(1, 2, 3)) * vol[s] for s in range(n))
        mag = sum(np.abs(got[s]).sum(axis=(1, 2, 3)) * vol[s] for s in range(n))
        assert np.all(np.abs(tot) <= 1e-14 * mag)


def test_quad26_linear_field_edge_and_corner_ghosts():
    """Edge and corner ghosts of a linear field follow the same closed form
    as the face ghosts (field at the source cell's centre, or at the ghost's
    own centre when finer leaves cover it)."""
    lv = _full_forest()
    nb0 = 3
    coef = np.array([-0.4, 0.9, 1.7])
    xyz = synth.forest_cell_centres(lv, nb0, N)
    U = [np.stack([2.0 + np.tensordot(coef, xyz[s], axes=1)] * 6) for s in range(len(lv))]
    fo = of.Forest(lv, nb0, N)
    seen = {"same": 0, "coarse": 0, "fine": 0}
    for s in range(0, len(lv), 7):
        L, b = int(lv[s, 0]), lv[s, 1:]
        gb = of.ghosted_block(fo, U, s, quad26=True)
        w = 1.0 / ((nb0 << L) * N)
        for c in [(-1, -1, 3), (-2, N + 1, -1), (N, -1, N + 1), (N + 1, N + 1, 0), (-3, -2, -1),
                  (4, N, N + 2), (-1, N, N)]:
            outside = sum(not (0 <= v < N) for v in c)
            assert outside >= 2
            centre = [((b[e] * N + c[e] + 0.5) * w) % 1.0 for e in range(3)]
            src = _contains(lv, nb0, centre)
            Ls = int(lv[src, 0])
            if Ls <= L:
                ws = 1.0 / ((nb0 << Ls) * N)
                at = [(np.floor(x / ws) + 0.5) * ws for x in centre]
                seen["same" if Ls == L else "coarse"] += 1
            else:
                at = centre
                seen["fine"] += 1
            got = gb[0, c[2] + 3, c[1] + 3, c[0] + 3]
            assert got == pytest.approx(2.0 + coef @ np.array(at), rel=0, abs=1e-14)
    assert min(seen.values()) > 0, seen


def test_quad26_mirror_symmetry():
    lv = _full_forest()
    U, dx0 = synth.smooth_forest_state(lv, 3, N, nf=6, seed=24)
    got, gam = of.rhs(lv, 3, list(U), dx0, mode=oracle.QUAD26)
    mv = lv.copy()
    mv[:, 2] = (3 << lv[:, 0]) - 1 - lv[:, 2]   # y -> 1 - y
    MU = U[:, :, :, ::-1, :].copy()
    MU[:, 2] *= -1
    mg, mgam = of.rhs(mv, 3, list(MU), dx0, mode=oracle.QUAD26)
    for s in range(len(lv)):
        back = mg[s][:, :, ::-1, :].copy()
        back[2] *= -1
        scale = np.abs(got[s]).max(axis=(1, 2, 3), keepdims=True)
        assert np.all(np.abs(back - got[s]) <= 1e-13 * scale)
    assert np.allclose(mgam, gam, rtol=1e-14, atol=0)


def test_full_balance_generator():
    lv = _full_forest()
    lmax = 2
    lo, w = _boxes(lv, 3, lmax)
    M = 3 << lmax
    owner = np.zeros((M, M, M), dtype=np.int64)
    for s, ((x, y, z), ww) in enumerate(zip(lo, w)):
        owner[z:z + ww, y:y + ww, x:x + ww] = s
    for o in [(i, j, k) for k in (-1, 0, 1) for j in (-1, 0, 1) for i in (-1, 0, 1) if (i, j, k) != (0, 0, 0)]:
        nb = np.roll(owner, shift=(-o[2], -o[1], -o[0]), axis=(0, 1, 2))
        assert np.abs(lv[owner, 0] - lv[nb, 0]).max() <= 1


def test_subset_evaluation_equals_the_full_one():
    """`only=` (used for sampled checks of large forests) gives the full
    evaluation's values for the chosen leaves, bit for bit."""
    lv = _forest(7, 0.25)
    U, dx0 = synth.smooth_forest_state(lv, NB0, N, nf=6, seed=25)
    full, fam = of.rhs(lv, NB0, list(U), dx0)
    pick = [0, 5, int(np.flatnonzero(lv[:, 0] == 0)[0]), int(np.flatnonzero(lv[:, 0] == 2)[0]), len(lv) - 1]
    part, pam = of.rhs(lv, NB0, list(U), dx0, only=pick)
    for s in pick:
        assert np.array_equal(part[s], full[s]) and pam[s] == fam[s]


@pytest.mark.parametrize("quad26", [False, True])
def test_forest_homogeneity_under_power_of_two_scaling(quad26):
    """The homogeneity pin on a three-level forest: the level transfer
    (copies and means of 8), the per-leaf RHS and the flux correction all
    scale exactly, so scaling rho, rho v, E, rho X by 4 and tau by 1/8 scales
    every leaf's dU/dt by the same factor, bit for bit (face-centre scheme,
    and the 26-point variant on a fully balanced forest)."""
    lv, nb0 = (_full_forest(), 3) if quad26 else (_forest(4, 0.25), NB0)
    mode = oracle.QUAD26 if quad26 else 0
    U, dx0 = synth.smooth_forest_state(lv, nb0, N, nf=7, seed=26)
    ref, ram = of.rhs(lv, nb0, list(U), dx0, mode=mode)
    V = U * 4.0
    V[:, 5] = U[:, 5] * 0.125
    got, gam = of.rhs(lv, nb0, list(V), dx0, mode=mode)
    assert np.array_equal(gam, ram)
    for s in range(len(lv)):
        for f in range(7):
            assert np.array_equal(got[s][f], ref[s][f] * (0.125 if f == 5 else 4.0)), (s, f)
