"""The seeded input recipes have the properties the design notes give them:
value ranges, field counts, mixes and sizes of the synthetic workloads that
stand in for the paper's runs (Sec. VI-A, Table I).  CPU only."""
import math

import numpy as np
import pytest

import synth

G53 = 5.0 / 3.0
ETA = 1e-3  # dual-energy switch threshold of the scheme's reading (Sec. IV-B)


def _states(U):
    """rho, v, E, internal energy and tau of a conserved array [f][...]."""
    rho, s, E, tau = U[0], U[1:4], U[4], U[5]
    eint = E - 0.5 * (s * s).sum(0) / rho
    return rho, s / rho, E, eint, tau


def test_item_seeds_are_independent_and_reproducible():
    a = synth.rng_for(20221012, 3).random(4)
    b = synth.rng_for(20221012, 3).random(4)
    c = synth.rng_for(20221012, 4).random(4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_iid_block_ranges():
    U = synth.iid_block(synth.rng_for(1, 0), 8, 11)
    assert U.shape == (11, 14, 14, 14)
    rho, v, E, eint, tau = _states(U)
    assert 0.5 <= rho.min() and rho.max() <= 2.0
    p = (G53 - 1.0) * eint
    assert 0.5 * (1 - 1e-12) <= p.min() and p.max() <= 2.0 * (1 + 1e-12)
    assert abs(v.std() - 0.1) < 0.005 and abs(v.mean()) < 0.005
    X = U[6:] / rho
    assert X.min() >= 0.0 and np.allclose(X.sum(0), 1.0, rtol=0, atol=1e-13)
    assert np.allclose(tau, np.power(eint, 1.0 / G53), rtol=1e-12)


def test_plain_domain_ranges():
    U = synth.plain_domain(seed=5, n=32, nf=8)
    rho, v, E, eint, tau = _states(U)
    # rho and p are rescaled onto [0.5, 2] exactly; each velocity component
    # has mean 0 and standard deviation 0.1
    assert rho.min() == pytest.approx(0.5, rel=1e-14) and rho.max() == pytest.approx(2.0, rel=1e-14)
    p = (G53 - 1.0) * eint
    assert p.min() == pytest.approx(0.5, rel=1e-12) and p.max() == pytest.approx(2.0, rel=1e-12)
    for d in range(3):
        assert v[d].std() == pytest.approx(0.1, rel=1e-12) and abs(v[d].mean()) < 1e-15
    assert np.allclose((U[6:] / rho).sum(0), 1.0, rtol=0, atol=1e-13)


def test_polytropes_atmosphere_is_in_the_tracer_branch():
    U = synth.polytropes(n=64)
    assert U.shape == (11, 64, 64, 64)
    rho, v, E, eint, tau = _states(U)
    atm = rho == 1e-10
    # the two stars fill 4/3 pi (0.35^3 + 0.25^3) / 8 = 3.06 % of the cube
    star_volume = 4.0 / 3.0 * math.pi * (0.35 ** 3 + 0.25 ** 3) / 8.0
    assert abs((1.0 - atm.mean()) - star_volume) < 0.003
    # The tracer branch (e < eta E) takes 97 % of the cells: the atmosphere,
    # except where the rotation is too slow to make its kinetic energy exceed
    # e (1/eta - 1), i.e. within R_c = sqrt(2 e (1/eta - 1) / (rho Omega^2))
    # of the rotation axis (about 0.03).  The stars stay out of it.
    switched = eint < ETA * E
    assert 0.965 < switched.mean() < 0.975
    assert not switched[~atm].any()
    c = -1.0 + (np.arange(64) + 0.5) * (2.0 / 64)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    omega = 0.3 / 0.45
    e_atm = 0.6 * 1e-10 ** G53 / (G53 - 1.0)
    rc2 = 2.0 * e_atm * (1.0 / ETA - 1.0) / (1e-10 * omega ** 2)
    assert 0.02 < math.sqrt(rc2) < 0.04
    assert np.array_equal(switched, atm & (x * x + y * y > rc2))
    # p = 0.6 rho^(5/3) and rigid rotation about z with Omega = 0.3/0.45
    p = (G53 - 1.0) * eint
    star = ~atm
    assert np.allclose(p[star], 0.6 * np.power(rho[star], G53), rtol=1e-10)
    assert np.allclose(v[0], -omega * y, rtol=1e-12, atol=1e-14)
    assert np.allclose(v[1], omega * x, rtol=1e-12, atol=1e-14)
    assert np.abs(v[2]).max() == 0.0


def test_uneven_batch_mix():
    leaves = synth.uneven_octree()
    assert len(leaves) == 4096
    N = np.array([l[0] for l in leaves])
    nf = np.array([l[1] for l in leaves])
    dx = np.array([l[2] for l in leaves])
    assert (N == 16).sum() == 1024 and (N == 8).sum() == 3072
    assert np.all(dx[N == 16] == 1.0 / 256) and np.all(dx[N == 8] == 1.0 / 512)
    assert set(nf.tolist()) == {6, 11}
    assert abs((nf == 11).mean() - 0.5) < 0.04  # Bernoulli(1/2): standard deviation 0.008
    # shuffled: the sizes are not in blocks
    assert np.count_nonzero(np.diff(N)) > 100
    # 5,767,168 cells, 8/11 of them in the 16^3 sub-grids
    cells = (N.astype(np.int64) ** 3).sum()
    assert cells == 5767168 and (N[N == 16].astype(np.int64) ** 3).sum() * 11 == cells * 8
    # a prefix keeps the order
    assert synth.uneven_octree(n_subgrids=100) == leaves[:100]


def test_serving_trace():
    t, sizes, nfs = synth.serving_trace(rate=20000.0, duration=1.0)
    assert np.all(np.diff(t) > 0) and t[0] >= 0.0 and t[-1] < 1.0
    # Poisson count: mean 20000, standard deviation ~141
    assert abs(t.size - 20000) < 6 * math.sqrt(20000)
    assert sizes.min() >= 1 and sizes.max() <= 64 and nfs.min() >= 6 and nfs.max() <= 11
    assert set(np.unique(nfs).tolist()) == set(range(6, 12))
    # exponential gaps: mean 1/rate
    assert np.diff(t).mean() == pytest.approx(1.0 / 20000.0, rel=0.05)


def test_bench_forest_leaf_counts():
    lv = synth.forest_leaves(16, 2, synth.sphere_refine((0.5, 0.5, 0.5), (0.35, 0.2)), balance="full")
    assert len(lv) == 21848
    levels = np.bincount(np.asarray(lv)[:, 0], minlength=3)
    assert levels.tolist() == [3032, 7040, 11776]
    # the leaves tile the cube: volumes (8^-level of a root block) sum to 16^3
    assert (8.0 ** -np.asarray(lv)[:, 0].astype(float)).sum() == 16 ** 3
    assert len(lv) * 8 ** 3 == 11186176


def test_star_region_bytes():
    # 1664 read cells + 512 written per 8^3 sub-grid, 11 fields: 374 B per cell
    assert synth.algorithmic_bytes(8, 11) == (1664 + 512) * 11 * 8 + 8
    assert (synth.algorithmic_bytes(8, 11) - 8) / 512 == 374.0
    # Table I: 14^3 - 8^3 ghost cells per sub-grid
    assert synth.ghost_cells(8) == 2232
