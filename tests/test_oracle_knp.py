"""Pins of the oracle's second flux, the central-upwind scheme with one-sided
local speeds (Kurganov, Noelle & Petrova 2001): the invariants the first
flux satisfies, plus its defining property that for supersonic flow (all
local speeds of one sign) it is the pure upwind flux."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import test_oracle_pins as pins

G53 = 5.0 / 3.0
KNP = oracle.FLUX_KNP


@pytest.mark.parametrize("prec", [0, 1])
def test_uniform_state_zero_rhs(prec):
    G = 14
    shp = (G, G, G)
    rng = np.random.default_rng(4)
    X = np.broadcast_to(rng.dirichlet(np.ones(5))[:, None, None, None], (5,) + shp)
    U = pins.block_from_states(pins.full(shp, 1.7), [pins.full(shp, c) for c in (0.4, -0.1, 0.2)],
                               pins.full(shp, 0.8), X)
    out, amax, fl = oracle.rhs_block(U, 3, G53, 0.125, prec + KNP)
    assert fl == 0 and np.all(out == 0)
    assert abs(amax - (0.4 + math.sqrt(G53 * 0.8 / 1.7))) <= (1e-14 if prec == 0 else 3e-7) * amax


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_cubic_density_is_advected_exactly(axis):
    N, g, h = 8, 3, 1.0 / 8
    G = N + 2 * g
    edges = np.arange(-g, N + g + 1) * h
    avg = pins._cubic_avg(edges[:-1], edges[1:])
    shp = (G, G, G)
    rho = np.broadcast_to(avg.reshape([G if (2 - a) == axis else 1 for a in range(3)]), shp).copy()
    v = np.array([0.3, -0.2, 0.1])
    U = pins.block_from_states(rho, [pins.full(shp, c) for c in v], pins.full(shp, 1.0))
    out, amax, fl = oracle.rhs_block(U, g, G53, h, KNP)
    xi = np.arange(N + 1) * h
    drho = (-v[axis] * (pins._cubic(xi[1:]) - pins._cubic(xi[:-1])) / h).reshape(
        [N if (2 - a) == axis else 1 for a in range(3)])
    assert pins.normwise(out[0], np.broadcast_to(drho, out[0].shape)) <= 1e-12
    for c in range(3):
        assert pins.normwise(out[1 + c], np.broadcast_to(v[c] * drho, out[0].shape)) <= 1e-12


def test_supersonic_flow_gets_the_upwind_flux():
    """u > c on both sides: am = 0, so Fhat = F(left state).  Across a density
    jump the left state is the upstream cell's value (both cells flattened),
    whereas the single-speed flux adds dissipation there."""
    q = np.array([1.0] * 7 + [2.5] * 7)
    shp = (7, 7, q.size)
    u, p = 3.0, 0.1
    U = pins.block_from_states(np.broadcast_to(q, shp).copy(),
                               [pins.full(shp, u), pins.full(shp, 0.0), pins.full(shp, 0.0)],
                               pins.full(shp, p))
    _, _, _, (fx, _, _) = oracle.rhs_block(U, 3, G53, 1.0, KNP, faces=True)
    _, _, _, (kx, _, _) = oracle.rhs_block(U, 3, G53, 1.0, 0, faces=True)
    left_rho = q[2:2 + fx.shape[-1]]  # cell i-1 of face i (line index i+2)
    np.testing.assert_allclose(fx[0, 0, 0], left_rho * u, rtol=1e-14)
    np.testing.assert_allclose(fx[1, 0, 0], left_rho * u * u + p, rtol=1e-14)
    jump = 7 - 3
    assert abs(kx[0, 0, 0, jump] - left_rho[jump] * u) > 0.1


@pytest.mark.parametrize("prec", [0, 1])
def test_periodic_conservation_and_symmetry(prec):
    glob = synth.plain_domain(seed=13, n=32, nf=11)
    blocks = list(synth.gather_blocks(glob, 8))
    outs, amax, flags = oracle.rhs_batch(blocks, G53, 1.0 / 32, prec + KNP, threads=4)
    tot = np.sum([o.sum(axis=(1, 2, 3)) for o in outs], axis=0)
    mag = np.sum([np.abs(o).sum(axis=(1, 2, 3)) for o in outs], axis=0)
    assert np.all(np.abs(tot) <= 1e-13 * mag)
    U, dx = synth.one_subgrid(seed=5, nf=11)
    out, am, _ = oracle.rhs_block(U, 3, G53, dx, prec + KNP)
    Um = np.flip(U, axis=3).copy()
    Um[1] *= -1
    om, amm, _ = oracle.rhs_block(Um, 3, G53, dx, prec + KNP)
    exp = np.flip(out, axis=3).copy()
    exp[1] *= -1
    for k in range(11):
        assert pins.normwise(om[k], exp[k]) <= (1e-13 if prec == 0 else 1e-6)


@pytest.mark.slow
def test_sod_tube_converges_with_knp():
    orig = oracle.rhs_block

    def knp_block(U, ghost=3, gamma=G53, dx=1.0, mode=0, faces=False):
        return orig(U, ghost, gamma, dx, mode | KNP, faces)

    oracle.rhs_block = knp_block
    try:
        errs = [pins._sod_run(n, 1.4)[0] for n in (64, 128, 256)]
    finally:
        oracle.rhs_block = orig
    kt = [pins._sod_run(n, 1.4)[0] for n in (64, 256)]
    assert errs[0] > errs[1] > errs[2] and errs[2] <= 3e-3
    assert min(math.log2(errs[i] / errs[i + 1]) for i in range(2)) >= 0.6
    assert errs[2] <= kt[1] * 1.05  # one-sided speeds are no more diffusive
