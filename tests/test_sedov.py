"""The Sedov point explosion (the paper's benchmark scenario, Sec. VI-A) on
the CPU: the similarity solution pinned by published constants and its own
invariants, and the oracle's SSP-RK3 run pinned against that solution."""
import math

import numpy as np
import pytest

import synth
from tests.sedov_exact import Sedov
from tests.sedov_run import from_domain, oracle_run, shock_measures, to_domain


@pytest.fixture(scope="module")
def sedov53():
    return Sedov(5.0 / 3.0)


def test_similarity_constants_match_the_literature():
    # Sedov's constant xi0 of R = xi0 (E t^2/rho0)^(1/5): 1.033 for gamma = 1.4
    # and 1.152 for gamma = 5/3 (three dimensions)
    assert abs(Sedov(1.4).xi0 - 1.033) < 1e-3
    assert abs(Sedov(5.0 / 3.0).xi0 - 1.152) < 1e-3


@pytest.mark.parametrize("g", [1.4, 5.0 / 3.0])
def test_similarity_profile_limits(g):
    s = Sedov(g)
    # strong-shock jump at xi = 1
    assert s.f[-1] == pytest.approx((g + 1) / (g - 1), rel=1e-12)
    assert s.phi[-1] == pytest.approx(2 / (g + 1), rel=1e-12)
    # centre: density vanishes, pressure stays finite, u/(Rdot xi) -> 1/gamma
    assert s.f[0] < 1e-10 and s.psi[0] > 0.1
    assert abs(s.phi[0] / s.xi[0] - 1.0 / g) < 0.03
    # density and velocity increase monotonically towards the shock
    assert np.all(np.diff(s.f) > 0) and np.all(np.diff(s.phi) > 0)


def test_similarity_profile_carries_the_blast_energy(sedov53):
    t = 0.04
    R = sedov53.shock_radius(t)
    r = np.linspace(0.0, R, 20001)[1:]
    rho, u, p = sedov53.profile(r, t)
    e = 0.5 * rho * u * u + p / (5.0 / 3.0 - 1.0)
    E = np.trapezoid(4.0 * math.pi * r * r * e, r)
    assert E == pytest.approx(1.0, rel=2e-3)
    # mass inside the shock equals the swept-up mass
    M = np.trapezoid(4.0 * math.pi * r * r * rho, r)
    assert M == pytest.approx(4.0 / 3.0 * math.pi * R ** 3, rel=2e-3)


def test_domain_layout_round_trip():
    glob, _ = synth.sedov_domain(n=16, nf=7)
    assert np.array_equal(from_domain(to_domain(glob, 8), 16), glob)


def test_initial_state_holds_the_blast_energy():
    glob, dx = synth.sedov_domain(n=16, nf=11, p0=0.0)
    assert glob[4].sum() * dx ** 3 == pytest.approx(1.0, rel=1e-14)
    assert np.all(glob[1:4] == 0)
    X = glob[6:] / glob[0]
    assert np.allclose(X.sum(axis=0), 1.0)


def test_oracle_sedov_run_against_the_similarity_solution(sedov53):
    t_end = sedov53.time_for_radius(0.35)
    res = {}
    for n in (16, 32):
        U, t, dts = oracle_run(n, t_end)
        dx = 1.0 / n
        assert t == pytest.approx(t_end, rel=1e-12)
        # conservation on the periodic cube: mass, momentum, energy, species
        assert U[0].sum() * dx ** 3 == pytest.approx(1.0, rel=1e-12)
        assert U[4].sum() * dx ** 3 == pytest.approx(1.0 + 1e-5 / (2.0 / 3.0), rel=1e-12)
        assert np.abs(U[1:4].sum(axis=(1, 2, 3))).max() * dx ** 3 < 1e-12
        # positive density everywhere; spherical symmetry of the result
        assert U[0].min() > 0
        assert np.abs(U[0] - U[0].transpose(1, 2, 0)).max() < 1e-10
        assert np.abs(U[0] - U[0][::-1]).max() < 1e-10
        res[n] = shock_measures(U[0], dx, sedov53, t)
    for n, (Rp, L1) in res.items():
        assert abs(Rp - 0.35) <= 1.0 / n, (n, Rp)
    assert res[32][1] < 0.85 * res[16][1]  # L1(rho) decreases with resolution
