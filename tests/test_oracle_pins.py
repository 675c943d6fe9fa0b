"""Pins of the CPU oracle against what the physics and mathematics fix.

Each test checks the oracle against something other than itself: an exact
closed form, an invariant, a symmetry, or convergence to an independent exact
solution (the Riemann problem, smooth advection).  The scheme is the one of
Sec. IV-B (PPM after Colella & Woodward 1984, central flux after Kurganov &
Tadmor 2000, Courant signal speed); Table I pins the bookkeeping.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests import exact_riemann as er

G53 = 5.0 / 3.0
HERE = os.path.dirname(os.path.abspath(__file__))


def block_from_states(rho, v, p, X=None, gamma=G53):
    return synth.conserved_from_states(rho, v[0], v[1], v[2], p, X, gamma)


def full(shape, val):
    return np.full(shape, float(val))


def normwise(a, b):
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() / scale


# ------------------------------------------------------------ uniform --
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("nf", [6, 11])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_uniform_state_has_zero_rhs_and_closed_form_speed(mode, nf, seed):
    rng = np.random.default_rng(seed)
    G = 14
    shp = (G, G, G)
    rho, p = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
    v = rng.normal(0.0, 0.3, 3)
    X = None
    if nf > 6:
        X = np.broadcast_to(rng.dirichlet(np.ones(nf - 6))[:, None, None, None], (nf - 6,) + shp)
    U = block_from_states(full(shp, rho), [full(shp, c) for c in v], full(shp, p), X)
    out, amax, fl = oracle.rhs_block(U, 3, G53, 0.125, mode)
    assert fl == 0
    assert np.all(out == 0.0)  # exactly: every face sees identical left/right states
    expect = np.abs(v).max() + math.sqrt(G53 * p / rho)
    assert abs(amax - expect) <= (1e-14 if mode == 0 else 3e-7) * expect


# --------------------------------------------- polynomial exactness --
def _cubic_avg(xl, xr):
    """Cell average of P(x) = 1 + 0.3x + 0.05x^2 + 0.01x^3 over [xl, xr]."""
    Q = lambda x: x + 0.15 * x ** 2 + 0.05 / 3 * x ** 3 + 0.0025 * x ** 4
    return (Q(xr) - Q(xl)) / (xr - xl)


def _cubic(x):
    return 1 + 0.3 * x + 0.05 * x ** 2 + 0.01 * x ** 3


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_cubic_density_is_advected_exactly(axis, mode):
    """PPM's unlimited face value is the 4th-order interpolant, exact for cell
    averages of a cubic; with uniform v and p the dissipation vanishes and
    d<rho>/dt = -v_a (P(x_{i+1/2}) - P(x_{i-1/2}))/dx holds to round-off.  All
    other fields follow from rho: s = rho v, E = p/(g-1) + rho|v|^2/2,
    tau = rho phi, rho_k = rho X_k."""
    N, g, h = 8, 3, 1.0 / 8
    G = N + 2 * g
    edges = (np.arange(-g, N + g + 1)) * h
    avg = _cubic_avg(edges[:-1], edges[1:])
    shp = (G, G, G)
    # axis 0 = x is the last array axis
    rho = np.broadcast_to(avg.reshape([G if (2 - a) == axis else 1 for a in range(3)]), shp).copy()
    v = np.array([0.3, -0.2, 0.1])
    p, phi = 1.0, 0.7
    nf = 11
    Xv = np.array([0.1, 0.2, 0.3, 0.15, 0.25])
    X = np.broadcast_to(Xv[:, None, None, None], (5,) + shp)
    U = block_from_states(rho, [full(shp, c) for c in v], full(shp, p), X)
    U[5] = rho * phi  # tau = rho * phi with constant phi
    out, amax, fl = oracle.rhs_block(U, g, G53, h, mode)
    assert fl == 0
    xi = np.arange(N + 1) * h
    drho = -v[axis] * (_cubic(xi[1:]) - _cubic(xi[:-1])) / h
    drho = drho.reshape([N if (2 - a) == axis else 1 for a in range(3)])
    exp = np.zeros_like(out)
    exp[0] = drho
    for c in range(3):
        exp[1 + c] = v[c] * drho
    exp[4] = 0.5 * np.dot(v, v) * drho
    exp[5] = phi * drho
    for k in range(5):
        exp[6 + k] = Xv[k] * drho
    if mode == 0:
        for f in range(nf):
            assert normwise(out[f], exp[f]) <= 1e-12, f
    else:
        # binary32 fluxes carry a few roundings of 2^-24 each, so the error of a
        # flux difference is bounded by a small multiple of eps32 * max|F| / dx
        _, _, _, faces = oracle.rhs_block(U, g, G53, h, 0, faces=True)
        for f in range(nf):
            fmax = max(np.abs(F[f]).max() for F in faces)
            assert np.abs(out[f] - exp[f]).max() <= 16 * 2.0 ** -24 * fmax / h, f


def test_linear_pressure_gives_exact_momentum_source():
    """At rest with a linear pressure ramp (uniform rho): face pressures are
    exact, the density and energy fluxes vanish and ds/dt = -grad p."""
    N, g, h = 8, 3, 0.1
    G = N + 2 * g
    shp = (G, G, G)
    c = (np.arange(G) - g + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    grad = np.array([0.3, -0.5, 0.2])
    p = 2.0 + grad[0] * x + grad[1] * y + grad[2] * z
    U = block_from_states(full(shp, 1.3), [full(shp, 0.0)] * 3, p)
    out, amax, fl = oracle.rhs_block(U, g, G53, h, 0)
    assert fl == 0
    assert np.abs(out[0]).max() <= 1e-13
    assert np.abs(out[4]).max() <= 1e-12
    for d in range(3):
        np.testing.assert_allclose(out[1 + d], -grad[d], rtol=0, atol=1e-12)


# ----------------------------------------- limiter, via face states --
def _passive_face_states(phi_line, u=0.5):
    """Recover the reconstructed face values of the passive scalar phi along x
    from the oracle's tau fluxes at u and -u (rho = p = 1):
      F(+u) = u(phiL+phiR)/2 - a(phiR-phiL)/2, F(-u) = -u(...)/2 - a(...)/2."""
    n = phi_line.size - 6
    shp = (7, 7, phi_line.size)
    res = []
    for uu in (u, -u):
        U = block_from_states(full(shp, 1.0), [full(shp, uu), full(shp, 0.0), full(shp, 0.0)],
                              full(shp, 1.0))
        U[5] = np.broadcast_to(phi_line, shp)
        _, amax, fl, (fx, fy, fz) = oracle.rhs_block(U, 3, G53, 1.0, 0, faces=True)
        res.append(fx[5, 0, 0, :])
        a = amax
    F1, F2 = res
    s = (F1 - F2) / u
    dd = -(F1 + F2) / a
    phiL = 0.5 * (s - dd)
    phiR = 0.5 * (s + dd)
    assert phiL.size == n + 1
    return phiL, phiR  # at faces i-1/2, i = 0..n


def test_limiter_keeps_monotone_profiles_monotone():
    rng = np.random.default_rng(7)
    for _ in range(20):
        q = np.cumsum(rng.exponential(1.0, 14) ** 3) + 1.0  # monotone, very uneven steps
        L, R = _passive_face_states(q)
        for i in range(L.size):  # face between cells i-1 and i (line index i+2, i+3)
            lo, hi = sorted((q[i + 2], q[i + 3]))
            for v in (L[i], R[i]):
                assert lo - 1e-12 * hi <= v <= hi + 1e-12 * hi
        # each interior cell's parabola (q-, q, q+) is monotone and has no
        # interior extremum: |q - (q- + q+)/2| <= |q+ - q-|/6 (CW84 eq. 1.10)
        for j in range(8):
            qm, qc, qp = R[j], q[j + 3], L[j + 1]
            assert (qp - qc) * (qc - qm) >= -1e-12
            assert abs(qc - 0.5 * (qm + qp)) <= abs(qp - qm) / 6 + 1e-12 * abs(qc)


def test_limiter_flattens_local_extrema():
    q = np.array([1.0, 1.1, 1.3, 1.6, 2.0, 1.7, 1.5, 1.4, 1.35, 1.3, 1.2, 1.1, 1.05, 1.0])
    L, R = _passive_face_states(q)
    j = 4 - 3  # cell with value 2.0 is interior cell 1
    assert abs(R[j] - 2.0) <= 1e-13 and abs(L[j + 1] - 2.0) <= 1e-13


def test_step_reduces_to_first_order_upwinded_states():
    """A single jump: all CW84 slopes vanish next to it and both adjacent cells
    are flattened, so the states at the jump are the two cell values."""
    q = np.array([1.0] * 7 + [3.0] * 7)
    L, R = _passive_face_states(q)
    i = 7 - 3  # face between line cells 6 and 7 is face i = 4
    assert abs(L[i] - 1.0) <= 1e-13 and abs(R[i] - 3.0) <= 1e-13


def test_cubic_face_values_are_exact():
    h = 0.1
    edges = np.arange(-3, 8 + 3 + 1) * h
    q = _cubic_avg(edges[:-1], edges[1:])
    L, R = _passive_face_states(q)
    xf = np.arange(9) * h
    np.testing.assert_allclose(L, _cubic(xf), rtol=0, atol=1e-12)
    np.testing.assert_allclose(R, _cubic(xf), rtol=0, atol=1e-12)


# ------------------------------------------------------- conservation --
@pytest.mark.parametrize("mode", [0, 1])
def test_periodic_domain_conserves_every_field(mode):
    n, N = 32, 8
    glob = synth.plain_domain(seed=11, n=n, nf=11)
    blocks = synth.gather_blocks(glob, N)
    outs, amax, flags = oracle.rhs_batch(list(blocks), G53, 1.0 / n, mode, threads=4)
    assert not flags.any()
    tot = np.sum([o.sum(axis=(1, 2, 3)) for o in outs], axis=0)
    mag = np.sum([np.abs(o).sum(axis=(1, 2, 3)) for o in outs], axis=0)
    assert np.all(np.abs(tot) <= 1e-13 * mag), (tot, mag)


def test_batch_equals_blocks():
    Us = synth.iid_batch(3, 8, 11, seed=3)
    outs, amax, flags = oracle.rhs_batch(Us, G53, 0.125, 0, threads=2)
    for s, U in enumerate(Us):
        o, a, f = oracle.rhs_block(U, 3, G53, 0.125, 0)
        assert np.array_equal(o, outs[s]) and a == amax[s]


# ---------------------------------------------------------- symmetry --
@pytest.mark.parametrize("mode", [0, 1])
def test_mirror_symmetry(mode):
    U, dx = synth.one_subgrid(seed=5, nf=11)
    out, amax, _ = oracle.rhs_block(U, 3, G53, dx, mode)
    for ax, f in ((3, 1), (2, 2), (1, 3)):  # array axis, momentum field flipped
        Um = np.flip(U, axis=ax).copy()
        Um[f] *= -1
        om, am, _ = oracle.rhs_block(Um, 3, G53, dx, mode)
        exp = np.flip(out, axis=ax).copy()
        exp[f] *= -1
        for k in range(U.shape[0]):
            assert normwise(om[k], exp[k]) <= (1e-13 if mode == 0 else 1e-6)
        assert am == amax


@pytest.mark.parametrize("mode", [0, 1])
def test_axis_permutation_symmetry(mode):
    U, dx = synth.one_subgrid(seed=6, nf=11)
    out, amax, _ = oracle.rhs_block(U, 3, G53, dx, mode)
    # swap x <-> y (array axes 3, 2) and momentum components 1, 2; same for x <-> z
    for axes, fields in (((3, 2), (1, 2)), ((3, 1), (1, 3)), ((2, 1), (2, 3))):
        Up = np.swapaxes(U, *axes).copy()
        Up[[fields[0], fields[1]]] = Up[[fields[1], fields[0]]]
        op, ap, _ = oracle.rhs_block(Up, 3, G53, dx, mode)
        exp = np.swapaxes(out, *axes).copy()
        exp[[fields[0], fields[1]]] = exp[[fields[1], fields[0]]]
        for k in range(U.shape[0]):
            assert normwise(op[k], exp[k]) <= (1e-13 if mode == 0 else 2e-6)
        assert ap == amax


# ------------------------------------------------------- dual energy --
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("ratio,uses_tau", [(5e-4, True), (2e-3, False)])
def test_dual_energy_switch(ratio, uses_tau, mode):
    """e = E - |s|^2/(2 rho); below eta*E (eta = 1e-3) the tracer gives
    e = tau^gamma.  A uniform state with tau deliberately inconsistent shows
    which branch fed the sound speed."""
    G = 14
    shp = (G, G, G)
    rho, vx = 1.2, 0.8
    ekin = 0.5 * rho * vx * vx
    E = ekin / (1.0 - ratio)
    eint = E - ekin
    tau = (3.0 * eint) ** (1.0 / G53)
    U = np.zeros((6,) + shp)
    U[0], U[1], U[4], U[5] = rho, rho * vx, E, tau
    out, amax, fl = oracle.rhs_block(U, 3, G53, 0.1, mode)
    assert fl == 0 and np.all(out == 0)
    e = 3.0 * eint if uses_tau else eint
    expect = vx + math.sqrt(G53 * (G53 - 1.0) * e / rho)
    assert abs(amax - expect) <= (1e-9 if mode == 0 else 1e-6) * expect


# ----------------------------------------------------- read region --
def test_only_the_star_region_is_read():
    U, dx = synth.one_subgrid(seed=9, nf=6)
    out, amax, fl = oracle.rhs_block(U, 3, G53, dx, 0)
    G, g, N = 14, 3, 8
    idx = np.arange(G) - g
    outside = (idx < 0) | (idx >= N)
    k, j, i = np.meshgrid(outside, outside, outside, indexing="ij")
    non_star = (k.astype(int) + j + i) >= 2
    assert non_star.sum() == G ** 3 - synth.star_cells(N)
    Un = U.copy()
    Un[:, non_star] = np.nan
    out2, amax2, fl2 = oracle.rhs_block(Un, 3, G53, dx, 0)
    assert fl2 == 0 and np.array_equal(out, out2) and amax == amax2
    # a bad value inside the star region is reported
    Ub = U.copy()
    Ub[0, 1, 5, 5] = -1.0  # z-ghost layer 2 cells out, interior x, y
    assert oracle.rhs_block(Ub, 3, G53, dx, 0)[2] & oracle.NONPHYS
    Ub = U.copy()
    Ub[4, 5, 5, 5] = np.inf
    assert oracle.rhs_block(Ub, 3, G53, dx, 0)[2] & oracle.NONPHYS


# ---------------------------------------------- mixed vs binary64 --
def test_mixed_form_error_is_small_on_smooth_data():
    glob = synth.plain_domain(seed=12, n=32, nf=11)
    blocks = list(synth.gather_blocks(glob, 8)[:8])
    o64, a64, _ = oracle.rhs_batch(blocks, G53, 1.0 / 32, 0)
    o32, a32, _ = oracle.rhs_batch(blocks, G53, 1.0 / 32, 1)
    for s in range(len(blocks)):
        for f in range(11):
            assert normwise(o32[s][f], o64[s][f]) <= 1e-5
    assert np.all(np.abs(a32 - a64) <= 1e-6 * a64)


# ----------------------------------------------------------- Table I --
def test_table1_bookkeeping():
    gold = json.load(open(os.path.join(HERE, "golden", "table1_bookkeeping.json")))
    g = gold["ghost_thickness"]
    for c in gold["cases"]:
        N = c["N"]
        assert synth.ghost_cells(N, g) == c["ghost_cells_per_subgrid"]
        assert c["leaf_subgrids"] * N ** 3 == c["overall_cells"]
        assert synth.kernel_calls_per_step(c["leaf_subgrids"]) == c["kernel_calls_per_step"]
        assert 2 * c["kernel_calls_per_step"] == c["transfers_per_step"]
        assert N + 2 * g == c["input_edge"]
        assert N + 2 == c["work_items_edge"]  # reconstruct/flux cover the innermost ghost layer
    assert synth.star_cells(8) == 1664 and synth.star_cells(16) == 8704


# ------------------------------------------- exact Riemann solution --
def test_exact_riemann_solver_satisfies_jump_conditions():
    g = 1.4
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us = er.star_state(*left, *right, g)
    # right-moving shock: Rankine-Hugoniot mass and momentum fluxes balance
    rhoR, uR, pR = right
    rs = er.sample(us + 1e-9, left, right, g)[0]
    S = (rs * us - rhoR * uR) / (rs - rhoR)
    mom_l = rs * us * us + ps - S * rs * us
    mom_r = rhoR * uR * uR + pR - S * rhoR * uR
    assert abs(mom_l - mom_r) <= 1e-10
    eL = ps / (g - 1) + 0.5 * rs * us * us
    eR = pR / (g - 1) + 0.5 * rhoR * uR * uR
    assert abs((eL + ps) * us - S * eL - ((eR + pR) * uR - S * eR)) <= 1e-10
    # left rarefaction: isentropic, Riemann invariant u + 2c/(g-1) constant
    rl = er.sample(us - 1e-9, left, right, g)[0]
    assert abs(ps / rl ** g - left[2] / left[0] ** g) <= 1e-10
    cL = math.sqrt(g * left[2] / left[0])
    cs = math.sqrt(g * ps / rl)
    assert abs(left[1] + 2 * cL / (g - 1) - (us + 2 * cs / (g - 1))) <= 1e-10


def _sod_run(nx, g, t_end=0.2, cfl=0.4, mode=0):
    ny = nz = 4
    gh = 3
    dx = 1.0 / nx
    xc = (np.arange(nx) + 0.5) * dx
    rho = np.where(xc < 0.5, 1.0, 0.125)
    p = np.where(xc < 0.5, 1.0, 0.1)
    shp = (nz, ny, nx)
    rho3 = np.broadcast_to(rho, shp)
    p3 = np.broadcast_to(p, shp)
    z = np.zeros(shp)
    U = synth.conserved_from_states(rho3, z, z, z, p3, None, g)

    def fill(Ui):
        Up = np.pad(Ui, ((0, 0), (gh, gh), (gh, gh), (0, 0)), mode="wrap")
        return np.pad(Up, ((0, 0), (0, 0), (0, 0), (gh, gh)), mode="edge")

    def L(Ui):
        out, amax, fl = oracle.rhs_block(fill(Ui), gh, g, dx, mode)
        assert fl == 0
        assert np.all(out[2] == 0) and np.all(out[3] == 0)  # no transverse momentum
        return out, amax

    t = 0.0
    while t < t_end - 1e-14:
        k1, amax = L(U)
        dt = min(cfl * dx / amax, t_end - t)
        U1 = U + dt * k1
        U2 = 0.75 * U + 0.25 * (U1 + dt * L(U1)[0])
        U = U / 3.0 + 2.0 / 3.0 * (U2 + dt * L(U2)[0])
        t += dt
    exact = er.cell_average_density(xc, dx, t_end, 0.5, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g)
    return np.sum(np.abs(U[0, 0, 0] - exact)) * dx, U


@pytest.mark.slow
@pytest.mark.parametrize("g", [1.4, G53])
def test_sod_tube_converges_to_exact_solution(g):
    errs = [_sod_run(n, g)[0] for n in (64, 128, 256)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[0] > errs[1] > errs[2]
    assert min(orders) >= 0.6, (errs, orders)
    assert errs[2] <= 3e-3, errs


# ------------------------------------------------ smooth advection order --
def _sine_avg(xl, xr, amp=0.2):
    return 1.0 + amp * (np.cos(2 * np.pi * xl) - np.cos(2 * np.pi * xr)) / (2 * np.pi * (xr - xl))


def _pulse_block(nx):
    gh = 3
    dx = 1.0 / nx
    edges = (np.arange(-gh, nx + gh + 1)) * dx
    rho = _sine_avg(edges[:-1], edges[1:])
    shp = (1 + 2 * gh, 1 + 2 * gh, nx + 2 * gh)
    rho3 = np.broadcast_to(rho, shp)
    o = np.ones(shp)
    z = np.zeros(shp)
    return synth.conserved_from_states(rho3, o, z, z, o, None, G53), dx


def test_smooth_pulse_rhs_converges_at_high_order():
    errs = []
    for nx in (16, 32, 64, 128):
        U, dx = _pulse_block(nx)
        out, amax, fl = oracle.rhs_block(U, 3, G53, dx, 0)
        xf = np.arange(nx + 1) * dx
        exact = -(0.2 * np.sin(2 * np.pi * xf[1:]) - 0.2 * np.sin(2 * np.pi * xf[:-1])) / dx
        errs.append(np.mean(np.abs(out[0, 0, 0] - exact)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert min(orders[1:]) >= 1.8, (errs, orders)


@pytest.mark.slow
def test_smooth_pulse_advection_converges():
    errs = []
    t_end = 0.25
    for nx in (16, 32, 64):
        U, dx = _pulse_block(nx)
        gh = 3
        Ui = U[:, gh:-gh, gh:-gh, gh:-gh].copy()

        def L(V):
            Vp = np.pad(V, ((0, 0), (gh, gh), (gh, gh), (gh, gh)), mode="wrap")
            return oracle.rhs_block(Vp, gh, G53, dx, 0)[:2]

        t = 0.0
        while t < t_end - 1e-14:
            k1, amax = L(Ui)
            dt = min(0.4 * dx / amax, t_end - t)
            U1 = Ui + dt * k1
            U2 = 0.75 * Ui + 0.25 * (U1 + dt * L(U1)[0])
            Ui = Ui / 3.0 + 2.0 / 3.0 * (U2 + dt * L(U2)[0])
            t += dt
        edges = np.arange(nx + 1) * dx - t_end
        exact = _sine_avg(edges[:-1], edges[1:])
        errs.append(np.mean(np.abs(Ui[0, 0, 0] - exact)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 1.8, (errs, orders)


@pytest.mark.parametrize("mode", [oracle.MODE_FP64, oracle.MODE_MIXED, oracle.FLUX_KNP, oracle.QUAD26])
def test_flux_homogeneity_under_power_of_two_scaling(mode):
    """The Euler fluxes are homogeneous of degree one in (rho, rho v, E,
    rho X) at fixed velocity, and the tau flux in tau: scaling those fields
    by lam and tau by mu (powers of two, so every step of the scheme scales
    exactly) scales each field's dU/dt by the same factor, bit for bit, and
    leaves the signal speed unchanged.  Thermal-dominated data keep the
    dual-energy switch off.  Fails for a wrong power of rho or p anywhere,
    species not weighted by rho, or a misplaced pressure term."""
    rng = synth.rng_for(91, 0)
    G, nf = 14, 8
    rho = rng.uniform(0.5, 2.0, (G, G, G))
    v = [rng.normal(0.0, 0.1, (G, G, G)) for _ in range(3)]
    p = rng.uniform(0.5, 2.0, (G, G, G))
    X = np.moveaxis(rng.dirichlet(np.ones(nf - 6), size=(G, G, G)), -1, 0)
    U = synth.conserved_from_states(rho, v[0], v[1], v[2], p, X)
    ref, ra, fl = oracle.rhs_block(U, 3, 5.0 / 3.0, 0.125, mode)
    assert not fl
    for lam, mu in ((4.0, 0.125), (0.25, 2.0)):
        V = U * lam
        V[5] = U[5] * mu
        got, ga, fl = oracle.rhs_block(V, 3, 5.0 / 3.0, 0.125, mode)
        assert not fl and ga == ra
        for f in range(nf):
            assert np.array_equal(got[f], ref[f] * (mu if f == 5 else lam)), (f, lam)
