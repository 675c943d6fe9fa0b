"""Pins of the oracle's 26-point variant (Sec. IV-B: PPM values at the face
centres, edge midpoints and vertices of every cell, central-upwind fluxes
there, Newton-Cotes quadrature over each face).

What fixes it without another implementation:
  * a uniform state gives exactly zero and the closed-form signal speed;
  * data that vary along one axis only make every quadrature point of a face
    see the same one-dimensional stencil, so the variant equals the
    face-centre scheme (weights summing to one);
  * conservation on a periodic domain, mirror and axis-permutation symmetry;
  * second-order convergence on diagonal waves, where the edge and vertex
    points matter;
  * the read region (a NaN outside it changes nothing);
  * the assembly (which cell, which line, which end, which weight) against a
    brute-force evaluation that pairs the two cells' reconstructed values at
    each quadrature point by the point's coordinates.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth

G53 = 5.0 / 3.0
Q = oracle.QUAD26


def _uniform(G=14, gamma=G53):
    shp = (G, G, G)
    return synth.conserved_from_states(np.full(shp, 1.3), np.full(shp, 0.2), np.full(shp, -0.1),
                                       np.full(shp, 0.05), np.full(shp, 0.9), np.full((5,) + shp, 0.2),
                                       gamma)


@pytest.mark.parametrize("mode", [Q, Q | oracle.MODE_MIXED, Q | oracle.FLUX_KNP])
def test_uniform_state_zero_rhs(mode):
    U = _uniform()
    out, amax, fl = oracle.rhs_block(U, 3, G53, 0.1, mode)
    assert fl == 0 and np.all(out == 0)
    c = np.sqrt(G53 * 0.9 / 1.3)
    ref = 0.2 + c
    assert amax == pytest.approx(ref, rel=1e-15 if not mode & 1 else 1e-6)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_one_dimensional_data_reduce_to_the_face_centre_scheme(axis):
    rng = synth.rng_for(5, axis)
    N, g = 8, 3
    G = N + 2 * g
    prof = {k: rng.uniform(0.5, 2.0, G) for k in ("rho", "p")}
    vel = rng.normal(0.0, 0.3, (3, G))
    shape = [1, 1, 1]
    shape[2 - axis] = G  # arrays are [z][y][x]
    b = lambda a: np.broadcast_to(a.reshape(shape), (G, G, G)).copy()
    U = synth.conserved_from_states(b(prof["rho"]), b(vel[0]), b(vel[1]), b(vel[2]), b(prof["p"]),
                                    None, G53)
    for mix in (0, oracle.MODE_MIXED):
        a, am_a, _ = oracle.rhs_block(U, g, G53, 0.125, mix)
        q, am_q, _ = oracle.rhs_block(U, g, G53, 0.125, mix | Q)
        tol = 1e-13 if mix == 0 else 1e-5
        for f in range(U.shape[0]):
            scale = max(np.abs(a[f]).max(), 1e-300)
            assert np.abs(q[f] - a[f]).max() <= tol * scale, (mix, f)
        # the signal speed also sees the edge and vertex points of the faces
        # parallel to the variation, so it can only grow
        assert am_q >= am_a


@pytest.mark.parametrize("mode", [Q, Q | oracle.MODE_MIXED])
def test_periodic_conservation(mode):
    glob = synth.plain_domain(seed=31, n=16, nf=11)
    blocks = synth.gather_blocks(glob, 8)
    outs, amax, fl = oracle.rhs_batch(list(blocks), G53, 1.0 / 16, mode, threads=4)
    assert not fl.any()
    tot = np.sum([o.sum(axis=(1, 2, 3)) for o in outs], axis=0)
    mag = np.sum([np.abs(o).sum(axis=(1, 2, 3)) for o in outs], axis=0)
    assert np.all(np.abs(tot) <= 1e-13 * mag)


def test_mirror_and_axis_permutation_symmetry():
    U = synth.iid_block(synth.rng_for(44, 0), 6, 8)
    out, amax, _ = oracle.rhs_block(U, 3, G53, 0.2, Q)
    # mirror x -> -x: reverse the x axis and negate s_x
    Um = U[:, :, :, ::-1].copy()
    Um[1] *= -1
    om, am_m, _ = oracle.rhs_block(Um, 3, G53, 0.2, Q)
    om = om[:, :, :, ::-1]
    om[1] *= -1
    scale = np.abs(out).max(axis=(1, 2, 3))[:, None, None, None]
    assert np.all(np.abs(om - out) <= 1e-13 * scale)
    assert am_m == pytest.approx(amax, rel=1e-15)
    # axis swaps: exchange two array axes and the matching momentum components
    for axes, fields in (((3, 2), (1, 2)), ((3, 1), (1, 3)), ((2, 1), (2, 3))):
        Up = np.swapaxes(U, *axes).copy()
        Up[[fields[0], fields[1]]] = Up[[fields[1], fields[0]]]
        op, am_p, _ = oracle.rhs_block(Up, 3, G53, 0.2, Q)
        exp = np.swapaxes(out, *axes).copy()
        exp[[fields[0], fields[1]]] = exp[[fields[1], fields[0]]]
        escale = np.abs(exp).max(axis=(1, 2, 3))[:, None, None, None]
        assert np.all(np.abs(op - exp) <= 1e-13 * escale)
        assert am_p == pytest.approx(amax, rel=1e-15)


def _wave_block(N, kvec, amp=0.01, v=(0.5, 0.3, 0.0)):
    """Cell averages of rho = 1 + amp sin(2 pi k.x) advected by uniform v at
    uniform pressure, and the exact d<rho>/dt."""
    G, dx = N + 6, 1.0 / N
    xc = (np.arange(G) - 3 + 0.5) * dx
    fac = np.prod([1.0 if k == 0 else np.sin(np.pi * k * dx) / (np.pi * k * dx) for k in kvec])
    ph = 2 * np.pi * (kvec[0] * xc[None, None, :] + kvec[1] * xc[None, :, None] + kvec[2] * xc[:, None, None])
    rho = 1 + amp * fac * np.sin(ph)
    shp = rho.shape
    U = synth.conserved_from_states(rho, np.full(shp, v[0]), np.full(shp, v[1]), np.full(shp, v[2]),
                                    np.full(shp, 1.0), None, G53)
    kv = sum(k * w for k, w in zip(kvec, v))
    return U, dx, -amp * 2 * np.pi * kv * fac * np.cos(ph)[3:-3, 3:-3, 3:-3]


@pytest.mark.parametrize("kvec", [(1, 1, 0), (1, 1, 1)])
def test_second_order_on_diagonal_waves(kvec):
    err = []
    for N in (16, 32, 64):
        U, dx, ex = _wave_block(N, kvec)
        r = oracle.rhs_block(U, 3, G53, dx, Q)[0][0]
        err.append(np.abs(r - ex).mean())
    orders = np.log2(np.array(err[:-1]) / np.array(err[1:]))
    assert np.all(orders >= 1.85), orders


def test_read_region():
    N = 6
    U = synth.iid_block(synth.rng_for(45, 0), N, 7)
    ref, am, fl = oracle.rhs_block(U, 3, G53, 0.2, Q)
    assert fl == 0
    G = N + 6
    read = np.zeros((G, G, G), dtype=bool)
    for z, y, x in itertools.product(range(G), repeat=3):
        c = np.array([x, y, z]) - 3
        far = np.sum((c == -3) | (c == N + 2))
        read[z, y, x] = far <= 1
    V = U.copy()
    V[:, ~read] = np.nan
    out, am2, fl2 = oracle.rhs_block(V, 3, G53, 0.2, Q)
    assert fl2 == 0 and np.array_equal(out, ref) and am2 == am
    W = U.copy()
    W[0, 0, 5, 4] = np.nan  # z = -3 with x, y in the interior: read
    assert oracle.rhs_block(W, 3, G53, 0.2, Q)[2] & oracle.NONPHYS


# ------------------------------------------------------------ brute force --
def _ppm5(q, eta=None):
    """PPM face values (q-, q+) of the middle cell of five line values."""
    def slope(a, b, c):
        dp, dm, dbar = c - b, b - a, 0.5 * (c - a)
        if dp * dm > 0:
            return np.copysign(min(abs(dbar), 2 * abs(dm), 2 * abs(dp)), dbar)
        return 0.0
    d = [slope(q[i - 1], q[i], q[i + 1]) for i in (1, 2, 3)]
    lo = 0.5 * (q[1] + q[2]) - (d[1] - d[0]) / 6.0
    hi = 0.5 * (q[2] + q[3]) - (d[2] - d[1]) / 6.0
    c = q[2]
    if (hi - c) * (c - lo) <= 0:
        return c, c
    D, m = hi - lo, c - 0.5 * (lo + hi)
    if D * m > D * D / 6:
        lo = 3 * c - 2 * hi
    elif D * m < -D * D / 6:
        hi = 3 * c - 2 * lo
    return lo, hi


def _prims(u, g):
    rho = u[0]
    e = u[4] - 0.5 * (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / rho
    if e < 1e-3 * u[4]:
        e = u[5] ** g
    return np.array([rho, u[1] / rho, u[2] / rho, u[3] / rho, (g - 1) * e] + [u[f] / rho for f in range(5, len(u))])


def _kt(wl, wr, d, g):
    def cons_flux(w):
        rho, v, p = w[0], w[1:4], w[4]
        E = p / (g - 1) + 0.5 * rho * v @ v
        U = np.concatenate([[rho], rho * v, [E], rho * w[5:]])
        u = v[d]
        F = U * u
        F[1 + d] += p
        F[4] += p * u
        return U, F, abs(u) + np.sqrt(g * p / rho)
    Ul, Fl, sl = cons_flux(wl)
    Ur, Fr, sr = cons_flux(wr)
    a = max(sl, sr)
    return 0.5 * (Fl + Fr) - 0.5 * a * (Ur - Ul), a


def test_assembly_against_brute_force():
    N, g = 2, G53
    U = synth.iid_block(synth.rng_for(46, 0), N, 7)
    G = N + 6
    W = np.zeros((G, G, G, U.shape[0]))
    for z, y, x in itertools.product(range(G), repeat=3):
        W[z, y, x] = _prims(U[:, z, y, x], g)
    # every cell next to an interior face: its value at each of its 26 surface points
    vals = {}
    for z, y, x in itertools.product(range(-1, N + 1), repeat=3):
        if sum(c < 0 or c >= N for c in (x, y, z)) > 1:
            continue
        for v in itertools.product((-1, 0, 1), repeat=3):
            if v == (0, 0, 0):
                continue
            line = [W[z + m * v[2] + 3, y + m * v[1] + 3, x + m * v[0] + 3] for m in range(-2, 3)]
            vals[(x, y, z, v)] = np.array([_ppm5([l[f] for l in line])[1] for f in range(W.shape[3])])
    # fluxes: for each interior face, 9 points with Simpson weights; states
    # found by the point's position relative to each cell's centre
    dUdt = np.zeros((U.shape[0], N, N, N))
    amax = 0.0
    for d in range(3):
        t1, t2 = [a for a in range(3) if a != d]
        for i in range(N + 1):
            for a, b in itertools.product(range(N), repeat=2):
                cl = [0, 0, 0]
                cl[d], cl[t1], cl[t2] = i - 1, a, b
                cr = list(cl)
                cr[d] += 1
                F = 0.0
                for o1, o2 in itertools.product((-1, 0, 1), repeat=2):
                    P = np.array(cl, dtype=float)
                    P[d] += 0.5
                    P[t1] += 0.5 * o1
                    P[t2] += 0.5 * o2
                    vl = tuple(int(round(2 * (P[k] - cl[k]))) for k in range(3))
                    vr = tuple(int(round(2 * (P[k] - cr[k]))) for k in range(3))
                    wl = vals[tuple(cl) + (vl,)]
                    # the right cell's value at P is the lower end of its line along -vr
                    line = [W[cr[2] - m * vr[2] + 3, cr[1] - m * vr[1] + 3, cr[0] - m * vr[0] + 3]
                            for m in range(-2, 3)]
                    wr = np.array([_ppm5([l[f] for l in line])[0] for f in range(W.shape[3])])
                    fh, sp = _kt(wl, wr, d, g)
                    amax = max(amax, sp)
                    F = F + (4 if o1 == 0 else 1) * (4 if o2 == 0 else 1) / 36.0 * fh
                for side, c in ((+1, cl), (-1, cr)):
                    if all(0 <= c[k] < N for k in range(3)):
                        dUdt[:, c[2], c[1], c[0]] -= side * F
    out, am, fl = oracle.rhs_block(U, 3, g, 1.0, Q)
    scale = np.abs(dUdt).max(axis=(1, 2, 3))[:, None, None, None]
    assert np.all(np.abs(out - dUdt) <= 1e-12 * scale)
    assert am == pytest.approx(amax, rel=1e-14)
