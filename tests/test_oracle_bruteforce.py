"""Brute-force pin of the oracle's indexing on the smallest sub-grid (N = 2).

A separate one-dimensional evaluation, written with plain Python floats over
an explicit list of the 8 cells of one line (2 interior cells and 3 ghosts on
each side), computes the face fluxes of that line: primitives of each cell,
CW84 slopes and face values, the parabola limiter, the Kurganov-Tadmor flux
at the line's 3 faces (Sec. IV-B's scheme in the face-centre reading).  It
knows nothing of the oracle's 3-D layout: the lines are cut out of the block
by explicit coordinates, and the momentum component along the line is picked
by name.  Every x, y and z line of random blocks (6 and 7 fields) must give
the oracle's face fluxes (face_out) to rounding, and the divergence of these
fluxes must give the oracle's dU/dt: a transposed index, a face shifted by
one, a swapped side or a wrong momentum component fails here.
"""
import math

import numpy as np
import pytest

import oracle
import synth

G53 = 5.0 / 3.0
ETA = 1e-3


def prim_cell(u, gamma):
    rho, s1, s2, s3, E, tau = u[:6]
    ekin = 0.5 * (s1 * s1 + s2 * s2 + s3 * s3) / rho
    e = E - ekin
    if e < ETA * E:
        e = tau ** gamma
    return [rho, s1 / rho, s2 / rho, s3 / rho, (gamma - 1.0) * e, tau / rho] + [x / rho for x in u[6:]]


def mc_slope(a, b, c):
    """CW84 limited slope of b between neighbours a and c."""
    dl, dr = b - a, c - b
    if dl * dr <= 0.0:
        return 0.0
    m = min(abs(0.5 * (c - a)), 2.0 * abs(dl), 2.0 * abs(dr))
    return m if c - a > 0 else -m


def ppm_states(q):
    """q: 8 values, cells -3..4.  Returns {cell: (q_minus, q_plus)} for
    cells -1, 0, 1, 2."""
    cell = {j: q[j + 3] for j in range(-3, 5)}
    slope = {j: mc_slope(cell[j - 1], cell[j], cell[j + 1]) for j in range(-2, 4)}
    face = {j: 0.5 * (cell[j] + cell[j + 1]) - (slope[j + 1] - slope[j]) / 6.0 for j in range(-2, 3)}
    st = {}
    for j in range(-1, 3):
        lo, hi, c = face[j - 1], face[j], cell[j]
        if (hi - c) * (c - lo) <= 0.0:
            lo = hi = c
        else:
            D, m = hi - lo, c - 0.5 * (lo + hi)
            if D * m > D * D / 6.0:
                lo = 3.0 * c - 2.0 * hi
            elif D * m < -D * D / 6.0:
                hi = 3.0 * c - 2.0 * lo
        st[j] = (lo, hi)
    return st


def kt_flux(wl, wr, axis, gamma):
    def parts(w):
        rho, vx, vy, vz, p = w[:5]
        un = (vx, vy, vz)[axis]
        E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
        U = [rho, rho * vx, rho * vy, rho * vz, E] + [rho * x for x in w[5:]]
        Fl = [rho * un, rho * vx * un, rho * vy * un, rho * vz * un, (E + p) * un] + [rho * x * un for x in w[5:]]
        Fl[1 + axis] += p
        return U, Fl, abs(un) + math.sqrt(gamma * p / rho)

    Ul, Fl, al = parts(wl)
    Ur, Fr, ar = parts(wr)
    a = max(al, ar)
    return [0.5 * (Fl[f] + Fr[f]) - 0.5 * a * (Ur[f] - Ul[f]) for f in range(len(Ul))], a


def line_fluxes(cells, axis, gamma):
    """cells: 8 conserved vectors along the line.  Returns the fluxes of the
    faces between cells (-1,0), (0,1), (1,2) and the largest speed."""
    W = [prim_cell(u, gamma) for u in cells]
    nf = len(W[0])
    st = [ppm_states([W[c][f] for c in range(8)]) for f in range(nf)]
    out, amax = [], 0.0
    for i in range(3):  # face between cells i-1 and i
        wl = [st[f][i - 1][1] for f in range(nf)]
        wr = [st[f][i][0] for f in range(nf)]
        F, a = kt_flux(wl, wr, axis, gamma)
        out.append(F)
        amax = max(amax, a)
    return out, amax


def block_sweeps(U, gamma):
    """Face fluxes of all lines of an N = 2 block: fx[f][z][y][i], fy[f][z][i][x],
    fz[f][i][y][x] for interior coordinates, face i between cells i-1 and i."""
    nf = U.shape[0]
    cell = lambda x, y, z: [float(U[f, z + 3, y + 3, x + 3]) for f in range(nf)]
    fx = np.zeros((nf, 2, 2, 3))
    fy = np.zeros((nf, 2, 3, 2))
    fz = np.zeros((nf, 3, 2, 2))
    amax = 0.0
    for a in range(2):
        for b in range(2):
            F, s = line_fluxes([cell(c, a, b) for c in range(-3, 5)], 0, gamma)  # x line at y=a, z=b
            amax = max(amax, s)
            for i in range(3):
                fx[:, b, a, i] = F[i]
            F, s = line_fluxes([cell(a, c, b) for c in range(-3, 5)], 1, gamma)  # y line at x=a, z=b
            amax = max(amax, s)
            for i in range(3):
                fy[:, b, i, a] = F[i]
            F, s = line_fluxes([cell(a, b, c) for c in range(-3, 5)], 2, gamma)  # z line at x=a, y=b
            amax = max(amax, s)
            for i in range(3):
                fz[:, i, b, a] = F[i]
    return fx, fy, fz, amax


@pytest.mark.parametrize("nf,seed", [(6, 1), (6, 2), (7, 3), (7, 4)])
def test_n2_sweeps_match_the_oracle(nf, seed):
    U = synth.iid_block(synth.rng_for(9090, seed), 2, nf)
    # larger velocities than the iid recipe, so that every term matters
    U[1:4] *= 8.0
    dx = 0.37
    fx, fy, fz, amax = block_sweeps(U, G53)
    out, oamax, flags, (ox, oy, oz) = oracle.rhs_block(U, 3, G53, dx, oracle.MODE_FP64, faces=True)
    assert flags == 0
    for mine, theirs in ((fx, ox), (fy, oy), (fz, oz)):
        scale = np.abs(theirs).max(axis=(1, 2, 3), keepdims=True)
        assert np.all(np.abs(mine - theirs) <= 1e-13 * scale)
    assert abs(amax - oamax) <= 1e-15 * oamax
    # divergence of the brute-force fluxes
    div = np.zeros((nf, 2, 2, 2))
    for z in range(2):
        for y in range(2):
            for x in range(2):
                Dx = fx[:, z, y, x + 1] - fx[:, z, y, x]
                Dy = fy[:, z, y + 1, x] - fy[:, z, y, x]
                Dz = fz[:, z + 1, y, x] - fz[:, z, y, x]
                div[:, z, y, x] = -((Dx + Dy) + Dz) / dx
    scale = np.abs(out).max(axis=(1, 2, 3), keepdims=True)
    assert np.all(np.abs(div - out) <= 1e-12 * scale)


def test_n2_sweep_sees_a_planted_index_error():
    """The comparison is sharp enough to see an off-by-one: shifting the brute
    force's x faces by one cell breaks the agreement."""
    U = synth.iid_block(synth.rng_for(9090, 5), 2, 6)
    U[1:4] *= 8.0
    fx, _, _, _ = block_sweeps(U, G53)
    _, _, _, (ox, _, _) = oracle.rhs_block(U, 3, G53, 0.37, oracle.MODE_FP64, faces=True)
    scale = np.abs(ox).max()
    assert np.abs(np.roll(fx, 1, axis=3) - ox).max() > 1e-6 * scale
    assert np.abs(fx.transpose(0, 2, 1, 3) - ox).max() > 1e-6 * scale
