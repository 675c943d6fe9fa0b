"""Oracle for the RHS of a multi-level forest of sub-grids (adaptive mesh).

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/``, only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it.  It
shares no code with the CUDA path: the ghost cells are located here by a
search over the leaves, not from the library's neighbour links.

A forest is a set of leaves (level L, bx, by, bz) of an octree over a
periodic cube of nb0^3 root blocks; every leaf holds N^3 cells of width
dx0 / 2^L, stored without ghost layers, U[s][f][z][y][x].  Its block
coordinates run over [0, nb0 2^L).

The paper's application discretises the fluid on a Cartesian adaptively
refined mesh and conserves mass, momentum and energy to machine precision
(Sec. III), but it states no formulas for the coupling of the levels.  The
readings taken here:

1. Ghost values.  A ghost cell of a level-L leaf takes the volume average,
   over that cell, of the composite field (the field that is constant on
   every cell of every leaf).  If a single leaf cell of level <= L contains
   it, that cell's value is taken (same level: a copy; coarser: piecewise
   constant prolongation).  Otherwise it is the mean of the averages of its
   eight children (restriction), added in the order k = i + 2 j + 4 k of the
   child offsets and multiplied by 1/8.
2. Each leaf's RHS is the single-block oracle on its ghosted block (face-
   centre scheme or the 26-point variant, Kurganov-Tadmor or Kurganov-
   Noelle-Petrova flux, binary64 or mixed).  The face-centre scheme reads
   the face ghost slabs only; the 26-point variant also reads edge and
   corner ghosts (every cell with each coordinate in [-3, N+2] and at most
   one of them at -3 or N+2), filled by the same rule.
3. Flux correction.  Where a level-L leaf meets four level-(L+1) leaves
   across a face, the flux through each coarse cell face is replaced by the
   area mean of the four fine fluxes through it (added in the order (0,0),
   (1,0), (0,1), (1,1) of the two tangential fine offsets, times 1/4):
   dU/dt += s (mean - F_coarse) / dx_L, s = +1 at the leaf's low face and
   -1 at its high face; the corrections of the x, y and z faces are added in
   that order.  Every face flux then enters once with each sign, so the sum
   of dU/dt dx_L^3 over all cells vanishes up to rounding.

Tangential axes of a face normal to d: (y, z) for x, (x, z) for y, (x, y)
for z.
"""
from __future__ import annotations

import numpy as np

from . import rhs_block

_TANG = ((1, 2), (0, 2), (0, 1))


class Forest:
    """Leaf lookup of a forest (a dict from (level, bx, by, bz) to the leaf)."""

    def __init__(self, leaves, nb0, N):
        self.leaves = np.asarray(leaves, dtype=np.int64).reshape(-1, 4)
        self.nb0, self.N = int(nb0), int(N)
        self.index = {tuple(int(v) for v in l): s for s, l in enumerate(self.leaves)}
        if len(self.index) != len(self.leaves):
            raise ValueError("duplicate leaves")

    def cells(self, L):
        """Cells per edge of the cube at level L."""
        return (self.nb0 << L) * self.N

    def leaf_at(self, L, g):
        """The leaf holding level-L cell g (global integer triple, wrapped
        periodically): (s, l, level-l cell index) for the leaf of level l <= L
        that contains it, or None when finer leaves cover it."""
        n = self.cells(L)
        g = tuple(int(c) % n for c in g)
        for l in range(L, -1, -1):
            c = tuple(v >> (L - l) for v in g)
            s = self.index.get((l,) + tuple(v // self.N for v in c))
            if s is not None:
                return s, l, c
        return None

    def local(self, s, c):
        """Local (x, y, z) of level cell c inside leaf s."""
        b = self.leaves[s, 1:]
        return tuple(int(c[d] - b[d] * self.N) for d in range(3))


def cell_average(forest, U, L, g):
    """Volume average of the composite field over level-L cell g (reading 1):
    a vector of n_fields values."""
    hit = forest.leaf_at(L, g)
    if hit is not None:
        s, _, c = hit
        x, y, z = forest.local(s, c)
        return U[s][:, z, y, x].astype(np.float64)
    acc = None
    for k in range(8):
        child = (2 * g[0] + (k & 1), 2 * g[1] + ((k >> 1) & 1), 2 * g[2] + (k >> 2))
        v = cell_average(forest, U, L + 1, child)
        acc = v if acc is None else acc + v
    return acc * 0.125


def ghosted_block(forest, U, s, ghost=3, quad26=False):
    """Leaf s with its ghost cells filled by reading 1: the face slabs
    (ghost layers deep) and, with quad26, the edge and corner cells the
    26-point variant reads; other ghost cells are zero.  Returns
    [nf][G][G][G]."""
    N = forest.N
    L = int(forest.leaves[s, 0])
    b = forest.leaves[s, 1:]
    nf = U[s].shape[0]
    G = N + 2 * ghost
    out = np.zeros((nf, G, G, G))
    out[:, ghost:ghost + N, ghost:ghost + N, ghost:ghost + N] = U[s]
    if quad26:
        r = range(-3, N + 3)
        for z in r:
            for y in r:
                for x in r:
                    c = (x, y, z)
                    if all(0 <= v < N for v in c):
                        continue
                    if sum(v in (-3, N + 2) for v in c) > 1:
                        continue
                    g = tuple(int(b[e]) * N + c[e] for e in range(3))
                    out[:, z + ghost, y + ghost, x + ghost] = cell_average(forest, U, L, g)
        return out
    for d in range(3):
        ta, tb = _TANG[d]
        for side in (0, 1):
            for depth in range(1, ghost + 1):
                cd = -depth if side == 0 else N - 1 + depth
                for jb in range(N):
                    for ja in range(N):
                        c = [0, 0, 0]
                        c[d], c[ta], c[tb] = cd, ja, jb
                        g = tuple(int(b[e]) * N + c[e] for e in range(3))
                        out[:, c[2] + ghost, c[1] + ghost, c[0] + ghost] = cell_average(forest, U, L, g)
    return out


def _face_flux(faces, d, c, i):
    """Flux vector through face i along d of the cell column through local c."""
    x, y, z = c
    if d == 0:
        return faces[0][:, z, y, i]
    if d == 1:
        return faces[1][:, z, i, x]
    return faces[2][:, i, y, x]


def rhs(leaves, nb0, U, dx0, gamma=5.0 / 3.0, mode=0, only=None):
    """dU/dt of every leaf (list of [nf][N][N][N]) and amax per leaf, with
    the flux correction of reading 3.  mode: the oracle's mode bits (binary32
    reconstruction and flux, one-sided flux, the 26-point variant).
    only: a list of leaves; then only those are evaluated (with the face
    fluxes of their finer neighbours for the correction) and the results are
    dicts keyed by leaf."""
    U = [np.asarray(u, dtype=np.float64) for u in U]
    N = U[0].shape[-1]
    fo = Forest(leaves, nb0, N)
    n = len(fo.leaves)
    cache = {}

    def leaf(s):
        """(uncorrected dU/dt, amax, face fluxes) of leaf s."""
        if s not in cache:
            dx = dx0 / (1 << int(fo.leaves[s, 0]))
            o, a, flags, fc = rhs_block(ghosted_block(fo, U, s, quad26=bool(mode & 4)), 3, gamma, dx, mode,
                                        faces=True)
            if flags:
                raise ValueError("oracle flagged leaf %d (flags %d)" % (s, flags))
            cache[s] = (o, a, fc)
        return cache[s]

    def corrected(s):
        """Reading 3: corrections at faces towards finer leaves, x then y then z."""
        o, a, fcs = leaf(s)
        L = int(fo.leaves[s, 0])
        b = fo.leaves[s, 1:]
        dx = dx0 / (1 << L)
        corr = [np.zeros_like(o) for _ in range(3)]
        for d in range(3):
            ta, tb = _TANG[d]
            for side in (0, 1):
                sgn = 1.0 if side == 0 else -1.0
                for jb in range(N):
                    for ja in range(N):
                        c = [0, 0, 0]
                        c[d], c[ta], c[tb] = (0 if side == 0 else N - 1), ja, jb
                        beyond = list(int(b[e]) * N + c[e] for e in range(3))
                        beyond[d] += -1 if side == 0 else 1
                        if fo.leaf_at(L, beyond) is not None:
                            continue  # same level or coarser: nothing to correct here
                        Fc = _face_flux(fcs, d, c, 0 if side == 0 else N)
                        acc = None
                        for t in range(4):
                            gf = [2 * v for v in beyond]
                            gf[d] += 1 if side == 0 else 0  # the fine cells touching the face
                            gf[ta] += t & 1
                            gf[tb] += t >> 1
                            hit = fo.leaf_at(L + 1, gf)
                            if hit is None or hit[1] != L + 1:
                                raise ValueError("forest is not 2:1 balanced at leaf %d" % s)
                            sf, _, cf = hit
                            Ff = _face_flux(leaf(sf)[2], d, fo.local(sf, cf), N if side == 0 else 0)
                            acc = Ff.copy() if acc is None else acc + Ff
                        mean = acc * 0.25
                        corr[d][:, c[2], c[1], c[0]] = sgn * (mean - Fc) / dx
        for d in range(3):
            o = o + corr[d]
        return o, a

    if only is not None:
        res = {s: corrected(int(s)) for s in only}
        return {s: r[0] for s, r in res.items()}, {s: r[1] for s, r in res.items()}
    outs, amax = [], np.zeros(n)
    for s in range(n):
        leaf(s)
    for s in range(n):
        o, amax[s] = corrected(s)
        outs.append(o)
    return outs, amax


def stage(leaves, nb0, U, U0, alpha, beta, dt, dx0, gamma=5.0 / 3.0, mode=0):
    """One explicit stage U_out = alpha U0 + beta (U + dt dU/dt) of every leaf."""
    dU, amax = rhs(leaves, nb0, U, dx0, gamma, mode)
    out = [alpha * np.asarray(u0) + beta * (np.asarray(u) + dt * du) for u, u0, du in zip(U, U0, dU)]
    return out, amax
