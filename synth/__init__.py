"""Seeded synthetic inputs for the hydro RHS workloads.

This module is shared by the tests, the benchmark and the oracle checks; it
holds none of the RHS arithmetic (no primitive recovery, reconstruction, flux
or divergence).  It only draws states and writes them in conserved form
(rho, momentum, total energy E = p/(gamma-1) + rho|v|^2/2, entropy tracer
tau = (p/(gamma-1))^(1/gamma), species densities rho*X_k), laid out as
ghosted blocks ``[n_fields][N+2g][N+2g][N+2g]`` with x fastest.

The paper's benchmark scenario (Sedov blast wave on 262144 cells, 512
sub-grids of 8^3 or 64 of 16^3; Sec. VI-A, Table I) is generated by the
application itself, not read from a dataset; these generators stand in for it
with the shapes of the paper's workloads:

  one_subgrid      one 8^3 sub-grid, 6 fields, iid cell states
  plain_domain     a 64^3 periodic domain cut into 512 sub-grids of 8^3 (the
                   262144 cells of Table I), 11 fields, smooth random fields
  uneven_octree    4096 leaves of a 3-level octree, 75 % 8^3 / 25 % 16^3,
                   6 or 11 fields per leaf, iid cell states, shuffled order
  polytropes       a 256^3 periodic domain (32768 sub-grids of 8^3) holding
                   two n = 1.5 polytropes on a 1e-10 atmosphere, 11 fields
  serving_trace    Poisson arrivals of tasks of 1..64 sub-grids
  sedov_domain     the point explosion itself: a periodic cube of gas at rest
                   with the blast energy put into the 8 cells at its centre
                   (the scenario of Sec. VI-A, here with 5 passive species)
  forest_leaves    leaves of a 2:1 balanced octree forest over a periodic
                   cube (random or around-a-point refinement), and
  smooth_forest_state  smooth random fields sampled at the forest's cells
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 20221012
GAMMA = 5.0 / 3.0
MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) used to derive per-item seeds."""
    x = (x + 0x9E3779B97F4A7C15) & MASK64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def rng_for(seed: int, item: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(splitmix64((seed ^ item) & MASK64)))


# --------------------------------------------------------------- states --
def conserved_from_states(rho, vx, vy, vz, p, X=None, gamma=GAMMA):
    """Stack a state given as density, velocity, pressure and mass fractions
    into the conserved field order (rho, sx, sy, sz, E, tau, rho*X_k)."""
    eint = p / (gamma - 1.0)
    fields = [rho, rho * vx, rho * vy, rho * vz,
              eint + 0.5 * rho * (vx * vx + vy * vy + vz * vz),
              np.power(eint, 1.0 / gamma)]
    if X is not None:
        for k in range(X.shape[0]):
            fields.append(rho * X[k])
    return np.stack(fields).astype(np.float64)


def iid_block(rng, N, nf, ghost=3, gamma=GAMMA):
    """iid cell states: rho ~ U[0.5,2], v_d ~ N(0, 0.1), p ~ U[0.5,2],
    species mass fractions ~ Dirichlet(1, ..., 1)."""
    G = N + 2 * ghost
    shp = (G, G, G)
    rho = rng.uniform(0.5, 2.0, shp)
    v = rng.normal(0.0, 0.1, (3,) + shp)
    p = rng.uniform(0.5, 2.0, shp)
    nsp = nf - 6
    X = None
    if nsp > 0:
        X = np.moveaxis(rng.dirichlet(np.ones(nsp), size=shp), -1, 0)
    return conserved_from_states(rho, v[0], v[1], v[2], p, X, gamma)


def one_subgrid(seed=BASE_SEED, N=8, nf=6, gamma=GAMMA):
    """One 8^3 sub-grid with 3 ghost layers (14^3), 6 fields; dx = 1/8."""
    return iid_block(rng_for(seed, 0), N, nf, 3, gamma), 1.0 / N


def iid_batch(n, N=8, nf=6, seed=BASE_SEED, gamma=GAMMA):
    """n independent iid sub-grids (sub-grid s drawn from splitmix64(seed ^ s))."""
    return [iid_block(rng_for(seed, s), N, nf, 3, gamma) for s in range(n)]


# ------------------------------------------------------ periodic domains --
def gather_blocks(glob, N, ghost=3, blocks=None):
    """Cut a periodic global array [nf][n][n][n] into ghosted N^3 sub-grids.

    blocks: iterable of (bx, by, bz) block coordinates (default: all, z-major).
    Returns an array [n_blocks][nf][G][G][G]."""
    nf, n = glob.shape[0], glob.shape[1]
    nb = n // N
    if blocks is None:
        blocks = [(bx, by, bz) for bz in range(nb) for by in range(nb) for bx in range(nb)]
    blocks = list(blocks)
    G = N + 2 * ghost
    out = np.empty((len(blocks), nf, G, G, G))
    r = np.arange(-ghost, N + ghost)
    for b, (bx, by, bz) in enumerate(blocks):
        ix = (bx * N + r) % n
        iy = (by * N + r) % n
        iz = (bz * N + r) % n
        out[b] = glob[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]]
    return out


def _fourier_field(rng, n, modes=8, kmax=4):
    """Sum of `modes` random periodic Fourier modes with wave numbers 1..kmax."""
    x = (np.arange(n) + 0.5) / n
    f = np.zeros((n, n, n))
    for _ in range(modes):
        k = rng.integers(-kmax, kmax + 1, 3)
        if not k.any():
            k[0] = 1
        ph = rng.uniform(0, 2 * np.pi)
        amp = rng.normal()
        f += amp * np.cos(2 * np.pi * (k[0] * x[None, None, :] + k[1] * x[None, :, None]
                                       + k[2] * x[:, None, None]) + ph)
    return f


def _rescale(f, lo, hi):
    return lo + (hi - lo) * (f - f.min()) / max(f.max() - f.min(), 1e-300)


def plain_domain(seed=BASE_SEED, n=64, nf=11, gamma=GAMMA):
    """64^3 periodic domain of smooth random fields (8 Fourier modes each,
    wave numbers 1-4): rho, p rescaled into [0.5, 2], velocity with standard
    deviation 0.1; species ~ Dirichlet(1) per cell.  dx = 1/n.
    Returns the global conserved array [nf][n][n][n]."""
    rng = rng_for(seed, 2)
    rho = _rescale(_fourier_field(rng, n), 0.5, 2.0)
    v = []
    for _ in range(3):
        f = _fourier_field(rng, n)
        v.append(0.1 * (f - f.mean()) / max(f.std(), 1e-300))
    p = _rescale(_fourier_field(rng, n), 0.5, 2.0)
    X = None
    if nf > 6:
        X = np.moveaxis(rng.dirichlet(np.ones(nf - 6), size=(n, n, n)), -1, 0)
    return conserved_from_states(rho, v[0], v[1], v[2], p, X, gamma)


def polytropes(seed=BASE_SEED, n=256, nf=11, gamma=GAMMA, dtype=np.float64):
    """Two n = 1.5 polytropes on [-1, 1]^3 (periodic), n^3 cells, dx = 2/n.

    rho = max(rho_c (1 - (r/R)^2)^1.5, 1e-10) around centres (+-0.45, 0, 0)
    with R = 0.35 and 0.25, rho_c = 1; p = K rho^(5/3), K = 0.6; rigid
    rotation v = Omega z x r with Omega = 0.3/0.45; species: one Dirichlet(1)
    draw per region (star A, star B, atmosphere) blended with the regions'
    density weights.  Returns the global conserved array [nf][n][n][n]."""
    rng = rng_for(seed, 4)
    dx = 2.0 / n
    c = -1.0 + (np.arange(n) + 0.5) * dx
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    K, floor, omega = 0.6, 1e-10, 0.3 / 0.45

    def profile(cx, R):
        r2 = ((x - cx) ** 2 + y ** 2 + z ** 2) / (R * R)
        return np.where(r2 < 1.0, np.power(np.clip(1.0 - r2, 0.0, None), 1.5), 0.0)

    wa = profile(0.45, 0.35)
    wb = profile(-0.45, 0.25)
    rho = np.maximum(wa + wb, floor)
    p = K * np.power(rho, 5.0 / 3.0)
    vx = -omega * y
    vy = omega * x
    vz = np.zeros_like(x)
    X = None
    nsp = nf - 6
    if nsp > 0:
        XA, XB, XC = (rng.dirichlet(np.ones(nsp)) for _ in range(3))
        wsum = wa + wb + floor
        X = (XA[:, None, None, None] * wa + XB[:, None, None, None] * wb
             + XC[:, None, None, None] * floor) / wsum
    U = conserved_from_states(rho, vx, vy, vz, p, X, gamma)
    return U.astype(dtype, copy=False)


# ---------------------------------------------------------------- octree --
def uneven_octree(seed=BASE_SEED, gamma=GAMMA, n_subgrids=None):
    """Leaves of a synthetic 3-level octree forest.

    1072 level-0 nodes of width 1/16: 1024 are leaves holding 16^3 sub-grids
    (dx = 1/256); 48 are refined twice (48 -> 384 -> 3072 leaves of width
    1/64 holding 8^3 sub-grids, dx = 1/512).  4096 leaves: 75 % 8^3, 25 %
    16^3; each leaf has 6 or 11 fields (Bernoulli 0.5); iid cell states; the
    batch order is shuffled.  Returns a list of (N, nf, dx, seed_item) tuples;
    call ``leaf_block`` to draw a leaf's data.  ``n_subgrids`` keeps a prefix
    of the shuffled list (smaller test batches with the same mix)."""
    rng = rng_for(seed, 3)
    leaves = [(16, 1.0 / 256)] * 1024 + [(8, 1.0 / 512)] * 3072
    nf = np.where(rng.random(len(leaves)) < 0.5, 6, 11)
    order = rng.permutation(len(leaves))
    out = [(leaves[i][0], int(nf[i]), leaves[i][1], int(i)) for i in order]
    if n_subgrids is not None:
        out = out[:n_subgrids]
    return out


def leaf_block(seed, leaf, gamma=GAMMA):
    N, nf, dx, item = leaf
    return iid_block(rng_for(seed, 1000 + item), N, nf, 3, gamma)


# --------------------------------------------------------------- serving --
def serving_trace(seed=BASE_SEED, rate=20000.0, duration=1.0, max_subgrids=64,
                  f_range=(6, 11)):
    """Poisson arrivals at `rate` tasks/s over `duration` s; each task holds
    U{1..max_subgrids} sub-grids of 8^3 with U{f_range} fields.
    Returns (arrival_times [s], n_subgrids per task, n_fields per task)."""
    rng = rng_for(seed, 5)
    n_est = int(rate * duration * 1.2 + 100)
    gaps = rng.exponential(1.0 / rate, n_est)
    t = np.cumsum(gaps)
    while t[-1] < duration:
        t = np.concatenate([t, t[-1] + np.cumsum(rng.exponential(1.0 / rate, n_est))])
    t = t[t < duration]
    sizes = rng.integers(1, max_subgrids + 1, t.size)
    nfs = rng.integers(f_range[0], f_range[1] + 1, t.size)
    return t, sizes, nfs


# ----------------------------------------------------------- bookkeeping --
def ghost_cells(N, ghost=3):
    """Ghost cells stored per sub-grid: (N+2g)^3 - N^3 (Table I)."""
    return (N + 2 * ghost) ** 3 - N ** 3


def star_cells(N, ghost=3):
    """Cells the scheme reads: interior plus 3-deep slabs on the six faces."""
    return N ** 3 + 6 * ghost * N * N


def algorithmic_bytes(N, nf, ghost=3):
    """Bytes per RHS of one sub-grid: read the star region once, write dU/dt
    once, write one double of signal speed."""
    return (star_cells(N, ghost) + N ** 3) * nf * 8 + 8


def kernel_calls_per_step(n_subgrids, kernels=5, iterations=3):
    """Launch count per time step of the non-aggregated code (Table I)."""
    return n_subgrids * kernels * iterations


def is_power_of_two_fraction(x):
    m, e = math.frexp(x)
    return m == 0.5


# ---------------------------------------------------------------- Sedov --
def sedov_domain(n=64, nf=11, gamma=GAMMA, E=1.0, rho0=1.0, p0=1e-5, seed=BASE_SEED):
    """Point explosion on the periodic cube [-1/2, 1/2]^3 with n^3 cells
    (dx = 1/n, n even): gas at rest with density rho0 and pressure p0, and the
    energy E added as internal energy, evenly, to the 2^3 cells that touch the
    centre.  Species (nf - 6 of them) carry uniform mass fractions drawn from a
    Dirichlet(1) distribution.  Returns (global array [nf][n][n][n], dx)."""
    if n % 2:
        raise ValueError("n must be even (the centre is a cell corner)")
    dx = 1.0 / n
    shp = (n, n, n)
    rho = np.full(shp, rho0)
    p = np.full(shp, p0)
    c = n // 2
    p[c - 1:c + 1, c - 1:c + 1, c - 1:c + 1] += (gamma - 1.0) * E / (8.0 * dx ** 3)
    X = None
    if nf > 6:
        x = rng_for(seed, 0xB1A57).dirichlet(np.ones(nf - 6))
        X = np.broadcast_to(x[:, None, None, None], (nf - 6,) + shp).copy()
    zero = np.zeros(shp)
    return conserved_from_states(rho, zero, zero, zero, p, X, gamma), dx


def cell_radii(n):
    """Distance of every cell centre of sedov_domain's cube from its centre."""
    x = (np.arange(n) + 0.5) / n - 0.5
    return np.sqrt(x[None, None, :] ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2)


# --------------------------------------------------------------- forests --
def _leaf_hash(seed, level, bx, by, bz):
    """Uniform number in [0, 1) fixed by the seed and the block (order-free)."""
    h = splitmix64((seed ^ (level << 60) ^ (bx << 40) ^ (by << 20) ^ bz) & MASK64)
    return (h >> 11) / float(1 << 53)


def forest_leaves(nb0, max_level, refine, seed=BASE_SEED, shuffle=True, balance="face"):
    """Leaves of a 2:1 face-balanced octree forest over the periodic unit cube
    cut into nb0^3 root blocks.

    refine(level, corner (x, y, z), width) -> bool says whether a block (unit-
    cube coordinates) is split; blocks at max_level are never split.  After
    that, any leaf with a face neighbour two or more levels finer is split
    until none is left (periodic neighbours included), so face neighbours
    differ by at most one level; balance="full" extends this to the edge and
    corner neighbours (all 26).  Returns an int32 array [n][4] of
    (level, bx, by, bz), block coordinates at the leaf's level in
    [0, nb0 2^level); shuffled by the seed unless shuffle is False (then
    sorted by level, bz, by, bx)."""
    leaves = set()
    stack = [(0, bx, by, bz) for bz in range(nb0) for by in range(nb0) for bx in range(nb0)]
    while stack:
        L, bx, by, bz = stack.pop()
        w = 1.0 / (nb0 << L)
        if L < max_level and refine(L, (bx * w, by * w, bz * w), w):
            stack.extend((L + 1, 2 * bx + i, 2 * by + j, 2 * bz + k)
                         for k in (0, 1) for j in (0, 1) for i in (0, 1))
        else:
            leaves.add((L, bx, by, bz))

    def covering(L, b):
        for l in range(L, -1, -1):
            key = (l,) + tuple(c >> (L - l) for c in b)
            if key in leaves:
                return key
        return None

    offsets = [o for o in ((i, j, k) for k in (-1, 0, 1) for j in (-1, 0, 1) for i in (-1, 0, 1))
               if (sum(map(abs, o)) == 1 if balance == "face" else any(o))]
    changed = True
    while changed:
        changed = False
        for leaf in sorted(leaves):
            if leaf not in leaves:
                continue
            L, b = leaf[0], leaf[1:]
            m = nb0 << L
            for o in offsets:
                q = [(b[e] + o[e]) % m for e in range(3)]
                c = covering(L, q)
                if c is not None and c[0] < L - 1:
                    leaves.discard(c)
                    cl, cb = c[0], c[1:]
                    for k in (0, 1):
                        for j in (0, 1):
                            for i in (0, 1):
                                leaves.add((cl + 1, 2 * cb[0] + i, 2 * cb[1] + j, 2 * cb[2] + k))
                    changed = True
    out = np.array(sorted(leaves, key=lambda t: (t[0], t[3], t[2], t[1])), dtype=np.int32).reshape(-1, 4)
    if shuffle:
        out = out[rng_for(seed, 0xF0CE57).permutation(len(out))]
    return out


def random_refine(seed, prob):
    """refine() predicate for forest_leaves: split a block with probability
    `prob`, decided by a hash of the seed and the block."""
    def f(level, corner, width):
        b = tuple(int(round(c / width)) for c in corner)
        return _leaf_hash(seed, level, *b) < prob
    return f


def sphere_refine(centre, radii):
    """refine() predicate: split a level-L block if it reaches within radii[L]
    of `centre` (periodic unit cube); refinement around a point, as a
    simulation refines around a blast or a star."""
    def f(level, corner, width):
        if level >= len(radii):
            return False
        d2 = 0.0
        for c, x0 in zip(corner, centre):
            # distance from the centre to the block along one axis, periodic
            lo = (c - x0) % 1.0
            hi = (x0 - c - width) % 1.0
            d = 0.0 if lo + width >= 1.0 or hi + width >= 1.0 else min(lo, hi)
            d2 += d * d
        return d2 < radii[level] ** 2
    return f


def forest_cell_centres(leaves, nb0, N):
    """Cell centres (unit-cube coordinates) of every leaf: array [n][3][N][N][N]
    (x, y, z) in the storage order [z][y][x]."""
    leaves = np.asarray(leaves).reshape(-1, 4)
    out = np.empty((len(leaves), 3, N, N, N))
    r = np.arange(N) + 0.5
    for s, (L, bx, by, bz) in enumerate(leaves):
        w = 1.0 / ((nb0 << int(L)) * N)
        out[s, 0] = ((bx * N + r) * w)[None, None, :]
        out[s, 1] = ((by * N + r) * w)[None, :, None]
        out[s, 2] = ((bz * N + r) * w)[:, None, None]
    return out


def smooth_forest_state(leaves, nb0, N, nf=11, seed=BASE_SEED, gamma=GAMMA):
    """Smooth periodic random fields sampled at the cell centres of a forest:
    rho and p = 1.25 + 0.75 f with f a sum of 6 Fourier modes (wave numbers
    1-3) normalised to |f| <= 1, so rho, p in [0.5, 2]; each velocity
    component 0.1 g (g likewise in [-1, 1]); species Dirichlet(1) per cell.
    Returns U [n_leaves][nf][N][N][N] (no ghost layers) and the root-level
    cell width dx0 = 1 / (nb0 N)."""
    rng = rng_for(seed, 0xF0E57)
    xyz = forest_cell_centres(leaves, nb0, N)

    def field():
        f = np.zeros(xyz.shape[:1] + xyz.shape[2:])
        amps = rng.normal(size=6)
        amps /= np.abs(amps).sum()
        for a in amps:
            k = rng.integers(-3, 4, 3)
            if not k.any():
                k[0] = 1
            ph = rng.uniform(0, 2 * np.pi)
            f += a * np.cos(2 * np.pi * (k[0] * xyz[:, 0] + k[1] * xyz[:, 1] + k[2] * xyz[:, 2]) + ph)
        return f

    rho = 1.25 + 0.75 * field()
    v = [0.1 * field() for _ in range(3)]
    p = 1.25 + 0.75 * field()
    X = None
    if nf > 6:
        X = np.moveaxis(rng.dirichlet(np.ones(nf - 6), size=rho.shape), -1, 0)
    U = conserved_from_states(rho, v[0], v[1], v[2], p, X, gamma)  # [nf][n][N][N][N]
    return np.ascontiguousarray(np.moveaxis(U, 0, 1)), 1.0 / (nb0 * N)


def sedov_forest(nb0=2, N=8, radii=(0.45, 0.25), nf=11, gamma=GAMMA, E=1.0, rho0=1.0, p0=1e-5,
                 seed=BASE_SEED):
    """The point explosion of sedov_domain on a forest refined around the
    centre of the periodic unit cube (sphere_refine with the given radii, so
    len(radii) levels of refinement at the centre): gas at rest, rho0, p0,
    and the energy E added as internal energy, evenly, to the 8 finest cells
    that touch the centre.  Returns (leaves, U [n][nf][N][N][N], dx0)."""
    leaves = forest_leaves(nb0, len(radii), sphere_refine((0.5, 0.5, 0.5), radii), seed=seed)
    xyz = forest_cell_centres(leaves, nb0, N)
    n = len(leaves)
    shp = (n, N, N, N)
    rho = np.full(shp, rho0)
    p = np.full(shp, p0)
    lmax = int(leaves[:, 0].max())
    dxf = 1.0 / ((nb0 << lmax) * N)
    near = np.all(np.abs(xyz - 0.5) < 0.75 * dxf, axis=1) & (leaves[:, 0] == lmax)[:, None, None, None]
    if near.sum() != 8:
        raise ValueError("the centre is not refined to the finest level")
    p[near] += (gamma - 1.0) * E / (8.0 * dxf ** 3)
    X = None
    if nf > 6:
        x = rng_for(seed, 0xB1A57).dirichlet(np.ones(nf - 6))
        X = np.broadcast_to(x[:, None, None, None, None], (nf - 6,) + shp).copy()
    zero = np.zeros(shp)
    U = conserved_from_states(rho, zero, zero, zero, p, X, gamma)
    return leaves, np.ascontiguousarray(np.moveaxis(U, 0, 1)), 1.0 / (nb0 * N)
