"""Cell states around the dual-energy switch (the reading of Sec. IV-B's
entropy tracer: e = E - |s|^2/(2 rho); where e < eta E the tracer gives
e = tau^gamma, eta = 1e-3).

Each state is built from rho and s with E placed at a chosen internal-to-total
energy ratio r = e/E, or at the last binary64 values on either side of the
switch as the binary64 definition evaluates it (E - (0.5 |s|^2)/rho against
eta*E, in that order of operations).  tau is inconsistent on purpose:
tau^gamma = k e with k = 4 or 1/4, so the two branches give pressures a factor
k apart and a branch taken differently shows as a large difference.

Test infrastructure: used by the oracle pin in test_oracle_pins and by the GPU
parity test of the switch window.
"""
from __future__ import annotations

import struct

import numpy as np

ETA = 1e-3
GAMMA = 5.0 / 3.0

# ratios e/E: far on both sides, the edges of the window in which the GPU
# re-evaluates the branch in the reference order (eta/2, 20 eta, and 1/4 for
# the binary32 form's internal energy), and within 2^-40 of the threshold
RATIOS = [5e-4, 2e-3,
          0.5 * ETA * (1 - 2.0 ** -52), 0.5 * ETA, 0.5 * ETA * (1 + 2.0 ** -52),
          20 * ETA * (1 - 2.0 ** -52), 20 * ETA, 20 * ETA * (1 + 2.0 ** -52),
          0.25 * (1 - 2.0 ** -30), 0.25, 0.25 * (1 + 2.0 ** -30),
          ETA * (1 - 2.0 ** -40), ETA * (1 + 2.0 ** -40)]
# binary64 steps from the first unswitched E (straddle_E): -2 and -1 are the
# two largest E that switch, 0 and 1 the two smallest that do not
STRADDLE = [-2, -1, 0, 1]


def _bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _flt(b):
    return struct.unpack("<d", struct.pack("<q", b))[0]


def eint_reference(rho, s1, s2, s3, E):
    """e = E - (0.5 |s|^2)/rho in the binary64 definition's order."""
    ssq = (s1 * s1 + s2 * s2) + s3 * s3
    return E - (0.5 * ssq) / rho


def switched(rho, s1, s2, s3, E):
    return eint_reference(rho, s1, s2, s3, E) < ETA * E


def straddle_E(rho, s1, s2, s3):
    """The smallest binary64 E for which the switch is not taken (so E with
    one binary64 step less is the largest for which it is)."""
    ssq = (s1 * s1 + s2 * s2) + s3 * s3
    ekin = (0.5 * ssq) / rho
    lo = ekin / (1.0 - ETA) * (1 - 1e-12)
    hi = ekin / (1.0 - ETA) * (1 + 1e-12)
    assert switched(rho, s1, s2, s3, lo) and not switched(rho, s1, s2, s3, hi)
    a, b = _bits(lo), _bits(hi)
    while b - a > 1:
        m = (a + b) // 2
        if switched(rho, s1, s2, s3, _flt(m)):
            a = m
        else:
            b = m
    return _flt(b)


def case_states(rng, n, low_density=False, gamma=GAMMA):
    """n cell states (rho, s1, s2, s3, E, tau) cycling over every ratio case
    and every straddle step.  Returns (states [n][6], expected_switch [n])."""
    cases = [("r", r) for r in RATIOS] + [("k", k) for k in STRADDLE]
    out = np.empty((n, 6))
    sw = np.empty(n, dtype=bool)
    for i in range(n):
        kind, val = cases[i % len(cases)]
        rho = float(rng.uniform(0.5, 2.0)) * (1e-10 if low_density else 1.0)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        vmag = float(rng.uniform(0.3, 1.5))
        s1, s2, s3 = (float(rho * vmag * c) for c in d)
        ekin = (0.5 * ((s1 * s1 + s2 * s2) + s3 * s3)) / rho
        if kind == "r":
            E = ekin / (1.0 - val)
        else:
            E = _flt(_bits(straddle_E(rho, s1, s2, s3)) + val)
        e = max(E - ekin, 1e-300)
        k = 4.0 if rng.uniform() < 0.5 else 0.25
        tau = (k * e) ** (1.0 / gamma)
        out[i] = (rho, s1, s2, s3, E, tau)
        sw[i] = switched(rho, s1, s2, s3, E)
    return out, sw


def window_block(rng, N=8, nf=6, ghost=3, low_density=False, gamma=GAMMA):
    """A ghosted block [nf][G][G][G] whose every cell is a switch-window state
    (species: rho times Dirichlet(1) fractions)."""
    G = N + 2 * ghost
    st, _ = case_states(rng, G ** 3, low_density, gamma)
    rng.shuffle(st)
    U = np.empty((nf, G, G, G))
    for f in range(6):
        U[f] = st[:, f].reshape(G, G, G)
    if nf > 6:
        X = rng.dirichlet(np.ones(nf - 6), size=G ** 3)
        for k in range(nf - 6):
            U[6 + k] = (st[:, 0] * X[:, k]).reshape(G, G, G)
    return U


def uniform_block(state, N=8, nf=6, ghost=3):
    """A block whose every cell holds one state (species 1/(nf-6) each)."""
    G = N + 2 * ghost
    U = np.empty((nf, G, G, G))
    for f in range(6):
        U[f] = state[f]
    for k in range(6, nf):
        U[k] = state[0] / (nf - 6)
    return U
