"""Pin of the mixed mode's primitive reading: the conserved values are
rounded to binary32 (to nearest, ties to even) and v = s/rho is a binary32
quotient of the rounded values; p = (gamma-1) e with e from the binary64
definition, rounded to binary32.

In a block holding one state, PPM returns the cell values unchanged and the
signal speed of the mixed mode is the binary32 value max_d |v_d| +
sqrt(gamma p / rho).  For states where the binary32 quotient of the rounded
values and the rounded binary64 quotient differ, the two readings give
different signal speeds, and the oracle's must be the first."""
import numpy as np

import oracle
import synth
from tests import dual_energy_cases as dec

f32 = np.float32
G53 = 5.0 / 3.0


def _amax32(rho32, v32, p32, gamma=G53):
    cs = np.sqrt(f32(gamma) * p32 / rho32)
    return max(abs(v) + cs for v in v32)


def test_mixed_mode_forms_binary32_quotients_of_rounded_values():
    rng = synth.rng_for(31337)
    found = 0
    while found < 12:
        rho = float(rng.uniform(0.5, 2.0))
        s = [float(x) for x in rng.normal(size=3) * 3.0]
        if f32(s[0]) / f32(rho) == f32(s[0] / rho):
            continue
        v = [x / rho for x in s]
        p = float(rng.uniform(0.5, 2.0))
        E = p / (G53 - 1.0) + 0.5 * rho * sum(x * x for x in v)
        tau = (p / (G53 - 1.0)) ** (1.0 / G53)
        state = (rho, s[0], s[1], s[2], E, tau)
        U = dec.uniform_block(state, N=2, nf=6)
        out, amax, flags = oracle.rhs_block(U, 3, G53, 0.5, oracle.MODE_MIXED)
        assert flags == 0 and np.all(out == 0.0)
        e = dec.eint_reference(*state[:5])
        p32 = f32((G53 - 1.0) * e)
        mine = _amax32(f32(rho), [f32(x) / f32(rho) for x in s], p32)
        other = _amax32(f32(rho), [f32(x / rho) for x in s], p32)
        assert amax == float(mine), (amax, mine)
        if mine != other:
            found += 1
