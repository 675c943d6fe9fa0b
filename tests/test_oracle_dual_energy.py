"""Pin of the oracle's dual-energy switch to the last binary64 step.

A block holding one state everywhere has zero dU/dt and largest signal speed
a = max_d |v_d| + sqrt(gamma p / rho), with p = (gamma - 1) e and e from the
branch the switch takes.  The states of tests/dual_energy_cases.py put E at
ratios e/E on both sides of eta = 1e-3 and at the last binary64 values on
either side of the switch, with an inconsistent tracer (tau^gamma = 4e or e/4),
so the two branches give signal speeds at least 1e-3 apart: the oracle's amax
shows which one it took, in both precision modes."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import dual_energy_cases as dec

G53 = 5.0 / 3.0


def _expected_amax(state, switched, gamma=G53):
    rho, s1, s2, s3, E, tau = state
    e = tau ** gamma if switched else dec.eint_reference(rho, s1, s2, s3, E)
    p = (gamma - 1.0) * e
    return max(abs(s1 / rho), abs(s2 / rho), abs(s3 / rho)) + math.sqrt(gamma * p / rho)


@pytest.mark.parametrize("low_density", [False, True])
def test_switch_is_taken_exactly_where_the_definition_puts_it(low_density):
    rng = synth.rng_for(4242, int(low_density))
    states, sw = dec.case_states(rng, 2 * (len(dec.RATIOS) + len(dec.STRADDLE)), low_density)
    # the straddle states do sit on both sides of the switch
    k = len(dec.RATIOS)
    assert list(sw[k:k + 4]) == [True, True, False, False]
    for st, s in zip(states, sw):
        U = dec.uniform_block(st, N=2, nf=7)
        for mode in (oracle.MODE_FP64, oracle.MODE_MIXED):
            out, amax, flags = oracle.rhs_block(U, 3, G53, 0.5, mode)
            assert flags == 0
            assert np.all(out == 0.0)
            want = _expected_amax(st, s)
            other = _expected_amax(st, not s)
            assert abs(other - want) > 1e-3 * want  # far beyond either tolerance
            tol = 1e-14 if mode == oracle.MODE_FP64 else 2e-6
            assert abs(amax - want) <= tol * want, (mode, s, amax, want, other)


def test_straddle_states_are_adjacent_binary64_values():
    rng = synth.rng_for(4243)
    for _ in range(20):
        rho = float(rng.uniform(0.5, 2.0))
        s = [float(x) for x in rng.normal(size=3)]
        Eb = dec.straddle_E(rho, *s)
        below = np.nextafter(Eb, 0.0)
        assert not dec.switched(rho, *s, Eb)
        assert dec.switched(rho, *s, below)
