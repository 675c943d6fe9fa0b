"""GPU parity at the dual-energy switch (Sec. IV-B's entropy tracer; the
reading e = E - |s|^2/(2 rho), e -> tau^gamma where e < 1e-3 E).

The kernels decide the branch from a fast estimate and re-evaluate it in the
reference order of operations near the threshold (binary64: within
[eta/2, 20 eta] E; mixed form: the binary32 internal energy is replaced by the
binary64 one below E/4).  These tests feed states at the edges of those
windows, within 2^-40 of the threshold and at the last binary64 values on
either side of it (tests/dual_energy_cases.py), with an inconsistent tracer so
that a branch taken differently from the oracle changes the pressure by a
factor 4:
  * blocks of one state each: dU/dt is exactly zero and the signal speed
    shows the branch; it must equal the oracle's (1e-14 binary64, 1e-6 mixed);
  * blocks mixing all states (ordinary and 1e-10 densities, 6 and 11 fields)
    against the oracle under the standard tolerances of both forms.
"""
import numpy as np
import pytest

import paper_2210_06438_gb300 as hydro
import synth
from tests import dual_energy_cases as dec
from tests import gpu_helpers as gh

pytestmark = pytest.mark.gpu
MIXED_FLAGS = [0, hydro.F_REGISTER_LOADS]


def _states():
    out = []
    for low in (False, True):
        st, sw = dec.case_states(synth.rng_for(515, int(low)), 2 * (len(dec.RATIOS) + len(dec.STRADDLE)), low)
        out += [(s, w) for s, w in zip(st, sw)]
    return out


@pytest.mark.parametrize("prec,flags", [(hydro.FP64, 0)] + [(hydro.FP32_FLUX_FP64_ACC, f) for f in MIXED_FLAGS])
def test_branch_of_every_window_state_matches_the_oracle(prec, flags):
    states = _states()
    blocks = [dec.uniform_block(s, N=8, nf=6) for s, _ in states]
    dxs = [0.125] * len(blocks)
    got, gam = gh.run_gpu(gh.to_dev(blocks), dxs, prec=prec, flags=flags)
    mode = 0 if prec == hydro.FP64 else 1
    ref, ram, fl = gh.oracle_ref(blocks, dxs, mode=mode)
    assert not fl.any()
    tol = 1e-14 if mode == 0 else 1e-6
    for i, ((s, w), g) in enumerate(zip(states, got)):
        assert np.all(g == 0.0), ("state", i)
        rel = abs(gam[i] - ram[i]) / ram[i]
        assert rel <= tol, ("state", i, "switched" if w else "not switched", gam[i], ram[i])
    gh._record("amax rel, window states", float(np.max(np.abs(gam - ram) / ram)) / tol)


@pytest.mark.parametrize("nf", [6, 11])
@pytest.mark.parametrize("low_density", [False, True])
@pytest.mark.parametrize("prec,flags", [(hydro.FP64, 0)] + [(hydro.FP32_FLUX_FP64_ACC, f) for f in MIXED_FLAGS])
def test_blocks_mixing_window_states(prec, flags, low_density, nf):
    rng = synth.rng_for(616, nf + 2 * int(low_density))
    blocks = [dec.window_block(rng, N=8, nf=nf, low_density=low_density) for _ in range(6)]
    blocks.append(dec.window_block(rng, N=16, nf=nf, low_density=low_density))
    dxs = [0.125] * 6 + [0.0625]
    got, gam = gh.run_gpu(gh.to_dev(blocks), dxs, prec=prec, flags=flags)
    rc, bad = hydro.status()
    assert rc == hydro.HYDRO_OK
    mode = 0 if prec == hydro.FP64 else 1
    ref, ram, fl = gh.oracle_ref(blocks, dxs, mode=mode)
    assert not fl.any()
    if mode == 0:
        gh.check_fp64(got, ref, gam, ram, blocks, dxs)
    else:
        gh.check_mixed(got, ref, gam, ram, blocks, dxs)
