"""The Courant step on the device (hydro_courant) and the stages that read dt
from device memory (hydro_domain_stage_dt, hydro_forest_stage_dt): the same
numbers as the host-side rule and the host-dt stages, and a CUDA-graph time
loop that reproduces the host-driven one bit for bit."""
import numpy as np
import pytest
import torch

import paper_2210_06438_gb300 as hydro
import synth
from bench import sedov_gpu_run

pytestmark = pytest.mark.gpu


def _clock(t=0.0, k=0):
    return torch.tensor([t, 0.0, float(k)], dtype=torch.float64, device="cuda")


def test_courant_matches_the_host_rule():
    rng = np.random.default_rng(61)
    n = 3001
    am = rng.uniform(0.5, 3.0, (3, n))
    am[1, 17] = 9.0  # the largest speed, in a middle row
    dx = 1.0 / 2 ** rng.integers(4, 8, n) * 0.9
    A = torch.from_numpy(am).cuda()
    D = torch.from_numpy(dx).cuda()
    hist = torch.zeros(8, dtype=torch.float64, device="cuda")
    c = _clock()
    hydro.courant(A, 3, n, n, c, 0.3, 10.0, dx_uniform=1.0 / 64, dt_hist=hist, hist_len=8)
    torch.cuda.synchronize()
    want = (0.3 * (1.0 / 64)) / am.max()
    assert c[1].item() == want and c[0].item() == want and c[2].item() == 1.0 and hist[0].item() == want
    hydro.courant(A, 3, n, n, c, 0.3, 10.0, dx=D, dt_hist=hist, hist_len=8)
    torch.cuda.synchronize()
    want2 = 0.3 * float((dx / am.max(axis=0)).min())
    assert c[1].item() == want2 and c[0].item() == want + want2 and c[2].item() == 2.0
    assert hist[1].item() == want2
    # the last step stops at t_end, later ones are zero
    c2 = _clock(t=10.0 - 1e-4)
    hydro.courant(A, 3, n, n, c2, 0.3, 10.0, dx_uniform=1.0)
    hydro.courant(A, 3, n, n, c2, 0.3, 10.0, dx_uniform=1.0)
    torch.cuda.synchronize()
    assert c2[0].item() == 10.0 and c2[1].item() == 0.0 and c2[2].item() == 2.0
    # rows wider than n (stride) and a single row
    W = torch.zeros((2, n + 5), dtype=torch.float64, device="cuda")
    W[:, :n] = A[:2]
    c3 = _clock()
    hydro.courant(W, 2, n + 5, n, c3, 0.5, 1.0, dx_uniform=0.25)
    torch.cuda.synchronize()
    assert c3[1].item() == (0.5 * 0.25) / am[:2].max()
    with pytest.raises(hydro.HydroError):
        hydro.courant(A, 3, n - 1, n, c, 0.3, 1.0, dx_uniform=1.0)


@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
@pytest.mark.parametrize("flags", [0, hydro.F_QUAD26])
def test_stage_dt_equals_stage(prec, flags):
    glob = synth.plain_domain(seed=62, n=32, nf=8)
    from tests.sedov_run import to_domain

    U = torch.from_numpy(to_domain(glob, 8)).cuda()
    U0 = U * 0.9
    nb, dx, dt = 4, 1.0 / 32, 3e-3
    a, b = torch.empty_like(U), torch.empty_like(U)
    am = torch.empty(nb ** 3, dtype=torch.float64, device="cuda")
    dtd = torch.tensor([dt], dtype=torch.float64, device="cuda")
    hydro.domain_stage(U, U0, 0.75, 0.25, dt, nb, 8, 8, dx, a, am, prec=prec, flags=flags)
    hydro.domain_stage_dt(U, U0, 0.75, 0.25, dtd, nb, 8, 8, dx, b, am, prec=prec, flags=flags)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # forests (the flux correction scales with beta dt too)
    lv = synth.forest_leaves(3, 2, synth.random_refine(1, 0.1), seed=1, balance="full")
    Uf, dx0 = synth.smooth_forest_state(lv, 3, 8, nf=7, seed=63)
    fo = hydro.Forest(lv, 3, 8, 7)
    Ud = torch.from_numpy(Uf).cuda()
    fa, fb = torch.empty_like(Ud), torch.empty_like(Ud)
    amf = torch.empty(len(lv), dtype=torch.float64, device="cuda")
    fo.stage(Ud, Ud, 1.0 / 3.0, 2.0 / 3.0, dt, dx0, fa, amf, prec=prec, flags=flags)
    fo.stage_dt(Ud, Ud, 1.0 / 3.0, 2.0 / 3.0, dtd, dx0, fb, amf, prec=prec, flags=flags)
    torch.cuda.synchronize()
    fo.close()
    assert torch.equal(fa, fb)


def test_graph_time_loop_equals_the_host_loop():
    """The Sedov run to t_end with the step on the device and graph replays
    gives the state of the host-driven loop fed the same dt sequence, bit
    for bit, and that sequence follows the host rule."""
    from tests.sedov_exact import Sedov

    t_end = Sedov(5.0 / 3.0).time_for_radius(0.3)
    g = sedov_gpu_run(n=32, prec=hydro.FP64, t_end=t_end)
    assert g["steps"] > 40 and g["t"] == pytest.approx(t_end, rel=1e-15, abs=0)
    h = sedov_gpu_run(n=32, prec=hydro.FP64, dts=g["dts"])
    assert torch.equal(g["U"], h["U"])
    assert sum(g["dts"]) == pytest.approx(t_end, rel=1e-12)
