"""The Sedov point explosion on the GPU through the domain form's fused
SSP-RK3 stages: the same trajectory as the oracle's run, conservation, and
convergence to the similarity solution (Sec. VI-A's benchmark scenario)."""
import numpy as np
import pytest

import paper_2210_06438_gb300 as hydro
from bench import sedov_gpu_run
from tests.sedov_exact import Sedov
from tests.sedov_run import from_domain, oracle_run, shock_measures

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def exact():
    return Sedov(5.0 / 3.0)


@pytest.fixture(scope="module")
def oracle32(exact):
    return oracle_run(32, exact.time_for_radius(0.35))


def _normwise(a, b):
    return max(np.abs(a[f] - b[f]).max() / np.abs(b[f]).max() for f in range(b.shape[0]))


def test_sedov_binary64_follows_the_oracle_trajectory(oracle32):
    U_ora, t, dts = oracle32
    r = sedov_gpu_run(n=32, prec=hydro.FP64, dts=dts)
    U = from_domain(r["U"].cpu().numpy(), 32)
    assert r["steps"] == len(dts)
    # ~100 steps of the 1e-12 RHS agreement
    assert _normwise(U, U_ora) < 1e-9
    # the GPU's own time-step rule picks the same steps to round-off
    own = sedov_gpu_run(n=32, prec=hydro.FP64, t_end=t)
    assert own["steps"] == len(dts)
    assert np.allclose(own["dts"], dts, rtol=1e-9)


def test_sedov_mixed_form_conserves_and_stays_close(oracle32):
    U_ora, t, dts = oracle32
    r = sedov_gpu_run(n=32, prec=hydro.FP32_FLUX_FP64_ACC, dts=dts)
    U = from_domain(r["U"].cpu().numpy(), 32)
    dx3 = (1.0 / 32) ** 3
    for f in (0, 4, 6, 10):
        assert abs(U[f].sum() - U_ora[f].sum()) * dx3 <= 1e-12 * np.abs(U_ora[f]).sum() * dx3
    assert np.abs(U[1:4].sum(axis=(1, 2, 3))).max() * dx3 < 1e-12
    assert np.abs(U[0] - U_ora[0]).max() / U_ora[0].max() < 1e-4


def test_sedov_converges_to_the_similarity_solution(exact):
    t_end = exact.time_for_radius(0.35)
    L1 = {}
    for n in (32, 64, 128):
        r = sedov_gpu_run(n=n, prec=hydro.FP64, t_end=t_end)
        rho = from_domain(r["U"].cpu().numpy(), n)[0]
        Rp, L1[n] = shock_measures(rho, 1.0 / n, exact, r["t"])
        assert abs(Rp - exact.shock_radius(r["t"])) <= 1.0 / n, (n, Rp)
        assert rho.min() > 0
    assert L1[64] < 0.8 * L1[32] and L1[128] < 0.8 * L1[64], L1


def test_sedov_with_the_26_point_variant(exact):
    """The paper's scheme on the paper's scenario: the binary64 26-point run
    follows the oracle's QUAD26 trajectory at 16^3 and puts the shock within a
    cell of R(t) at 32^3, spherically symmetric."""
    import oracle

    t_end = exact.time_for_radius(0.35)
    U_ora, t, dts = oracle_run(16, t_end, mode=oracle.QUAD26)
    r = sedov_gpu_run(n=16, prec=hydro.FP64, dts=dts, flags=hydro.F_QUAD26)
    U = from_domain(r["U"].cpu().numpy(), 16)
    assert _normwise(U, U_ora) < 1e-9
    r = sedov_gpu_run(n=32, prec=hydro.FP64, t_end=t_end, flags=hydro.F_QUAD26)
    rho = from_domain(r["U"].cpu().numpy(), 32)[0]
    Rp, L1 = shock_measures(rho, 1.0 / 32, exact, r["t"])
    assert abs(Rp - exact.shock_radius(r["t"])) <= 1.0 / 32
    assert np.abs(rho - rho.transpose(1, 2, 0)).max() < 1e-10 * rho.max()
