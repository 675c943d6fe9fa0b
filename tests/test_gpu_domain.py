"""The domain form: ghost shells gathered in the kernel from the neighbouring
sub-grids of a periodic cube stored without ghosts, and the fused explicit
stage.  Checked against the oracle on the equivalent ghosted sub-grids, and a
full SSP-RK3 step against the oracle's."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_06438_gb300 as hydro
import synth
from tests import gpu_helpers as gh

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0


def domain_layout(glob, N):
    """[nf][n][n][n] periodic array -> [s][nf][N][N][N], s = bx + nb (by + nb bz)."""
    nf, n = glob.shape[0], glob.shape[1]
    nb = n // N
    a = glob.reshape(nf, nb, N, nb, N, nb, N)          # f, bz, z, by, y, bx, x
    a = a.transpose(1, 3, 5, 0, 2, 4, 6)                # bz, by, bx, f, z, y, x
    return np.ascontiguousarray(a.reshape(nb ** 3, nf, N, N, N)), nb


def from_domain(arr, nb, N):
    nf = arr.shape[1]
    a = arr.reshape(nb, nb, nb, nf, N, N, N).transpose(3, 0, 4, 1, 5, 2, 6)
    return np.ascontiguousarray(a.reshape(nf, nb * N, nb * N, nb * N))


@pytest.mark.parametrize("N,n", [(8, 32), (16, 32), (12, 24), (3, 9), (2, 6), (8, 8)])
@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_domain_rhs_matches_the_ghosted_subgrids(N, n, prec):
    glob = synth.plain_domain(seed=17, n=n, nf=11)
    dom, nb = domain_layout(glob, N)
    dx = 1.0 / n
    U = torch.from_numpy(dom).cuda()
    out = torch.full_like(U, float("nan"))
    am = torch.full((nb ** 3,), float("nan"), dtype=torch.float64, device="cuda")
    hydro.domain_rhs(U, nb, N, 11, dx, out, am, prec=prec)
    torch.cuda.synchronize()
    blocks = list(synth.gather_blocks(glob, N))  # the same sub-grid order, with ghosts
    mode = 0 if prec == hydro.FP64 else 1
    ref, ram, fl = gh.oracle_ref(blocks, [dx] * len(blocks), mode=mode)
    got = [o for o in out.cpu().numpy()]
    if mode == 0:
        gh.check_fp64(got, ref, am.cpu().numpy(), ram, blocks, [dx] * len(blocks))
    else:
        gh.check_mixed(got, ref, am.cpu().numpy(), ram, blocks, [dx] * len(blocks))
    # the same kernel arithmetic as the ghosted entry point
    g, gam = gh.run_gpu(gh.to_dev(blocks), [dx] * len(blocks), prec=prec)
    for a, b in zip(got, g):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_fused_stage_equals_rhs_then_update(prec):
    glob = synth.plain_domain(seed=19, n=32, nf=8)
    dom, nb = domain_layout(glob, 8)
    U = torch.from_numpy(dom).cuda()
    U0 = U * 1.01
    dx, dt = 1.0 / 32, 1e-3
    L = torch.empty_like(U)
    am = torch.empty(nb ** 3, dtype=torch.float64, device="cuda")
    hydro.domain_rhs(U, nb, 8, 8, dx, L, am, prec=prec)
    out = torch.empty_like(U)
    am2 = torch.empty_like(am)
    hydro.domain_stage(U, U0, 0.75, 0.25, dt, nb, 8, 8, dx, out, am2, prec=prec)
    torch.cuda.synchronize()
    ref = 0.75 * U0 + 0.25 * (U + dt * L)
    # per field, normwise: a few roundings of the largest term
    err = (out - ref).abs().amax(dim=(0, 2, 3, 4))
    scale = ref.abs().amax(dim=(0, 2, 3, 4))
    assert float((err / scale).max()) <= 4e-16
    assert torch.equal(am, am2)


def test_rk3_step_matches_the_oracle():
    """Three fused stages (Shu-Osher SSP-RK3) on a smooth periodic 32^3 domain
    against the oracle's RHS of the gathered sub-grids with the same stages."""
    n, N, nf = 32, 8, 6
    glob = synth.plain_domain(seed=23, n=n, nf=nf)
    dx = 1.0 / n
    dom, nb = domain_layout(glob, N)
    U = torch.from_numpy(dom).cuda()
    U1, U2, U3 = (torch.empty_like(U) for _ in range(3))
    am = torch.empty(nb ** 3, dtype=torch.float64, device="cuda")
    hydro.domain_rhs(U, nb, N, nf, dx, U1, am)
    torch.cuda.synchronize()
    dt = 0.4 * dx / float(am.max())
    hydro.domain_stage(U, U, 0.0, 1.0, dt, nb, N, nf, dx, U1, am)
    hydro.domain_stage(U1, U, 0.75, 0.25, dt, nb, N, nf, dx, U2, am)
    hydro.domain_stage(U2, U, 1.0 / 3.0, 2.0 / 3.0, dt, nb, N, nf, dx, U3, am)
    torch.cuda.synchronize()

    def L(state):
        blocks = list(synth.gather_blocks(state, N))
        outs, _, _ = oracle.rhs_batch(blocks, G53, dx, 0, threads=8)
        return from_domain(np.stack(outs), nb, N)

    V = glob
    V1 = V + dt * L(V)
    V2 = 0.75 * V + 0.25 * (V1 + dt * L(V1))
    V3 = V / 3.0 + 2.0 / 3.0 * (V2 + dt * L(V2))
    got = from_domain(U3.cpu().numpy(), nb, N)
    for f in range(nf):
        assert np.abs(got[f] - V3[f]).max() <= 1e-13 * max(np.abs(V3[f]).max(), 1.0)


def test_domain_argument_checks():
    U = torch.zeros(8, 6, 8, 8, 8, dtype=torch.float64, device="cuda")
    am = torch.empty(8, dtype=torch.float64, device="cuda")
    with pytest.raises(hydro.HydroError):
        hydro.domain_rhs(U, 2, 8, 6, 0.1, U, am)  # output aliases input
    with pytest.raises(hydro.HydroError):
        hydro.domain_rhs(U, 2, 8, 5, 0.1, torch.empty_like(U), am)


@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_domain_with_the_one_sided_flux(prec):
    """HYDRO_F_KNP in the domain form against the oracle's KNP mode on the
    gathered sub-grids."""
    n, N = 16, 8
    glob = synth.plain_domain(seed=29, n=n, nf=11)
    dom, nb = domain_layout(glob, N)
    dx = 1.0 / n
    U = torch.from_numpy(dom).cuda()
    out = torch.empty_like(U)
    am = torch.empty(nb ** 3, dtype=torch.float64, device="cuda")
    hydro.domain_rhs(U, nb, N, 11, dx, out, am, prec=prec, flags=hydro.F_KNP)
    torch.cuda.synchronize()
    blocks = list(synth.gather_blocks(glob, N))
    mode = oracle.FLUX_KNP + (0 if prec == hydro.FP64 else 1)
    ref, ram, _ = gh.oracle_ref(blocks, [dx] * len(blocks), mode=mode)
    got = [o for o in out.cpu().numpy()]
    if prec == hydro.FP64:
        gh.check_fp64(got, ref, am.cpu().numpy(), ram, blocks, [dx] * len(blocks))
    else:
        gh.check_mixed(got, ref, am.cpu().numpy(), ram, blocks, [dx] * len(blocks))


@pytest.mark.parametrize("N,n", [(8, 16), (12, 24)])
@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_domain_with_the_26_point_variant(N, n, prec):
    """HYDRO_F_QUAD26 in the domain form gives the bits of the ghosted entry
    point on the gathered sub-grids (which the oracle pins separately); the
    fused stage applies on top of it."""
    glob = synth.plain_domain(seed=31, n=n, nf=9)
    dom, nb = domain_layout(glob, N)
    dx = 1.0 / n
    U = torch.from_numpy(dom).cuda()
    out = torch.empty_like(U)
    am = torch.empty(nb ** 3, dtype=torch.float64, device="cuda")
    hydro.domain_rhs(U, nb, N, 9, dx, out, am, prec=prec, flags=hydro.F_QUAD26)
    torch.cuda.synchronize()
    blocks = list(synth.gather_blocks(glob, N))
    g, gam = gh.run_gpu(gh.to_dev(blocks), [dx] * len(blocks), prec=prec, flags=hydro.F_QUAD26)
    for a, b in zip(out.cpu().numpy(), g):
        assert np.array_equal(a, b)
    assert np.array_equal(am.cpu().numpy(), gam)
    st = torch.empty_like(U)
    hydro.domain_stage(U, U, 0.0, 1.0, 1e-3, nb, N, 9, dx, st, am, prec=prec, flags=hydro.F_QUAD26)
    torch.cuda.synchronize()
    ref = U + 1e-3 * out
    err = (st - ref).abs().amax(dim=(0, 2, 3, 4)) / ref.abs().amax(dim=(0, 2, 3, 4))
    assert float(err.max()) <= 4e-16
