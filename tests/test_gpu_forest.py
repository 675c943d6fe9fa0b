"""GPU parity of the forest entry points (multi-level ghost slabs, fused tile
kernel, flux correction) against the forest oracle, in both precision
forms, with both fluxes, the fused stage, 8^3 and 16^3 leaves; plus the
one-level forest against the periodic domain kernel bit for bit, exact
zeros on constant states and conservation across levels."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_06438_gb300 as hydro
import synth
from oracle import forest as of
from tests import gpu_helpers as gh

pytestmark = pytest.mark.gpu
MX = hydro.FP32_FLUX_FP64_ACC


def _forest(nb0=2, seed=7, prob=0.25, max_level=2):
    return synth.forest_leaves(nb0, max_level, synth.random_refine(seed, prob), seed=seed)


def _run(lv, nb0, U, dx0, prec, flags=0, stage=None):
    n, nf, N = U.shape[0], U.shape[1], U.shape[-1]
    fo = hydro.Forest(lv, nb0, N, nf)
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    out = torch.full_like(Ud, float("nan"))
    am = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    if stage is None:
        fo.rhs(Ud, dx0, out, am, prec=prec, flags=flags)
    else:
        U0, a, b, dt = stage
        fo.stage(Ud, torch.from_numpy(U0).cuda(), a, b, dt, dx0, out, am, prec=prec, flags=flags)
    torch.cuda.synchronize()
    info = fo.info()
    fo.close()
    return list(out.cpu().numpy()), am.cpu().numpy(), info


def _dxs(lv, dx0):
    return [dx0 / (1 << int(L)) for L in lv[:, 0]]


def _check(prec, got, gam, ref, ram, U, dxs):
    if prec == hydro.FP64:
        return gh.check_fp64(got, ref, gam, ram, list(U), dxs)
    return gh.check_mixed(got, ref, gam, ram, list(U), dxs)


@pytest.mark.parametrize("prec", [hydro.FP64, MX])
@pytest.mark.parametrize("N,nb0,seed,prob,nf", [(8, 2, 7, 0.25, 11), (8, 2, 4, 0.25, 6), (16, 1, 3, 0.6, 7),
                                                (12, 1, 3, 0.6, 10), (6, 2, 4, 0.25, 8)])
def test_forest_rhs_matches_oracle(prec, N, nb0, seed, prob, nf):
    lv = _forest(nb0, seed, prob)
    assert len(set(lv[:, 0])) >= 2
    U, dx0 = synth.smooth_forest_state(lv, nb0, N, nf=nf, seed=31 + seed)
    got, gam, info = _run(lv, nb0, U, dx0, prec)
    ref, ram = of.rhs(lv, nb0, list(U), dx0, mode=0 if prec == hydro.FP64 else oracle.MODE_MIXED)
    _check(prec, got, gam, ref, ram, U, _dxs(lv, dx0))
    kind, _ = hydro.forest_links(lv, nb0, N)
    assert info["n_level_faces"] == sum(k != 0 for row in kind for k in row) > 0
    assert info["n_reflux_leaves"] == sum(any(k == 1 for k in row) for row in kind) > 0


@pytest.mark.parametrize("N,nb0,seed,prob", [(12, 1, 3, 0.6), (8, 2, 7, 0.25)])
def test_mixed_forest_kernel_families_bitwise(N, nb0, seed, prob):
    """The pipelined mixed kernel (default) and the register-load one give
    the same bits on forests, partial tiles included, for the RHS and a
    stage."""
    lv = _forest(nb0, seed, prob)
    U, dx0 = synth.smooth_forest_state(lv, nb0, N, nf=11, seed=47)
    a = _run(lv, nb0, U, dx0, MX)
    b = _run(lv, nb0, U, dx0, MX, flags=hydro.F_REGISTER_LOADS)
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(x, y)
    assert np.array_equal(a[1], b[1])
    st = (U * 0.5, 0.75, 0.25, 1e-3)
    a = _run(lv, nb0, U, dx0, MX, stage=st, flags=hydro.F_KNP)
    b = _run(lv, nb0, U, dx0, MX, stage=st, flags=hydro.F_KNP | hydro.F_REGISTER_LOADS)
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(x, y)


def test_forest_one_sided_flux():
    lv = _forest()
    U, dx0 = synth.smooth_forest_state(lv, 2, 8, nf=9, seed=41)
    got, gam, _ = _run(lv, 2, U, dx0, hydro.FP64, flags=hydro.F_KNP)
    ref, ram = of.rhs(lv, 2, list(U), dx0, mode=oracle.FLUX_KNP)
    gh.check_fp64(got, ref, gam, ram, list(U), _dxs(lv, dx0))


@pytest.mark.parametrize("prec", [hydro.FP64, MX])
def test_forest_stage_matches_oracle(prec):
    lv = _forest(2, 4, 0.25)
    U, dx0 = synth.smooth_forest_state(lv, 2, 8, nf=8, seed=42)
    U0, _ = synth.smooth_forest_state(lv, 2, 8, nf=8, seed=43)
    a, b, dt = 0.75, 0.25, 2e-3
    got, gam, _ = _run(lv, 2, U, dx0, prec, stage=(U0, a, b, dt))
    mode = 0 if prec == hydro.FP64 else oracle.MODE_MIXED
    ref, ram = of.stage(lv, 2, list(U), list(U0), a, b, dt, dx0, mode=mode)
    dU, _ = of.rhs(lv, 2, list(U), dx0, mode=mode)
    dxs = _dxs(lv, dx0)
    for s in range(len(lv)):
        Umax = np.abs(U[s]).reshape(U.shape[1], -1).max(axis=1)
        for f in range(U.shape[1]):
            # the state's rounding plus beta dt times the RHS gate of the form
            if mode == 0:
                rt = 1e-12 * max(np.abs(dU[s][f]).max(), ram[s] * Umax[f] / dxs[s])
            else:
                rt = 64 * 2.0 ** -24 * 2 * ram[s] * (Umax[f] + (Umax[4] if 1 <= f <= 4 else 0)) / dxs[s]
            tol = 4e-16 * np.abs(ref[s][f]).max() + b * dt * rt
            assert np.abs(got[s][f] - ref[s][f]).max() <= tol, (s, f)
    assert np.allclose(gam, ram, rtol=1e-14 if mode == 0 else 1e-6, atol=0)


@pytest.mark.parametrize("prec", [hydro.FP64, MX])
def test_one_level_forest_equals_domain_kernel(prec):
    nb0, N = 3, 8
    lv = synth.forest_leaves(nb0, 0, lambda *a: False, seed=6)
    glob = synth.plain_domain(seed=44, n=nb0 * N, nf=11)
    blocks = synth.gather_blocks(glob, N, blocks=[tuple(l[1:]) for l in lv])
    U = np.ascontiguousarray(blocks[:, :, 3:-3, 3:-3, 3:-3])
    dx0 = 1.0 / (nb0 * N)
    got, gam, info = _run(lv, nb0, U, dx0, prec)
    assert info["n_level_faces"] == 0 and info["n_reflux_leaves"] == 0
    # the domain kernel on the cube in its own order s = bx + nb (by + nb bz)
    order = [int(x + nb0 * (y + nb0 * z)) for _, x, y, z in lv]
    dom = np.empty_like(U)
    dom[order] = U
    Ud = torch.from_numpy(dom).cuda()
    out = torch.empty_like(Ud)
    am = torch.empty(len(lv), dtype=torch.float64, device="cuda")
    hydro.domain_rhs(Ud, nb0, N, 11, dx0, out, am, prec=prec)
    torch.cuda.synchronize()
    o, a = out.cpu().numpy(), am.cpu().numpy()
    for s in range(len(lv)):
        assert np.array_equal(got[s], o[order[s]])
        assert gam[s] == a[order[s]]


@pytest.mark.parametrize("prec", [hydro.FP64, MX])
def test_constant_state_exact_zero(prec):
    lv = _forest(2, 4, 0.25)
    n, N = len(lv), 8
    shp = (n, N, N, N)
    X = np.full((2,) + shp, 0.5)
    Uc = synth.conserved_from_states(np.full(shp, 0.8), np.full(shp, -0.3), np.full(shp, 0.1),
                                     np.full(shp, 0.2), np.full(shp, 1.7), X)
    U = np.ascontiguousarray(np.moveaxis(Uc, 0, 1))
    got, gam, _ = _run(lv, 2, U, 1.0 / 16, prec)
    for o in got:
        assert np.all(o == 0.0)


@pytest.mark.parametrize("prec", [hydro.FP64, MX])
def test_conservation_across_levels(prec):
    lv = _forest(2, 7, 0.25)
    U, dx0 = synth.smooth_forest_state(lv, 2, 8, nf=11, seed=45)
    got, _, _ = _run(lv, 2, U, dx0, prec)
    vol = np.array(_dxs(lv, dx0)) ** 3
    tot = sum(got[s].sum(axis=(1, 2, 3)) * vol[s] for s in range(len(lv)))
    mag = sum(np.abs(got[s]).sum(axis=(1, 2, 3)) * vol[s] for s in range(len(lv)))
    assert np.all(np.abs(tot) <= (1e-14 if prec == hydro.FP64 else 1e-12) * mag), tot / mag


def test_forest_rk3_step_in_a_cuda_graph():
    """The forest entry points allocate nothing after their first call, so a
    whole SSP-RK3 step (9 launches) records into a CUDA graph; its replay
    gives the bits of the direct calls."""
    lv = _forest(2, 7, 0.25)
    U_h, dx0 = synth.smooth_forest_state(lv, 2, 8, nf=11, seed=46)
    fo = hydro.Forest(lv, 2, 8, 11)
    U = torch.from_numpy(U_h).cuda()
    W1, W2, W3 = torch.empty_like(U), torch.empty_like(U), torch.empty_like(U)
    am = torch.empty((3, len(lv)), dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())  # after the copies above

    def step(out):
        fo.stage(U, U, 0.0, 1.0, 1e-4, dx0, W1, am[0], stream=st)
        fo.stage(W1, U, 0.75, 0.25, 1e-4, dx0, W2, am[1], stream=st)
        fo.stage(W2, U, 1.0 / 3.0, 2.0 / 3.0, 1e-4, dx0, out, am[2], stream=st)

    with torch.cuda.stream(st):
        step(W3)  # first calls: kernel attributes, status word
        torch.cuda.synchronize()
        ref, ref_am = W3.clone(), am.clone()
        W3.zero_()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            step(W3)
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(W3, ref) and torch.equal(am, ref_am)
    fo.close()


# ------------------------------------------------- 26-point variant --
def _full_forest():
    return synth.forest_leaves(3, 2, synth.random_refine(1, 0.1), seed=1, balance="full")


@pytest.mark.parametrize("prec", [hydro.FP64, MX])
@pytest.mark.parametrize("case", ["three_levels_8", "two_levels_16", "two_levels_12", "three_levels_6"])
def test_quad26_forest_matches_oracle(prec, case):
    if case == "three_levels_8":
        lv, nb0, N, nf = _full_forest(), 3, 8, 7
    elif case == "three_levels_6":  # the smallest leaf: a 3-cell slab is half a finer leaf
        lv, nb0, N, nf = _full_forest(), 3, 6, 8
    else:  # 16^3 (two tiles per edge) and 12^3 (partial tiles)
        N = 16 if case == "two_levels_16" else 12
        lv, nb0, nf = synth.forest_leaves(1, 2, synth.random_refine(3, 0.6), seed=3, balance="full"), 1, 6
    U, dx0 = synth.smooth_forest_state(lv, nb0, N, nf=nf, seed=48)
    got, gam, info = _run(lv, nb0, U, dx0, prec, flags=hydro.F_QUAD26)
    assert info["quad26"] == 1
    mode = oracle.QUAD26 | (0 if prec == hydro.FP64 else oracle.MODE_MIXED)
    ref, ram = of.rhs(lv, nb0, list(U), dx0, mode=mode)
    _check(prec, got, gam, ref, ram, U, _dxs(lv, dx0))
    vol = np.array(_dxs(lv, dx0)) ** 3
    tot = sum(got[s].sum(axis=(1, 2, 3)) * vol[s] for s in range(len(lv)))
    mag = sum(np.abs(got[s]).sum(axis=(1, 2, 3)) * vol[s] for s in range(len(lv)))
    assert np.all(np.abs(tot) <= (1e-14 if prec == hydro.FP64 else 1e-12) * mag)


def test_quad26_forest_stage_and_one_sided_flux():
    lv = _full_forest()
    U, dx0 = synth.smooth_forest_state(lv, 3, 8, nf=6, seed=49)
    U0, _ = synth.smooth_forest_state(lv, 3, 8, nf=6, seed=50)
    a, b, dt = 1.0 / 3.0, 2.0 / 3.0, 1e-3
    got, gam, _ = _run(lv, 3, U, dx0, hydro.FP64, flags=hydro.F_QUAD26 | hydro.F_KNP, stage=(U0, a, b, dt))
    mode = oracle.QUAD26 | oracle.FLUX_KNP
    ref, ram = of.stage(lv, 3, list(U), list(U0), a, b, dt, dx0, mode=mode)
    dU, _ = of.rhs(lv, 3, list(U), dx0, mode=mode)
    dxs = _dxs(lv, dx0)
    for s in range(len(lv)):
        Umax = np.abs(U[s]).reshape(6, -1).max(axis=1)
        for f in range(6):
            rt = 1e-12 * max(np.abs(dU[s][f]).max(), ram[s] * Umax[f] / dxs[s])
            assert np.abs(got[s][f] - ref[s][f]).max() <= 4e-16 * np.abs(ref[s][f]).max() + b * dt * rt
    assert np.allclose(gam, ram, rtol=1e-14, atol=0)


@pytest.mark.parametrize("prec", [hydro.FP64, MX])
def test_quad26_one_level_forest_equals_domain_kernel(prec):
    nb0, N = 2, 8
    lv = synth.forest_leaves(nb0, 0, lambda *a: False, seed=8)
    glob = synth.plain_domain(seed=51, n=nb0 * N, nf=9)
    blocks = synth.gather_blocks(glob, N, blocks=[tuple(l[1:]) for l in lv])
    U = np.ascontiguousarray(blocks[:, :, 3:-3, 3:-3, 3:-3])
    dx0 = 1.0 / (nb0 * N)
    got, gam, _ = _run(lv, nb0, U, dx0, prec, flags=hydro.F_QUAD26)
    order = [int(x + nb0 * (y + nb0 * z)) for _, x, y, z in lv]
    dom = np.empty_like(U)
    dom[order] = U
    Ud = torch.from_numpy(dom).cuda()
    out = torch.empty_like(Ud)
    am = torch.empty(len(lv), dtype=torch.float64, device="cuda")
    hydro.domain_rhs(Ud, nb0, N, 9, dx0, out, am, prec=prec, flags=hydro.F_QUAD26)
    torch.cuda.synchronize()
    o, a = out.cpu().numpy(), am.cpu().numpy()
    for s in range(len(lv)):
        assert np.array_equal(got[s], o[order[s]])
        assert gam[s] == a[order[s]]


def test_quad26_needs_full_balance():
    lv = _forest(2, 7, 0.25)  # balanced across faces only
    U, dx0 = synth.smooth_forest_state(lv, 2, 8, nf=6)
    fo = hydro.Forest(lv, 2, 8, 6)
    assert fo.info()["quad26"] == 0
    Ud = torch.from_numpy(U).cuda()
    out = torch.empty_like(Ud)
    am = torch.empty(len(lv), dtype=torch.float64, device="cuda")
    with pytest.raises(hydro.HydroError) as ei:
        fo.rhs(Ud, dx0, out, am, flags=hydro.F_QUAD26)
    assert ei.value.code == hydro.HYDRO_EINVAL
    fo.close()


@pytest.mark.parametrize("flags", [0, hydro.F_QUAD26])
def test_forest_nonphysical_input_is_flagged(flags):
    """A negative density inside one leaf is recorded in the status word with
    that leaf's index (the ghost transfers pass it on unflagged: only the
    tile that reads the cell flags it); the call completes and the word
    clears when read."""
    lv = _full_forest()
    U, dx0 = synth.smooth_forest_state(lv, 3, 8, nf=6, seed=52)
    # a cell of a coarsest-level leaf four cells from its faces: neighbours of
    # the same level read three cells deep and finer ones two, so only the
    # leaf itself reads it
    s_bad = int(np.flatnonzero(lv[:, 0] == 0)[0])
    U[s_bad, 0, 4, 4, 4] = -1.0
    hydro.status()  # clear
    got, gam, _ = _run(lv, 3, U, dx0, hydro.FP64, flags=flags)
    rc, bad = hydro.status()
    assert rc == hydro.HYDRO_ENONPHYS and bad == s_bad
    hydro.status()
    assert hydro.status() == (hydro.HYDRO_OK, -1)


def test_forest_argument_checks():
    lv = _forest(2, 4, 0.25)
    U, dx0 = synth.smooth_forest_state(lv, 2, 8, nf=6)
    fo = hydro.Forest(lv, 2, 8, 6)
    Ud = torch.from_numpy(U).cuda()
    out = torch.empty_like(Ud)
    am = torch.empty(len(lv), dtype=torch.float64, device="cuda")
    for kw in (dict(flags=16), dict(dx0=-1.0), dict(gamma=1.0), dict(out=Ud)):
        with pytest.raises(hydro.HydroError) as ei:
            fo.rhs(Ud, kw.get("dx0", dx0), kw.get("out", out), am, gamma=kw.get("gamma", 5.0 / 3.0),
                   flags=kw.get("flags", 0))
        assert ei.value.code == hydro.HYDRO_EINVAL
    fo.close()


# ------------------------------------------------------- Sedov on a forest --
def test_sedov_on_a_forest():
    """The point explosion on a forest refined around the centre (levels 1
    and 2, 64^3 cells' resolution at the centre): two steps follow the
    forest oracle's; the run to R = 0.35 conserves mass and energy to
    rounding across the level boundaries the shock crosses, keeps the mirror
    symmetry, and puts the density peak within a cell of the similarity
    solution's shock radius."""
    from bench import sedov_forest_run
    from tests.sedov_exact import Sedov
    from tests.sedov_run import forest_shock_measures, oracle_forest_steps

    ex = Sedov(5.0 / 3.0)
    r2 = sedov_forest_run(prec=hydro.FP64, dts=[2e-5, 2e-5])
    leaves, U0, dx0 = synth.sedov_forest()
    ref = oracle_forest_steps(leaves, 2, list(U0), dx0, r2["dts"])
    got = r2["U"].cpu().numpy()
    for s in range(len(leaves)):
        for f in range(U0.shape[1]):
            assert np.abs(got[s][f] - ref[s][f]).max() <= 1e-11 * np.abs(ref[s][f]).max() + 1e-300
    r = sedov_forest_run(prec=hydro.FP64, t_end=ex.time_for_radius(0.35))
    U = r["U"].cpu().numpy()
    lv = r["leaves"]
    vol = (dx0 / (1 << lv[:, 0].astype(np.int64))) ** 3
    tot0 = (U0.sum(axis=(2, 3, 4)) * vol[:, None]).sum(axis=0)
    tot = (U.sum(axis=(2, 3, 4)) * vol[:, None]).sum(axis=0)
    mag = (np.abs(U).sum(axis=(2, 3, 4)) * vol[:, None]).sum(axis=0)
    for f in (0, 4, 5, 6, 10):
        assert abs(tot[f] - tot0[f]) <= 1e-12 * mag[f], (f, tot[f] - tot0[f])
    for f in (1, 2, 3):
        assert abs(tot[f]) <= 1e-12 * mag[0]
    # mirror x -> 1 - x maps the forest onto itself
    key = {tuple(int(v) for v in l): s for s, l in enumerate(lv)}
    worst = 0.0
    for s, (L, bx, by, bz) in enumerate(lv):
        m = key[(int(L), int((2 << int(L)) - 1 - bx), int(by), int(bz))]
        worst = max(worst, np.abs(U[s, 0] - U[m, 0, :, :, ::-1]).max())
    assert worst <= 1e-9 * U[:, 0].max()
    Rp, L1 = forest_shock_measures(lv, 2, U[:, 0], ex, r["t"])
    assert abs(Rp - ex.shock_radius(r["t"])) <= 1.0 / 32, (Rp, ex.shock_radius(r["t"]))
    assert U[:, 0].min() > 0 and L1 < 0.5


@pytest.mark.slow
@pytest.mark.parametrize("prec", [hydro.FP64, MX])
def test_bench_forest_full_size_sampled(prec):
    """The forest of the benchmark (21848 leaves of 8^3 in three levels, 11.2M
    cells, 11 fields) through the same entry point and launch shapes as
    bench.forest_forms; sampled leaves of every kind (each level, coarse
    leaves corrected by finer neighbours, fine leaves next to coarser ones)
    against the forest oracle evaluated for those leaves only."""
    nb0, radii = 16, (0.35, 0.2)
    lv = synth.forest_leaves(nb0, 2, synth.sphere_refine((0.5, 0.5, 0.5), radii), balance="full")
    U, dx0 = synth.smooth_forest_state(lv, nb0, 8, nf=11)
    got, gam, info = _run(lv, nb0, U, dx0, prec)
    assert info["n_leaves"] == 21848
    kind, _ = hydro.forest_links(lv, nb0, 8)
    rng = np.random.default_rng(53)
    groups = [np.flatnonzero(lv[:, 0] == L) for L in range(3)]
    groups.append(np.array([s for s in range(len(lv)) if 1 in kind[s]]))   # corrected by finer leaves
    groups.append(np.array([s for s in range(len(lv)) if -1 in kind[s]]))  # next to coarser leaves
    pick = sorted({int(x) for g in groups for x in rng.choice(g, 4, replace=False)})
    mode = 0 if prec == hydro.FP64 else oracle.MODE_MIXED
    ref, ram = of.rhs(lv, nb0, U, dx0, mode=mode, only=pick)
    _check(prec, [got[s] for s in pick], gam[pick], [ref[s] for s in pick], np.array([ram[s] for s in pick]),
           U[pick], [dx0 / (1 << int(lv[s, 0])) for s in pick])


@pytest.mark.parametrize("prec,flags", [(hydro.FP64, 0), (MX, 0), (hydro.FP64, hydro.F_QUAD26)])
def test_forest_homogeneity_under_power_of_two_scaling(prec, flags):
    """Level transfers, tiles and flux correction scale exactly: rho, rho v,
    E, rho X times 4 and tau times 1/8 scale every leaf's dU/dt by the same
    factor on the GPU, bit for bit, and leave amax unchanged."""
    lv = _full_forest()
    U, dx0 = synth.smooth_forest_state(lv, 3, 8, nf=7, seed=54)
    ref, ra, _ = _run(lv, 3, U, dx0, prec, flags=flags)
    V = U * 4.0
    V[:, 5] = U[:, 5] * 0.125
    got, ga, _ = _run(lv, 3, V, dx0, prec, flags=flags)
    assert np.array_equal(ga, ra)
    for s in range(len(lv)):
        for f in range(7):
            assert np.array_equal(got[s][f], ref[s][f] * (0.125 if f == 5 else 4.0)), (s, f)
