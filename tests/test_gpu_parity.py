"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs, for every workload shape and the edge cases."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_06438_gb300 as hydro
import synth
from tests import gpu_helpers as gh

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0


def _both(blocks, dxs, prec=hydro.FP64, **kw):
    dev = gh.to_dev(blocks)
    got, gam = gh.run_gpu(dev, dxs, prec=prec, **kw)
    return got, gam


# ------------------------------------------------------- one sub-grid --
@pytest.mark.parametrize("nf", [6, 11])
def test_one_subgrid_fp64(nf):
    U, dx = synth.one_subgrid(nf=nf)
    got, gam = _both([U], [dx])
    ref, ram, fl = gh.oracle_ref([U], [dx])
    assert not fl.any()
    gh.check_fp64(got, ref, gam, ram, [U], [dx])
    rc, bad = hydro.status()
    assert rc == hydro.HYDRO_OK


# the mixed form has two kernel families: the pipelined default and the
# register-load kernels (HYDRO_F_REGISTER_LOADS)
MIXED_KERNELS = [0, hydro.F_REGISTER_LOADS]


@pytest.mark.parametrize("flags", MIXED_KERNELS)
@pytest.mark.parametrize("nf", [6, 11])
def test_one_subgrid_mixed(nf, flags):
    U, dx = synth.one_subgrid(nf=nf)
    got, gam = _both([U], [dx], prec=hydro.FP32_FLUX_FP64_ACC, flags=flags)
    ref, ram, _ = gh.oracle_ref([U], [dx], mode=1)
    gh.check_mixed(got, ref, gam, ram, [U], [dx])


# ------------------------------------------------------ plain domain --
@pytest.mark.parametrize("prec,flags", [(hydro.FP64, 0)] +
                         [(hydro.FP32_FLUX_FP64_ACC, f) for f in MIXED_KERNELS])
def test_plain_aggregation_512_subgrids(prec, flags):
    glob = synth.plain_domain(n=64, nf=11)
    blocks = synth.gather_blocks(glob, 8)
    dxs = [1.0 / 64] * len(blocks)
    got, gam = _both(list(blocks), dxs, prec=prec, flags=flags)
    mode = 0 if prec == hydro.FP64 else 1
    ref, ram, fl = gh.oracle_ref(list(blocks), dxs, mode=mode)
    assert not fl.any()
    if mode == 0:
        gh.check_fp64(got, ref, gam, ram, blocks, dxs)
    else:
        gh.check_mixed(got, ref, gam, ram, blocks, dxs)
        # against the binary64 oracle: the flux-scaled binary32 bound, and a
        # normwise cap just above the scheme's own error here -- the oracle's
        # mixed mode differs from its binary64 mode by 1.44e-5 normwise on this
        # domain (the error grows with the cancellation in the flux
        # differences, i.e. with resolution)
        ref64, ram64, _ = gh.oracle_ref(list(blocks), dxs, mode=0)
        gh.check_mixed(got, ref64, gam, ram64, blocks, dxs, ulps=16, label="mixed vs fp64")
        nw = gh.normwise_vs(got, ref64)
        gh._record("mixed vs fp64 normwise", nw)
        assert nw <= 2e-5
    # periodic domain: the GPU result conserves every field on its own
    tot = np.sum([o.sum(axis=(1, 2, 3)) for o in got], axis=0)
    mag = np.sum([np.abs(o).sum(axis=(1, 2, 3)) for o in got], axis=0)
    assert np.all(np.abs(tot) <= 1e-13 * mag)


# ------------------------------------------------------- uneven batch --
@pytest.mark.parametrize("prec,flags", [(hydro.FP64, 0)] +
                         [(hydro.FP32_FLUX_FP64_ACC, f) for f in MIXED_KERNELS])
def test_uneven_octree_batch(prec, flags):
    leaves = synth.uneven_octree(n_subgrids=48)
    assert {l[0] for l in leaves} == {8, 16} and {l[1] for l in leaves} == {6, 11}
    blocks = [synth.leaf_block(synth.BASE_SEED, l) for l in leaves]
    dxs = [l[2] for l in leaves]
    got, gam = _both(blocks, dxs, prec=prec, flags=flags)
    mode = 0 if prec == hydro.FP64 else 1
    ref, ram, _ = gh.oracle_ref(blocks, dxs, mode=mode)
    if mode == 0:
        gh.check_fp64(got, ref, gam, ram, blocks, dxs)
    else:
        gh.check_mixed(got, ref, gam, ram, blocks, dxs)


# --------------------------------------------------------- edge cases --
@pytest.mark.parametrize("N", [2, 3, 5, 12, 16, 17])
def test_ragged_sizes_and_partial_tiles(N):
    blocks = [synth.iid_block(synth.rng_for(7, N), N, 8)]
    dxs = [0.3]
    got, gam = _both(blocks, dxs)
    ref, ram, _ = gh.oracle_ref(blocks, dxs)
    gh.check_fp64(got, ref, gam, ram, blocks, dxs)


@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
@pytest.mark.parametrize("N", [33, hydro.HYDRO_MAX_N])
def test_large_and_largest_subgrids(N, prec):
    """One sub-grid of many tiles: N = 33 (5 tiles per edge, the last one
    cell wide) and the largest accepted edge (32768 tiles sharing one
    signal-speed slot), against the oracle in both precisions."""
    blocks = [synth.iid_block(synth.rng_for(99, N), N, 8)]
    dxs = [1.0 / N]
    got, gam = gh.run_gpu(gh.to_dev(blocks), dxs, prec=prec)
    mode = 0 if prec == hydro.FP64 else 1
    ref, ram, fl = gh.oracle_ref(blocks, dxs, mode=mode)
    assert not fl.any()
    if mode == 0:
        gh.check_fp64(got, ref, gam, ram, blocks, dxs)
    else:
        gh.check_mixed(got, ref, gam, ram, blocks, dxs)


@pytest.mark.parametrize("flags", MIXED_KERNELS)
@pytest.mark.parametrize("N", [2, 3, 5, 12, 16, 17])
def test_ragged_sizes_and_partial_tiles_mixed(N, flags):
    blocks = [synth.iid_block(synth.rng_for(7, N), N, 8 + N % 4),
              synth.iid_block(synth.rng_for(70, N), N, 6)]
    dxs = [0.3, 0.25]
    got, gam = _both(blocks, dxs, prec=hydro.FP32_FLUX_FP64_ACC, flags=flags)
    ref, ram, _ = gh.oracle_ref(blocks, dxs, mode=1)
    gh.check_mixed(got, ref, gam, ram, blocks, dxs)


def test_mixed_kernel_families_agree_bitwise():
    """The pipelined and the register-load kernels run the same arithmetic in
    the same order, so they agree bit for bit, as do the tuned plans that
    are restricted to either family."""
    leaves = synth.uneven_octree(n_subgrids=40)
    blocks = [synth.leaf_block(synth.BASE_SEED + 1, l) for l in leaves]
    blocks += [synth.iid_block(synth.rng_for(11, N), N, 7 + N % 5) for N in (3, 5, 12)]
    dxs = [l[2] for l in leaves] + [0.2, 0.3, 0.125]
    dev = gh.to_dev(blocks)
    mx = hydro.FP32_FLUX_FP64_ACC
    a, aam = gh.run_gpu(dev, dxs, prec=mx)
    b, bam = gh.run_gpu(dev, dxs, prec=mx, flags=hydro.F_REGISTER_LOADS)
    c, cam = gh.run_gpu(dev, dxs, prec=mx, form="plan",
                        plan_kw={"autotune": True, "flags": hydro.PLAN_PIPELINED})
    d, dam = gh.run_gpu(dev, dxs, prec=mx, form="plan",
                        plan_kw={"autotune": True, "flags": hydro.PLAN_REGISTER_LOADS})
    for other, oam in ((b, bam), (c, cam), (d, dam)):
        for s in range(len(blocks)):
            assert np.array_equal(other[s], a[s]), s
        assert np.array_equal(oam, aam)


@pytest.mark.parametrize("prec,flags", [(hydro.FP64, 0), (hydro.FP64, hydro.F_QUAD26),
                                        (hydro.FP32_FLUX_FP64_ACC, 0),
                                        (hydro.FP32_FLUX_FP64_ACC, hydro.F_REGISTER_LOADS)])
def test_wider_ghost_layer_is_ignored_beyond_three(prec, flags):
    U4 = synth.iid_block(synth.rng_for(8, 0), 8, 7, ghost=4)
    U4[:, 0, :, :] = np.nan  # the 4th layer is never read
    U4[:, :, -1, :] = np.nan
    dev = gh.to_dev([U4])
    got, gam = gh.run_gpu(dev, [0.1], ghost=4, prec=prec, flags=flags)
    U3 = U4[:, 1:-1, 1:-1, 1:-1].copy()
    mode = (0 if prec == hydro.FP64 else oracle.MODE_MIXED) + (oracle.QUAD26 if flags & hydro.F_QUAD26 else 0)
    ref, ram, _ = oracle.rhs_batch([U3], G53, 0.1, mode)
    if prec == hydro.FP64:
        gh.check_fp64(got, ref, gam, ram, [U3], [0.1])
    else:
        gh.check_mixed(got, ref, gam, ram, [U3], [0.1])


def test_every_field_count():
    blocks = [synth.iid_block(synth.rng_for(9, f), 8, f) for f in range(6, 12)]
    dxs = [0.125] * len(blocks)
    got, gam = _both(blocks, dxs)
    ref, ram, _ = gh.oracle_ref(blocks, dxs)
    gh.check_fp64(got, ref, gam, ram, blocks, dxs)


def test_empty_batch_is_a_noop():
    desc = hydro.descriptors([])
    hydro.rhs(desc, None, None, n=0)


def test_invalid_arguments_are_rejected():
    U = torch.zeros(6, 14, 14, 14, dtype=torch.float64, device="cuda")
    out = torch.empty(6 * 512, dtype=torch.float64, device="cuda")
    am = torch.empty(1, dtype=torch.float64, device="cuda")
    bad = [
        dict(items=[(U, 0.1, 1, 6)]),          # N < 2
        dict(items=[(U, 0.1, 8, 5)]),          # too few fields
        dict(items=[(U, 0.1, 8, 12)]),         # too many fields
        dict(items=[(U, -0.1, 8, 6)]),         # dx <= 0
        dict(items=[(U, 0.1, 8, 6)], ghost=2),
        dict(items=[(U, 0.1, 8, 6)], gamma=1.0),
        dict(items=[(U, 0.1, 8, 6)], N=16),    # uniform-batch mismatch
        dict(items=[(0, 0.1, 8, 6)]),          # NULL input
    ]
    for b in bad:
        desc = hydro.descriptors(b["items"])
        with pytest.raises(hydro.HydroError) as ei:
            hydro.rhs(desc, out, am, ghost=b.get("ghost", 3), gamma=b.get("gamma", G53),
                      N=b.get("N", 0))
        assert ei.value.code == hydro.HYDRO_EINVAL


def test_nonphysical_input_is_flagged_not_fatal():
    blocks = synth.iid_batch(4, 8, 6, seed=21)
    blocks[2] = blocks[2].copy()
    blocks[2][0, 1, 6, 6] = -1.0  # negative density in a z-ghost layer of sub-grid 2
    blocks[3] = blocks[3].copy()
    blocks[3][0, 0, 0, 0] = np.nan  # a corner cell: outside the read region
    hydro.status()  # clear
    got, gam = _both(blocks, [0.1] * 4)
    rc, bad = hydro.status()
    assert rc == hydro.HYDRO_ENONPHYS and bad == 2
    ref, ram, fl = gh.oracle_ref(blocks, [0.1] * 4)
    assert fl[2] and not fl[3]
    gh.check_fp64([got[i] for i in (0, 1, 3)], [ref[i] for i in (0, 1, 3)], gam[[0, 1, 3]],
                  ram[[0, 1, 3]], [blocks[i] for i in (0, 1, 3)], [0.1] * 3)
    rc, bad = hydro.status()
    assert rc == hydro.HYDRO_OK and bad == -1


# -------------------------------------------- forms agree bitwise --
def test_uniform_state_gives_exact_zero_on_gpu():
    shp = (22, 22, 22)
    U = synth.conserved_from_states(np.full(shp, 1.3), np.full(shp, 0.2), np.full(shp, -0.1),
                                    np.full(shp, 0.05), np.full(shp, 0.9), None)
    for prec in (hydro.FP64, hydro.FP32_FLUX_FP64_ACC):
        got, gam = _both([U, U[:, 4:-4, 4:-4, 4:-4].copy()], [0.1, 0.1], prec=prec)
        assert np.all(got[0] == 0) and np.all(got[1] == 0)


@pytest.mark.parametrize("N,F", [(8, 11), (12, 9), (16, 6), (5, 7)])
@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_uniform_batch_work_list_built_on_the_device(N, F, prec):
    """hydro_rhs_ex builds the work list of a batch of one N and one field
    count on the device from the descriptors; a plan builds it on the host.
    Both lists must describe the same tiles: the results agree bit for bit
    (widths that are powers of two and others, partial and several tiles)."""
    n = 10
    blocks = [synth.iid_block(synth.rng_for(515, s), N, F) for s in range(n)]
    dxs = [1.0 / 64, 0.3, 2.0 ** -9, 1.0 / 3.0, 0.125] * 2
    dev = gh.to_dev(blocks)
    direct, dam = gh.run_gpu(dev, dxs, prec=prec)
    plan, pam = gh.run_gpu(dev, dxs, prec=prec, form="plan")
    for s in range(n):
        assert np.array_equal(direct[s], plan[s]), s
    assert np.array_equal(dam, pam)
    want, want_am, fl = gh.oracle_ref(blocks, dxs, mode=0 if prec == hydro.FP64 else 1)
    assert not fl.any()
    if prec == hydro.FP64:
        gh.check_fp64(direct, want, dam, want_am, blocks, dxs)
    else:
        gh.check_mixed(direct, want, dam, want_am, blocks, dxs)


@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_alone_in_batch_per_subgrid_and_plan_are_bitwise_equal(prec):
    leaves = synth.uneven_octree(n_subgrids=24)
    blocks = [synth.leaf_block(synth.BASE_SEED, l) for l in leaves]
    dxs = [l[2] for l in leaves]
    dev = gh.to_dev(blocks)
    batch, bam = gh.run_gpu(dev, dxs, prec=prec)
    streams = [torch.cuda.Stream() for _ in range(4)]
    per, pam = gh.run_gpu(dev, dxs, prec=prec, form="per_subgrid", streams=streams)
    plan, plam = gh.run_gpu(dev, dxs, prec=prec, form="plan")
    tuned, tam = gh.run_gpu(dev, dxs, prec=prec, form="plan", plan_kw={"autotune": True})
    for s in (0, 5, 17):
        alone, aam = gh.run_gpu([dev[s]], [dxs[s]], prec=prec)
        assert np.array_equal(alone[0], batch[s]) and aam[0] == bam[s]
    for other, oam in ((per, pam), (plan, plam), (tuned, tam)):
        for s in range(len(blocks)):
            assert np.array_equal(other[s], batch[s]), s
        assert np.array_equal(oam, bam)
    again, agam = gh.run_gpu(dev, dxs, prec=prec)
    for s in range(len(blocks)):
        assert np.array_equal(again[s], batch[s])


# ------------------------------------- polytropes at full size, sampled --
@pytest.mark.slow
def test_polytropes_full_size_sampled():
    """The 32768-sub-grid polytrope workload at full size through a tuned
    plan (the configuration the benchmark times): sampled sub-grids against
    the oracle, all sub-grids for conservation and finiteness."""
    from bench import polytrope_batch

    batch = polytrope_batch(n=256)
    dxs = [batch.dx] * batch.n
    for prec in (hydro.FP64, hydro.FP32_FLUX_FP64_ACC):
        p = hydro.Plan(batch.desc, ghost=3, gamma=G53, prec=prec, autotune=True, n=batch.n)
        out = torch.empty(batch.out_doubles, dtype=torch.float64, device="cuda")
        amax = torch.empty(batch.n, dtype=torch.float64, device="cuda")
        p.execute(out, amax)
        rc, bad = hydro.status()
        assert rc == hydro.HYDRO_OK
        o = out.view(batch.n, 11, 8, 8, 8)
        assert torch.isfinite(o).all()
        tot = o.sum(dim=(0, 2, 3, 4)).cpu().numpy()
        mag = o.abs().sum(dim=(0, 2, 3, 4)).cpu().numpy()
        assert np.all(np.abs(tot) <= 1e-12 * mag), (tot, mag)
        rng = np.random.default_rng(5)
        sample = np.sort(rng.choice(batch.n, 96, replace=False))
        blocks = [batch.blocks[s].cpu().numpy() for s in sample]
        got = [o[s].cpu().numpy() for s in sample]
        gam = amax.cpu().numpy()[sample]
        mode = 0 if prec == hydro.FP64 else 1
        ref, ram, fl = gh.oracle_ref(blocks, [batch.dx] * len(sample), mode=mode)
        if mode == 0:
            gh.check_fp64(got, ref, gam, ram, blocks, [batch.dx] * len(sample))
        else:
            gh.check_mixed(got, ref, gam, ram, blocks, [batch.dx] * len(sample))
        p.close()
        del out, amax


# ---------------------------------------------- inputs in pinned host memory --
@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_pinned_host_buffers_are_read_in_place(prec):
    """Descriptors and outputs may point into pinned host memory: the kernels
    read and write it in place over the host link, with the same bits as
    device buffers (both mixed kernel families, plans and direct calls)."""
    leaves = synth.uneven_octree(n_subgrids=24)
    blocks = [synth.leaf_block(synth.BASE_SEED + 2, l) for l in leaves]
    dxs = [l[2] for l in leaves]
    dev = gh.to_dev(blocks)
    host = [torch.from_numpy(np.ascontiguousarray(b)).pin_memory() for b in blocks]
    ref, ram = gh.run_gpu(dev, dxs, prec=prec)
    items = [(h, dx, h.shape[1] - 6, h.shape[0]) for h, dx in zip(host, dxs)]
    desc = hydro.descriptors(items)
    n = len(items)
    out = torch.full((hydro.output_doubles(desc, n),), float("nan"), dtype=torch.float64).pin_memory()
    amax = torch.full((n,), float("nan"), dtype=torch.float64).pin_memory()
    flag_sets = [0] if prec == hydro.FP64 else [0, hydro.F_REGISTER_LOADS]
    for flags in flag_sets:
        out.fill_(float("nan"))
        hydro.rhs(desc, out, amax, prec=prec, n=n, flags=flags)
        torch.cuda.synchronize()
        off = 0
        for s, (h, dx, N, F) in enumerate(items):
            m = F * N ** 3
            assert np.array_equal(out[off:off + m].numpy().reshape(F, N, N, N), ref[s]), s
            off += m
        assert np.array_equal(amax.numpy(), ram)
    p = hydro.Plan(desc, prec=prec, autotune=True, n=n)
    out.fill_(float("nan"))
    p.execute(out, amax)
    torch.cuda.synchronize()
    p.close()
    assert np.array_equal(amax.numpy(), ram)
    assert np.array_equal(out[:ref[0].size].numpy().reshape(ref[0].shape), ref[0])


@pytest.mark.parametrize("prec,flags", [(hydro.FP64, 0), (hydro.FP32_FLUX_FP64_ACC, 0), (hydro.FP64, hydro.F_QUAD26),
                                        (hydro.FP32_FLUX_FP64_ACC, hydro.F_REGISTER_LOADS)])
def test_flux_homogeneity_under_power_of_two_scaling(prec, flags):
    """The property the oracle pin checks, on the GPU path: rho, rho v, E,
    rho X scaled by lam and tau by mu (powers of two, thermal data) scale each
    field's dU/dt by exactly that factor and leave amax unchanged, bit for
    bit, through every kernel step (seeds, Newton steps, conversions)."""
    rng = synth.rng_for(92, 0)
    G, nf, n = 14, 8, 6
    blocks = []
    for _ in range(n):
        rho = rng.uniform(0.5, 2.0, (G, G, G))
        v = [rng.normal(0.0, 0.1, (G, G, G)) for _ in range(3)]
        p = rng.uniform(0.5, 2.0, (G, G, G))
        X = np.moveaxis(rng.dirichlet(np.ones(nf - 6), size=(G, G, G)), -1, 0)
        blocks.append(synth.conserved_from_states(rho, v[0], v[1], v[2], p, X))
    ref, ra = gh.run_gpu(gh.to_dev(blocks), [0.125] * n, prec=prec, flags=flags)
    for lam, mu in ((4.0, 0.125), (0.25, 2.0)):
        scaled = []
        for b in blocks:
            V = b * lam
            V[5] = b[5] * mu
            scaled.append(V)
        got, ga = gh.run_gpu(gh.to_dev(scaled), [0.125] * n, prec=prec, flags=flags)
        assert np.array_equal(ga, ra)
        for s in range(n):
            for f in range(nf):
                assert np.array_equal(got[s][f], ref[s][f] * (mu if f == 5 else lam)), (s, f, lam)
