"""GPU parity of the 26-point quadrature variant (HYDRO_F_QUAD26, Sec. IV-B)
against the oracle's QUAD26 mode, in both precision forms, with partial
tiles, the one-sided flux, plans and conservation."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_06438_gb300 as hydro
import synth
from tests import gpu_helpers as gh

pytestmark = pytest.mark.gpu
Q = oracle.QUAD26
MX = hydro.FP32_FLUX_FP64_ACC


def _check(prec, blocks, dxs, knp=False, **kw):
    flags = hydro.F_QUAD26 | (hydro.F_KNP if knp else 0)
    got, gam = gh.run_gpu(gh.to_dev(blocks), dxs, prec=prec, flags=flags, **kw)
    mode = Q | (oracle.FLUX_KNP if knp else 0) | (0 if prec == hydro.FP64 else oracle.MODE_MIXED)
    ref, ram, fl = gh.oracle_ref(blocks, dxs, mode=mode)
    assert not fl.any()
    if prec == hydro.FP64:
        gh.check_fp64(got, ref, gam, ram, blocks, dxs)
    else:
        gh.check_mixed(got, ref, gam, ram, blocks, dxs)
    return got, gam


@pytest.mark.parametrize("prec", [hydro.FP64, MX])
@pytest.mark.parametrize("nf", [6, 11])
def test_one_subgrid(prec, nf):
    U, dx = synth.one_subgrid(nf=nf)
    _check(prec, [U], [dx])


@pytest.mark.parametrize("prec", [hydro.FP64, MX])
def test_uneven_octree_batch(prec):
    leaves = synth.uneven_octree(n_subgrids=24)
    assert {l[0] for l in leaves} == {8, 16}
    blocks = [synth.leaf_block(synth.BASE_SEED, l) for l in leaves]
    _check(prec, blocks, [l[2] for l in leaves])


@pytest.mark.parametrize("N", [3, 5, 12])
def test_ragged_sizes_and_partial_tiles(N):
    blocks = [synth.iid_block(synth.rng_for(17, N), N, 6 + N % 6)]
    for prec in (hydro.FP64, MX):
        _check(prec, blocks, [0.2])


def test_one_sided_flux():
    blocks = synth.iid_batch(6, 8, 11, seed=51)
    _check(hydro.FP64, list(blocks), [0.125] * 6, knp=True)


def test_uniform_state_exact_zero_and_plan_matches_direct_call():
    shp = (14, 14, 14)
    U = synth.conserved_from_states(np.full(shp, 1.3), np.full(shp, 0.2), np.full(shp, -0.1),
                                    np.full(shp, 0.05), np.full(shp, 0.9), None)
    for prec in (hydro.FP64, MX):
        got, _ = gh.run_gpu(gh.to_dev([U]), [0.1], prec=prec, flags=hydro.F_QUAD26)
        assert np.all(got[0] == 0)
    blocks = synth.iid_batch(10, 8, 8, seed=52)
    dev = gh.to_dev(list(blocks))
    for prec in (hydro.FP64, MX):
        a, aam = gh.run_gpu(dev, [0.125] * 10, prec=prec, flags=hydro.F_QUAD26)
        b, bam = gh.run_gpu(dev, [0.125] * 10, prec=prec, form="plan",
                            plan_kw={"autotune": True, "flags": hydro.PLAN_QUAD26})
        for s in range(10):
            assert np.array_equal(a[s], b[s])
        assert np.array_equal(aam, bam)


def test_periodic_conservation():
    glob = synth.plain_domain(seed=53, n=32, nf=11)
    blocks = list(synth.gather_blocks(glob, 8))
    for prec in (hydro.FP64, MX):
        got, _ = gh.run_gpu(gh.to_dev(blocks), [1.0 / 32] * len(blocks), prec=prec, flags=hydro.F_QUAD26)
        tot = np.sum([o.sum(axis=(1, 2, 3)) for o in got], axis=0)
        mag = np.sum([np.abs(o).sum(axis=(1, 2, 3)) for o in got], axis=0)
        assert np.all(np.abs(tot) <= 1e-13 * mag)


@pytest.mark.parametrize("flags", [hydro.F_QUAD26, hydro.F_QUAD26 | hydro.F_KNP, hydro.F_KNP])
@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_per_subgrid_form_with_flags_gives_the_aggregated_bits(prec, flags):
    """hydro_rhs_per_subgrid_ex: one launch per sub-grid over a stream pool
    runs the flux variant of its flags with the aggregated form's bits."""
    blocks = [torch.from_numpy(synth.iid_block(synth.rng_for(808, s), N, F)).cuda()
              for s, (N, F) in enumerate([(8, 11), (16, 6), (5, 8), (8, 7), (12, 11)])]
    desc = hydro.descriptors([(b, 0.2, b.shape[1] - 6, b.shape[0]) for b in blocks])
    n = len(blocks)
    nout = hydro.output_doubles(desc, n)
    ref = torch.empty(nout, dtype=torch.float64, device="cuda")
    ram = torch.empty(n, dtype=torch.float64, device="cuda")
    hydro.rhs(desc, ref, ram, prec=prec, n=n, flags=flags)
    out = torch.full((nout,), float("nan"), dtype=torch.float64, device="cuda")
    am = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    pool = [torch.cuda.Stream() for _ in range(3)]
    for st in pool:  # the pool's streams do not order themselves after the fills above
        st.wait_stream(torch.cuda.current_stream())
    hydro.rhs_per_subgrid(desc, out, am, pool, prec=prec, n=n, flags=flags)
    torch.cuda.synchronize()
    assert torch.equal(out, ref) and torch.equal(am, ram)
