"""GPU parity of the one-sided central-upwind flux (HYDRO_F_KNP) against the
oracle's KNP mode, in both precision forms, and its plan/serving paths."""
import numpy as np
import pytest
import torch

import oracle
import paper_2210_06438_gb300 as hydro
import synth
from tests import gpu_helpers as gh

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,flags", [(hydro.FP64, 0), (hydro.FP32_FLUX_FP64_ACC, 0),
                                        (hydro.FP32_FLUX_FP64_ACC, hydro.F_REGISTER_LOADS)])
def test_knp_parity_uneven_batch(prec, flags):
    leaves = synth.uneven_octree(n_subgrids=40)
    blocks = [synth.leaf_block(synth.BASE_SEED, l) for l in leaves]
    dxs = [l[2] for l in leaves]
    got, gam = gh.run_gpu(gh.to_dev(blocks), dxs, prec=prec, flags=hydro.F_KNP | flags)
    mode = (0 if prec == hydro.FP64 else 1) + oracle.FLUX_KNP
    ref, ram, _ = gh.oracle_ref(blocks, dxs, mode=mode)
    if prec == hydro.FP64:
        gh.check_fp64(got, ref, gam, ram, blocks, dxs)
    else:
        gh.check_mixed(got, ref, gam, ram, blocks, dxs)
    # the two fluxes differ (KNP is not the single-speed flux)
    kt, _ = gh.run_gpu(gh.to_dev(blocks), dxs, prec=prec)
    assert max(np.abs(a - b).max() for a, b in zip(got, kt)) > 0


def test_knp_plan_and_server_match_direct_call():
    blocks = synth.iid_batch(12, 8, 11, seed=41)
    dev = gh.to_dev(blocks)
    dxs = [0.125] * 12
    direct, dam = gh.run_gpu(dev, dxs, flags=hydro.F_KNP)
    plan, pam = gh.run_gpu(dev, dxs, form="plan", plan_kw={"knp": True, "autotune": True})
    for a, b in zip(direct, plan):
        assert np.array_equal(a, b)
    assert np.array_equal(dam, pam)
    desc = hydro.descriptors([(b, 0.125, 8, 11) for b in dev])
    out = torch.empty(hydro.output_doubles(desc), dtype=torch.float64, device="cuda")
    am = torch.empty(12, dtype=torch.float64, device="cuda")
    srv = hydro.Server(knp=True)
    rc, t = srv.submit(desc, out, am, n=12)
    assert rc == hydro.HYDRO_OK and srv.wait(t) == hydro.HYDRO_OK
    srv.close()
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.array_equal(o, np.concatenate([d.ravel() for d in direct]))
