"""Inputs that start 8 but not 16 bytes aligned.  The mixed form's pipelined
kernel stages full tiles by 16-byte copies where the stored rows allow it
(ghosted blocks with even G and odd ghost width, ghost-free domains and
forest leaves of even N, 16-byte aligned blocks) and by one 8-byte copy per
cell otherwise.  The same data placed 8 bytes off must give the same bits
through the second path as through the first."""
import numpy as np
import pytest
import torch

import paper_2210_06438_gb300 as hydro
import synth
from tests import gpu_helpers as gh

pytestmark = pytest.mark.gpu
MX = hydro.FP32_FLUX_FP64_ACC


def _shifted(a):
    """A device copy of array `a` whose first element sits 8 bytes past a
    16-byte boundary (torch allocations are 256-byte aligned)."""
    a = np.ascontiguousarray(a)
    flat = torch.empty(a.size + 1, dtype=torch.float64, device="cuda")
    view = flat[1:].view(a.shape)
    view.copy_(torch.from_numpy(a))
    assert view.data_ptr() % 16 == 8
    return view


@pytest.mark.parametrize("prec", [hydro.FP64, MX])
def test_ghosted_blocks_off_the_16_byte_grid(prec):
    host = [synth.iid_block(synth.rng_for(606, s), 8, 11) for s in range(24)]
    dxs = [1.0 / 64, 0.3] * 12
    aligned = gh.to_dev(host)
    shifted = [_shifted(b) for b in host]
    a, aam = gh.run_gpu(aligned, dxs, prec=prec)
    b, bam = gh.run_gpu(shifted, dxs, prec=prec)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(aam, bam)


@pytest.mark.parametrize("N,n", [(8, 32), (16, 32)])
def test_domain_off_the_16_byte_grid(N, n):
    glob = synth.plain_domain(seed=23, n=n, nf=11)
    nb = n // N
    dom = glob.reshape(11, nb, N, nb, N, nb, N).transpose(1, 3, 5, 0, 2, 4, 6).reshape(nb ** 3, 11, N, N, N)
    outs = []
    for U in (torch.from_numpy(np.ascontiguousarray(dom)).cuda(), _shifted(dom)):
        out = torch.full(U.shape, float("nan"), dtype=torch.float64, device="cuda")
        am = torch.full((nb ** 3,), float("nan"), dtype=torch.float64, device="cuda")
        hydro.domain_rhs(U, nb, N, 11, 1.0 / n, out, am, prec=MX)
        torch.cuda.synchronize()
        outs.append((out.cpu().numpy(), am.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_forest_leaves_off_the_16_byte_grid():
    lv = synth.forest_leaves(2, 2, synth.random_refine(7, 0.25), seed=7)
    U, dx0 = synth.smooth_forest_state(lv, 2, 8, nf=11, seed=38)
    n = U.shape[0]
    outs = []
    for Ud in (torch.from_numpy(np.ascontiguousarray(U)).cuda(), _shifted(U)):
        fo = hydro.Forest(lv, 2, 8, 11)
        out = torch.full(Ud.shape, float("nan"), dtype=torch.float64, device="cuda")
        am = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        fo.rhs(Ud, dx0, out, am, prec=MX)
        torch.cuda.synchronize()
        fo.close()
        outs.append((out.cpu().numpy(), am.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
