"""hydro_rhs_noalloc, the entry point for callers that cannot allocate device
memory: real-time loops in which an allocation (which may synchronise the
whole device) is not allowed, and processes whose device memory belongs to
another allocator that must not be bypassed or has handed all of it out.

Called through the C ABI twice in a row on the same batch, its results must
equal those of hydro_rhs_ex, the allocating entry point, bit for bit (its
register-load kernel has the same per-cell arithmetic), and match the oracle
under the parity tolerances of the other GPU tests.  A call made after the
first one must leave the device's free memory and torch's allocated bytes
unchanged.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

import paper_2210_06438_gb300 as hydro
import synth
from tests import gpu_helpers as gh

pytestmark = pytest.mark.gpu


def _batch(N, F, n):
    host = [synth.iid_block(synth.rng_for(77, s), N, F) for s in range(n)]
    blocks = [torch.from_numpy(b).cuda() for b in host]
    dxs = [1.0 / (8 * N), 0.3] * (n // 2) + [1.0 / (8 * N)] * (n % 2)  # power-of-two and not
    desc = hydro.descriptors([(b, dx, N, F) for b, dx in zip(blocks, dxs)])
    return host, blocks, dxs, desc


@pytest.mark.parametrize("N,F,n", [(8, 11, 64), (16, 6, 9)])
@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_noalloc_matches_the_allocating_entry_point_twice(N, F, n, prec):
    host, blocks, dxs, desc = _batch(N, F, n)
    nout = hydro.output_doubles(desc, n)
    ref = torch.empty(nout, dtype=torch.float64, device="cuda")
    ref_am = torch.empty(n, dtype=torch.float64, device="cuda")
    hydro.rhs(desc, ref, ref_am, N=N, n_fields=F, prec=prec, n=n)
    outs = []
    for _ in range(2):
        out = torch.full((nout,), float("nan"), dtype=torch.float64, device="cuda")
        am = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        hydro.rhs_noalloc(desc, out, am, N=N, n_fields=F, prec=prec, n=n)
        torch.cuda.synchronize()
        assert torch.equal(out, ref) and torch.equal(am, ref_am)
        outs.append((out, am))
    # and against the oracle under the standard gates of the two forms
    mode = 0 if prec == hydro.FP64 else 1
    want, want_am, fl = gh.oracle_ref(host, dxs, mode=mode)
    assert not fl.any()
    o = outs[1][0].cpu().numpy()
    got = [o[s * F * N ** 3:(s + 1) * F * N ** 3].reshape(F, N, N, N) for s in range(n)]
    if mode == 0:
        gh.check_fp64(got, want, outs[1][1].cpu().numpy(), want_am, host, dxs)
    else:
        gh.check_mixed(got, want, outs[1][1].cpu().numpy(), want_am, host, dxs)


@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_noalloc_allocates_no_device_memory(prec):
    _, blocks, dxs, desc = _batch(8, 11, 200)
    n = 200
    out = torch.empty(hydro.output_doubles(desc, n), dtype=torch.float64, device="cuda")
    am = torch.empty(n, dtype=torch.float64, device="cuda")
    hydro.rhs_noalloc(desc, out, am, N=8, n_fields=11, prec=prec, n=n)  # first call: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        hydro.rhs_noalloc(desc, out, am, N=8, n_fields=11, prec=prec, n=n)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_rejects_batches_beyond_its_scratch():
    d = hydro.descriptors([(8, 0.1, 8, 6)] * (hydro.NOALLOC_MAX_SUBGRIDS + 1))
    with pytest.raises(hydro.HydroError) as ei:
        hydro.rhs_noalloc(d, 8, 8, N=8, n_fields=6)
    assert ei.value.code == hydro.HYDRO_ETOOBIG
    mixed = hydro.descriptors([(8, 0.1, 8, 6), (8, 0.1, 16, 6)])
    with pytest.raises(hydro.HydroError) as ei:
        hydro.rhs_noalloc(mixed, 8, 8, N=8, n_fields=6)
    assert ei.value.code == hydro.HYDRO_EINVAL
    one = hydro.descriptors([(8, 0.1, 8, 6)])
    with pytest.raises(hydro.HydroError) as ei:  # 0 ("any") is not accepted here
        hydro.rhs_noalloc(one, 8, 8, N=0, n_fields=6)
    assert ei.value.code == hydro.HYDRO_EINVAL
