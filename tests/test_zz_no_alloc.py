"""hydro_rhs_noalloc, the entry point for callers that cannot allocate
(graph capture that forbids allocation, real-time loops, processes whose
device memory belongs to another allocator).  Called through the C ABI twice
in a row on the same batch, its results must equal those of hydro_rhs_ex, the
allocating entry point, within the parity tolerance of the GPU tests (they are
normally bitwise equal: the same kernel code with the same per-cell
arithmetic).  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

import paper_2210_06438_gb300 as hydro
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,F,n", [(8, 11, 64), (16, 6, 9)])
@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_noalloc_matches_the_allocating_entry_point_twice(N, F, n, prec):
    blocks = [torch.from_numpy(synth.iid_block(synth.rng_for(77, s), N, F)).cuda() for s in range(n)]
    dxs = [1.0 / (8 * N), 0.3] * (n // 2) + [1.0 / (8 * N)] * (n % 2)  # power-of-two and not
    desc = hydro.descriptors([(b, dx, N, F) for b, dx in zip(blocks, dxs)])
    nout = hydro.output_doubles(desc, n)
    ref = torch.empty(nout, dtype=torch.float64, device="cuda")
    ref_am = torch.empty(n, dtype=torch.float64, device="cuda")
    hydro.rhs(desc, ref, ref_am, N=N, n_fields=F, prec=prec, n=n)
    for _ in range(2):
        out = torch.full((nout,), float("nan"), dtype=torch.float64, device="cuda")
        am = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        hydro.rhs_noalloc(desc, out, am, N=N, n_fields=F, prec=prec, n=n)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        # the GPU parity tolerance: 1e-12 of the per-(sub-grid, field) scale
        o = out.view(n, F, -1)
        r = ref.view(n, F, -1)
        scale = r.abs().amax(dim=2).clamp_min(1e-300)
        assert float(((o - r).abs().amax(dim=2) / scale).max()) <= 1e-12
        assert float(((am - ref_am).abs() / ref_am.abs().clamp_min(1e-300)).max()) <= 1e-14


def test_noalloc_rejects_batches_beyond_its_scratch():
    d = hydro.descriptors([(8, 0.1, 8, 6)] * (hydro.NOALLOC_MAX_SUBGRIDS + 1))
    with pytest.raises(hydro.HydroError) as ei:
        hydro.rhs_noalloc(d, 8, 8, N=8, n_fields=6)
    assert ei.value.code == hydro.HYDRO_ETOOBIG
    mixed = hydro.descriptors([(8, 0.1, 8, 6), (8, 0.1, 16, 6)])
    with pytest.raises(hydro.HydroError) as ei:
        hydro.rhs_noalloc(mixed, 8, 8, N=8, n_fields=6)
    assert ei.value.code == hydro.HYDRO_EINVAL
