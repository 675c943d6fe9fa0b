"""Direct calls (hydro_rhs_ex, hydro_rhs_per_subgrid) from several host
threads at once, on their own streams: each thread's results must be those
of the same call made alone, bit for bit.  The library takes a work-list
slot per call (four slots, each with its own lock) instead of one process
lock, so the calls build their work lists and wait for their slots
concurrently; ctypes releases the interpreter lock during each call."""
import threading

import numpy as np
import pytest
import torch

import paper_2210_06438_gb300 as hydro
import synth

pytestmark = pytest.mark.gpu


def _batch(seed, n, N, F):
    blocks = [torch.from_numpy(synth.iid_block(synth.rng_for(seed, s), N, F)).cuda() for s in range(n)]
    desc = hydro.descriptors([(b, 0.1, N, F) for b in blocks])
    return blocks, desc


@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_direct_calls_from_several_threads(prec):
    specs = [(901, 40, 8, 11), (902, 9, 16, 6), (903, 33, 8, 6), (904, 5, 12, 9), (905, 64, 8, 7),
             (906, 3, 16, 11)]
    batches = [_batch(*sp) for sp in specs]
    refs = []
    for (blocks, desc), (_, n, N, F) in zip(batches, specs):
        out = torch.empty(hydro.output_doubles(desc, n), dtype=torch.float64, device="cuda")
        am = torch.empty(n, dtype=torch.float64, device="cuda")
        hydro.rhs(desc, out, am, prec=prec, n=n)
        torch.cuda.synchronize()
        refs.append((out.clone(), am.clone()))
    streams = [torch.cuda.Stream() for _ in specs]
    results = [None] * len(specs)
    errors = []

    def work(i):
        try:
            blocks, desc = batches[i]
            _, n, N, F = specs[i]
            outs = []
            for rep in range(12):
                with torch.cuda.stream(streams[i]):  # the fills run on the call's own stream
                    out = torch.full((hydro.output_doubles(desc, n),), float("nan"), dtype=torch.float64,
                                     device="cuda")
                    am = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
                if rep % 3 == 2:
                    hydro.rhs_per_subgrid(desc, out, am, [streams[i]], prec=prec, n=n)
                else:
                    hydro.rhs(desc, out, am, prec=prec, n=n, stream=streams[i])
                outs.append((out, am))
            streams[i].synchronize()
            results[i] = outs
        except Exception as e:  # reported by the main thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(specs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    torch.cuda.synchronize()
    for i, outs in enumerate(results):
        for out, am in outs:
            assert torch.equal(out, refs[i][0]) and torch.equal(am, refs[i][1]), ("batch", i)
    rc, bad = hydro.status()
    assert rc == hydro.HYDRO_OK
