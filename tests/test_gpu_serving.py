"""The serving loop on the GPU: tasks submitted while others run are batched
into shared launches, and every task's result is the same alone and in the
mix (the same kernel arithmetic, so bitwise); budget admission and rejection."""
import time

import numpy as np
import pytest
import torch

import paper_2210_06438_gb300 as hydro
import synth

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0


def _pool(n=24, seed=31):
    rng = np.random.default_rng(seed)
    blocks, meta = [], []
    for s in range(n):
        N = 16 if s % 6 == 5 else 8
        F = int(rng.integers(6, 12))
        blocks.append(torch.from_numpy(synth.iid_block(synth.rng_for(seed, s), N, F)).cuda())
        meta.append((N, F, 1.0 / (8 * N)))
    return blocks, meta


@pytest.mark.parametrize("flags", [0, hydro.F_QUAD26, hydro.F_KNP])
@pytest.mark.parametrize("prec", [hydro.FP64, hydro.FP32_FLUX_FP64_ACC])
def test_results_are_identical_alone_and_in_the_mix(prec, flags):
    blocks, meta = _pool()
    rng = np.random.default_rng(3)
    tasks = []
    for t in range(40):
        k = int(rng.integers(1, 6))
        ids = rng.choice(len(blocks), k, replace=False)
        items = [(blocks[i], meta[i][2], meta[i][0], meta[i][1]) for i in ids]
        desc = hydro.descriptors(items)
        nout = hydro.output_doubles(desc, k)
        tasks.append((desc, k, torch.full((nout,), float("nan"), dtype=torch.float64, device="cuda"),
                      torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")))
    srv = hydro.Server(n_streams=3, max_batch=12, prec=prec, flags=flags)
    tickets = []
    for i, (desc, k, out, am) in enumerate(tasks):
        rc, t = srv.submit(desc, out, am, n=k)
        assert rc == hydro.HYDRO_OK
        tickets.append(t)
        if i % 7 == 0:
            time.sleep(0.0005)
    for t in tickets:
        assert srv.wait(t, 30_000_000_000) == hydro.HYDRO_OK
    torch.cuda.synchronize()
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(tasks) and st["launches"] < len(tasks)  # aggregation happened
    assert st["max_subgrids_per_launch"] <= 12
    for desc, k, out, am in tasks:
        ref = torch.empty_like(out)
        ram = torch.empty_like(am)
        hydro.rhs(desc, ref, ram, prec=prec, n=k, flags=flags)
        torch.cuda.synchronize()
        assert torch.equal(out, ref) and torch.equal(am, ram)


def test_budget_admission_on_the_gpu():
    blocks, meta = _pool(8)
    items = [(blocks[i], meta[i][2], meta[i][0], meta[i][1]) for i in range(2)]
    desc = hydro.descriptors(items)
    nout = hydro.output_doubles(desc, 2)
    one = sum(((m[0] + 6) ** 3 + m[0] ** 3) * m[1] * 8 + 8 for m in meta[:2])
    srv = hydro.Server(n_streams=4, budget_bytes=2 * one)
    outs = [torch.empty(nout, dtype=torch.float64, device="cuda") for _ in range(10)]
    ams = [torch.empty(2, dtype=torch.float64, device="cuda") for _ in range(10)]
    ts = [srv.submit(desc, outs[i], ams[i], n=2)[1] for i in range(10)]
    for t in ts:
        assert srv.wait(t, 30_000_000_000) == hydro.HYDRO_OK
    st = srv.stats()
    assert st["peak_bytes_in_flight"] <= 2 * one and st["completed"] == 10
    big = hydro.descriptors([(blocks[i], meta[i][2], meta[i][0], meta[i][1]) for i in range(8)])
    rc, _ = srv.submit(big, outs[0], ams[0], n=8)
    assert rc == hydro.HYDRO_EBUDGET
    srv.close()
    torch.cuda.synchronize()
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
