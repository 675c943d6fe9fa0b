#!/usr/bin/env python3
"""Benchmark of the aggregated hydro RHS on one GB300 (or N replicas).

Workload (default): 32768 sub-grids of 8^3 (256^3 cells, 11 fields: rho,
momentum, E, tau and 5 species) holding two n = 1.5 polytropes on a 1e-10
atmosphere; inputs ~7.9 GB on the device, far larger than L2.

Metric: cell-updates/s of one RHS evaluation (interior cells x evaluations /
s).  `value` is the binary64 aggregated form (one tuned, graph-replayed launch
per step); the JSON line also carries the mixed binary32/binary64 form, the
per-sub-grid launch form, the end-to-end number through the C ABI with host
buffers, the roofline of the dominant kernel and the oracle timed on the host
cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

GAMMA = 5.0 / 3.0
METRIC = "cell-updates/s (aggregated FP64 hydro RHS: PPM + Kurganov-Tadmor)"
WORKLOAD = "polytropes: 32768 sub-grids of 8^3 + 3 ghost layers (256^3 cells), 11 FP64 fields"


# ------------------------------------------------------------ workloads --
class Batch:
    pass


def polytrope_batch(n=256, nf=11, N=8, device="cuda", chunk=2048):
    """Ghosted sub-grids of the polytrope domain, resident on the device.

    The global periodic array is drawn on the host (synth.polytropes), copied
    once, and cut into ghosted blocks on the device with index gathers."""
    import torch

    import paper_2210_06438_gb300 as hydro

    glob = synth.polytropes(n=n, nf=nf)
    gd = torch.from_numpy(glob).to(device)
    del glob
    nb = n // N
    S = nb ** 3
    G = N + 6
    blocks = torch.empty((S, nf, G, G, G), dtype=torch.float64, device=device)
    r = torch.arange(-3, N + 3, device=device)
    ids = torch.arange(S, device=device)
    bx, by, bz = ids % nb, (ids // nb) % nb, ids // (nb * nb)
    for s0 in range(0, S, chunk):
        sl = slice(s0, min(S, s0 + chunk))
        ix = (bx[sl, None] * N + r[None, :]) % n
        iy = (by[sl, None] * N + r[None, :]) % n
        iz = (bz[sl, None] * N + r[None, :]) % n
        g = gd[:, iz[:, :, None, None], iy[:, None, :, None], ix[:, None, None, :]]
        blocks[sl] = g.permute(1, 0, 2, 3, 4)
    del gd
    torch.cuda.synchronize()
    b = Batch()
    b.n, b.N, b.nf, b.dx = S, N, nf, 2.0 / n
    b.blocks = blocks
    b.desc = hydro.descriptors([(int(blocks[s].data_ptr()), b.dx, N, nf) for s in range(S)])
    b.out_doubles = S * nf * N ** 3
    b.cells = S * N ** 3
    b.alg_bytes = S * synth.algorithmic_bytes(N, nf)
    return b


# -------------------------------------------------- algorithmic counts --
def fp64_ops_per_cell(N=8, F=11):
    """Floating-point operations (add, sub, mul, div, sqrt; comparisons and
    selections not counted) of the reference definition per interior cell:
      primitives  (F + 9) per read cell,  (N^3 + 18 N^2) read cells
      PPM         per line and field: (N+4) slopes x 6 + (N+3) faces x 5
                  + (N+2) limited cells x 10;  3 N^2 lines
      flux        10 F + 26 per face;  3 N^2 (N+1) faces
      divergence  6 F per cell"""
    n3 = N ** 3
    prim = (F + 9) * (n3 + 18 * N * N)
    ppm = 3 * N * N * F * ((N + 4) * 6 + (N + 3) * 5 + (N + 2) * 10)
    flux = 3 * N * N * (N + 1) * (10 * F + 26)
    div = 6 * F * n3
    return (prim + ppm + flux + div) / n3


def fp64_peak_gflops(sm_mhz, n_sm=152):
    """binary64 FMA pipe: 2 DFMA per SM per clock (measured on this GPU:
    1.6-2.0 per clock), i.e. 4 flop per SM per clock."""
    return n_sm * 4 * sm_mhz * 1e-3


# ---------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.first = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
            return
        # nvidia-smi takes a moment to start: wait (up to 2 s) for its first
        # sample so that the timed region that follows is sampled throughout
        t_end = time.perf_counter() + 2.0
        while not self.lines and self.proc.poll() is None and time.perf_counter() < t_end:
            time.sleep(0.01)
        self.first = len(self.lines)  # samples before this one were taken before the region

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[self.first:] or self.lines
        for ln in lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- timing --
def time_steps(fn, steps, warmup, stream):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def time_flushed(fn, steps, warmup, stream, flush=None):
    """Per-step CUDA-event times (ms) of fn on `stream`, with an L2 flush
    (a write of a buffer larger than L2) before every step, outside the
    events.  Returns (median, p10, p90)."""
    import torch

    for _ in range(warmup):
        fn()
    ts = []
    for _ in range(steps):
        if flush is not None:
            flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return (float(np.median(ts)), float(np.percentile(ts, 10)), float(np.percentile(ts, 90)))


def fp64_probe_peak(stream, reps=7, iters=20000):
    """Measured binary64 peak (GFLOP/s): the library's fused multiply-add
    probe (hydro_probe_fp64), timed with CUDA events on `stream`, median of
    `reps` launches after one warm-up launch."""
    import torch

    import paper_2210_06438_gb300 as hydro

    hydro.probe_fp64(4, 1000, stream)
    ts = []
    n = 0.0
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        n = hydro.probe_fp64(4, iters, stream)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ms = float(np.median(ts))
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return {"gflops": 2.0 * n / (ms * 1e-3) * 1e-9, "ms": ms, "fma_per_launch": n, "sms": n_sm,
            "launches": reps}


def normwise_error(got, ref, ref_amax, batch):
    """max over (sub-grid, field) of max|got - ref| / max(max|ref|, S), with
    the flux-divergence floor S = amax * max|U_f| / dx of the parity tests."""
    g = got.view(batch.n, batch.nf, -1)
    r = ref.view(batch.n, batch.nf, -1)
    umax = batch.blocks.abs().amax(dim=(2, 3, 4))
    floor = ref_amax[:, None] * umax / batch.dx
    scale = torch_max(r.abs().amax(dim=2), floor).clamp_min(1e-300)
    return float(((g - r).abs().amax(dim=2) / scale).max())


def torch_max(a, b):
    import torch

    return torch.maximum(a, b)


def conservation_drift(out, batch):
    """|sum of dU/dt| / sum |dU/dt| over the periodic domain, worst field."""
    o = out.view(batch.n, batch.nf, -1)
    return float((o.sum(dim=(0, 2)) / o.abs().sum(dim=(0, 2)).clamp_min(1e-300)).abs().max())


def max_over_ranks(values, world, device="cuda"):
    """Element-wise maximum of per-rank timings (all ranks get the result)."""
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def kernel_source_digest(path):
    """sha256 of a CUDA source with // comments and blank lines removed (so
    that the record follows code changes, not comment edits)."""
    import hashlib
    import re

    lines = []
    for line in open(path, encoding="utf-8"):
        line = re.sub(r"//.*", "", line).rstrip()
        if line:
            lines.append(line)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def recorded_traffic(form, n_tiles):
    """DRAM bytes of one launch from the committed ncu record, scaled to
    n_tiles; None unless the kernel source's code still matches the record."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
        src = os.path.join(ROOT, "paper_2210_06438_gb300", "csrc", "hydro_kernels.cuh")
        if kernel_source_digest(src) != rec["kernel_code_sha256"]:
            return None
        return rec["forms"][form]["bytes_per_tile"] * n_tiles
    except Exception:
        return None


def recorded_counts(form):
    """The committed ncu record of a form (bytes and instruction counts per
    tile), or None unless the kernel source's code still matches it."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
        src = os.path.join(ROOT, "paper_2210_06438_gb300", "csrc", "hydro_kernels.cuh")
        if kernel_source_digest(src) != rec["kernel_code_sha256"]:
            return None
        return rec["forms"][form]
    except Exception:
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# --------------------------------------------------------------- serving --
def serving_run(rate, duration, per_task, budget=40 << 30, n_streams=4, max_batch=4096,
                pool_per_f=96, ring_bytes=4 << 30, seed=synth.BASE_SEED, prec=0):
    """Replay a Poisson task stream (synth.serving_trace) through the server.

    Sub-grid states live in a device pool (pool_per_f sub-grids of 8^3 for each
    field count 6..11); each task draws its sub-grids from the pool of its field
    count and writes into its own slice of an output ring.  Tasks are submitted
    at their arrival times from this thread.  Returns throughput and latency
    percentiles (completion - arrival, host monotonic clock)."""
    import torch

    import paper_2210_06438_gb300 as hydro

    t_arr, sizes, nfs = synth.serving_trace(seed, rate=rate, duration=duration)
    rng = np.random.default_rng(seed)
    pools = {}
    for F in range(6, 12):
        blk = torch.empty((pool_per_f, F, 14, 14, 14), dtype=torch.float64, device="cuda")
        for i in range(pool_per_f):
            blk[i] = torch.from_numpy(synth.iid_block(synth.rng_for(seed, 7000 + 100 * F + i), 8, F))
        pools[F] = blk
    ring = torch.empty(ring_bytes // 8, dtype=torch.float64, device="cuda")
    ring_am = torch.empty(1 << 20, dtype=torch.float64, device="cuda")
    descs = []
    for k in range(t_arr.size):
        F = int(nfs[k])
        ids = rng.integers(0, pool_per_f, int(sizes[k]))
        descs.append(hydro.descriptors([(int(pools[F][i].data_ptr()), 1.0 / 64, 8, F) for i in ids]))
    srv = hydro.Server(budget_bytes=budget, max_batch=max_batch, n_streams=n_streams,
                       per_task=per_task, prec=prec)
    off = 0
    aoff = 0
    slot_owner = {}
    tickets = []
    t0 = time.perf_counter() + 0.05
    for k in range(t_arr.size):
        n = int(sizes[k])
        need = n * int(nfs[k]) * 512
        if off + need > ring.numel():
            off = 0
        if aoff + n > ring_am.numel():
            aoff = 0
        prev = slot_owner.get(off)
        if prev is not None:
            srv.wait(prev)
        while time.perf_counter() < t0 + t_arr[k]:
            pass
        rc, t = srv.submit(descs[k], int(ring.data_ptr()) + 8 * off, int(ring_am.data_ptr()) + 8 * aoff, n=n)
        if rc != hydro.HYDRO_OK:
            raise RuntimeError("submit failed: %d" % rc)
        tickets.append((t, n))
        slot_owner[off] = t
        off += need
        aoff += n
    for t, _ in tickets:
        srv.wait(t)
    torch.cuda.synchronize()
    lat, first, last, cells = [], None, None, 0
    for t, n in tickets:
        ts, tl, td = srv.times(t)
        lat.append((td - ts) * 1e-3)
        first = ts if first is None else min(first, ts)
        last = td if last is None else max(last, td)
        cells += n * 512
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    return {"tasks": len(tickets), "offered_tasks_per_s": rate, "duration_s": duration,
            "cell_updates_per_s": cells / ((last - first) * 1e-9),
            "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
            "mean_us": float(lat.mean()), "launches": st["launches"],
            "max_subgrids_per_launch": st["max_subgrids_per_launch"],
            "peak_bytes_in_flight": st["peak_bytes_in_flight"], "per_task": per_task}


# ------------------------------------------------------------- Sedov --
def rk3_device_loop(step_pair, clock, t_end, stream, chunk=16):
    """A time loop with the step computed on the device.  step_pair(forward)
    runs one step (hydro_courant, then three *_stage_dt launches) from one
    state buffer to the other (forward: first to second).  Two CUDA graphs of
    `chunk` (even) steps are recorded, one per buffer the state starts in,
    so a replay leaves it where it was.  Returns run(), which advances to
    t_end: graph replays while t_end is more than 2 chunk dt away, single
    steps after that (the device clamps the last dt to t_end), with one host
    read of the clock per replay or step; run() returns (steps, whether the
    final state is in the second buffer)."""
    import torch

    assert chunk % 2 == 0
    graphs = {}
    for first in (True, False):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for i in range(chunk):
                step_pair(first == (i % 2 == 0))
        graphs[first] = g

    def run():
        t, dt_last, k, at_first = 0.0, 0.0, 0, True
        while t < t_end:
            if dt_last > 0.0 and t_end - t > 2.0 * chunk * dt_last:
                graphs[at_first].replay()
            else:
                step_pair(at_first)
                at_first = not at_first
            stream.synchronize()
            c = clock.cpu()
            t, dt_last, k = float(c[0]), float(c[1]), int(c[2])
        return k, not at_first

    return run


def sedov_gpu_run(n=64, prec=0, cfl=0.3, t_end=None, dts=None, gamma=5.0 / 3.0, flags=0,
                  stream=None):
    """The Sedov point explosion (synth.sedov_domain, 11 fields) integrated on
    the GPU with SSP-RK3 steps of three fused stages of the domain form
    (ghost shells gathered in the kernel), to t_end or along `dts`.  The time
    step follows the rule of tests/sedov_run.py (dt = cfl dx / the largest
    signal speed of the previous step's stages); to t_end it is computed on
    the device (hydro_courant) and the steps are replayed from CUDA graphs
    (rk3_device_loop), along `dts` the host passes each dt.  Returns a dict
    with the final state (device, domain layout), t, the steps' dt and the
    wall time."""
    import torch

    import paper_2210_06438_gb300 as hydro
    from tests.sedov_run import to_domain

    glob, dx = synth.sedov_domain(n=n, nf=11, gamma=gamma)
    N, nf = 8, 11
    nb = n // N
    U = torch.from_numpy(to_domain(glob, N)).cuda()
    W1, W2 = torch.empty_like(U), torch.empty_like(U)
    am = torch.empty((3, nb ** 3), dtype=torch.float64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    kw = dict(gamma=gamma, prec=prec, stream=st, flags=flags)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dts is None:
        # the time step on the device (hydro_courant + hydro_domain_stage_dt), CUDA-graph replay
        st = stream if stream is not None else torch.cuda.Stream()
        kw["stream"] = st
        A, B = U, torch.empty_like(U)
        clock = torch.zeros(3, dtype=torch.float64, device="cuda")
        hist = torch.zeros(1 << 16, dtype=torch.float64, device="cuda")
        dtp = clock[1:2]

        def step_pair(forward):
            src, dst = (A, B) if forward else (B, A)
            hydro.courant(am, 3, nb ** 3, nb ** 3, clock, cfl, t_end, dx_uniform=dx, dt_hist=hist,
                          hist_len=hist.numel(), stream=st)
            hydro.domain_stage_dt(src, src, 0.0, 1.0, dtp, nb, N, nf, dx, W1, am[0], **kw)
            hydro.domain_stage_dt(W1, src, 0.75, 0.25, dtp, nb, N, nf, dx, W2, am[1], **kw)
            hydro.domain_stage_dt(W2, src, 1.0 / 3.0, 2.0 / 3.0, dtp, nb, N, nf, dx, dst, am[2], **kw)

        torch.cuda.synchronize()
        hydro.domain_rhs(A, nb, N, nf, dx, W1, am[0], **kw)  # first call on the device: setup
        run = rk3_device_loop(step_pair, clock, t_end, st)
        st.synchronize()
        with torch.cuda.stream(st):
            ev0.record(st)
            hydro.domain_rhs(A, nb, N, nf, dx, W1, am[0], **kw)  # a_0
            am[1:].copy_(am[0].expand(2, -1))
            k, flipped = run()
            ev1.record(st)
        st.synchronize()
        c = clock.cpu()
        return {"U": B if flipped else A, "t": float(c[0]), "dts": hist[:k].cpu().tolist(), "steps": k,
                "ms": ev0.elapsed_time(ev1), "n": n, "dx": dx}
    ev0.record(st)
    hydro.domain_rhs(U, nb, N, nf, dx, W1, am[0], **kw)
    a_next = float(am[0].max())
    t, used, k = 0.0, [], 0
    while (dts is not None and k < len(dts)) or (dts is None and t < t_end):
        dt = dts[k] if dts is not None else min(cfl * dx / a_next, t_end - t)
        hydro.domain_stage(U, U, 0.0, 1.0, dt, nb, N, nf, dx, W1, am[0], **kw)
        hydro.domain_stage(W1, U, 0.75, 0.25, dt, nb, N, nf, dx, W2, am[1], **kw)
        hydro.domain_stage(W2, U, 1.0 / 3.0, 2.0 / 3.0, dt, nb, N, nf, dx, W1, am[2], **kw)
        U, W1 = W1, U
        a_next = float(am.max())  # host sync: the next step's dt
        t += dt
        used.append(dt)
        k += 1
    ev1.record(st)
    torch.cuda.synchronize()
    return {"U": U, "t": t, "dts": used, "steps": k, "ms": ev0.elapsed_time(ev1), "n": n, "dx": dx}


def sedov_forest_run(nb0=2, N=8, radii=(0.45, 0.25), prec=0, cfl=0.3, t_end=None, dts=None,
                     gamma=5.0 / 3.0, flags=0, stream=None):
    """The point explosion on a forest refined around the centre
    (synth.sedov_forest, 11 fields), integrated with SSP-RK3 steps of three
    forest stages (ghost slabs across levels, fused tiles, flux correction),
    to t_end or along `dts`.  One global step for all levels: dt = cfl min
    over leaves of dx_leaf / a_leaf, a_leaf the leaf's largest signal speed
    over the previous step's stages (to t_end: on the device, steps replayed
    from CUDA graphs, as in sedov_gpu_run).  Returns a dict with the final
    state (device, [n][nf][N^3]), the leaves, t, the steps' dt and the wall
    time."""
    import torch

    import paper_2210_06438_gb300 as hydro

    leaves, U0, dx0 = synth.sedov_forest(nb0=nb0, N=N, radii=radii, gamma=gamma)
    nf = U0.shape[1]
    fo = hydro.Forest(leaves, nb0, N, nf)
    U = torch.from_numpy(U0).cuda()
    W1, W2 = torch.empty_like(U), torch.empty_like(U)
    n = len(leaves)
    am = torch.empty((3, n), dtype=torch.float64, device="cuda")
    dxs = torch.tensor([dx0 / (1 << int(L)) for L in leaves[:, 0]], dtype=torch.float64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    kw = dict(gamma=gamma, prec=prec, stream=st, flags=flags)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dts is None:
        # the time step on the device (hydro_courant + hydro_forest_stage_dt), CUDA-graph replay
        st = stream if stream is not None else torch.cuda.Stream()
        kw["stream"] = st
        A, B = U, torch.empty_like(U)
        clock = torch.zeros(3, dtype=torch.float64, device="cuda")
        hist = torch.zeros(1 << 16, dtype=torch.float64, device="cuda")
        dtp = clock[1:2]

        def step_pair(forward):
            src, dst = (A, B) if forward else (B, A)
            hydro.courant(am, 3, n, n, clock, cfl, t_end, dx=dxs, dt_hist=hist, hist_len=hist.numel(),
                          stream=st)
            fo.stage_dt(src, src, 0.0, 1.0, dtp, dx0, W1, am[0], **kw)
            fo.stage_dt(W1, src, 0.75, 0.25, dtp, dx0, W2, am[1], **kw)
            fo.stage_dt(W2, src, 1.0 / 3.0, 2.0 / 3.0, dtp, dx0, dst, am[2], **kw)

        torch.cuda.synchronize()
        fo.rhs(A, dx0, W1, am[0], **kw)  # first call on the device: setup
        run = rk3_device_loop(step_pair, clock, t_end, st)
        st.synchronize()
        with torch.cuda.stream(st):
            ev0.record(st)
            fo.rhs(A, dx0, W1, am[0], **kw)  # a_0
            am[1:].copy_(am[0].expand(2, -1))
            k, flipped = run()
            ev1.record(st)
        st.synchronize()
        c = clock.cpu()
        info = fo.info()
        fo.close()
        return {"U": B if flipped else A, "leaves": leaves, "t": float(c[0]), "dts": hist[:k].cpu().tolist(),
                "steps": k, "ms": ev0.elapsed_time(ev1), "nb0": nb0, "dx0": dx0, "info": info}
    ev0.record(st)
    fo.rhs(U, dx0, W1, am[0], **kw)
    a_leaf = am[0].clone()
    t, used, k = 0.0, [], 0
    while (dts is not None and k < len(dts)) or (dts is None and t < t_end):
        dt = dts[k] if dts is not None else min(cfl * float((dxs / a_leaf).min()), t_end - t)
        fo.stage(U, U, 0.0, 1.0, dt, dx0, W1, am[0], **kw)
        fo.stage(W1, U, 0.75, 0.25, dt, dx0, W2, am[1], **kw)
        fo.stage(W2, U, 1.0 / 3.0, 2.0 / 3.0, dt, dx0, W1, am[2], **kw)
        U, W1 = W1, U
        a_leaf = am.max(dim=0).values
        t += dt
        used.append(dt)
        k += 1
    ev1.record(st)
    torch.cuda.synchronize()
    info = fo.info()
    fo.close()
    return {"U": U, "leaves": leaves, "t": t, "dts": used, "steps": k, "ms": ev0.elapsed_time(ev1),
            "nb0": nb0, "dx0": dx0, "info": info}


def forest_forms(steps, warmup, stream, nb0=16, radii=(0.35, 0.2), N=8, nf=11, gamma=5.0 / 3.0):
    """The RHS of an adaptive forest: leaves of three levels refined around
    the cube's centre (synth.sphere_refine; 128^3 cells' resolution at level
    0, 512^3 at the centre), smooth random fields (synth.smooth_forest_state),
    11 fields.  Each RHS is three launches: ghost slabs across levels, the
    fused tile kernel, the flux correction.  Also one SSP-RK3 step of three
    forest stages.  Value: leaf cell-updates/s."""
    import torch

    import paper_2210_06438_gb300 as hydro

    leaves = synth.forest_leaves(nb0, len(radii), synth.sphere_refine((0.5, 0.5, 0.5), radii), balance="full")
    U_h, dx0 = synth.smooth_forest_state(leaves, nb0, N, nf=nf)
    U = torch.from_numpy(U_h).cuda()
    del U_h
    out, tmp = torch.empty_like(U), torch.empty_like(U)
    n = len(leaves)
    am = torch.empty(n, dtype=torch.float64, device="cuda")
    vol = torch.tensor([(dx0 / (1 << int(L))) ** 3 for L in leaves[:, 0]], dtype=torch.float64,
                       device="cuda")
    fo = hydro.Forest(leaves, nb0, N, nf)
    cells = n * N ** 3
    res = {}
    for name, prec in (("fp64_forest", hydro.FP64), ("mixed_forest", hydro.FP32_FLUX_FP64_ACC)):
        ms = time_steps(lambda: fo.rhs(U, dx0, out, am, gamma=gamma, prec=prec, stream=stream), steps,
                        warmup, stream)
        w = (out * vol[:, None, None, None, None]).sum(dim=(0, 2, 3, 4))
        a = (out.abs() * vol[:, None, None, None, None]).sum(dim=(0, 2, 3, 4))
        res[name] = {"value": cells / (ms * 1e-3), "ms": ms,
                     "conservation_drift": float((w / a.clamp_min(1e-300)).abs().max())}

    def rk3(prec):
        dt = 1e-5
        fo.stage(U, U, 0.0, 1.0, dt, dx0, out, am, gamma=gamma, prec=prec, stream=stream)
        fo.stage(out, U, 0.75, 0.25, dt, dx0, tmp, am, gamma=gamma, prec=prec, stream=stream)
        fo.stage(tmp, U, 1.0 / 3.0, 2.0 / 3.0, dt, dx0, out, am, gamma=gamma, prec=prec, stream=stream)

    ms = time_steps(lambda: rk3(hydro.FP64), max(1, steps // 2), 1, stream)
    res["fp64_forest_rk3_step"] = {"value": 3 * cells / (ms * 1e-3), "ms": ms,
                                   "note": "three forest stages; value = stage cell-updates/s"}
    if fo.info()["quad26"]:
        for name, prec in (("fp64_forest_quad26", hydro.FP64), ("mixed_forest_quad26", hydro.FP32_FLUX_FP64_ACC)):
            ms = time_steps(lambda: fo.rhs(U, dx0, out, am, gamma=gamma, prec=prec, stream=stream,
                                           flags=hydro.F_QUAD26), max(1, steps // 3), 1, stream)
            w = (out * vol[:, None, None, None, None]).sum(dim=(0, 2, 3, 4))
            a = (out.abs() * vol[:, None, None, None, None]).sum(dim=(0, 2, 3, 4))
            res[name] = {"value": cells / (ms * 1e-3), "ms": ms,
                         "conservation_drift": float((w / a.clamp_min(1e-300)).abs().max()),
                         "note": "the 26-point variant: gather of every leaf's ghosted block, "
                                 "26-point tiles, flux correction"}
    info = fo.info()
    fo.close()
    levels = np.bincount(leaves[:, 0]).tolist()
    res["fp64_forest"]["workload"] = {
        "leaves": n, "leaves_by_level": levels, "cells": cells, "N": N, "fields": nf, "nb0": nb0,
        "refine_radii": list(radii), "level_faces": info["n_level_faces"],
        "reflux_leaves": info["n_reflux_leaves"], "forest_device_bytes": info["device_bytes"],
        "note": "sphere refinement around the centre, 2:1 balanced across faces, edges and corners, "
                "periodic; smooth random fields"}
    return res


def sedov_forest_form(prec, nb0=4, radii=(0.42, 0.36), flags=0):
    """The Sedov blast on a forest refined around the centre: level-2
    resolution (128^3 cells' width at nb0 = 4) where the shock runs, level 1
    outside; measures against the similarity solution as for sedov_form."""
    from tests.sedov_exact import Sedov
    from tests.sedov_run import forest_shock_measures

    ex = Sedov(5.0 / 3.0)
    r = sedov_forest_run(nb0=nb0, radii=radii, prec=prec, t_end=ex.time_for_radius(0.35), flags=flags)
    lv = r["leaves"]
    Rp, L1 = forest_shock_measures(lv, nb0, r["U"][:, 0].cpu().numpy(), ex, r["t"])
    cells = len(lv) * 512
    return {"value": 3 * cells * r["steps"] / (r["ms"] * 1e-3), "unit": "stage cell-updates/s",
            "steps": r["steps"], "ms": r["ms"], "t_end": r["t"], "R_peak": Rp,
            "R_exact": ex.shock_radius(r["t"]), "L1_rho": L1, "cells": cells,
            "leaves_by_level": np.bincount(lv[:, 0]).tolist(),
            "note": "Sedov blast to R = 0.35 on a forest refined around the centre (%d leaves of 8^3, "
                    "11 fields, radii %s), SSP-RK3 of forest stages, one global dt" % (len(lv), list(radii))}


def sedov_form(n, prec, flags=0):
    """One Sedov run at n^3 with its measures against the similarity solution."""
    from tests.sedov_exact import Sedov
    from tests.sedov_run import from_domain, shock_measures

    ex = Sedov(5.0 / 3.0)
    r = sedov_gpu_run(n=n, prec=prec, t_end=ex.time_for_radius(0.35), flags=flags)
    rho = from_domain(r["U"].cpu().numpy(), n)[0]
    Rp, L1 = shock_measures(rho, r["dx"], ex, r["t"])
    return {"value": 3 * n ** 3 * r["steps"] / (r["ms"] * 1e-3), "unit": "stage cell-updates/s",
            "steps": r["steps"], "ms": r["ms"], "t_end": r["t"], "R_peak": Rp,
            "R_exact": ex.shock_radius(r["t"]), "L1_rho": L1,
            "note": "Sedov blast to R = 0.35 on %d^3 cells (%d sub-grids of 8^3, 11 fields), "
                    "SSP-RK3 of fused domain stages, dt from the signal speed (host sync per step)"
                    % (n, (n // 8) ** 3)}


# ---------------------------------------------------------- cpu baseline --
def oracle_small_configs(seconds=1.5):
    """The oracle on the two small workloads: one 8^3 sub-grid with 6 fields
    (iid cells) and the 64^3 periodic domain of 512 sub-grids with 11 fields
    (smooth fields), at one thread and at all host cores."""
    U1, dx1 = synth.one_subgrid(nf=6)
    glob = synth.plain_domain(n=64, nf=11)
    blocks = list(synth.gather_blocks(glob, 8))
    res = {}
    for name, bl, dx in (("one_subgrid_8^3_6_fields", [U1], dx1), ("plain_domain_64^3_11_fields", blocks, 1.0 / 64)):
        r1, _, _ = oracle_sample_rate(bl, dx, seconds=seconds, threads=1)
        ra, thr, _ = oracle_sample_rate(bl, dx, seconds=seconds)
        res[name] = {"one_core": r1, "all_cores": ra, "cores": thr, "unit": "cell-updates/s"}
    return res


def oracle_sample_parity(blocks_host, dx, gpu):
    """The GPU results of the benchmark workload against the oracle on the
    CPU-baseline sample (each sub-grid whole): binary64 form against the
    oracle's binary64 mode under the 1e-12 gate of the parity tests, the
    mixed form's normwise error against the binary64 oracle (per sub-grid and
    field, max|gpu - oracle| / max(max|oracle|, amax max|U_f| / dx), worst
    over the sample) and against
    the oracle's mixed mode in binary32 ulps of the flux-divergence scale."""
    import oracle

    threads = os.cpu_count() or 1
    ref, ram, fl = oracle.rhs_batch(blocks_host, GAMMA, dx, 0, threads=threads)
    ref1, ram1, _ = oracle.rhs_batch(blocks_host, GAMMA, dx, 1, threads=threads)
    n = len(blocks_host)
    nf = blocks_host[0].shape[0]
    r0 = np.stack([r.reshape(nf, -1) for r in ref])
    r1 = np.stack([r.reshape(nf, -1) for r in ref1])
    umax = np.stack([np.abs(b).reshape(nf, -1).max(axis=1) for b in blocks_host])
    floor = ram[:, None] * umax / dx
    fp64 = (np.abs(gpu["fp64"] - r0).max(axis=2) / np.maximum(np.maximum(np.abs(r0).max(axis=2), floor),
                                                               1e-300)).max()
    # normwise with the parity tests' flux-divergence floor (exact zeros of
    # uniform regions must not divide by zero)
    mx = (np.abs(gpu["mixed"] - r0).max(axis=2) / np.maximum(np.maximum(np.abs(r0).max(axis=2), floor),
                                                              1e-300)).max()
    S32 = 2.0 * ram1[:, None] * (umax + np.where((np.arange(nf) >= 1) & (np.arange(nf) <= 4), umax[:, 4:5], 0.0))
    ulps = (np.abs(gpu["mixed"] - r1).max(axis=2) / (2.0 ** -24 * S32 / dx)).max()
    return {"subgrids": n, "oracle_flags": int(fl.any()),
            "fp64_vs_oracle_err_over_1e-12": float(fp64 / 1e-12),
            "fp64_amax_rel": float((np.abs(gpu["fp64_amax"] - ram) / ram).max()),
            "mixed_vs_oracle_fp64_normwise": float(mx),
            "mixed_vs_oracle_mixed_ulps_of_S32": float(ulps),
            "mixed_amax_rel_vs_oracle_mixed": float((np.abs(gpu["mixed_amax"] - ram1) / ram1).max())}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    import subprocess

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample_rate(blocks_host, dx, seconds=10.0, threads=None, mode=0):
    """The oracle (as it stands) over a sample of sub-grids, repeated until
    `seconds` of wall time; returns (cells/s, threads, repetitions)."""
    import oracle

    threads = threads or os.cpu_count() or 1
    cells = sum(b.shape[1] - 6 for b in blocks_host[:1]) ** 3 * len(blocks_host)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.rhs_batch(blocks_host, GAMMA, dx, mode, threads=threads)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return cells * reps / el, threads, reps


# ------------------------------------------------------------ reference --
def run_reference(args, rank, world):
    """The reference arm: the oracle timed on the host cores."""
    if rank != 0:
        return
    import oracle

    oracle.build()
    n_sample = args.ref_sample
    n = args.domain
    glob = synth.polytropes(n=n, nf=11)  # the workload itself; a sample of its sub-grids per step
    nb = n // 8
    idx = np.linspace(0, nb ** 3 - 1, n_sample).astype(int)
    blocks = list(synth.gather_blocks(glob, 8, blocks=[(i % nb, (i // nb) % nb, i // (nb * nb)) for i in idx]))
    del glob
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.rhs_batch(blocks, GAMMA, 2.0 / n, 0, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.rhs_batch(blocks, GAMMA, 2.0 / n, 0, threads=threads)
    el = time.perf_counter() - t0
    cells = n_sample * 512
    value = cells * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "%d evenly spaced sub-grids of the workload per step"
                   % n_sample},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": threads,
                         "kind": "oracle",
                         "sample": "%d sub-grids of 8^3, 11 fields, per step" % n_sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ smaller workloads --
def small_workloads(stream, steps, warmup, streams_pool):
    """The three smaller workloads of the benchmark suite, each timed on the
    GPU in the aggregated form and the one-launch-per-sub-grid form:

      one_subgrid  one 8^3 sub-grid, 6 fields (iid states): per-call latency
                   of hydro_rhs_ex and of a graph-replayed plan (p50/p99 of
                   >= 200 calls, host wall clock and device events) -- the
                   paper's context is one Reconstruct (~300 us) and one Flux
                   (~150 us) launch for one 8^3 sub-grid on an A100 (Sec. V-A)
      plain_512    the 64^3 periodic domain (512 sub-grids of 8^3, 11 fields,
                   smooth random fields; Table I's 262144 cells): one fused
                   plan vs 512 per-sub-grid launches on 1/4/16/128 streams
      uneven_4096  the 3-level octree batch (3072 8^3 + 1024 16^3 sub-grids,
                   6 or 11 fields, shuffled): autotuned plan vs per-sub-grid
                   launches on 128 streams
    Every timed step of plain_512 and one_subgrid follows an L2 flush (a 512
    MB write); uneven_4096's inputs (1.3 GB) exceed L2."""
    import time

    import torch

    import paper_2210_06438_gb300 as hydro

    flush = torch.empty(64 << 20, dtype=torch.float64, device="cuda")  # 512 MB > L2
    res = {}
    precs = (("fp64", hydro.FP64), ("mixed", hydro.FP32_FLUX_FP64_ACC))

    # ---- one sub-grid
    U, dx = synth.one_subgrid(nf=6)
    Ud = torch.from_numpy(U).cuda()
    desc = hydro.descriptors([(Ud, dx, 8, 6)])
    out = torch.empty(6 * 512, dtype=torch.float64, device="cuda")
    am = torch.empty(1, dtype=torch.float64, device="cuda")
    one = {"cells": 512}
    for name, prec in precs:
        plan = hydro.Plan(desc, ghost=3, gamma=GAMMA, prec=prec, stream=stream)
        for form, call in (("rhs_ex", lambda: hydro.rhs(desc, out, am, ghost=3, gamma=GAMMA, prec=prec,
                                                        stream=stream)),
                           ("plan", lambda: plan.execute(out, am, stream))):
            for _ in range(20):
                call()
            torch.cuda.synchronize()
            wall, dev = [], []
            for _ in range(max(200, steps)):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                t0 = time.perf_counter()
                a.record(stream)
                call()
                b.record(stream)
                b.synchronize()
                wall.append((time.perf_counter() - t0) * 1e6)
                dev.append(a.elapsed_time(b) * 1e3)
            one["%s_%s" % (name, form)] = {
                "wall_us_p50": float(np.percentile(wall, 50)), "wall_us_p99": float(np.percentile(wall, 99)),
                "device_us_p50": float(np.percentile(dev, 50)), "device_us_p99": float(np.percentile(dev, 99)),
                "calls": len(wall)}
        plan.close()
    one["note"] = ("call-to-completion latency of one 8^3 sub-grid (6 fields); wall: host clock around the "
                   "call and the stream synchronisation; device: CUDA events around the call")
    res["one_subgrid"] = one
    del Ud, out

    # ---- 512 sub-grids of the 64^3 periodic domain
    glob = synth.plain_domain(n=64, nf=11)
    blocks = torch.from_numpy(np.ascontiguousarray(synth.gather_blocks(glob, 8))).cuda()
    n = blocks.shape[0]
    desc = hydro.descriptors([(int(blocks[s].data_ptr()), 1.0 / 64, 8, 11) for s in range(n)])
    out = torch.empty(n * 11 * 512, dtype=torch.float64, device="cuda")
    am = torch.empty(n, dtype=torch.float64, device="cuda")
    cells = n * 512
    plain = {"cells": cells, "subgrids": n, "inputs_bytes": blocks.numel() * 8}
    for name, prec in precs:
        plan = hydro.Plan(desc, ghost=3, gamma=GAMMA, prec=prec, autotune=True, stream=stream, n=n)
        ms, p10, p90 = time_flushed(lambda: plan.execute(out, am, stream), max(steps, 20), warmup, stream, flush)
        plan.close()
        ent = {"fused_ms": ms, "fused_ms_p10_p90": [p10, p90], "fused_value": cells / (ms * 1e-3)}
        for k in (1, 4, 16, len(streams_pool)):
            def per_sub(k=k):
                hydro.rhs_per_subgrid(desc, out, am, streams_pool[:k], ghost=3, gamma=GAMMA, prec=prec, n=n)
            per_sub()
            torch.cuda.synchronize()
            t = []
            for _ in range(max(3, min(steps, 10))):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                per_sub()
                torch.cuda.synchronize()
                t.append((time.perf_counter() - t0) * 1e3)
            ent["per_subgrid_ms_streams_%d" % k] = float(np.median(t))
        best = min(v for kk, v in ent.items() if kk.startswith("per_subgrid_ms"))
        ent["per_subgrid_best_value"] = cells / (best * 1e-3)
        ent["fused_over_best_per_subgrid"] = best / ms
        plain[name] = ent
    plain["note"] = ("64^3 periodic domain, 512 sub-grids of 8^3, 11 fields; fused: autotuned plan, one "
                     "graph replay, CUDA events; per-sub-grid: 512 launches (hydro_rhs_per_subgrid) on a "
                     "round-robin stream pool, host clock to completion; L2 flushed before every step")
    res["plain_512"] = plain
    del blocks, out

    # ---- uneven octree batch
    leaves = synth.uneven_octree()
    host = [synth.leaf_block(synth.BASE_SEED, l) for l in leaves]
    dev_blocks = [torch.from_numpy(b).cuda() for b in host]
    del host
    desc = hydro.descriptors([(b, l[2], l[0], l[1]) for b, l in zip(dev_blocks, leaves)])
    n = len(leaves)
    cells = int(sum(l[0] ** 3 for l in leaves))
    out = torch.empty(hydro.output_doubles(desc, n), dtype=torch.float64, device="cuda")
    am = torch.empty(n, dtype=torch.float64, device="cuda")
    alg = int(sum(synth.algorithmic_bytes(l[0], l[1]) for l in leaves))
    uneven = {"cells": cells, "subgrids": n, "n8": int(sum(l[0] == 8 for l in leaves)),
              "n16": int(sum(l[0] == 16 for l in leaves)), "alg_bytes": alg}
    for name, prec in precs:
        plan = hydro.Plan(desc, ghost=3, gamma=GAMMA, prec=prec, autotune=True, stream=stream, n=n)
        info = plan.info()
        ms, p10, p90 = time_flushed(lambda: plan.execute(out, am, stream), max(steps, 10), warmup, stream)
        plan.close()
        ms_ex = time_steps(lambda: hydro.rhs(desc, out, am, ghost=3, gamma=GAMMA, prec=prec, stream=stream, n=n),
                           max(steps, 10), warmup, stream)
        def per_sub():
            hydro.rhs_per_subgrid(desc, out, am, streams_pool, ghost=3, gamma=GAMMA, prec=prec, n=n)
        per_sub()
        torch.cuda.synchronize()
        t = []
        for _ in range(max(3, min(steps, 5))):
            t0 = time.perf_counter()
            per_sub()
            torch.cuda.synchronize()
            t.append((time.perf_counter() - t0) * 1e3)
        ms_ps = float(np.median(t))
        uneven[name] = {"plan_ms": ms, "plan_ms_p10_p90": [p10, p90], "plan_value": cells / (ms * 1e-3),
                        "plan_gbs_alg": alg / (ms * 1e-3) * 1e-9,
                        "rhs_ex_ms": ms_ex, "rhs_ex_value": cells / (ms_ex * 1e-3),
                        "per_subgrid_ms": ms_ps, "per_subgrid_value": cells / (ms_ps * 1e-3),
                        "streams": len(streams_pool), "plan": {k: info[k] for k in (
                            "threads_per_cta", "ctas_per_sm", "lines_per_chunk", "n_tiles", "n_candidates")}}
    uneven["note"] = ("3-level octree, 75 % 8^3 / 25 % 16^3 sub-grids, 6 or 11 fields each, shuffled; plan: "
                      "autotuned, graph replay (CUDA events); rhs_ex: direct call per step (work list "
                      "built and cost-sorted on the host each call); per-sub-grid: one launch each on "
                      "the stream pool (host clock)")
    res["uneven_4096"] = uneven
    del dev_blocks, out, flush
    torch.cuda.empty_cache()
    return res


# ------------------------------------------------------------------ ours --
def run_ours(args, rank, world):
    import torch

    import paper_2210_06438_gb300 as hydro

    hydro.load(build_if_missing=True)
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    batch = polytrope_batch(n=args.domain)
    cells = batch.cells
    out = torch.empty(batch.out_doubles, dtype=torch.float64, device=dev)
    amax = torch.empty(batch.n, dtype=torch.float64, device=dev)

    plan64 = hydro.Plan(batch.desc, ghost=3, gamma=GAMMA, prec=hydro.FP64, autotune=True,
                        stream=stream, n=batch.n)
    planmx = hydro.Plan(batch.desc, ghost=3, gamma=GAMMA, prec=hydro.FP32_FLUX_FP64_ACC,
                        autotune=True, stream=stream, n=batch.n)
    info64, infomx = plan64.info(), planmx.info()
    hydro.status(stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    hbm_peak_early = measured_peaks().get("hbm_gbs", 6800.0)

    # ---- headline: binary64 aggregated form
    for _ in range(args.warmup):
        plan64.execute(out, amax, stream)
    barrier()
    clk = ClockSampler(dev.index)
    clk.start()
    ms64 = time_steps(lambda: plan64.execute(out, amax, stream), args.steps, 0, stream)
    clocks = clk.stop()
    barrier()
    rc, bad = hydro.status(stream)
    if rc != hydro.HYDRO_OK:
        raise RuntimeError("nonphysical input flagged in sub-grid %d" % bad)
    fp64_peak = fp64_probe_peak(stream)
    out64 = out.clone()
    amax64 = amax.clone()
    drift64 = conservation_drift(out64, batch)
    msmx = time_steps(lambda: planmx.execute(out, amax, stream), args.steps, args.warmup, stream)
    mixed_err = normwise_error(out, out64, amax64, batch)
    drift = conservation_drift(out, batch)
    # the GPU results of the sub-grids the CPU-baseline leg samples, kept for
    # its comparison with the oracle
    sample_idx = np.linspace(0, batch.n - 1, args.cpu_sample).astype(int)
    ti = torch.from_numpy(sample_idx).to(dev)
    gpu_sample = {"fp64": out64.view(batch.n, batch.nf, -1)[ti].cpu().numpy(),
                  "fp64_amax": amax64[ti].cpu().numpy(),
                  "mixed": out.view(batch.n, batch.nf, -1)[ti].cpu().numpy(),
                  "mixed_amax": amax[ti].cpu().numpy()}
    del out64

    # ---- per-sub-grid launch form (strategy-2 analogue), 128-stream pool
    pool = [torch.cuda.Stream(device=dev) for _ in range(args.streams)]

    def per_sub(prec, streams):
        hydro.rhs_per_subgrid(batch.desc, out, amax, streams, ghost=3, gamma=GAMMA, prec=prec,
                              n=batch.n)

    def timed_pool(prec, steps, streams=pool):
        for _ in range(1):
            per_sub(prec, streams)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            per_sub(prec, streams)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / steps * 1e3

    ps_steps = max(1, min(args.steps, 3))
    ms_ps64 = timed_pool(hydro.FP64, ps_steps)
    ms_psmx = timed_pool(hydro.FP32_FLUX_FP64_ACC, ps_steps)
    # the stream-pool sweep of the per-sub-grid form (binary64)
    ps_sweep = {str(k): timed_pool(hydro.FP64, 1, pool[:k]) for k in (1, 4, 16) if k <= len(pool)}
    ps_sweep[str(len(pool))] = ms_ps64

    # ---- the maximum-aggregation knob of strategy 3 (Sec. V-D, VI-B): the same
    # sub-grids in launches of A sub-grids each (hydro_rhs_ex on consecutive
    # slices of the descriptor array, round-robin over 8 streams)
    agg_sweep = {"1": {"ms": ps_sweep.get("16", ms_ps64), "launches": batch.n,
                       "note": "one launch per sub-grid (hydro_rhs_per_subgrid, 16 streams)"}}
    sg_size = ctypes.sizeof(hydro.Subgrid)
    desc_base = ctypes.addressof(batch.desc)
    per_sub_doubles = batch.nf * 512

    def run_agg(A, streams):
        for k, i in enumerate(range(0, batch.n, A)):
            d = ctypes.cast(desc_base + i * sg_size, ctypes.POINTER(hydro.Subgrid))
            hydro.rhs(d, out.data_ptr() + i * per_sub_doubles * 8, amax.data_ptr() + i * 8, ghost=3,
                      gamma=GAMMA, prec=hydro.FP64, stream=streams[k % len(streams)], n=min(A, batch.n - i))

    for A in (16, 64, 256, 1024, 4096, batch.n):
        run_agg(A, pool[:8])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run_agg(A, pool[:8])
        torch.cuda.synchronize()
        ms_a = (time.perf_counter() - t0) * 1e3
        agg_sweep[str(A)] = {"ms": ms_a, "launches": -(-batch.n // A)}
    for v in agg_sweep.values():
        v["value"] = cells * world / (v["ms"] * 1e-3)

    # ---- the smaller workloads of the suite (one sub-grid, 512, the uneven batch)
    small = {} if args.no_small else small_workloads(stream, args.steps, args.warmup, pool)

    # ---- per-replay distribution of the headline plan (CUDA events around each replay)
    reps = []
    for _ in range(50):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan64.execute(out, amax, stream)
        e1.record(stream)
        e1.synchronize()
        reps.append(e0.elapsed_time(e1))
    rep_pct = {"p10": float(np.percentile(reps, 10)), "p50": float(np.percentile(reps, 50)),
               "p90": float(np.percentile(reps, 90)), "replays": len(reps)}

    # ---- domain form: the same cells stored without ghosts, ghost shells
    # gathered in the kernel; and one SSP-RK3 step of three fused stages
    dom = batch.blocks[:, :, 3:-3, 3:-3, 3:-3].contiguous()
    dout = torch.empty_like(dom)
    dtmp = torch.empty_like(dom)
    nbd = args.domain // 8

    def dom_rhs(prec):
        hydro.domain_rhs(dom, nbd, 8, batch.nf, batch.dx, dout, amax, prec=prec, stream=stream)

    def rk3_step(prec):
        dt = 1e-4
        hydro.domain_stage(dom, dom, 0.0, 1.0, dt, nbd, 8, batch.nf, batch.dx, dout, amax, prec=prec,
                           stream=stream)
        hydro.domain_stage(dout, dom, 0.75, 0.25, dt, nbd, 8, batch.nf, batch.dx, dtmp, amax, prec=prec,
                           stream=stream)
        hydro.domain_stage(dtmp, dom, 1.0 / 3.0, 2.0 / 3.0, dt, nbd, 8, batch.nf, batch.dx, dout, amax,
                           prec=prec, stream=stream)

    ms_dom64 = time_steps(lambda: dom_rhs(hydro.FP64), args.steps, args.warmup, stream)
    ms_dommx = time_steps(lambda: dom_rhs(hydro.FP32_FLUX_FP64_ACC), args.steps, args.warmup, stream)
    ms_rk64 = time_steps(lambda: rk3_step(hydro.FP64), max(1, args.steps // 2), 1, stream)
    ms_rkmx = time_steps(lambda: rk3_step(hydro.FP32_FLUX_FP64_ACC), max(1, args.steps // 2), 1, stream)
    dom_bytes = batch.n * (synth.star_cells(8) + 512) * batch.nf * 8
    del dom, dout, dtmp

    # ---- the 26-point quadrature variant on the same sub-grids
    quad = {}
    if not args.no_quad26:
        for name, prec in (("fp64_quad26", hydro.FP64), ("mixed_quad26", hydro.FP32_FLUX_FP64_ACC)):
            pq = hydro.Plan(batch.desc, ghost=3, gamma=GAMMA, prec=prec, autotune=True, stream=stream,
                            n=batch.n, flags=hydro.PLAN_QUAD26)
            msq = time_steps(lambda: pq.execute(out, amax, stream), max(1, args.steps // 3), 1, stream)
            quad[name] = {"value": cells * world / (msq * 1e-3), "ms": msq,
                          "conservation_drift": conservation_drift(out, batch),
                          "note": "fluxes at 9 points per face (26 per cell), Simpson weights"}
            pq.close()

    # ---- an adaptive forest of three refinement levels
    forest = {}
    if not args.no_forest:
        forest = forest_forms(args.steps, args.warmup, stream)

    # ---- the Sedov point explosion (the paper's scenario) on the 64^3 cube
    sedov = {}
    if not args.no_sedov:
        sedov = {"sedov_fp64_64": sedov_form(64, hydro.FP64),
                 "sedov_mixed_64": sedov_form(64, hydro.FP32_FLUX_FP64_ACC),
                 "sedov_fp64_quad26_64": sedov_form(64, hydro.FP64, hydro.F_QUAD26),
                 "sedov_mixed_quad26_64": sedov_form(64, hydro.FP32_FLUX_FP64_ACC, hydro.F_QUAD26),
                 "sedov_fp64_128": sedov_form(128, hydro.FP64)}
        if not args.no_forest:
            sedov["sedov_fp64_forest"] = sedov_forest_form(hydro.FP64)
            sedov["sedov_mixed_forest"] = sedov_forest_form(hydro.FP32_FLUX_FP64_ACC)

    # ---- end to end through the C ABI with host buffers.  Inputs and outputs
    # live in pinned host memory; the plan's descriptors point there and the
    # kernel reads the read region (and writes dU/dt) in place over the host
    # link (NVLink-C2C on GB300), so the transfers overlap the arithmetic.  The
    # step ends with the host reading the result (the largest signal speed).
    host_in = torch.empty(batch.blocks.shape, dtype=torch.float64, pin_memory=True)
    host_in.copy_(batch.blocks)
    host_out = torch.empty(batch.out_doubles, dtype=torch.float64, pin_memory=True)
    host_amax = torch.empty(batch.n, dtype=torch.float64, pin_memory=True)
    bstride = host_in[0].numel() * 8
    hdesc = hydro.descriptors([(int(host_in.data_ptr()) + s * bstride, batch.dx, batch.N, batch.nf)
                               for s in range(batch.n)])
    plan_host = hydro.Plan(hdesc, ghost=3, gamma=GAMMA, prec=hydro.FP64, autotune=True, stream=stream,
                           n=batch.n)
    info_host = {k: plan_host.info()[k] for k in ("threads_per_cta", "ctas_per_sm", "lines_per_chunk",
                                                  "prefetch")}
    e2e_read = []

    def e2e_step():
        plan_host.execute(host_out, host_amax, stream)
        stream.synchronize()
        e2e_read.append(float(host_amax.max()))

    e2e_steps = max(1, min(args.steps, 5))
    ms_e2e = time_steps(e2e_step, e2e_steps, 1, stream)
    plan64.execute(out, amax, stream)
    torch.cuda.synchronize()
    e2e_same = bool(torch.equal(host_out, out.cpu())) and bool(torch.equal(host_amax, amax.cpu()))
    plan_host.close()

    # the same with explicit copies (device buffers, one copy each way)
    def e2e_copy_step():
        batch.blocks.copy_(host_in, non_blocking=True)
        plan64.execute(out, amax, stream)
        host_out.copy_(out, non_blocking=True)
        host_amax.copy_(amax, non_blocking=True)
        stream.synchronize()
        e2e_read.append(float(host_amax.max()))

    ms_e2e_copy = time_steps(e2e_copy_step, e2e_steps, 1, stream)
    h2d = batch.n * synth.star_cells(batch.N) * batch.nf * 8  # cells the kernel reads
    h2d_copy = batch.blocks.numel() * 8
    d2h = (batch.out_doubles + batch.n) * 8
    del host_in, host_out

    # ---- serving: Poisson task stream, continuous batching vs one launch per task
    serving = None
    if not args.no_serving:
        serving_run(args.rate, 0.3, per_task=False)  # warm-up (first use of the pools), not reported
        serving = {
            "aggregated": serving_run(args.rate, args.serve_seconds, per_task=False),
            "per_task": serving_run(args.rate, args.serve_seconds, per_task=True),
            # at four times the rate the one-launch-per-task form runs out of capacity
            "stress_x4_aggregated": serving_run(4 * args.rate, args.serve_seconds / 2, per_task=False),
            "stress_x4_per_task": serving_run(4 * args.rate, args.serve_seconds / 2, per_task=True),
            # the mixed precision form at the same rate
            "aggregated_mixed": serving_run(args.rate, args.serve_seconds, per_task=False, prec=1),
            "per_task_mixed": serving_run(args.rate, args.serve_seconds, per_task=True, prec=1),
        }

    # ---- max over ranks
    (ms64, msmx, ms_ps64, ms_psmx, ms_e2e, ms_dom64, ms_dommx, ms_rk64, ms_rkmx, ms_e2e_copy) = max_over_ranks(
        [ms64, msmx, ms_ps64, ms_psmx, ms_e2e, ms_dom64, ms_dommx, ms_rk64, ms_rkmx, ms_e2e_copy], world,
        device=dev)
    if rank != 0:
        return

    # ---- roofline of the dominant kernel (the binary64 tile kernel)
    peaks = measured_peaks()
    flops = fp64_ops_per_cell(8, 11) * cells
    peak_fp64 = fp64_peak["gflops"]
    ach = flops / (ms64 * 1e-3) * 1e-9
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    n_sm = fp64_peak["sms"]
    roof = {"bound": "alu", "achieved": ach, "peak": peak_fp64, "unit": "GFLOP/s (fp64)",
            "frac": ach / peak_fp64, "traffic": recorded_traffic("fp64", info64["n_tiles"]),
            "peak_source": "measured: hydro_probe_fp64 (independent binary64 FMAs on all %d SMs, CUDA "
                           "events, median of %d launches of %.2f ms) = %.2f DFMA/clk/SM at the sampled "
                           "median SM clock; derived nominal 2 DFMA/clk/SM x %d SMs x %.0f MHz = %.1f GFLOP/s"
                           % (n_sm, fp64_peak["launches"], fp64_peak["ms"],
                              peak_fp64 * 1e9 / 2 / n_sm / ((clocks.get("sm_mhz") or 2070.0) * 1e6),
                              n_sm, clocks.get("sm_mhz") or 2070.0,
                              fp64_peak_gflops(clocks.get("sm_mhz") or 2070.0, n_sm)),
            "hbm": {"achieved_gbs": batch.alg_bytes / (ms64 * 1e-3) * 1e-9, "peak_gbs": hbm_peak,
                    "frac": batch.alg_bytes / (ms64 * 1e-3) * 1e-9 / hbm_peak,
                    "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}}
    # the kernel's own binary64-pipe instructions (ncu record) at the probe's
    # rate (one fused multiply-add = one pipe instruction, two flops)
    rc64 = recorded_counts("fp64")
    if rc64 and "fp64_pipe_thread_instructions_per_tile" in rc64:
        pipe_ops = rc64["fp64_pipe_thread_instructions_per_tile"] * info64["n_tiles"]
        floor_ms = pipe_ops / (peak_fp64 * 1e9 / 2) * 1e3
        roof["fp64_pipe"] = {"thread_instructions": pipe_ops, "floor_ms": floor_ms, "frac": floor_ms / ms64,
                             "source": "sm__thread_inst_executed_pipe_fp64_pred_on.sum per tile (ncu record) at "
                                       "the measured probe rate"}
    # the dense-block figure beside the algorithmic one: every ghosted block
    # read whole ((N + 2g)^3 cells) plus dU/dt, the bytes a kernel reading
    # whole blocks would move
    dense_bytes = batch.n * ((batch.N + 6) ** 3 + batch.N ** 3) * batch.nf * 8
    mixed_roof = {"bound": "hbm", "achieved": batch.alg_bytes / (msmx * 1e-3) * 1e-9,
                  "peak": hbm_peak, "unit": "GB/s",
                  "traffic": recorded_traffic("mixed", infomx["n_tiles"]),
                  "alg_bytes": batch.alg_bytes,
                  "frac": batch.alg_bytes / (msmx * 1e-3) * 1e-9 / hbm_peak,
                  "dense_block_bytes": dense_bytes,
                  "dense_block_frac": dense_bytes / (msmx * 1e-3) * 1e-9 / hbm_peak,
                  "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    # the bound that holds for this kernel: instruction issue (ncu record of
    # its warp instructions per tile; 4 per clock per SM)
    rcmx = recorded_counts("mixed")
    if rcmx and "warp_instructions_per_tile" in rcmx:
        insts = rcmx["warp_instructions_per_tile"] * infomx["n_tiles"]
        mhz = clocks.get("sm_mhz") or 2070.0
        floor_ms = insts / (4.0 * n_sm * mhz * 1e6) * 1e3
        mixed_roof["issue"] = {"warp_instructions": insts, "floor_ms": floor_ms, "frac": floor_ms / msmx,
                               "source": "smsp__inst_executed.sum per tile (ncu record), 4 issues per clock "
                                         "per SM at the sampled SM clock"}

    # ---- oracle on the host cores (bounded sample of the same workload)
    cpu = None
    if not args.no_cpu_baseline:
        idx = np.linspace(0, batch.n - 1, args.cpu_sample).astype(int)
        host_blocks = [batch.blocks[int(i)].cpu().numpy() for i in idx]
        rate, thr, reps = oracle_sample_rate(host_blocks, batch.dx, seconds=args.cpu_seconds)
        sample_parity = oracle_sample_parity(host_blocks, batch.dx, gpu_sample)
        one = host_blocks[::max(1, len(host_blocks) // 128)]
        rate1, _, reps1 = oracle_sample_rate(one, batch.dx, seconds=min(3.0, args.cpu_seconds), threads=1)
        cpu = {"value": rate, "unit": "cell-updates/s", "cores": thr, "kind": "oracle",
               "sample": "%d evenly spaced sub-grids of the workload, %d passes, FP64, OpenMP over "
                         "sub-grids" % (len(idx), reps),
               "one_core": {"value": rate1, "sample": "%d of those sub-grids, %d passes, 1 thread"
                                                      % (len(one), reps1)},
               "cpu_model": cpu_model(), "other_workloads": oracle_small_configs(),
               "parity_on_sample": sample_parity}

    value = cells * world / (ms64 * 1e-3)
    line = {
        "metric": METRIC,
        "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "subgrids": batch.n, "cells": cells,
                   "inputs_bytes": batch.blocks.numel() * 8, "l2": "inputs (7.9 GB) > L2",
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "plan_fp64": info64, "plan_mixed": infomx},
        "e2e": {"value": cells * world / (ms_e2e * 1e-3), "unit": "cell-updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
                "how": "inputs and outputs in pinned host memory, read and written in place by the "
                       "kernel over NVLink-C2C (h2d = the read region's bytes); result read on the host",
                "bitwise_equal_to_device_run": e2e_same, "plan": info_host,
                "explicit_copies": {"value": cells * world / (ms_e2e_copy * 1e-3), "ms_per_step": ms_e2e_copy,
                                    "h2d_bytes_per_step": h2d_copy, "d2h_bytes_per_step": d2h}},
        "gpu_launches": args.steps,
        "roofline": roof,
        "forms": {
            "fp64_aggregated": {"value": value, "ms": ms64, "conservation_drift": drift64,
                                "replay_ms": rep_pct},
            "mixed_aggregated": {"value": cells * world / (msmx * 1e-3), "ms": msmx,
                                 "roofline": mixed_roof, "max_rel_err_vs_fp64_gpu": mixed_err,
                                 "max_rel_err_vs_fp64_oracle": (cpu or {}).get("parity_on_sample", {}).get(
                                     "mixed_vs_oracle_fp64_normwise"),
                                 "conservation_drift": drift},
            "fp64_per_subgrid": {"value": cells * world / (ms_ps64 * 1e-3), "ms": ms_ps64,
                                 "streams": args.streams, "launches": batch.n,
                                 "ms_by_streams": ps_sweep},
            "fp64_by_subgrids_per_launch": agg_sweep,
            "fp64_domain": {"value": cells * world / (ms_dom64 * 1e-3), "ms": ms_dom64,
                            "note": "ghost shells gathered in the kernel from ghost-free storage"},
            "mixed_domain": {"value": cells * world / (ms_dommx * 1e-3), "ms": ms_dommx,
                             "hbm_frac": dom_bytes / (ms_dommx * 1e-3) * 1e-9 / hbm_peak_early},
            "fp64_rk3_step": {"value": 3 * cells * world / (ms_rk64 * 1e-3), "ms": ms_rk64,
                              "note": "three fused SSP-RK3 stages; value = stage cell-updates/s"},
            "mixed_rk3_step": {"value": 3 * cells * world / (ms_rkmx * 1e-3), "ms": ms_rkmx},
            **quad,
            **forest,
            **small,
            **sedov,
            "mixed_per_subgrid": {"value": cells * world / (ms_psmx * 1e-3), "ms": ms_psmx,
                                  "streams": args.streams, "launches": batch.n},
        },
        "clocks": clocks,
        "cpu_baseline": cpu,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)


def run_profile_forest(args, nb0=16, radii=(0.35, 0.2), N=8, nf=11):
    """The forest RHS of forest_forms for ncu: `warmup` untimed and `steps`
    timed calls, each three launches (level transfer, tiles, flux correction;
    the 26-point variant: gather, tiles, flux correction)."""
    import torch

    import paper_2210_06438_gb300 as hydro

    stream = torch.cuda.current_stream()
    leaves = synth.forest_leaves(nb0, len(radii), synth.sphere_refine((0.5, 0.5, 0.5), radii), balance="full")
    U_h, dx0 = synth.smooth_forest_state(leaves, nb0, N, nf=nf)
    U = torch.from_numpy(U_h).cuda()
    out = torch.empty_like(U)
    am = torch.empty(len(leaves), dtype=torch.float64, device="cuda")
    fo = hydro.Forest(leaves, nb0, N, nf)
    prec = hydro.FP64 if args.profile in ("forest64", "forest64_quad26") else hydro.FP32_FLUX_FP64_ACC
    flags = hydro.F_QUAD26 if args.profile.endswith("quad26") else 0
    ms = time_steps(lambda: fo.rhs(U, dx0, out, am, prec=prec, stream=stream, flags=flags), args.steps,
                    args.warmup, stream)
    rc, bad = hydro.status(stream)
    info = fo.info()
    fo.close()
    print(json.dumps({"profile": args.profile, "ms": ms, "cells": len(leaves) * N ** 3, "status": rc,
                      "launches_before_timed": 3 * args.warmup, "forest": info}), flush=True)


def run_profile(args):
    """A short run of one form for ncu: the tuned plan, `warmup` untimed and
    `steps` timed executions.  Prints how many launches of the tile kernel
    precede the timed ones (autotuner candidates x 4 + warm-ups), the value to
    give ncu's --launch-skip."""
    import torch

    import paper_2210_06438_gb300 as hydro

    hydro.load(build_if_missing=True)
    stream = torch.cuda.current_stream()
    if args.profile.startswith("forest"):
        return run_profile_forest(args)
    batch = polytrope_batch(n=args.domain)
    if args.profile.startswith("domain"):
        # the domain form: the same cells stored without ghosts, the ghost
        # shells gathered in the kernel (one launch per call, no tuning)
        prec = hydro.FP64 if args.profile == "domain64" else hydro.FP32_FLUX_FP64_ACC
        dom = batch.blocks[:, :, 3:-3, 3:-3, 3:-3].contiguous()
        del batch.blocks
        dout = torch.empty_like(dom)
        amax = torch.empty(batch.n, dtype=torch.float64, device="cuda")
        nbd = args.domain // batch.N
        ms = time_steps(lambda: hydro.domain_rhs(dom, nbd, batch.N, batch.nf, batch.dx, dout, amax, prec=prec,
                                                 stream=stream), args.steps, args.warmup, stream)
        rc, bad = hydro.status(stream)
        print(json.dumps({"profile": args.profile, "domain": args.domain, "subgrids": batch.n, "ms": ms,
                          "alg_bytes": batch.alg_bytes, "status": rc, "launches_before_timed": args.warmup,
                          "kernel": "rhs_domain_kernel" if prec == hydro.FP64 else "rhs_domain_pipe"}),
              flush=True)
        return
    prec = hydro.FP64 if args.profile.startswith("fp64") else hydro.FP32_FLUX_FP64_ACC
    flags = hydro.PLAN_QUAD26 if args.profile.endswith("quad26") else 0
    plan = hydro.Plan(batch.desc, ghost=3, gamma=GAMMA, prec=prec, autotune=True, stream=stream,
                      n=batch.n, flags=flags)
    info = plan.info()
    out = torch.empty(batch.out_doubles, dtype=torch.float64, device="cuda")
    amax = torch.empty(batch.n, dtype=torch.float64, device="cuda")
    ms = time_steps(lambda: plan.execute(out, amax, stream), args.steps, args.warmup, stream)
    rc, bad = hydro.status(stream)
    # launches of the kernel the plan runs before the timed ones (ncu's
    # --launch-skip with a kernel-name filter): the autotuner times every
    # candidate 4 times; the pipelined mixed kernel (the only one with over
    # 200 KB of shared memory) is one candidate among register-load ones, the
    # other plans' candidates all share a kernel name
    pipe = prec != hydro.FP64 and not flags and info["smem_bytes"] > 200 * 1024
    print(json.dumps({"profile": args.profile, "domain": args.domain, "subgrids": batch.n,
                      "ms": ms, "alg_bytes": batch.alg_bytes,
                      "gbs": batch.alg_bytes / (ms * 1e-3) * 1e-9, "status": rc,
                      "launches_before_timed": (4 if pipe else 4 * info["n_candidates"]) + args.warmup,
                      "kernel": "rhs_tiles_pipe" if pipe else ("rhs_quad" if flags else "rhs_tiles_kernel"),
                      "plan": info}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--domain", type=int, default=256, help="cells per edge of the domain")
    ap.add_argument("--streams", type=int, default=128)
    ap.add_argument("--cpu-sample", type=int, default=2048)
    ap.add_argument("--ref-sample", type=int, default=2048,
                    help="sub-grids per step of the reference (oracle) arm")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-sedov", action="store_true", help="skip the Sedov blast runs")
    ap.add_argument("--no-forest", action="store_true", help="skip the adaptive-forest forms")
    ap.add_argument("--no-quad26", action="store_true", help="skip the 26-point quadrature forms")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the smaller workloads (one sub-grid, 512 sub-grids, the uneven batch)")
    ap.add_argument("--rate", type=float, default=20000.0, help="serving arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--profile", choices=["fp64", "mixed", "fp64_quad26", "mixed_quad26", "domain64", "domainmx",
                                          "forest64", "forestmx", "forest64_quad26", "forestmx_quad26"],
                    default=None,
                    help="short run of one form for ncu (no JSON bench line)")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
        return
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch

        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group(backend)
    if world > 1:
        # replicas: the scaling run times the headline and the forms beside it;
        # the serving, Sedov and 26-point runs stay single-GPU extras
        args.no_serving = args.no_sedov = args.no_quad26 = args.no_forest = args.no_small = True
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch

        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
