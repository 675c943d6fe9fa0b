"""Host-side arithmetic of bench.py, without a GPU: the algorithmic operation
count of the binary64 roofline, the parity figures the CPU-baseline leg
reports, the gate that ties the committed ncu record to the kernel source,
and the clock record."""
import json
import os
import threading

import numpy as np
import pytest

import bench
import oracle
import synth


def test_algorithmic_flops_per_cell():
    # N = 8, F = 11 (per interior cell of the definition): primitives
    # (F + 9) on each of 1664 read cells; PPM per line and field 12 slopes x 6
    # + 11 faces x 5 + 10 limited cells x 10 on 3 x 64 lines; flux 10 F + 26
    # on 3 x 64 x 9 faces; divergence 6 F
    total = 20 * 1664 + 3 * 64 * 11 * (72 + 55 + 100) + 3 * 64 * 9 * 136 + 6 * 11 * 512
    assert bench.fp64_ops_per_cell(8, 11) == total / 512 == 1526.375
    for N in (2, 8, 16):
        # the read cells are the star region, the faces those the oracle returns
        assert N ** 3 + 18 * N * N == synth.star_cells(N)
        U = synth.iid_block(synth.rng_for(5, N), N, 6)
        _, _, _, (fx, fy, fz) = oracle.rhs_block(U, dx=0.1, faces=True)
        assert (fx.size + fy.size + fz.size) // 6 == 3 * N * N * (N + 1)


def _gpu_from_oracle(blocks, dx):
    r0, a0, _ = oracle.rhs_batch(blocks, dx=dx, mode=oracle.MODE_FP64)
    r1, a1, _ = oracle.rhs_batch(blocks, dx=dx, mode=oracle.MODE_MIXED)
    nf = blocks[0].shape[0]
    return {"fp64": np.stack([r.reshape(nf, -1) for r in r0]), "fp64_amax": np.array(a0),
            "mixed": np.stack([r.reshape(nf, -1) for r in r1]), "mixed_amax": np.array(a1)}


def test_sample_parity_figures():
    blocks = [synth.iid_block(synth.rng_for(71, s), 8, 11) for s in range(3)]
    dx = 1.0 / 64
    gpu = _gpu_from_oracle(blocks, dx)
    p = bench.oracle_sample_parity(blocks, dx, gpu)
    assert p["subgrids"] == 3 and p["oracle_flags"] == 0
    assert p["fp64_vs_oracle_err_over_1e-12"] == 0.0 and p["fp64_amax_rel"] == 0.0
    assert p["mixed_vs_oracle_mixed_ulps_of_S32"] == 0.0 and p["mixed_amax_rel_vs_oracle_mixed"] == 0.0
    # the mixed mode's own distance from binary64: small, not zero
    assert 0.0 < p["mixed_vs_oracle_fp64_normwise"] < 1e-4
    # an error planted in one binary64 result shows at its size relative to
    # that (sub-grid, field)'s scale
    s, f, i = 1, 2, 100
    scale = max(np.abs(gpu["fp64"][s, f]).max(),
                gpu["fp64_amax"][s] * np.abs(blocks[s][f]).max() / dx)
    gpu["fp64"][s, f, i] += 3e-12 * scale
    p = bench.oracle_sample_parity(blocks, dx, gpu)
    assert p["fp64_vs_oracle_err_over_1e-12"] == pytest.approx(3.0, rel=1e-3)


def test_ncu_record_follows_the_code_not_the_comments(tmp_path, monkeypatch):
    a = tmp_path / "a.cuh"
    b = tmp_path / "b.cuh"
    a.write_text("int f(int x) {\n  return x + 1;  // one\n}\n")
    b.write_text("// a header comment\nint f(int x) {\n\n  return x + 1;  // another\n}\n")
    assert bench.kernel_source_digest(str(a)) == bench.kernel_source_digest(str(b))
    b.write_text("int f(int x) {\n  return x + 2;\n}\n")
    assert bench.kernel_source_digest(str(a)) != bench.kernel_source_digest(str(b))
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))
    monkeypatch.setattr(bench, "kernel_source_digest", lambda p: rec["kernel_code_sha256"])
    assert bench.recorded_traffic("fp64", 32768) == rec["forms"]["fp64"]["bytes_per_tile"] * 32768
    assert bench.recorded_counts("mixed") == rec["forms"]["mixed"]
    monkeypatch.setattr(bench, "kernel_source_digest", lambda p: "0" * 64)
    assert bench.recorded_traffic("fp64", 32768) is None and bench.recorded_counts("mixed") is None


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler(lines, first):
    c = bench.ClockSampler(0)
    c.proc = _Done()
    c.t = threading.Thread(target=lambda: None)
    c.t.start()
    c.lines = list(lines)
    c.first = first
    return c.stop()


def test_clock_record():
    idle = "1005, 2070, 120.5, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active"
    busy = ["2070, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "2040, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "2055, 2070, 1395.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "[N/A]"]
    # the sample taken before the timed region is left out
    r = _sampler([idle] + busy, 1)
    assert r == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    # no sample inside the region: all samples
    assert _sampler([idle], 1)["samples"] == 1
    slow = "1500, 2070, 700.0, 0x8, Active, Not Active, Not Active, Not Active"
    assert _sampler([slow, busy[0]], 0)["reasons"] == ["hw_slowdown"]
    assert _sampler([], 0)["reasons"] == ["no samples"]
