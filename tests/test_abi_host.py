"""Host-side checks of the C ABI (no GPU): the library builds for sm_103a,
loads, exports every function include/hydro.h declares, and rejects invalid
arguments before touching the device."""
import ctypes
import os
import re

import pytest

import paper_2210_06438_gb300 as hydro
from paper_2210_06438_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "hydro.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hydro_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return hydro.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20, names
    so = ctypes.CDLL(_build.LIB)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_strerror_and_version(lib):
    assert hydro.strerror(hydro.HYDRO_ENONPHYS).startswith("nonphysical")
    assert hydro.strerror(12345) == "unknown status"
    assert lib.hydro_version() >= 100


def test_output_length(lib):
    d = hydro.descriptors([(8, 0.1, 8, 6), (16, 0.1, 16, 11), (24, 0.1, 5, 7)])
    assert hydro.output_doubles(d) == 6 * 512 + 11 * 4096 + 7 * 125
    bad = hydro.descriptors([(8, 0.1, 1, 6)])
    with pytest.raises(hydro.HydroError):
        hydro.output_doubles(bad)


@pytest.mark.parametrize("kw", [
    dict(items=[(8, 0.1, 1, 6)]), dict(items=[(8, 0.1, 8, 5)]), dict(items=[(8, 0.1, 8, 12)]),
    dict(items=[(8, -0.1, 8, 6)]), dict(items=[(8, float("nan"), 8, 6)]),
    dict(items=[(8, 0.1, 8, 6)], ghost=2), dict(items=[(8, 0.1, 8, 6)], gamma=1.0),
    dict(items=[(8, 0.1, 8, 6)], N=16), dict(items=[(8, 0.1, 8, 6)], n_fields=7),
    dict(items=[(0, 0.1, 8, 6)]), dict(items=[(12, 0.1, 8, 6)]),  # misaligned input
    dict(items=[(8, 0.1, 300, 6)]),
])
def test_invalid_arguments_rejected_without_device(lib, kw):
    desc = hydro.descriptors(kw["items"])
    with pytest.raises(hydro.HydroError) as ei:
        hydro.rhs(desc, 64, 64, ghost=kw.get("ghost", 3), gamma=kw.get("gamma", 5.0 / 3.0),
                  N=kw.get("N", 0), n_fields=kw.get("n_fields", 0))
    assert ei.value.code == hydro.HYDRO_EINVAL


def test_plan_and_server_argument_checks(lib):
    with pytest.raises(hydro.HydroError):
        hydro.Plan(hydro.descriptors([(8, 0.1, 8, 6)]), ghost=1)
    with pytest.raises(hydro.HydroError):
        hydro.Server(budget_bytes=0, dry_run_ns=1000)
    with pytest.raises(hydro.HydroError):
        hydro.Server(n_streams=0, dry_run_ns=1000)


def test_time_step_entry_points_check_arguments_before_the_device(lib):
    """hydro_courant and the stages that read dt from device memory refuse bad
    arguments without touching a GPU."""
    P = 0x10000  # an aligned address that is never dereferenced
    bad = [
        dict(amax=0), dict(n_rows=0), dict(row_stride=3), dict(n=0), dict(cfl=0.0),
        dict(cfl=float("nan")), dict(clock=0), dict(dx=0, dx_uniform=0.0), dict(hist_len=4, dt_hist=0),
        dict(amax=P + 4),  # misaligned
    ]
    for kw in bad:
        a = dict(amax=P, n_rows=3, row_stride=8, n=8, dx=0, dx_uniform=0.1, cfl=0.3, t_end=1.0, clock=P,
                 dt_hist=0, hist_len=0)
        a.update(kw)
        rc = lib.hydro_courant(a["amax"], a["n_rows"], a["row_stride"], a["n"], a["dx"], a["dx_uniform"],
                               a["cfl"], a["t_end"], a["clock"], a["dt_hist"], a["hist_len"], None)
        assert rc == hydro.HYDRO_EINVAL, kw
    # a null dt pointer
    assert lib.hydro_domain_stage_dt(P, P, 0.0, 1.0, None, 4, 8, 6, 0.1, 5.0 / 3.0, P * 2, P, 0, None,
                                     0) == hydro.HYDRO_EINVAL
    assert lib.hydro_forest_stage_dt(None, P, P, 0.0, 1.0, P, 0.1, 5.0 / 3.0, P * 2, P, 0, None,
                                     0) == hydro.HYDRO_EINVAL


def test_fp64_probe_checks_arguments_before_the_device(lib):
    """hydro_probe_fp64 refuses bad arguments without touching a GPU."""
    n = ctypes.c_double(0.0)
    assert lib.hydro_probe_fp64(0, 100, None, ctypes.byref(n)) == hydro.HYDRO_EINVAL
    assert lib.hydro_probe_fp64(65, 100, None, ctypes.byref(n)) == hydro.HYDRO_EINVAL
    assert lib.hydro_probe_fp64(4, 0, None, ctypes.byref(n)) == hydro.HYDRO_EINVAL
    assert lib.hydro_probe_fp64(4, 100, None, None) == hydro.HYDRO_EINVAL


def test_per_subgrid_and_server_flags_are_checked(lib):
    """Unknown flag bits are refused before any device work."""
    d = hydro.descriptors([(8, 0.1, 8, 6)])
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.hydro_rhs_per_subgrid_ex(d, 1, 3, 5.0 / 3.0, 64, 64, 0, arr, 1, 1 << 10) == hydro.HYDRO_EINVAL
    with pytest.raises(hydro.HydroError):
        hydro.Server(dry_run_ns=1000, flags=hydro.F_REGISTER_LOADS)


def test_buffers_must_be_dense_binary64():
    """The binding passes a tensor's address only when the C ABI's plain
    binary64 array reading of it is the tensor's own layout."""
    import torch

    from paper_2210_06438_gb300 import binding

    a = torch.zeros(4, 6, dtype=torch.float64)
    assert binding._ptr(a) == a.data_ptr() and binding._ptr(a[1]) == a[1].data_ptr()
    assert binding._ptr(None) == 0 and binding._ptr(4096) == 4096
    with pytest.raises(TypeError):
        binding._ptr(a.float())
    with pytest.raises(ValueError):
        binding._ptr(a.t())
    with pytest.raises(ValueError):
        binding._ptr(a[:, :3])
    # the check comes before the library is called
    desc = hydro.descriptors([(4096, 0.1, 8, 6)])
    with pytest.raises(TypeError):
        hydro.rhs(desc, torch.zeros(6 * 512, dtype=torch.float32), a[0])
