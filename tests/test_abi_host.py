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
