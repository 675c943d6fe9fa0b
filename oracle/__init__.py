"""CPU oracle for the per-sub-grid hydro RHS (test infrastructure).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_2210_06438_gb300``) never imports it, and the two share
no code.

The arithmetic lives in ``hydro_oracle.c`` (plain C, binary64,
``-O2 -ffp-contract=off``); this module compiles it with gcc on first use and
wraps it with ctypes.  What it computes, step by step, is the scheme named in
Sec. IV-B of the paper (Euler equations; PPM reconstruction; central-upwind
flux of Kurganov & Tadmor; Courant signal speed) with the readings listed in
the C file's header.

Functions
---------
rhs_block(U, ghost, gamma, dx, mode)        any nx*ny*nz block, returns (dUdt, amax, flags)
rhs_block_faces(...)                        also returns the face fluxes per direction
rhs_batch(Us, gamma, dx, mode, threads)     list of cubic sub-grids, OpenMP over sub-grids
forest.rhs / forest.stage                   multi-level forests of sub-grids: ghost cells
                                            across levels and the flux correction
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hydro_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

NONPHYS = 1
EINVAL = 2
MODE_FP64 = 0
MODE_MIXED = 1
FLUX_KT = 0   # Kurganov-Tadmor (single speed)
FLUX_KNP = 2  # Kurganov-Noelle-Petrova (one-sided speeds); add to the mode
QUAD26 = 4    # fluxes at 9 points per face (26 per cell) with Simpson weights; add to the mode

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.ora_rhs_block.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, dp, dp, dp]
            lib.ora_rhs_block.restype = ctypes.c_int
            lib.ora_rhs_batch.argtypes = [ctypes.POINTER(dp), ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int), dp, ctypes.c_int64,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                          ctypes.POINTER(dp), dp,
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_int]
            lib.ora_rhs_batch.restype = ctypes.c_int
            lib.ora_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def rhs_block(U, ghost=3, gamma=5.0 / 3.0, dx=1.0, mode=MODE_FP64, faces=False):
    """RHS of one block.

    U: float64 array [nf][nz+2g][ny+2g][nx+2g] (x fastest).
    Returns (dUdt [nf][nz][ny][nx], amax, flags) and, if ``faces``, the face
    fluxes (fx [nf][nz][ny][nx+1], fy [nf][nz][ny+1][nx], fz [nf][nz+1][ny][nx]).
    """
    lib = _load()
    U = np.ascontiguousarray(U, dtype=np.float64)
    nf, gz, gy, gx = U.shape
    nx, ny, nz = gx - 2 * ghost, gy - 2 * ghost, gz - 2 * ghost
    out = np.zeros((nf, nz, ny, nx), dtype=np.float64)
    amax = np.zeros(1, dtype=np.float64)
    nfx = nf * nz * ny * (nx + 1)
    nfy = nf * nz * (ny + 1) * nx
    nfz = nf * (nz + 1) * ny * nx
    fbuf = np.zeros(nfx + nfy + nfz, dtype=np.float64) if faces else None
    flags = lib.ora_rhs_block(_dptr(U), nx, ny, nz, ghost, nf, float(gamma), float(dx), int(mode),
                              _dptr(out), _dptr(amax),
                              _dptr(fbuf) if faces else ctypes.POINTER(ctypes.c_double)())
    if flags & EINVAL:
        raise ValueError("oracle rejected the block arguments")
    if not faces:
        return out, float(amax[0]), flags
    fx = fbuf[:nfx].reshape(nf, nz, ny, nx + 1)
    fy = fbuf[nfx:nfx + nfy].reshape(nf, nz, ny + 1, nx)
    fz = fbuf[nfx + nfy:].reshape(nf, nz + 1, ny, nx)
    return out, float(amax[0]), flags, (fx, fy, fz)


def rhs_batch(Us, gamma=5.0 / 3.0, dx=None, mode=MODE_FP64, ghost=3, threads=1):
    """RHS of a list of cubic sub-grids (each [nf][G][G][G]); OpenMP over sub-grids.

    Returns (list of dUdt arrays, amax array, flags array)."""
    lib = _load()
    n = len(Us)
    Us = [np.ascontiguousarray(u, dtype=np.float64) for u in Us]
    N = np.array([u.shape[1] - 2 * ghost for u in Us], dtype=np.int32)
    nf = np.array([u.shape[0] for u in Us], dtype=np.int32)
    if dx is None:
        dx = np.ones(n)
    dx = np.ascontiguousarray(np.broadcast_to(np.asarray(dx, dtype=np.float64), (n,)))
    outs = [np.zeros((int(nf[s]), int(N[s]), int(N[s]), int(N[s]))) for s in range(n)]
    amax = np.zeros(n)
    flags = np.zeros(n, dtype=np.int32)
    PP = ctypes.POINTER(ctypes.c_double) * max(n, 1)
    uptr = PP(*[_dptr(u) for u in Us])
    optr = PP(*[_dptr(o) for o in outs])
    lib.ora_rhs_batch(uptr, N.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      nf.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(dx), n, ghost,
                      float(gamma), int(mode), optr, _dptr(amax),
                      flags.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(threads))
    return outs, amax, flags


def max_threads() -> int:
    return int(_load().ora_max_threads())
