"""Drivers of the Sedov point-explosion workload: SSP-RK3 steps of the RHS on
the periodic cube of synth.sedov_domain, with the time-step rule

    dt_n = cfl * dx / a_n,   a_0 = amax(U^0),
    a_n = max of amax over the three stage evaluations of step n-1,

and the measures taken against the similarity solution (tests/sedov_exact.py):
the radius of the peak of the radially binned density, and the L1 norm of
the density error over the cube.

`oracle_run` integrates with the CPU oracle (test infrastructure);
`to_domain` / `from_domain` convert between the global array and the
domain layout [s][f][N^3] (s = bx + nb (by + nb bz)) that the GPU's domain
entry points take.
"""
from __future__ import annotations

import numpy as np

import synth


def to_domain(glob, N):
    nf, n = glob.shape[0], glob.shape[1]
    nb = n // N
    a = glob.reshape(nf, nb, N, nb, N, nb, N).transpose(1, 3, 5, 0, 2, 4, 6)
    return np.ascontiguousarray(a.reshape(nb ** 3, nf, N, N, N))


def from_domain(dom, n):
    S, nf, N = dom.shape[0], dom.shape[1], dom.shape[2]
    nb = n // N
    a = dom.reshape(nb, nb, nb, nf, N, N, N).transpose(3, 0, 4, 1, 5, 2, 6)
    return np.ascontiguousarray(a.reshape(nf, n, n, n))


def shock_measures(rho, dx, exact, t):
    """(R_peak, L1(rho)) of a density field [n][n][n] at time t."""
    n = rho.shape[0]
    r = synth.cell_radii(n)
    rho_ex, _, _ = exact.profile(r, t)
    bins = np.arange(0.0, 0.5, dx / 2)
    idx = np.digitize(r.ravel(), bins)
    cnt = np.bincount(idx, minlength=len(bins) + 1)
    prof = np.bincount(idx, rho.ravel(), minlength=len(bins) + 1) / np.maximum(cnt, 1)
    rb = (np.arange(len(prof)) - 0.5) * dx / 2
    return float(rb[np.argmax(prof)]), float(np.abs(rho - rho_ex).mean())


def oracle_run(n, t_end, gamma=5.0 / 3.0, cfl=0.3, mode=0, nf=11, threads=8, dts=None):
    """Integrate the oracle's RHS to t_end (or along the given dt sequence).
    Returns (global state, t, list of dt)."""
    import oracle

    U, dx = synth.sedov_domain(n=n, nf=nf, gamma=gamma)
    N = 8
    nb = n // N

    def rhs(U):
        outs, am, fl = oracle.rhs_batch(list(synth.gather_blocks(U, N)), gamma, dx, mode,
                                        threads=threads)
        if fl.any():
            raise RuntimeError("nonphysical state in the Sedov run")
        D = from_domain(np.stack(outs).reshape(nb ** 3, nf, N, N, N), n)
        return D, float(am.max())

    t, used = 0.0, []
    a_next = None
    k = 0
    while (dts is not None and k < len(dts)) or (dts is None and t < t_end):
        D, a0 = rhs(U)
        if a_next is None:
            a_next = a0
        dt = dts[k] if dts is not None else min(cfl * dx / a_next, t_end - t)
        U1 = U + dt * D
        D1, a1 = rhs(U1)
        U2 = 0.75 * U + 0.25 * (U1 + dt * D1)
        D2, a2 = rhs(U2)
        U = U / 3.0 + 2.0 / 3.0 * (U2 + dt * D2)
        a_next = max(a0, a1, a2)
        t += dt
        used.append(dt)
        k += 1
    return U, t, used


# ------------------------------------------------------------------ forests --
def forest_shock_measures(leaves, nb0, rho, exact, t):
    """(R_peak, L1(rho)) of the density of a forest (rho [n][N][N][N], the
    leaves of synth.sedov_forest): cells binned by the radius of their centre
    from the cube's centre, averaged with volume weights; L1 volume-weighted."""
    N = rho.shape[-1]
    xyz = synth.forest_cell_centres(leaves, nb0, N)
    r = np.sqrt(((xyz - 0.5) ** 2).sum(axis=1))
    vol = (1.0 / ((nb0 << leaves[:, 0].astype(np.int64)) * N)) ** 3
    w = np.broadcast_to(vol[:, None, None, None], r.shape)
    rho_ex, _, _ = exact.profile(r, t)
    dxf = 1.0 / ((nb0 << int(leaves[:, 0].max())) * N)
    bins = np.arange(0.0, 0.5, dxf)
    idx = np.digitize(r.ravel(), bins)
    cnt = np.bincount(idx, w.ravel(), minlength=len(bins) + 1)
    prof = np.bincount(idx, (rho * w).ravel(), minlength=len(bins) + 1) / np.maximum(cnt, 1e-300)
    rb = (np.arange(len(prof)) - 0.5) * dxf
    L1 = float((np.abs(rho - rho_ex) * w).sum() / w.sum())
    return float(rb[np.argmax(prof)]), L1


def oracle_forest_steps(leaves, nb0, U, dx0, dts, gamma=5.0 / 3.0, mode=0):
    """SSP-RK3 steps of the forest oracle along the given dt sequence."""
    from oracle import forest as of

    U = [np.asarray(u, dtype=np.float64) for u in U]
    for dt in dts:
        U1, _ = of.stage(leaves, nb0, U, U, 0.0, 1.0, dt, dx0, gamma, mode)
        U2, _ = of.stage(leaves, nb0, U1, U, 0.75, 0.25, dt, dx0, gamma, mode)
        U, _ = of.stage(leaves, nb0, U2, U, 1.0 / 3.0, 2.0 / 3.0, dt, dx0, gamma, mode)
    return U
