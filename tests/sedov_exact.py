"""Self-similar solution of the spherical point explosion (Sedov-Taylor blast
wave) in an ideal gas at rest with zero pressure.

Written from the similarity reduction of the spherical Euler equations (Sedov
1959; Landau & Lifshitz, Fluid Mechanics, Sec. 106).  With the shock radius
R(t) = xi0 (E t^2 / rho0)^(1/5), alpha = dlnR/dlnt = 2/5, Rdot = alpha R / t and
xi = r / R, the ansatz

    rho = rho0 f(xi),   u = Rdot phi(xi),   p = rho0 Rdot^2 psi(xi)

turns mass, momentum and entropy conservation into three ordinary
differential equations in xi,

    (phi - xi) f'   + f phi'     = -2 f phi / xi
    (phi - xi) phi' + psi' / f   = (1 - alpha)/alpha * phi
    psi'/psi - gamma f'/f        = 2 (1 - alpha) / (alpha (phi - xi)),

integrated inward from the strong-shock (Rankine-Hugoniot) values at xi = 1,
f = (g+1)/(g-1), phi = psi = 2/(g+1).  Energy conservation fixes xi0:

    1 = 4 pi alpha^2 xi0^5 int_0^1 (f phi^2 / 2 + psi / (g - 1)) xi^2 dxi.

Test infrastructure only (an exact solution to check the scheme against).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp

ALPHA = 0.4  # R ~ t^(2/5) in three dimensions


def _rhs(xi, y, g):
    f, phi, psi = y
    a = ALPHA
    w = phi - xi
    # unknowns f', phi', psi' of the linear system above
    #   w f' + f phi'               = -2 f phi / xi
    #   w phi' + psi'/f             = (1-a)/a phi
    #   -g/f f' + psi'/psi          = 2 (1-a) / (a w)
    A = np.array([[w, f, 0.0],
                  [0.0, w, 1.0 / f],
                  [-g / f, 0.0, 1.0 / psi]])
    b = np.array([-2.0 * f * phi / xi, (1.0 - a) / a * phi, 2.0 * (1.0 - a) / (a * w)])
    return np.linalg.solve(A, b)


class Sedov:
    """Profiles f, phi, psi on xi in (xi_min, 1] and the constant xi0."""

    def __init__(self, gamma, xi_min=1e-3, n=4000):
        g = float(gamma)
        self.gamma = g
        y0 = [(g + 1.0) / (g - 1.0), 2.0 / (g + 1.0), 2.0 / (g + 1.0)]
        xs = np.linspace(1.0, xi_min, n)
        sol = solve_ivp(_rhs, (1.0, xi_min), y0, t_eval=xs, args=(g,), method="LSODA",
                        rtol=1e-10, atol=1e-13)
        if not sol.success:
            raise RuntimeError(sol.message)
        self.xi = sol.t[::-1]
        self.f, self.phi, self.psi = (sol.y[k][::-1] for k in range(3))
        integrand = (0.5 * self.f * self.phi ** 2 + self.psi / (g - 1.0)) * self.xi ** 2
        # the inner part (xi < xi_min) holds a negligible share of the energy
        I = np.trapezoid(integrand, self.xi)
        self.energy_integral = I
        self.xi0 = (1.0 / (4.0 * math.pi * ALPHA ** 2 * I)) ** 0.2

    def shock_radius(self, t, E=1.0, rho0=1.0):
        return self.xi0 * (E * t * t / rho0) ** 0.2

    def time_for_radius(self, R, E=1.0, rho0=1.0):
        return (R / self.xi0) ** 2.5 * math.sqrt(rho0 / E)

    def profile(self, r, t, E=1.0, rho0=1.0):
        """rho, u, p at radii r (array) at time t; ambient state outside R."""
        R = self.shock_radius(t, E, rho0)
        Rdot = ALPHA * R / t
        xi = np.asarray(r, dtype=float) / R
        inside = xi <= 1.0
        xc = np.clip(xi, self.xi[0], 1.0)
        rho = np.where(inside, rho0 * np.interp(xc, self.xi, self.f), rho0)
        u = np.where(inside, Rdot * np.interp(xc, self.xi, self.phi), 0.0)
        p = np.where(inside, rho0 * Rdot ** 2 * np.interp(xc, self.xi, self.psi), 0.0)
        return rho, u, p
