"""Host-side Peng-Robinson helpers for setting up initial fields (not part of the time step).

The equal-area (Maxwell) construction on the isotherm of Eq. 49 gives the coexisting
liquid and vapour densities that the workloads place on either side of an interface.
"""
from __future__ import annotations

import math

import numpy as np


def critical_temperature(a: float, b: float, R: float) -> float:
    """Tc with the paper's rounded PR constants: a = 0.45724 R^2 Tc^2/pc, b = 0.0778 R Tc/pc."""
    return 0.0778 * a / (0.45724 * b * R)


def pressure(rho, T, a, b, R, acentric):
    Tc = critical_temperature(a, b, R)
    kap = 0.37464 + 1.54226 * acentric - 0.26992 * acentric ** 2
    theta = (1.0 + kap * (1.0 - np.sqrt(T / Tc))) ** 2
    return rho * R * T / (1.0 - b * rho) - a * theta * rho ** 2 / (1.0 + 2.0 * b * rho - (b * rho) ** 2)


def coexistence(T: float, a: float = 2 / 49, b: float = 2 / 21, R: float = 1.0, acentric: float = 0.344):
    """(rho_l, rho_v, p_sat) at temperature T by equal areas in the p-v plane."""
    from scipy.integrate import quad
    from scipy.optimize import brentq

    P = lambda r: float(pressure(r, T, a, b, R, acentric))
    rr = np.linspace(1e-4, 0.999 / b, 20001)
    pp = pressure(rr, T, a, b, R, acentric)
    d = np.diff(pp)
    idx = np.where(np.sign(d[1:]) != np.sign(d[:-1]))[0]
    if len(idx) < 2:
        raise ValueError("no coexistence above Tc")
    r_max, r_min = rr[idx[0] + 1], rr[idx[1] + 1]
    lo, hi = max(P(r_min), 1e-12), P(r_max)

    def roots(ps):
        return (brentq(lambda r: P(r) - ps, 0.1 * ps / (R * T), r_max),
                brentq(lambda r: P(r) - ps, r_min, 0.9999 / b))

    def area(ps):
        rv, rl = roots(ps)
        return quad(lambda r: (ps - P(r)) / (r * r), rv, rl, epsabs=1e-14, epsrel=1e-13, limit=200)[0]

    ps = brentq(area, lo * (1 + 1e-9) + 1e-15, hi * (1 - 1e-9), xtol=1e-16, rtol=1e-14)
    rv, rl = roots(ps)
    return rl, rv, ps
