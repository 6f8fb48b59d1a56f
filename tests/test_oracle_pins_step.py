"""Pins of one full oracle time step and of the two phase-change terms of Eq. 18.

* The D3Q19 MRT collision of every node of a random 4^3 periodic lattice (Eqs. 1, 3, 5-10), with
  non-unit relaxation times, sigma != 0 and gravity, written here in population space as the
  explicit matrix products of Eq. 1, f* = f - M^-1 Lambda M (f - f_eq) + M^-1 (I - Lambda/2) M G,
  with M built in this file from the polynomial rows that Eq. 5 implies and inverted by numpy;
  f* is read back from the oracle's streamed state (Eq. 4 undone on the periodic lattice).
  psi (Eq. 8 with the Peng-Robinson EOS of Eq. 49) and F_m (Eq. 7) of the same step are pinned
  against sums over the velocity set of Eq. 2.
* The compression term -T/(rho c_V) (dp/dT)_rho div u of Eq. 18: a small-amplitude sound wave in a
  supercritical fluid is adiabatic; continuity and Eq. 17 without diffusion give
  dT' = R T0 / (c_V rho0 (1 - b rho0)) drho' for the wave's Fourier mode.
* The conduction term chi grad(rho c_V) . grad T / (rho c_V) of Eq. 18: in a static fluid (flow
  frozen) with a fixed density profile rho(x) between two Eq. 51 walls, the steady temperature
  solves d/dx (rho dT/dx) = 0 (Eq. 17 with lambda = rho c_V chi), i.e. T(x) follows the integral
  of 1/rho, not a straight line.

Each check would fail for a dropped term, a flipped sign, a missing factor 1/c_V, 1/rho or
(1 - b rho), or a swapped relaxation rate.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle
import workloads as W

# velocity set of Eq. 2 as printed (columns of the 3 x 19 matrix)
E19 = np.array([
    [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
    [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
    [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]]).T
CS2 = 1.0 / 3.0


def moment_matrix():
    """Rows: the raw velocity moments whose equilibria Eq. 5 lists, in its order."""
    ex, ey, ez = (E19[:, k].astype(float) for k in range(3))
    rows = [np.ones(19), ex, ey, ez, ex ** 2 + ey ** 2 + ez ** 2, 2 * ex ** 2 - ey ** 2 - ez ** 2,
            ey ** 2 - ez ** 2, ex * ey, ex * ez, ey * ez, ex ** 2 * ey, ex * ey ** 2, ex ** 2 * ez,
            ex * ez ** 2, ey ** 2 * ez, ey * ez ** 2, ex ** 2 * ey ** 2, ex ** 2 * ez ** 2, ey ** 2 * ez ** 2]
    return np.array(rows)


def eq5(rho, u):
    ux, uy, uz = u
    u2 = ux * ux + uy * uy + uz * uz
    phi = rho * CS2 * CS2 * (1 - 1.5 * u2)
    return np.array([
        rho, rho * ux, rho * uy, rho * uz, rho + rho * u2,
        rho * (2 * ux * ux - uy * uy - uz * uz), rho * (uy * uy - uz * uz),
        rho * ux * uy, rho * ux * uz, rho * uy * uz,
        rho * CS2 * uy + rho * ux * ux * uy, rho * CS2 * ux + rho * uy * uy * ux,
        rho * CS2 * uz + rho * ux * ux * uz, rho * CS2 * ux + rho * uz * uz * ux,
        rho * CS2 * uz + rho * uy * uy * uz, rho * CS2 * uy + rho * uz * uz * uy,
        phi + rho * CS2 * (ux * ux + uy * uy), phi + rho * CS2 * (ux * ux + uz * uz),
        phi + rho * CS2 * (uy * uy + uz * uz)])


def eq9(F, u, Fm, psi2, sigma, tau_e):
    Fx, Fy, Fz = F
    ux, uy, uz = u
    return np.array([
        0.0, Fx, Fy, Fz, 2 * (F @ u) + 6 * sigma * (Fm @ Fm) / (psi2 * (tau_e - 0.5)),
        2 * (2 * Fx * ux - Fy * uy - Fz * uz), 2 * (Fy * uy - Fz * uz),
        Fx * uy + Fy * ux, Fx * uz + Fz * ux, Fy * uz + Fz * uy,
        CS2 * Fy, CS2 * Fx, CS2 * Fz, CS2 * Fx, CS2 * Fz, CS2 * Fy,
        2 * CS2 * (ux * Fx + uy * Fy), 2 * CS2 * (ux * Fx + uz * Fz), 2 * CS2 * (uy * Fy + uz * Fz)])


def critical_T(a, b, R):
    """Tc from the Peng-Robinson constants a = 0.45724 R^2 Tc^2 / pc, b = 0.0778 R Tc / pc."""
    return 0.0778 * a / (0.45724 * b * R)


def p_pr(rho, T, a, b, R, omega):
    """Eq. 49."""
    Tc = critical_T(a, b, R)
    theta = (1 + (0.37464 + 1.54226 * omega - 0.26992 * omega ** 2) * (1 - np.sqrt(T / Tc))) ** 2
    return rho * R * T / (1 - b * rho) - a * theta * rho ** 2 / (1 + 2 * b * rho - b * b * rho ** 2)


def test_mrt_collision_of_a_random_lattice_bruteforce():
    """Every node of a random 4^3 periodic lattice after one oracle step equals the population-
    space matrix products of Eq. 1 (Eqs. 3, 5, 6, 9, 10), to FP64 round-off."""
    n = 4
    s = W.LatticeSetup(n, n, n, sigma=0.0931, tau_e=1.1, tau_v=0.7, tau_q=1.3, tau_pi=0.9,
                       gravity=(1.5e-4, -2.5e-4, 3.5e-4), rho_buoy=1.4)
    N = n ** 3
    Tc = critical_T(s.a, s.b, s.R)
    M = moment_matrix()
    Minv = np.linalg.inv(M)
    w = Minv @ eq5(1.0, np.zeros(3))         # rest-state weights: 1/3, 1/18, 1/36
    # a random non-equilibrium state: f = w rho (1 + noise), g = w_T T
    rho0 = W.uniform(101, N, 0.9, 2.2)
    f = (w[None, :] * rho0[:, None]) * (1 + W.uniform(102, N * 19, -0.2, 0.2).reshape(N, 19))
    T0 = W.uniform(103, N, 0.86 * Tc, 0.95 * Tc)
    wT = np.array([1 - s.d] + [s.d / 6] * 6)
    g = wT[None, :] * T0[:, None]
    o = oracle.Oracle(s)
    o.init(np.ones(s.shape), np.full(s.shape, 0.9 * Tc))
    o.set_pops(f, g)
    o.step(1)
    f1, _ = o.pops()
    d = o.diag()
    # undo the periodic streaming of Eq. 4: f*_a(x) = f_a(x + e_a, t + 1)
    idx = np.arange(N).reshape(s.shape)            # [z, y, x]
    fstar = np.empty((N, 19))
    for a in range(19):
        ex, ey, ez = E19[a]
        src = np.roll(idx, shift=(-ez, -ey, -ex), axis=(0, 1, 2)).reshape(-1)
        fstar[:, a] = f1[src, a]
    # psi of Eq. 8 (G = -1, c = 1) and F_m of Eq. 7 by direct sums over Eq. 2's velocities
    rho = f.sum(axis=1)
    T = g.sum(axis=1)
    psi = np.sqrt(2 * (rho * CS2 - p_pr(rho, T, s.a, s.b, s.R, s.acentric)))
    assert np.max(np.abs(psi - d["psi"].reshape(-1))) < 1e-14 * np.max(psi)
    wgt = np.where((E19 ** 2).sum(1) == 1, 1 / 6, np.where((E19 ** 2).sum(1) == 2, 1 / 12, 0.0))
    psi3 = psi.reshape(s.shape)
    Fm = np.zeros((N, 3))
    for a in range(1, 19):
        ex, ey, ez = E19[a]
        nb = np.roll(psi3, shift=(-ez, -ey, -ex), axis=(0, 1, 2)).reshape(-1)
        Fm += wgt[a] * nb[:, None] * E19[a][None, :].astype(float)
    Fm *= psi[:, None]                              # -G psi(x) sum w psi(x + e) e, G = -1
    assert np.max(np.abs(Fm - d["Fm"].reshape(N, 3))) < 1e-14 * np.max(np.abs(Fm))
    Lam = np.diag([1, 1, 1, 1, 1 / s.tau_e] + [1 / s.tau_v] * 5 + [1 / s.tau_q] * 6 + [1 / s.tau_pi] * 3)
    I = np.eye(19)
    err = 0.0
    for i in range(N):
        F = Fm[i] + (rho[i] - s.rho_buoy) * np.asarray(s.gravity)
        u = (E19.T @ f[i] + 0.5 * F) / rho[i]                         # Eq. 10
        feq = Minv @ eq5(rho[i], u)
        G = Minv @ eq9(F, u, Fm[i], psi[i] ** 2, s.sigma, s.tau_e)
        expect = f[i] - Minv @ Lam @ M @ (f[i] - feq) + Minv @ (I - 0.5 * Lam) @ M @ G
        err = max(err, float(np.max(np.abs(expect - fstar[i]))))
    assert err < 1e-13 * float(np.max(np.abs(fstar)))
    # a swapped rate pair (tau_q <-> tau_pi) moves f* far beyond that round-off
    Lsw = np.diag([1, 1, 1, 1, 1 / s.tau_e] + [1 / s.tau_v] * 5 + [1 / s.tau_pi] * 6 + [1 / s.tau_q] * 3)
    F = Fm[0] + (rho[0] - s.rho_buoy) * np.asarray(s.gravity)
    u = (E19.T @ f[0] + 0.5 * F) / rho[0]
    feq = Minv @ eq5(rho[0], u)
    wrong = f[0] - Minv @ Lsw @ M @ (f[0] - feq)
    right = f[0] - Minv @ Lam @ M @ (f[0] - feq)
    assert np.max(np.abs(wrong - right)) > 1e4 * err


def _mode(field, L, k=1):
    x = np.arange(L)
    return np.sum(field * np.exp(-2j * math.pi * k * x / L)) * 2 / L


def test_compression_work_of_eq18_in_an_adiabatic_sound_wave():
    """Eq. 18's -T/(rho cV) (dp/dT)_rho div u with (dp/dT)_rho = rho R / (1 - b rho): in a sound wave
    of a supercritical fluid (T0 = 1.1 Tc, rho0 = 3) the temperature mode follows the density
    mode as dT' = R T0 / (cV rho0 (1 - b rho0)) drho' (continuity + Eq. 17, diffusion negligible)."""
    L = 128
    s = W.LatticeSetup(L, 1, 1, sigma=W.SIGMA_STAR, chi_or_lambda=0.002, cV=5.0)
    Tc = critical_T(s.a, s.b, s.R)
    rho0, T0 = 3.0, 1.1 * Tc
    x = np.arange(L)
    rho = np.broadcast_to(rho0 * (1 + 1e-3 * np.cos(2 * math.pi * x / L)), s.shape).copy()
    o = oracle.Oracle(s)
    o.init(rho, np.full(s.shape, T0))
    K = s.R * T0 / (s.cV * rho0 * (1 - s.b * rho0))
    r0 = _mode(rho.reshape(-1), L)
    dr, dT = [], []
    for _ in range(40):
        o.step(10)
        m = o.moments()
        dr.append((_mode(m["rho"].reshape(-1), L) - r0).real)
        dT.append(_mode(m["T"].reshape(-1) - T0, L).real)
    dr, dT = np.array(dr), np.array(dT)
    assert np.max(np.abs(dr)) > 0.6 * 1e-3 * rho0          # the wave has swung through most of its range
    slope = float(dT @ dr / (dr @ dr))
    assert abs(slope / K - 1) < 0.01, (slope, K)


def test_density_weighted_conduction_of_eq18_in_a_static_fluid():
    """Eq. 18's chi grad(rho cV).grad T / (rho cV) with the flow frozen: between Eq. 51 walls at
    x = -1/2 and L - 1/2 the steady temperature over a fixed density profile rho(x) solves
    d/dx (rho dT/dx) = 0, T = T_a + (T_b - T_a) int dx / rho / int_0^L dx / rho."""
    L = 64
    Ta, Tb = 0.90, 0.82
    s = W.LatticeSetup(L, 1, 1, sigma=W.SIGMA_STAR, flow_off=1, chi_or_lambda=0.3,
                       bc=(W.BC_WALL, W.BC_WALL, 0, 0, 0, 0),
                       T_wall_over_Tc=(Ta, Tb, 0.86, 0.86, 0.86, 0.86))
    Tc = critical_T(s.a, s.b, s.R)
    prof = lambda xx: 3.5 + 2.5 * np.cos(math.pi * (xx + 0.5) / L)   # flat at both walls
    x = np.arange(L, dtype=float)
    rho = np.broadcast_to(prof(x), s.shape).copy()
    lin = Ta + (Tb - Ta) * (x + 0.5) / L
    o = oracle.Oracle(s)
    o.init(rho, np.broadcast_to(lin * Tc, s.shape).copy())
    o.step(16000)
    Tn = o.moments()["T"].reshape(-1) / Tc
    total = quad(lambda xx: 1.0 / prof(xx), -0.5, L - 0.5)[0]
    closed = np.array([Ta + (Tb - Ta) * quad(lambda xx: 1.0 / prof(xx), -0.5, xi)[0] / total for xi in x])
    bend = np.max(np.abs(closed - lin))
    assert bend > 0.1 * abs(Tb - Ta)                        # far from the uniform-density straight line
    assert np.max(np.abs(Tn - closed)) < 0.02 * bend, (np.max(np.abs(Tn - closed)), bend)
