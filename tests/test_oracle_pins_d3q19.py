"""Pins of the oracle's temperature LB on the D3Q19 lattice (thermal_q = 19): the BGK equation of
Eq. 19 with the standard D3Q19 weights and cs_T^2 = 1/3 (Sec. III.B), chi = (tau_g - 1/2) / 3,
grad T from the first moment of g (the D3Q19 form of Eq. 45), the source of Eqs. 23-24.

* periodic conduction: a sine mode decays as exp(-chi k^2 t);
* two Eq. 51 faces at different temperatures: the linear steady profile;
* two steps from a random temperature field (frozen uniform fluid, so phi_s = 0): the BGK
  recursion written population by population with its own streaming over the velocity set;
* a temperature wave carried by a uniform flow: phi_s with the first-moment grad T advects it at
  the flow speed and diffuses it at chi;
* the D3Q7 and D3Q19 lattices give the same decay rate for the same chi.
"""
import math

import numpy as np

import oracle
import workloads as W

E19 = np.array([
    [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
    [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
    [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]]).T
W19 = np.where((E19 ** 2).sum(1) == 0, 1 / 3, np.where((E19 ** 2).sum(1) == 1, 1 / 18, 1 / 36))


def _setup(**kw):
    base = dict(nx=1, ny=1, nz=1, sigma=W.SIGMA_STAR, thermal_q=19)
    base.update(kw)
    return W.LatticeSetup(**base)


def _mode(field, L, k=1):
    x = np.arange(L)
    return np.sum(field * np.exp(-2j * math.pi * k * x / L)) * 2 / L


def _decay(q, chi, L=64, t=1500):
    s = _setup(nx=L, flow_off=1, chi_or_lambda=chi, thermal_q=q)
    Tc = oracle.Tc_of(s)
    x = np.arange(L)
    T0, A = 0.86 * Tc, 0.01 * Tc
    T = np.broadcast_to(T0 + A * np.sin(2 * np.pi * x / L), s.shape).copy()
    o = oracle.Oracle(s)
    o.init(np.full(s.shape, 0.38), T)
    o.step(t)
    Tn = o.moments()["T"].reshape(-1)
    o.close()
    return abs(_mode(Tn - T0, L)) / A, abs(Tn.mean() - T0)


def test_d3q19_conduction_decay_rate():
    chi, L, t = 0.08, 64, 1500
    ratio, drift = _decay(19, chi, L, t)
    expect = math.exp(-chi * (2 * math.pi / L) ** 2 * t)
    assert abs(ratio / expect - 1) < 0.01, (ratio, expect)
    assert drift < 1e-14   # energy conserved to round-off


def test_d3q7_and_d3q19_decay_alike():
    r7, _ = _decay(7, 0.05)
    r19, _ = _decay(19, 0.05)
    assert abs(r7 / r19 - 1) < 0.01, (r7, r19)


def test_d3q19_anti_bounce_back_linear_profile():
    nz = 16
    s = _setup(nz=nz, flow_off=1, chi_or_lambda=0.08, bc=(0, 0, 0, 0, W.BC_THERMAL_ONLY, W.BC_THERMAL_ONLY),
               T_wall_over_Tc=(0.86, 0.86, 0.86, 0.86, 0.90, 0.82))
    Tc = oracle.Tc_of(s)
    o = oracle.Oracle(s)
    o.init(np.full(s.shape, 0.38), np.full(s.shape, 0.86 * Tc))
    o.step(20000)
    Tn = o.moments()["T"].reshape(-1)
    o.close()
    z = np.arange(nz) + 0.5
    expect = (0.90 + (0.82 - 0.90) * z / nz) * Tc
    assert np.max(np.abs(Tn - expect)) < 1e-3 * (0.08 * Tc)


def test_d3q19_two_steps_bruteforce():
    """Frozen uniform fluid (phi_s = 0): g+ = g - (g - w T) / tau_g, then g(x + e, t + 1) = g+(x, t),
    twice, on a random periodic 5 x 4 x 3 temperature field."""
    nx, ny, nz = 5, 4, 3
    chi = 0.07
    s = _setup(nx=nx, ny=ny, nz=nz, flow_off=1, chi_or_lambda=chi)
    Tc = oracle.Tc_of(s)
    T0 = (0.86 + 0.05 * W.uniform(71, nx * ny * nz)).reshape(s.shape) * Tc
    o = oracle.Oracle(s)
    o.init(np.full(s.shape, 0.38), T0)
    o.step(2)
    _, g_orc = o.pops()
    o.close()
    tau = chi * 3.0 + 0.5
    g = W19[None, None, None, :] * T0[..., None]           # [z, y, x, a]
    for _ in range(2):
        T = g.sum(-1, keepdims=True)
        gp = g - (g - W19 * T) / tau
        g = np.empty_like(gp)
        for a in range(19):
            ex, ey, ez = E19[a]
            g[..., a] = np.roll(gp[..., a], shift=(ez, ey, ex), axis=(0, 1, 2))
    assert np.max(np.abs(g.reshape(-1, 19) - g_orc)) < 1e-15 * Tc


def test_d3q19_advected_temperature_wave():
    L, U, chi = 64, 0.05, 0.05
    s = _setup(nx=L, chi_or_lambda=chi, cV=1e9)
    Tc = oracle.Tc_of(s)
    x = np.arange(L)
    T0, A = 0.86 * Tc, 1e-4 * Tc
    T = np.broadcast_to(T0 + A * np.sin(2 * np.pi * x / L), s.shape).copy()
    u = np.zeros((3,) + s.shape)
    u[0] = U
    o = oracle.Oracle(s)
    o.init(np.full(s.shape, 0.38), T, u)
    t = 640
    o.step(t)
    c = _mode(o.moments()["T"].reshape(-1) - T0, L)
    o.close()
    k = 2 * math.pi / L
    assert abs(abs(c) / (A * math.exp(-chi * k * k * t)) - 1) < 0.02
    phase = math.remainder(np.angle(c) - (-math.pi / 2 - k * U * t), 2 * math.pi)
    assert abs(phase) < 0.02 * k * U * t
