"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the FP64 oracle.

This module holds no arithmetic of the lattice Boltzmann method itself: no equation of
state, no equilibrium, no collision.  It only builds initial density / temperature /
velocity fields of the shapes used by the paper's three tests (Sec. IV.A static and
evaporating droplet, Sec. IV.B heated-surface droplet, Sec. IV.C pool boiling), and the
lattice parameter sets of the workloads.  Coexistence densities (which need the equation
of state) are passed in by the caller; each side computes them with its own code.

Layout convention for every field: numpy array of shape (nz, ny, nx), x fastest, i.e.
node index = x + nx * (y + ny * z).

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out from its published
definition; uniform doubles take the top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

MASTER_SEED = 20220116

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n successive splitmix64 outputs for a generator started at `seed` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n doubles uniform in [lo, hi) from splitmix64(seed)."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def _coords(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def _min_image(d: np.ndarray, n: int, periodic: bool) -> np.ndarray:
    if not periodic:
        return d
    return d - n * np.round(d / n)


def tanh_profile(r: np.ndarray, R0: float, W: float, inside: float, outside: float) -> np.ndarray:
    """Diffuse-interface profile: `inside` for r << R0, `outside` for r >> R0.

    rho(r) = (in + out)/2 - (in - out)/2 tanh(2 (r - R0) / W).  The workloads use W = 4,
    i.e. tanh((r - R0)/2): an "interface width 2" read as the tanh length scale.
    """
    return 0.5 * (inside + outside) - 0.5 * (inside - outside) * np.tanh(2.0 * (r - R0) / W)


def droplet(shape, R0: float, W: float, rho_in: float, rho_out: float,
            periodic=(True, True, True), center=None) -> np.ndarray:
    """Spherical drop (or bubble if rho_in < rho_out) centred at (n/2, n/2, n/2)."""
    nz, ny, nx = shape
    x, y, z = _coords(shape)
    cx, cy, cz = center if center is not None else (nx / 2.0, ny / 2.0, nz / 2.0)
    dx = _min_image(x - cx, nx, periodic[0])
    dy = _min_image(y - cy, ny, periodic[1])
    dz = _min_image(z - cz, nz, periodic[2])
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    return tanh_profile(r, R0, W, rho_in, rho_out)


def slab(shape, half_thickness: float, W: float, rho_in: float, rho_out: float,
         axis: int = 2) -> np.ndarray:
    """Flat liquid slab normal to `axis` (0=x, 1=y, 2=z), centred, periodic minimum image."""
    x, y, z = _coords(shape)
    c = [x, y, z][axis]
    n = shape[2 - axis]
    d = np.abs(_min_image(c - n / 2.0, n, True))
    return tanh_profile(d, half_thickness, W, rho_in, rho_out)


def pool(shape, height: float, W: float, rho_l: float, rho_v: float) -> np.ndarray:
    """Liquid pool filling z < height, vapour above."""
    _, _, z = _coords(shape)
    return tanh_profile(z, height, W, rho_l, rho_v)


def add_noise(field_: np.ndarray, seed: int, amp: float) -> np.ndarray:
    """Add uniform noise in [-amp, amp) drawn from splitmix64(seed), in node order."""
    flat = field_.reshape(-1)
    return (flat + uniform(seed, flat.size, -amp, amp)).reshape(field_.shape)


# ----------------------------------------------------------------------------------------
# Lattice parameter sets of the workloads (values of Sec. IV; where the paper is silent the value
# is a reading stated beside it)
# ----------------------------------------------------------------------------------------

BC_PERIODIC, BC_WALL, BC_OUTFLOW, BC_THERMAL_ONLY = 0, 1, 2, 3


@dataclass
class LatticeSetup:
    """Plain parameter record; each side maps it onto its own parameter struct."""
    nx: int
    ny: int
    nz: int
    bc: Tuple[int, int, int, int, int, int] = (0, 0, 0, 0, 0, 0)   # -x,+x,-y,+y,-z,+z
    T_wall_over_Tc: Tuple[float, ...] = (0.86,) * 6
    hot_dT_over_Tc: float = 0.0
    hot_sigma: float = 10.0
    a: float = 2.0 / 49.0
    b: float = 2.0 / 21.0
    R: float = 1.0
    acentric: float = 0.344
    sigma: float = 0.0
    tau_e: float = 1.25
    tau_v: float = 0.8
    tau_q: float = 1.0
    tau_pi: float = 1.0
    cV: float = 5.0
    d: float = 0.95
    varsigma_q: float = 1.0
    varsigma_pi: float = 1.0
    lambda_mode: int = 0          # 0: constant chi, 1: constant lambda
    chi_or_lambda: float = 0.08
    gravity: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    flow_off: int = 0             # f frozen: a static fluid (u = 0, div u = 0; conduction only)
    thermal_off: int = 0          # g frozen (isothermal phase)
    rho_buoy: float = 0.0         # > 0: fixed reference density of the buoyancy force (else rho_ave)
    thermal_bgk: int = 0          # 1: BGK D3Q7 collision (one rate 1/varsigma_T) instead of MRT
    divu_mode: int = 0            # 1: finite-difference div u in the interior, Eq. 48 next to solid faces
    wall_rho: float = 0.0         # > 0: virtual density of the solid layer below the -z wall (wetting)
    wall_rho_patch: float = 0.0   # virtual density inside the patch around (nx/2, ny/2)
    wall_patch_half: float = 0.0  # half side of the square patch; 0: no patch
    wall_scheme: int = 0          # 1: rho_w = max(phi rho_ave - drho, rho_ave / 10) from the fluid layer
    wall_phi: float = 0.0
    wall_drho: float = 0.0
    wall_phi_patch: float = 0.0
    wall_drho_patch: float = 0.0
    thermal_q: int = 7            # thermal lattice: 7 (D3Q7 MRT, Eqs. 37-43) or 19 (Eq. 19 BGK on D3Q19)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n_nodes(self):
        return self.nx * self.ny * self.nz


# Thermodynamic-consistency constant of Eq. 9.  The paper does not print its value; it is
# chosen once by the flat-interface calibration script in oracle/ and frozen here.
SIGMA_STAR = 0.1125
# The same calibration for a = 1/49, the EOS constant of the paper's droplet tests (Sec. IV.A).
SIGMA_STAR_A1_49 = 0.1175


def static_droplet(n: int = 32, R0: float = 8.0, W: float = 4.0) -> Dict:
    """Static droplet, n^3 periodic, uniform T = 0.86 Tc (Sec. IV.A spurious-current test)."""
    s = LatticeSetup(n, n, n, sigma=SIGMA_STAR)
    return dict(name=f"static_droplet_{n}^3", setup=s, kind="droplet", R0=R0, W=W,
                Tr_drop=0.86, Tr_gas=0.86)


def evaporation(n: int = 128, R0: float = 24.0, W: float = 4.0) -> Dict:
    """Droplet at 0.86 Tc in vapour held at 0.95 Tc by Dirichlet faces (Sec. IV.A D^2 law).

    EOS constant a = 1/49 as in the paper's D^2 test, with its own calibrated sigma* (with
    a = 2/49 the 128^3 case diverges within 2000 steps)."""
    s = LatticeSetup(n, n, n, bc=(BC_THERMAL_ONLY,) * 6, T_wall_over_Tc=(0.95,) * 6,
                     a=1.0 / 49.0, sigma=SIGMA_STAR_A1_49, lambda_mode=1, chi_or_lambda=0.2)
    return dict(name=f"droplet_evaporation_{n}^3", setup=s, kind="droplet", R0=R0, W=W,
                Tr_drop=0.86, Tr_gas=0.95)


# Saturated vapour density of the Peng-Robinson EOS (a = 2/49, b = 2/21, R = 1, acentric 0.344)
# at 0.86 Tc from the Maxwell equal-area construction (the EOS pin of the oracle tests checks it).
RHO_V_086 = 0.37968


def pool_boiling(nx: int = 200, ny: int = 200, nz: int = 300, height: float = 100.0,
                 hot_sigma: float = 10.0, g: float = 3e-5, W: float = 4.0,
                 rho_buoy: float = RHO_V_086) -> Dict:
    """Pool boiling: bottom wall with a Gaussian hot spot, top outflow (Sec. IV.C).

    The top is open, so the buoyancy force takes the ambient saturated vapour as its reference
    density, F_b = (rho - rho_v) g: the vapour column is force-free and the liquid is carried by
    the bottom wall.  (With the closed-box reference rho_ave the vapour column is driven up
    through the open top; the run drains mass and cools until it diverges.)"""
    s = LatticeSetup(nx, ny, nz, bc=(BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC,
                                     BC_WALL, BC_OUTFLOW),
                     T_wall_over_Tc=(0.86,) * 6, hot_dT_over_Tc=0.10, hot_sigma=hot_sigma,
                     sigma=SIGMA_STAR, lambda_mode=0, chi_or_lambda=0.08,
                     gravity=(0.0, 0.0, -g), rho_buoy=rho_buoy)
    return dict(name=f"pool_boiling_{nx}x{ny}x{nz}", setup=s, kind="pool", height=height,
                W=W, Tr_liquid=0.86)


def pool_boiling_downscaled() -> Dict:
    """64x64x96 copy of the pool-boiling case, geometry scaled by 0.32."""
    return pool_boiling(64, 64, 96, height=32.0, hot_sigma=3.2)


# Parameters of the improved virtual-density wall (scheme 1: rho_w = phi rho_ave - drho) chosen by
# a sessile-droplet sweep on this model (contact angle from the droplet's cap) to give about
# 37 degrees (hydrophilic, phi) and 130 degrees (hydrophobic, drho), the two angles of the
# nucleate boiling test (Sec. IV.C).
WET_PHI_37 = 1.40
WET_DRHO_130 = 0.284


def nucleate_boiling(nx: int = 200, ny: int = 200, nz: int = 280, liquid: float = 200.0,
                     patch_side: float = 55.0, g: float = 1.5e-5, W: float = 4.0) -> Dict:
    """Bubble nucleation and departure (Sec. IV.C): saturated liquid (0 <= z <= liquid) under its
    vapour at 0.86 Tc, bottom wall at 0.96 Tc with a hydrophobic square patch at its centre and a
    hydrophilic rest, bounce-back at the top and the bottom, periodic x and y, chi = 0.08, and
    buoyancy against the domain-mean density."""
    s = LatticeSetup(nx, ny, nz, bc=(BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC,
                                     BC_WALL, BC_WALL),
                     T_wall_over_Tc=(0.86, 0.86, 0.86, 0.86, 0.96, 0.86), hot_dT_over_Tc=0.0,
                     sigma=SIGMA_STAR, lambda_mode=0, chi_or_lambda=0.08,
                     gravity=(0.0, 0.0, -g), rho_buoy=0.0,
                     wall_scheme=1, wall_phi=WET_PHI_37, wall_drho=0.0, wall_phi_patch=1.0,
                     wall_drho_patch=WET_DRHO_130, wall_patch_half=0.5 * patch_side)
    return dict(name=f"nucleate_boiling_{nx}x{ny}x{nz}", setup=s, kind="pool", height=liquid,
                W=W, Tr_liquid=0.86)


def heated_surface_droplet(nx: int = 200, ny: int = 200, nz: int = 100, R0: float = 30.0,
                           W: float = 4.0) -> Dict:
    """Droplet evaporation on a heated surface (Sec. IV.B): a hemispherical drop of radius 30 at
    the centre of a bottom wall at 0.87 Tc (contact angle about 88 degrees: a scheme-1 wall with
    phi = 1, drho = 0.005), open top held at T_sat = 0.86 Tc, periodic x and y, no gravity,
    chi = 0.02, and the EOS constant and sigma* of the droplet tests (a = 1/49).  The paper runs
    the first 10^4 steps without the thermal model (thermal_off); the contact-line pinning of
    its hysteresis window is set by the caller through the wettability map.  The vapour starts at
    0.42 rather than the flat-interface coexistence density 0.38: the drop's Laplace pressure
    holds its vapour above saturation, and a vapour started at 0.38 takes the whole drop up in
    this 4M-node box while it settles."""
    s = LatticeSetup(nx, ny, nz, bc=(BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC,
                                     BC_WALL, BC_OUTFLOW),
                     T_wall_over_Tc=(0.86, 0.86, 0.86, 0.86, 0.87, 0.86), hot_dT_over_Tc=0.0,
                     a=1.0 / 49.0, sigma=SIGMA_STAR_A1_49, lambda_mode=0, chi_or_lambda=0.02,
                     gravity=(0.0, 0.0, 0.0), wall_scheme=1, wall_phi=1.0, wall_drho=0.005)
    return dict(name=f"heated_surface_droplet_{nx}x{ny}x{nz}", setup=s, kind="sessile", R0=R0,
                W=W, Tr_drop=0.86, Tr_gas=0.86, rho_gas=0.42)


def batch_instances(count: int = 256, seed: int = MASTER_SEED) -> List[Dict]:
    """Ensemble of periodic droplets (even i) and flat slabs (odd i) of uneven size.

    The EOS constant is a = 1/49, as in the paper's droplet tests (Sec. IV.A), with its own
    calibrated sigma*, and the initial tanh interface is 6 lattice units wide.  (With a = 2/49, or
    with narrower initial interfaces, the larger droplets below 0.85 Tc diverge within 50 steps:
    the start-up compression wave converges on the droplet centre and the phase-change source
    amplifies it.)"""
    out = []
    for i in range(count):
        r = uniform(seed + i, 4)
        L = 24 + int(r[0] * 73)                      # U{24..96}
        Tr = 0.80 + 0.10 * r[1]
        R_frac = 0.20 + 0.15 * r[2]
        s = LatticeSetup(L, L, L, a=1.0 / 49.0, sigma=SIGMA_STAR_A1_49)
        out.append(dict(name=f"inst{i}", setup=s, kind="droplet" if i % 2 == 0 else "slab",
                        R0=R_frac * L, W=6.0, Tr_drop=Tr, Tr_gas=Tr, noise=1e-3,
                        noise_seed=seed + 1000003 + i))
    return out


def build_fields(case: Dict, Tc: float, rho_l: float, rho_v: float,
                 rho_l_gas: Optional[float] = None):
    """Initial (rho, T, u) of a case; Tc and coexistence densities come from the caller.

    Returns float64 arrays rho (nz,ny,nx), T (nz,ny,nx) and u = None (fluid at rest).
    """
    s: LatticeSetup = case["setup"]
    shape = s.shape
    periodic = (s.bc[0] != BC_WALL and s.bc[0] != BC_OUTFLOW,
                s.bc[2] != BC_WALL and s.bc[2] != BC_OUTFLOW,
                s.bc[4] != BC_WALL and s.bc[4] != BC_OUTFLOW)
    kind = case["kind"]
    if kind == "droplet":
        rho = droplet(shape, case["R0"], case["W"], rho_l, rho_v, periodic=periodic)
        if case["Tr_drop"] == case["Tr_gas"]:
            T = np.full(shape, case["Tr_drop"] * Tc)
        else:
            nz, ny, nx = shape
            x, y, z = _coords(shape)
            r = np.sqrt((x - nx / 2.0) ** 2 + (y - ny / 2.0) ** 2 + (z - nz / 2.0) ** 2)
            T = np.where(r <= case["R0"], case["Tr_drop"] * Tc, case["Tr_gas"] * Tc)
    elif kind == "slab":
        rho = slab(shape, case["R0"], case["W"], rho_l, rho_v, axis=2)
        T = np.full(shape, case["Tr_drop"] * Tc)
    elif kind == "sessile":   # hemisphere on the -z wall (the wall plane is z = -1/2)
        nz, ny, nx = shape
        rho = droplet(shape, case["R0"], case["W"], rho_l, case.get("rho_gas", rho_v), periodic=periodic,
                      center=(nx / 2.0, ny / 2.0, -0.5))
        T = np.full(shape, case["Tr_drop"] * Tc)
    elif kind == "pool":
        rho = pool(shape, case["height"], case["W"], rho_l, rho_v)
        T = np.full(shape, case["Tr_liquid"] * Tc)
    else:
        raise ValueError(kind)
    if case.get("noise"):
        rho = add_noise(rho, case["noise_seed"], case["noise"])
    return np.ascontiguousarray(rho), np.ascontiguousarray(T), None


def random_state(shape, seed: int, rho_lo=0.5, rho_hi=6.0, T_lo=0.055, T_hi=0.068):
    """Smooth-free random (rho, T) fields for small brute-force parity cases."""
    n = int(np.prod(shape))
    rho = uniform(seed, n, rho_lo, rho_hi).reshape(shape)
    T = uniform(seed + 7919, n, T_lo, T_hi).reshape(shape)
    return rho, T
