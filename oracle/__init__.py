"""ctypes front end of the FP64 CPU oracle (lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and by the
CPU-baseline leg of bench.py.  The CUDA path never imports it and it never imports the
CUDA path; the only module both use is `workloads` (seeded inputs, no method arithmetic).

Every function follows the passage cited in lbm_oracle.c.  `maxwell()` is the
equal-area construction on the Peng-Robinson isotherm (Eq. 49), used to place the
initial coexisting densities and to check the paper's rho_l ~ 6.5, rho_g ~ 0.38 at
0.86 Tc (Sec. IV.A).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liblbm_oracle.so")
_LIB32 = os.path.join(_LIB_DIR, "liblbm_oracle_f32.so")   # same source, -DORC_REAL=float
_lock = threading.Lock()
_lib = None
_lib32 = None


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("bc", C.c_int * 6),
        ("T_wall", C.c_double * 6),
        ("hot_dT", C.c_double), ("hot_sigma", C.c_double),
        ("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("acentric", C.c_double),
        ("sigma", C.c_double),
        ("tau_e", C.c_double), ("tau_v", C.c_double), ("tau_q", C.c_double), ("tau_pi", C.c_double),
        ("cV", C.c_double), ("d", C.c_double), ("varsigma_q", C.c_double), ("varsigma_pi", C.c_double),
        ("lambda_mode", C.c_int), ("chi_or_lambda", C.c_double),
        ("g", C.c_double * 3),
        ("flow_off", C.c_int), ("thermal_off", C.c_int),
        ("rho_buoy", C.c_double),
        ("thermal_bgk", C.c_int),
        ("divu_mode", C.c_int),
        ("wall_rho", C.c_double), ("wall_rho_patch", C.c_double), ("wall_patch_half", C.c_double),
        ("wall_scheme", C.c_int), ("wall_phi", C.c_double), ("wall_drho", C.c_double),
        ("wall_phi_patch", C.c_double), ("wall_drho_patch", C.c_double),
        ("thermal_q", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE arithmetic, OpenMP over z-planes): the FP64
    oracle, and the FP32 build of the same source that the tests use to measure rounding floors."""
    with _lock:
        for out, extra in ((_LIB, []), (_LIB32, ["-DORC_REAL=float"])):
            if (not force and os.path.exists(out)
                    and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
                continue
            os.makedirs(_LIB_DIR, exist_ok=True)
            tmp = out + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu99", *extra, "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, out)
        return _LIB


def lib(precision: str = "f64"):
    global _lib, _lib32
    if precision == "f32":
        if _lib32 is None:
            build()
            _lib32 = _bind(C.CDLL(_LIB32))
        return _lib32
    if _lib is None:
        build()
        _lib = _bind(C.CDLL(_LIB))
    return _lib


def _bind(L):
    """Declare the argument and return types of the oracle's exported functions."""
    dp = C.POINTER(C.c_double)
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.POINTER(OrcParams)]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_init.argtypes = [C.c_void_p, dp, dp, dp]
    L.orc_step.argtypes = [C.c_void_p, C.c_int]
    L.orc_moments.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
    L.orc_get_pops.argtypes = [C.c_void_p, dp, dp]
    L.orc_set_pops.argtypes = [C.c_void_p, dp, dp]
    L.orc_set_wall_map.argtypes = [C.c_void_p, dp, dp]
    L.orc_get_diag.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, dp]
    L.orc_get_rho_ave.restype = C.c_double
    L.orc_get_rho_ave.argtypes = [C.c_void_p]
    L.orc_set_rho_ave.argtypes = [C.c_void_p, C.c_double]
    L.orc_Tc.restype = C.c_double
    L.orc_Tc.argtypes = [C.POINTER(OrcParams)]
    L.orc_p_eos.restype = C.c_double
    L.orc_p_eos.argtypes = [C.POINTER(OrcParams), C.c_double, C.c_double]
    L.orc_matrix_M.argtypes = [dp]
    L.orc_matrix_N.argtypes = [dp]
    L.orc_matrix_Ninv.argtypes = [dp]
    L.orc_velocities19.argtypes = [C.POINTER(C.c_int)]
    L.orc_invert.argtypes = [C.c_int, dp, dp]
    L.orc_collide_node.argtypes = [C.POINTER(OrcParams), dp, dp, dp, C.c_double, dp, dp]
    L.orc_feq.argtypes = [C.c_double, dp, dp]
    L.orc_force_pops.argtypes = [C.POINTER(OrcParams), dp, dp, dp, C.c_double, dp]
    L.orc_fd_divergence.argtypes = [C.POINTER(OrcParams), dp, dp]
    L.orc_fd_divergence.restype = None
    L.orc_num_threads.restype = C.c_int
    L.orc_set_num_threads.argtypes = [C.c_int]
    L.orc_set_num_threads.restype = None
    return L


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def params_from_setup(s) -> OrcParams:
    """Map a workloads.LatticeSetup onto the oracle's parameter struct (its own Tc)."""
    p = OrcParams()
    p.nx, p.ny, p.nz = s.nx, s.ny, s.nz
    for k in range(6):
        p.bc[k] = int(s.bc[k])
    p.a, p.b, p.R, p.acentric = s.a, s.b, s.R, s.acentric
    Tc = lib().orc_Tc(C.byref(p))
    for k in range(6):
        p.T_wall[k] = s.T_wall_over_Tc[k] * Tc
    p.hot_dT = s.hot_dT_over_Tc * Tc
    p.hot_sigma = s.hot_sigma
    p.sigma = s.sigma
    p.tau_e, p.tau_v, p.tau_q, p.tau_pi = s.tau_e, s.tau_v, s.tau_q, s.tau_pi
    p.cV, p.d, p.varsigma_q, p.varsigma_pi = s.cV, s.d, s.varsigma_q, s.varsigma_pi
    p.lambda_mode, p.chi_or_lambda = s.lambda_mode, s.chi_or_lambda
    for k in range(3):
        p.g[k] = s.gravity[k]
    p.flow_off, p.thermal_off = s.flow_off, s.thermal_off
    p.rho_buoy = s.rho_buoy
    p.thermal_bgk = int(s.thermal_bgk)
    p.divu_mode = int(getattr(s, "divu_mode", 0))
    p.wall_rho = float(getattr(s, "wall_rho", 0.0))
    p.wall_rho_patch = float(getattr(s, "wall_rho_patch", 0.0))
    p.wall_patch_half = float(getattr(s, "wall_patch_half", 0.0))
    p.wall_scheme = int(getattr(s, "wall_scheme", 0))
    for k in ("wall_phi", "wall_drho", "wall_phi_patch", "wall_drho_patch"):
        setattr(p, k, float(getattr(s, k, 0.0)))
    p.thermal_q = int(getattr(s, "thermal_q", 7))
    return p


def Tc_of(s) -> float:
    p = OrcParams()
    p.a, p.b, p.R, p.acentric = s.a, s.b, s.R, s.acentric
    return lib().orc_Tc(C.byref(p))


def p_eos(s, rho: float, T: float) -> float:
    p = OrcParams()
    p.a, p.b, p.R, p.acentric = s.a, s.b, s.R, s.acentric
    return lib().orc_p_eos(C.byref(p), float(rho), float(T))


def maxwell(s, T: float, tol: float = 1e-13):
    """Coexisting (rho_l, rho_v, p_sat) of Eq. 49 at temperature T by equal areas.

    Solves p(rho_v) = p(rho_l) = p_sat and  int_{rho_v}^{rho_l} (p_sat - p) / rho^2 drho = 0
    (equal areas in the p - v plane) with scipy's root finder and quadrature.
    """
    from scipy.integrate import quad
    from scipy.optimize import brentq

    P = lambda r: p_eos(s, r, T)
    # spinodal points: extrema of p(rho) on (0, 1/b)
    rr = np.linspace(1e-4, 0.999 / s.b, 20001)
    pp = np.array([P(r) for r in rr])
    dp = np.diff(pp)
    idx = np.where(np.sign(dp[1:]) != np.sign(dp[:-1]))[0]
    if len(idx) < 2:
        raise ValueError("supercritical temperature: no coexistence")
    r_max, r_min = rr[idx[0] + 1], rr[idx[1] + 1]
    p_lo, p_hi = max(P(r_min), 1e-12), P(r_max)

    def roots(ps):
        rv = brentq(lambda r: P(r) - ps, 0.1 * ps / (s.R * T), r_max)
        rl = brentq(lambda r: P(r) - ps, r_min, 0.9999 / s.b)
        return rv, rl

    def area(ps):
        rv, rl = roots(ps)
        val, _ = quad(lambda r: (ps - P(r)) / (r * r), rv, rl, epsabs=1e-14, epsrel=1e-13, limit=200)
        return val

    ps = brentq(area, p_lo * (1 + 1e-9) + 1e-15, p_hi * (1 - 1e-9), xtol=tol * 1e-3, rtol=1e-14)
    rv, rl = roots(ps)
    return rl, rv, ps


class Oracle:
    """One FP64 lattice: init(rho, T[, u]) -> step(n) -> moments().

    precision="f32" runs the FP32 build of the same source (rounding-floor measurements only).
    """

    def __init__(self, setup, precision: str = "f64"):
        self.setup = setup
        self.params = params_from_setup(setup)
        self.N = setup.n_nodes
        self.shape = setup.shape
        self._L = lib(precision)
        self._h = self._L.orc_create(C.byref(self.params))
        if not self._h:
            raise MemoryError("orc_create failed")

    def close(self):
        if self._h:
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def init(self, rho, T, u=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(-1)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        rc = self._L.orc_init(self._h, _dp(rho), _dp(T), _dp(uu))
        if rc:
            raise RuntimeError(f"orc_init rc={rc}")

    def step(self, n: int = 1):
        rc = self._L.orc_step(self._h, int(n))
        if rc:
            raise FloatingPointError(f"oracle step failed rc={rc} (non-finite or psi^2 <= 0)")

    def moments(self):
        out = [np.empty(self.N) for _ in range(5)]
        rc = self._L.orc_moments(self._h, *[_dp(a) for a in out])
        if rc:
            raise FloatingPointError(f"oracle moments failed rc={rc}")
        rho, ux, uy, uz, T = [a.reshape(self.shape) for a in out]
        return dict(rho=rho, ux=ux, uy=uy, uz=uz, T=T)

    @property
    def thermal_q(self):
        return 19 if int(getattr(self.setup, "thermal_q", 7)) == 19 else 7

    def pops(self):
        q = self.thermal_q
        f = np.empty(self.N * 19)
        g = np.empty(self.N * q)
        self._L.orc_get_pops(self._h, _dp(f), _dp(g))
        return f.reshape(self.N, 19), g.reshape(self.N, q)

    def set_pops(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
        self._L.orc_set_pops(self._h, _dp(f), _dp(g))

    def set_wall_map(self, phi, drho):
        """(phi, drho) of a scheme-1 wetting wall per (x, y), arrays of ny x nx."""
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        drho = np.ascontiguousarray(drho, dtype=np.float64).reshape(-1)
        assert phi.size == drho.size == self.shape[1] * self.shape[2]
        if self._L.orc_set_wall_map(self._h, _dp(phi), _dp(drho)) != 0:
            raise ValueError("wall map: phi must be > 0 and drho >= 0")

    def diag(self):
        """div u (Eq. 48, or finite differences in divu_mode 1), grad T (Eq. 45), grad rho, F_m, phi_s,
        psi of the last step."""
        N = self.N
        d = dict(divu=np.empty(N), gradT=np.empty(3 * N), gradrho=np.empty(3 * N),
                 Fm=np.empty(3 * N), phis=np.empty(N), psi=np.empty(N))
        self._L.orc_get_diag(self._h, _dp(d["divu"]), _dp(d["gradT"]), _dp(d["gradrho"]),
                           _dp(d["Fm"]), _dp(d["phis"]), _dp(d["psi"]))
        for k in ("gradT", "gradrho", "Fm"):
            d[k] = d[k].reshape(self.shape + (3,))
        for k in ("divu", "phis", "psi"):
            d[k] = d[k].reshape(self.shape)
        return d

    @property
    def rho_ave(self):
        return self._L.orc_get_rho_ave(self._h)


def matrices():
    """M (19x19, rows of Eq. 5), its generic inverse, N and N^-1 (Eqs. 38, 41), velocities."""
    L = lib()
    M = np.empty(19 * 19)
    L.orc_matrix_M(_dp(M))
    Mi = np.empty(19 * 19)
    L.orc_invert(19, _dp(M), _dp(Mi))
    N = np.empty(49)
    Ni = np.empty(49)
    L.orc_matrix_N(_dp(N))
    L.orc_matrix_Ninv(_dp(Ni))
    e = (C.c_int * 57)()
    L.orc_velocities19(e)
    return dict(M=M.reshape(19, 19), Minv=Mi.reshape(19, 19), N=N.reshape(7, 7),
                Ninv=Ni.reshape(7, 7), e19=np.array(list(e)).reshape(19, 3))


def collide_node(setup, f, F, Fm, psi2):
    p = params_from_setup(setup)
    f = np.ascontiguousarray(f, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    Fm = np.ascontiguousarray(Fm, dtype=np.float64)
    fs = np.empty(19)
    u = np.empty(3)
    lib().orc_collide_node(C.byref(p), _dp(f), _dp(F), _dp(Fm), float(psi2), _dp(fs), _dp(u))
    return fs, u


def feq(rho, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(19)
    lib().orc_feq(float(rho), _dp(u), _dp(out))
    return out


def force_pops(setup, F, u, Fm, psi2):
    p = params_from_setup(setup)
    out = np.empty(19)
    lib().orc_force_pops(C.byref(p), _dp(np.ascontiguousarray(F, dtype=np.float64)),
                         _dp(np.ascontiguousarray(u, dtype=np.float64)),
                         _dp(np.ascontiguousarray(Fm, dtype=np.float64)), float(psi2), _dp(out))
    return out


def fd_divergence(setup, u: np.ndarray) -> np.ndarray:
    """The oracle's isotropic finite-difference divergence of a given velocity field u (shape
    (3, nz, ny, nx)) at every node, neighbours wrapped or mirrored by the setup's faces."""
    p = params_from_setup(setup)
    ui = np.ascontiguousarray(np.moveaxis(np.asarray(u, dtype=np.float64), 0, -1).reshape(-1))
    out = np.empty(setup.n_nodes, dtype=np.float64)
    lib().orc_fd_divergence(C.byref(p), _dp(ui), _dp(out))
    return out.reshape(setup.shape)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the oracle's following calls (OpenMP)."""
    lib().orc_set_num_threads(int(n))
