"""Thin ctypes binding of the C-ABI in include/lbm.h (same names, argument marshalling only).

Every step of the lattice update runs in the CUDA kernels of libgb300lbm.so; there is no
CPU fallback.  If the library is missing this module raises at import of `lib()`.
Field arguments may be numpy arrays (host memory; copied inside the call) or CUDA torch
tensors (device memory; used in place).  All fields are float32, shape (nz, ny, nx) or
flat, node index x + nx*(y + ny*z); a velocity field is (3, nz, ny, nx).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ESTATE, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_EBOUNDS = 0, -1, -2, -3, -4, -5, -6, -7
LBM_NOALLOC_MAX_ELEMENTS = 1 << 31
LBM_BC_PERIODIC, LBM_BC_WALL, LBM_BC_OUTFLOW, LBM_BC_THERMAL_ONLY = 0, 1, 2, 3
LBM_FP32, LBM_BF16_SHIFTED, LBM_FP16_SHIFTED = 0, 1, 2
LBM_KERNEL_AUTO, LBM_KERNEL_TWO_PASS, LBM_KERNEL_FUSED, LBM_KERNEL_FUSED_TMA = 0, 1, 2, 3


class LbmParams(C.Structure):
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
        ("g", C.c_double * 3), ("rho_buoy", C.c_double),
        ("flow_off", C.c_int), ("thermal_off", C.c_int),
        ("precision", C.c_int), ("rho_ref", C.c_double), ("T_ref", C.c_double),
        ("kernel", C.c_int), ("use_graph", C.c_int), ("use_tma", C.c_int), ("check_nonfinite", C.c_int),
        ("cuda_stream", C.c_void_p),
        ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t), ("test_stall", C.c_int),
        ("thermal_bgk", C.c_int), ("divu_mode", C.c_int),
        ("wall_rho", C.c_double), ("wall_rho_patch", C.c_double), ("wall_patch_half", C.c_double),
        ("wall_scheme", C.c_int), ("wall_phi", C.c_double), ("wall_drho", C.c_double),
        ("wall_phi_patch", C.c_double), ("wall_drho_patch", C.c_double),
        ("thermal_q", C.c_int),
    ]


# every symbol include/lbm.h declares
EXPORTS = ["lbm_params_default", "lbm_eos_critical", "lbm_workspace_bytes", "lbm_create",
           "lbm_init_fields", "lbm_step", "lbm_get_moments", "lbm_get_totals", "lbm_steps_done",
           "lbm_kernel_in_use",
           "lbm_step_profiled", "lbm_plan_shapes", "lbm_get_plan", "lbm_select_plan", "lbm_autotune",
           "lbm_destroy", "lbm_status_str", "lbm_last_error", "lbm_field_sum_noalloc",
           "lbm_state_bytes", "lbm_save_state", "lbm_load_state", "lbm_set_wall_map",
           "lbm_batch_create", "lbm_batch_nodes", "lbm_batch_init_fields", "lbm_batch_step", "lbm_batch_autotune",
           "lbm_batch_plan", "lbm_batch_select_plan", "lbm_batch_get_moments", "lbm_batch_get_totals",
           "lbm_batch_steps_done", "lbm_batch_launches_per_step", "lbm_batch_destroy"]

_lib = None


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libgb300lbm.so (building it from source if needed); raise if it cannot be had."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library {_build.LIB} is missing: build it with paper_2201_06039_gb300.build")
    L = C.CDLL(_build.LIB)
    P = C.POINTER(LbmParams)
    vp, fp, dp = C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_double)
    L.lbm_params_default.argtypes = [P]
    L.lbm_params_default.restype = None
    L.lbm_eos_critical.argtypes = [P, dp, dp]
    L.lbm_workspace_bytes.argtypes = [P]
    L.lbm_workspace_bytes.restype = C.c_size_t
    L.lbm_create.argtypes = [P, C.POINTER(vp)]
    L.lbm_init_fields.argtypes = [vp, vp, vp, vp]
    L.lbm_step.argtypes = [vp, C.c_int]
    L.lbm_get_moments.argtypes = [vp, vp, vp, vp, vp, vp]
    L.lbm_get_totals.argtypes = [vp, dp, dp, dp]
    L.lbm_steps_done.argtypes = [vp]
    L.lbm_steps_done.restype = C.c_longlong
    L.lbm_state_bytes.argtypes = [vp]
    L.lbm_state_bytes.restype = C.c_size_t
    L.lbm_save_state.argtypes = [vp, vp, C.c_size_t]
    L.lbm_load_state.argtypes = [vp, vp, C.c_size_t]
    L.lbm_set_wall_map.argtypes = [vp, vp, vp]
    L.lbm_kernel_in_use.argtypes = [vp]
    L.lbm_step_profiled.argtypes = [vp, C.c_int, dp, C.POINTER(C.c_int)]
    L.lbm_plan_shapes.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int]
    L.lbm_get_plan.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.lbm_select_plan.argtypes = [vp, C.c_int, C.c_int]
    L.lbm_autotune.argtypes = [vp, C.c_int, dp]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_status_str.argtypes = [C.c_int]
    L.lbm_status_str.restype = C.c_char_p
    L.lbm_field_sum_noalloc.argtypes = [vp, C.c_longlong, dp, vp]
    L.lbm_last_error.argtypes = []
    L.lbm_last_error.restype = C.c_char_p
    ip = C.POINTER(C.c_int)
    L.lbm_batch_create.argtypes = [P, C.c_int, ip, C.POINTER(vp)]
    L.lbm_batch_nodes.argtypes = [vp, C.c_int]
    L.lbm_batch_nodes.restype = C.c_longlong
    L.lbm_batch_init_fields.argtypes = [vp, vp, vp, vp]
    L.lbm_batch_step.argtypes = [vp, C.c_int]
    L.lbm_batch_autotune.argtypes = [vp, C.c_int, dp]
    L.lbm_batch_plan.argtypes = [vp, ip, ip, ip, ip]
    L.lbm_batch_select_plan.argtypes = [vp, C.c_int, C.c_int]
    L.lbm_batch_get_moments.argtypes = [vp, vp, vp, vp, vp, vp]
    L.lbm_batch_get_totals.argtypes = [vp, dp]
    L.lbm_batch_steps_done.argtypes = [vp]
    L.lbm_batch_steps_done.restype = C.c_longlong
    L.lbm_batch_launches_per_step.argtypes = [vp]
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != LBM_OK:
        L = lib(False)
        raise LbmError(rc, f"{what}: {L.lbm_status_str(rc).decode()}: {L.lbm_last_error().decode()}")


def _ptr(a):
    """Raw pointer of a numpy array (host) or a torch tensor (device or host)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"], "fields must be contiguous float32"
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        assert a.dtype == torch.float32 and a.is_contiguous(), "fields must be contiguous float32"
        return a.data_ptr()
    raise TypeError(type(a))


# ------------------------------------------------------------------- the C-ABI, same names
def lbm_params_default() -> LbmParams:
    p = LbmParams()
    lib().lbm_params_default(C.byref(p))
    return p


def lbm_eos_critical(p: LbmParams):
    Tc, pc = C.c_double(), C.c_double()
    _check(lib().lbm_eos_critical(C.byref(p), C.byref(Tc), C.byref(pc)), "lbm_eos_critical")
    return Tc.value, pc.value


def lbm_workspace_bytes(p: LbmParams) -> int:
    return int(lib().lbm_workspace_bytes(C.byref(p)))


def lbm_create(p: LbmParams):
    h = C.c_void_p()
    _check(lib().lbm_create(C.byref(p), C.byref(h)), "lbm_create")
    return h


def lbm_init_fields(ctx, rho, T, u=None):
    _check(lib().lbm_init_fields(ctx, _ptr(rho), _ptr(T), _ptr(u)), "lbm_init_fields")


def lbm_step(ctx, n: int):
    _check(lib().lbm_step(ctx, int(n)), "lbm_step")


def lbm_get_moments(ctx, rho=None, ux=None, uy=None, uz=None, T=None):
    _check(lib().lbm_get_moments(ctx, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(uz), _ptr(T)), "lbm_get_moments")


def lbm_get_totals(ctx):
    m, t, r = C.c_double(), C.c_double(), C.c_double()
    _check(lib().lbm_get_totals(ctx, C.byref(m), C.byref(t), C.byref(r)), "lbm_get_totals")
    return m.value, t.value, r.value


def lbm_steps_done(ctx) -> int:
    return int(lib().lbm_steps_done(ctx))


def lbm_state_bytes(ctx) -> int:
    return int(lib().lbm_state_bytes(ctx))


def lbm_save_state(ctx) -> np.ndarray:
    """Checkpoint of the context's state as a host byte array."""
    buf = np.empty(lbm_state_bytes(ctx), dtype=np.uint8)
    _check(lib().lbm_save_state(ctx, buf.ctypes.data, buf.nbytes), "lbm_save_state")
    return buf


def lbm_load_state(ctx, buf: np.ndarray):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().lbm_load_state(ctx, buf.ctypes.data, buf.nbytes), "lbm_load_state")


def lbm_set_wall_map(ctx, phi, drho):
    """(phi, drho) of a scheme-1 wetting wall per (x, y): float32 arrays of ny x nx (numpy or torch)."""
    _check(lib().lbm_set_wall_map(ctx, _ptr(phi), _ptr(drho)), "lbm_set_wall_map")


def lbm_kernel_in_use(ctx) -> int:
    return int(lib().lbm_kernel_in_use(ctx))


def lbm_step_profiled(ctx, n: int):
    ms = (C.c_double * 3)()
    cnt = (C.c_int * 3)()
    _check(lib().lbm_step_profiled(ctx, int(n), ms, cnt), "lbm_step_profiled")
    return list(ms), list(cnt)


def lbm_plan_shapes():
    """[(tile_w, tile_h), ...] of the TMA kernel's tile shapes, by shape index."""
    n = int(lib().lbm_plan_shapes(None, None, 0))
    w = (C.c_int * n)()
    h = (C.c_int * n)()
    lib().lbm_plan_shapes(w, h, n)
    return list(zip(list(w), list(h)))


def lbm_get_plan(ctx):
    """(shape, zchunk, items, ctas) of the TMA plan in use; shape -1 without the TMA kernel."""
    v = [C.c_int() for _ in range(4)]
    _check(lib().lbm_get_plan(ctx, *[C.byref(x) for x in v]), "lbm_get_plan")
    return tuple(x.value for x in v)


def lbm_select_plan(ctx, shape: int, zchunk: int = 0):
    _check(lib().lbm_select_plan(ctx, int(shape), int(zchunk)), "lbm_select_plan")


def lbm_autotune(ctx, steps: int) -> float:
    ms = C.c_double()
    _check(lib().lbm_autotune(ctx, int(steps), C.byref(ms)), "lbm_autotune")
    return ms.value


def lbm_field_sum_noalloc(field, n: int, stream=None) -> float:
    """FP64 sum of n float32 values at device pointer `field` (int) or a CUDA float32 tensor,
    using no device allocation (see include/lbm.h).

    With a tensor, n must not exceed its element count, and the call runs with the tensor's device
    current and, unless `stream` is given, on torch's current stream of that device (the stream
    torch's own kernels that produced the field ran on).  With a raw pointer the current device
    is used and `stream` None means the legacy default stream."""
    if isinstance(field, int):
        ptr = field
        st = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
        out = C.c_double()
        _check(lib().lbm_field_sum_noalloc(ptr, int(n), C.byref(out), st), "lbm_field_sum_noalloc")
        return out.value
    import torch
    if not field.is_cuda:
        raise ValueError("lbm_field_sum_noalloc: field must be a CUDA tensor")
    if field.dtype != torch.float32 or not field.is_contiguous():
        raise ValueError("lbm_field_sum_noalloc: field must be a contiguous float32 tensor")
    if not 0 <= int(n) <= field.numel():
        raise ValueError(f"lbm_field_sum_noalloc: n = {n} outside 0..{field.numel()} (the tensor's elements)")
    with torch.cuda.device(field.device):
        if stream is None:
            st = torch.cuda.current_stream(field.device).cuda_stream
        else:
            st = stream if isinstance(stream, int) else stream.cuda_stream
        out = C.c_double()
        _check(lib().lbm_field_sum_noalloc(_ptr(field), int(n), C.byref(out), st), "lbm_field_sum_noalloc")
    return out.value


def lbm_destroy(ctx):
    if ctx:
        lib().lbm_destroy(ctx)


def lbm_batch_create(common: LbmParams, dims):
    """dims: sequence of (nx, ny, nz) per instance."""
    flat = (C.c_int * (3 * len(dims)))(*[int(v) for d in dims for v in d])
    b = C.c_void_p()
    _check(lib().lbm_batch_create(C.byref(common), len(dims), flat, C.byref(b)), "lbm_batch_create")
    return b


def lbm_batch_nodes(b, instance: int = -1) -> int:
    return lib().lbm_batch_nodes(b, instance)


def lbm_batch_init_fields(b, rho, T, u=None):
    _check(lib().lbm_batch_init_fields(b, _ptr(rho), _ptr(T), _ptr(u)), "lbm_batch_init_fields")


def lbm_batch_step(b, n: int):
    _check(lib().lbm_batch_step(b, n), "lbm_batch_step")


def lbm_batch_autotune(b, steps: int) -> float:
    ms = C.c_double()
    _check(lib().lbm_batch_autotune(b, steps, C.byref(ms)), "lbm_batch_autotune")
    return ms.value


def lbm_batch_plan(b):
    v = [C.c_int() for _ in range(4)]
    _check(lib().lbm_batch_plan(b, *[C.byref(x) for x in v]), "lbm_batch_plan")
    return dict(tile_rows=v[0].value, z_split=v[1].value, items=v[2].value, ctas=v[3].value)


def lbm_batch_select_plan(b, tile_rows: int, z_split: int):
    """Select a work plan: tile rows 4 or 8, columns split into 1, 2 or 4 z-chunks; (0, 0) selects
    the TMA mode (one TMA-kernel launch per instance over 48 streams)."""
    _check(lib().lbm_batch_select_plan(b, tile_rows, z_split), "lbm_batch_select_plan")


def lbm_batch_get_moments(b, rho=None, ux=None, uy=None, uz=None, T=None):
    _check(lib().lbm_batch_get_moments(b, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(uz), _ptr(T)), "lbm_batch_get_moments")


def lbm_batch_get_totals(b, n_instances: int) -> np.ndarray:
    out = np.zeros(2 * n_instances, dtype=np.float64)
    _check(lib().lbm_batch_get_totals(b, out.ctypes.data_as(C.POINTER(C.c_double))), "lbm_batch_get_totals")
    return out.reshape(n_instances, 2)


def lbm_batch_steps_done(b) -> int:
    return lib().lbm_batch_steps_done(b)


def lbm_batch_launches_per_step(b) -> int:
    """Kernel launches one step of the current plan enqueues (1 for a persistent batched plan)."""
    n = lib().lbm_batch_launches_per_step(b)
    _check(n if n < 0 else 0, "lbm_batch_launches_per_step")
    return n


def lbm_batch_destroy(b):
    if b:
        lib().lbm_batch_destroy(b)


# ------------------------------------------------------------------- convenience
def params_from_setup(setup, **overrides) -> LbmParams:
    """Map a workloads.LatticeSetup onto lbm_params (temperatures scaled by this library's Tc)."""
    p = lbm_params_default()
    p.nx, p.ny, p.nz = setup.nx, setup.ny, setup.nz
    for k in range(6):
        p.bc[k] = int(setup.bc[k])
    p.a, p.b, p.R, p.acentric = setup.a, setup.b, setup.R, setup.acentric
    Tc, _ = lbm_eos_critical(p)
    for k in range(6):
        p.T_wall[k] = setup.T_wall_over_Tc[k] * Tc
    p.hot_dT = setup.hot_dT_over_Tc * Tc
    p.hot_sigma = setup.hot_sigma
    p.sigma = setup.sigma
    p.tau_e, p.tau_v, p.tau_q, p.tau_pi = setup.tau_e, setup.tau_v, setup.tau_q, setup.tau_pi
    p.cV, p.d, p.varsigma_q, p.varsigma_pi = setup.cV, setup.d, setup.varsigma_q, setup.varsigma_pi
    p.lambda_mode, p.chi_or_lambda = setup.lambda_mode, setup.chi_or_lambda
    for k in range(3):
        p.g[k] = setup.gravity[k]
    p.flow_off, p.thermal_off = setup.flow_off, setup.thermal_off
    p.rho_buoy = getattr(setup, "rho_buoy", 0.0)
    p.thermal_bgk = int(getattr(setup, "thermal_bgk", 0))
    p.divu_mode = int(getattr(setup, "divu_mode", 0))
    p.wall_rho = getattr(setup, "wall_rho", 0.0)
    p.wall_rho_patch = getattr(setup, "wall_rho_patch", 0.0)
    p.wall_patch_half = getattr(setup, "wall_patch_half", 0.0)
    p.wall_scheme = getattr(setup, "wall_scheme", 0)
    for k in ("wall_phi", "wall_drho", "wall_phi_patch", "wall_drho_patch"):
        setattr(p, k, getattr(setup, k, 0.0))
    p.thermal_q = int(getattr(setup, "thermal_q", 7))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Lattice:
    """One lattice on the current CUDA device; device memory comes from torch."""

    def __init__(self, params: LbmParams, stream=None):
        import torch
        self.params = params
        self.shape = (params.nz, params.ny, params.nx)
        self.N = params.nx * params.ny * params.nz
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        params.cuda_stream = self.stream.cuda_stream
        nbytes = lbm_workspace_bytes(params)
        if nbytes == 0:
            _check(LBM_EINVAL, "lbm_workspace_bytes")
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self._ws.data_ptr()
        params.workspace = (base + 255) & ~255
        params.workspace_bytes = nbytes
        self.ctx = lbm_create(params)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho, T, u=None):
        def f32(a):
            if a is None or not isinstance(a, np.ndarray):
                return a
            return np.ascontiguousarray(a, dtype=np.float32)
        lbm_init_fields(self.ctx, f32(rho), f32(T), f32(u))

    def step(self, n: int = 1):
        lbm_step(self.ctx, n)

    def moments(self):
        """Host copies of rho, ux, uy, uz, T (float32 numpy, shape (nz, ny, nx))."""
        out = {k: np.empty(self.shape, dtype=np.float32) for k in ("rho", "ux", "uy", "uz", "T")}
        lbm_get_moments(self.ctx, out["rho"], out["ux"], out["uy"], out["uz"], out["T"])
        return out

    def totals(self):
        return lbm_get_totals(self.ctx)

    @property
    def kernel(self):
        return lbm_kernel_in_use(self.ctx)

    @property
    def steps_done(self):
        return lbm_steps_done(self.ctx)

    def save_state(self) -> np.ndarray:
        return lbm_save_state(self.ctx)

    def load_state(self, buf: np.ndarray):
        lbm_load_state(self.ctx, buf)

    def set_wall_map(self, phi, drho):
        def f32(a):
            return np.ascontiguousarray(a, dtype=np.float32) if isinstance(a, np.ndarray) else a
        lbm_set_wall_map(self.ctx, f32(phi), f32(drho))

    @property
    def plan(self):
        """(shape, zchunk, items, ctas) of the TMA plan in use (shape -1: no TMA kernel)."""
        return lbm_get_plan(self.ctx)

    def select_plan(self, shape: int, zchunk: int = 0):
        lbm_select_plan(self.ctx, shape, zchunk)

    def plan_key(self) -> str:
        """Cache key of the plan choice: lattice size, storage, faces, wetting wall and the GPU."""
        import torch
        p = self.params
        wet = int(p.wall_scheme == 1 or p.wall_rho > 0)
        dev = torch.cuda.get_device_name(torch.cuda.current_device()).replace(" ", "_")
        return (f"{p.nx}x{p.ny}x{p.nz}/prec{p.precision}/bc{''.join(str(int(b)) for b in p.bc)}"
                f"/wet{wet}/{dev}")

    def autotune(self, steps: int = 10, cache: str = None) -> dict:
        """Pick the TMA plan by timing (lbm_autotune), or take it from the JSON file `cache` if that
        holds an entry for this lattice (plan_key).  A fresh measurement is written to `cache`.
        Returns {"shape", "zchunk", "ms_per_step" (None when taken from the cache), "cached"}."""
        import json
        key = self.plan_key()
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as fh:
                table = json.load(fh)
        hit = table.get(key)
        if hit is not None:
            self.select_plan(hit["shape"], hit["zchunk"])
            return dict(shape=hit["shape"], zchunk=hit["zchunk"], ms_per_step=None, cached=True)
        ms = lbm_autotune(self.ctx, steps)
        shape, zchunk, _, _ = self.plan
        if cache:
            table[key] = dict(shape=shape, zchunk=zchunk, ms_per_step=ms, steps=steps)
            d = os.path.dirname(os.path.abspath(cache))
            os.makedirs(d, exist_ok=True)
            tmp = cache + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(table, fh, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return dict(shape=shape, zchunk=zchunk, ms_per_step=ms, cached=False)


class Batch:
    """Batched ensemble of independent lattices (same model constants, uneven sizes)."""

    def __init__(self, common: LbmParams, dims, stream=None):
        import torch
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        common.cuda_stream = self.stream.cuda_stream
        common.workspace = None
        common.workspace_bytes = 0
        self.b = lbm_batch_create(common, self.dims)
        self.sizes = [lbm_batch_nodes(self.b, k) for k in range(len(self.dims))]
        self.N = lbm_batch_nodes(self.b, -1)

    def close(self):
        if getattr(self, "b", None):
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho, T, u=None):
        """rho, T: per-instance arrays (shape (nz, ny, nx)) or one concatenated float32 array."""
        def cat(a):
            if a is None or not isinstance(a, (list, tuple)):
                return a if a is None or not isinstance(a, np.ndarray) else np.ascontiguousarray(a, np.float32)
            return np.ascontiguousarray(np.concatenate([np.asarray(x, np.float32).ravel() for x in a]))
        lbm_batch_init_fields(self.b, cat(rho), cat(T), cat(u))

    def step(self, n: int = 1):
        lbm_batch_step(self.b, n)

    def autotune(self, steps: int = 3) -> float:
        return lbm_batch_autotune(self.b, steps)

    @property
    def plan(self):
        return lbm_batch_plan(self.b)

    def select_plan(self, tile_rows: int, z_split: int):
        lbm_batch_select_plan(self.b, tile_rows, z_split)

    def moments(self):
        """Per-instance dicts of host float32 arrays rho, ux, uy, uz, T (shape (nz, ny, nx))."""
        flat = {k: np.empty(self.N, dtype=np.float32) for k in ("rho", "ux", "uy", "uz", "T")}
        lbm_batch_get_moments(self.b, flat["rho"], flat["ux"], flat["uy"], flat["uz"], flat["T"])
        out, off = [], 0
        for (nx, ny, nz), n in zip(self.dims, self.sizes):
            out.append({k: v[off:off + n].reshape(nz, ny, nx) for k, v in flat.items()})
            off += n
        return out

    def totals(self):
        return lbm_batch_get_totals(self.b, len(self.dims))
