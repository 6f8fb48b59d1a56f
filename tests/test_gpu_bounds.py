"""The bounds-checked build of the library (libgb300lbm_bounds.so, -DLBM_BOUNDS_CHECK) on small
lattices, through the C-ABI with host buffers.

In that build every population, field and shared-memory index of the update is checked before
use; an index outside its buffer is recorded (and the access skipped, so nothing faults) and
lbm_step returns LBM_EBOUNDS.  This is the stand-in for a memory checker: on 4^3 and 8^3 lattices
(periodic, walled and open faces; the generic, two-pass and TMA kernels) no index may fall
outside its buffer, the result must match the FP64 oracle (within the parity bar of the other
multi-step tests), and the checks must not change a bit of the result of the release build.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from tests._parity import bars, fp32_floor, rel_errors, run_oracle

pytestmark = pytest.mark.gpu

STEPS = 20


def _bounds_lib():
    from paper_2201_06039_gb300 import build as B
    from paper_2201_06039_gb300 import lbm
    B.build(variants=("bounds",))
    L = C.CDLL(B.BOUNDS_LIB)
    vp = C.c_void_p
    P = C.POINTER(lbm.LbmParams)
    L.lbm_create.argtypes = [P, C.POINTER(vp)]
    L.lbm_init_fields.argtypes = [vp, vp, vp, vp]
    L.lbm_step.argtypes = [vp, C.c_int]
    L.lbm_get_moments.argtypes = [vp, vp, vp, vp, vp, vp]
    L.lbm_kernel_in_use.argtypes = [vp]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_last_error.restype = C.c_char_p
    return L


def _run(L, params, rho, T, steps):
    ctx = C.c_void_p()
    rc = L.lbm_create(C.byref(params), C.byref(ctx))
    assert rc == 0, L.lbm_last_error()
    r = np.ascontiguousarray(rho, dtype=np.float32)
    t = np.ascontiguousarray(T, dtype=np.float32)
    assert L.lbm_init_fields(ctx, r.ctypes.data, t.ctypes.data, None) == 0, L.lbm_last_error()
    for _ in range(steps):                      # one step a call: every step's flag is checked
        rc = L.lbm_step(ctx, 1)
        assert rc == 0, (rc, L.lbm_last_error())
    out = {k: np.empty(r.shape, dtype=np.float32) for k in ("rho", "ux", "uy", "uz", "T")}
    assert L.lbm_get_moments(ctx, *[out[k].ctypes.data for k in ("rho", "ux", "uy", "uz", "T")]) == 0
    kernel = L.lbm_kernel_in_use(ctx)
    L.lbm_destroy(ctx)
    return out, kernel


CASES = {
    "periodic_4": lambda: (W.LatticeSetup(4, 4, 4, sigma=W.SIGMA_STAR, gravity=(0, 0, -3e-5)), 4),
    "periodic_8": lambda: (W.LatticeSetup(8, 8, 8, sigma=W.SIGMA_STAR), 8),
    "walls_8": lambda: (W.LatticeSetup(8, 8, 8, sigma=W.SIGMA_STAR, gravity=(0, 0, -3e-5),
                                       bc=(0, 0, 0, 0, W.BC_WALL, W.BC_OUTFLOW), hot_dT_over_Tc=0.1,
                                       hot_sigma=2.0), 8),
    "box_walls_8": lambda: (W.LatticeSetup(8, 8, 8, sigma=W.SIGMA_STAR,
                                           bc=(W.BC_WALL, W.BC_WALL, W.BC_THERMAL_ONLY, W.BC_THERMAL_ONLY,
                                               W.BC_WALL, W.BC_WALL)), 8),
}


@pytest.mark.parametrize("variant", [dict(kernel=1), dict(kernel=2, use_tma=0), dict(kernel=2, use_tma=1)],
                         ids=["two_pass", "fused", "fused_tma"])
@pytest.mark.parametrize("case", list(CASES))
def test_bounds_checked_build_small_lattices(case, variant):
    from paper_2201_06039_gb300 import lbm
    L = _bounds_lib()
    s, n = CASES[case]()
    rho, T = W.random_state(s.shape, 4242 + n, rho_lo=0.36, rho_hi=0.44, T_lo=0.060, T_hi=0.064)
    rho = rho.astype(np.float32).astype(np.float64)
    T = T.astype(np.float32).astype(np.float64)
    p = lbm.params_from_setup(s, use_graph=0, check_nonfinite=1, **variant)
    got, kernel = _run(L, p, rho, T, STEPS)
    # the release build computes the same bits
    ref_lat = lbm.Lattice(lbm.params_from_setup(s, use_graph=0, check_nonfinite=1, **variant))
    ref_lat.init(rho.astype(np.float32), T.astype(np.float32))
    ref_lat.step(STEPS)
    rel = ref_lat.moments()
    assert ref_lat.kernel == kernel
    ref_lat.close()
    for k in rel:
        assert np.array_equal(got[k], rel[k]), k
    orc = run_oracle(s, rho, T, None, STEPS)
    err = rel_errors(got, orc)
    bar = bars(fp32_floor(s, rho, T, None, STEPS, ref=orc))   # the velocities here are ~1e-6
    assert all(err[k] <= bar[k] for k in err), (err, bar)
