"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every symbol that
include/lbm.h declares, and validates parameters on the host (no GPU calls)."""
import ctypes as C
import os
import re
import subprocess

import pytest

import paper_2201_06039_gb300 as G
from paper_2201_06039_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = lbm.lib()
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    assert sorted(lbm.EXPORTS) == names
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.lib_path()], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    assert set(names) <= exported


def test_library_is_built_for_sm103a_only():
    from paper_2201_06039_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert build.up_to_date()


def test_params_default_matches_paper_constants():
    p = G.lbm_params_default()
    assert (p.tau_e, p.tau_v, p.tau_q, p.tau_pi) == (1.25, 0.8, 1.0, 1.0)
    assert (p.cV, p.d, p.varsigma_q, p.varsigma_pi) == (5.0, 0.95, 1.0, 1.0)
    assert abs(p.a - 2 / 49) < 1e-15 and abs(p.b - 2 / 21) < 1e-15 and p.acentric == 0.344
    Tc, pc = G.lbm_eos_critical(p)
    assert abs(Tc - 0.0778 * p.a / (0.45724 * p.b * p.R)) < 1e-15
    assert abs(pc - 0.0778 * p.R * Tc / p.b) < 1e-15


def test_workspace_bytes_counts_state():
    p = G.lbm_params_default()
    p.nx, p.ny, p.nz = 32, 16, 8
    N = 32 * 16 * 8
    nb = G.lbm_workspace_bytes(p)
    assert nb >= N * (2 * 26 * 4 + 8 + 4)
    p.precision = G.LBM_BF16_SHIFTED
    assert G.lbm_workspace_bytes(p) < nb


@pytest.mark.parametrize("field,value", [("nx", 0), ("tau_v", 0.5), ("d", 1.5), ("precision", 7),
                                         ("kernel", 9), ("chi_or_lambda", -1.0), ("divu_mode", 2)])
def test_invalid_params_rejected_on_host(field, value):
    p = G.lbm_params_default()
    p.nx = p.ny = p.nz = 8
    setattr(p, field, value)
    with pytest.raises(G.LbmError) as ei:
        G.lbm_create(p)
    assert ei.value.status == G.LBM_EINVAL
    assert G.lbm_workspace_bytes(p) == 0


def test_finite_difference_divu_needs_the_two_pass_kernels():
    p = G.lbm_params_default()
    p.nx = p.ny = p.nz = 8
    p.divu_mode = 1
    p.kernel = G.LBM_KERNEL_FUSED
    with pytest.raises(G.LbmError) as ei:
        G.lbm_create(p)
    assert ei.value.status == G.LBM_EINVAL and "two-pass" in str(ei.value)
    q = G.lbm_params_default()
    q.divu_mode = 1
    with pytest.raises(G.LbmError) as ei:
        G.lbm_batch_create(q, [(8, 8, 8)])
    assert ei.value.status == G.LBM_EINVAL


@pytest.mark.parametrize("bottom,rho_w,rho_p,radius", [(0, 0.5, 0.0, 0.0), (1, -0.1, 0.0, 0.0),
                                                       (1, 0.5, 0.0, 3.0), (1, 0.0, 0.3, 3.0),
                                                       (1, 0.5, 0.3, -1.0)])
def test_wetting_wall_parameters_checked(bottom, rho_w, rho_p, radius):
    """A virtual wall density needs a -z wall; a patch needs both densities positive."""
    p = G.lbm_params_default()
    p.nx = p.ny = p.nz = 8
    if bottom:
        p.bc[4] = p.bc[5] = G.LBM_BC_WALL
    p.wall_rho, p.wall_rho_patch, p.wall_patch_half = rho_w, rho_p, radius
    with pytest.raises(G.LbmError) as ei:
        G.lbm_create(p)
    assert ei.value.status == G.LBM_EINVAL


@pytest.mark.parametrize("kw", [dict(wall_scheme=2), dict(wall_scheme=1, wall_phi=0.0),
                                dict(wall_scheme=1, wall_phi=1.1, wall_drho=-0.5),
                                dict(wall_scheme=1, wall_phi=1.1, wall_rho=2.0),
                                dict(wall_scheme=1, wall_phi=1.1, wall_patch_half=3.0),
                                dict(wall_scheme=1, wall_phi=1.1, wall_patch_half=3.0, wall_phi_patch=1.0,
                                     wall_drho_patch=-1.0),
                                dict(wall_scheme=1, wall_phi=1.1, bottom=0)])
def test_wetting_scheme1_parameters_checked(kw):
    """Scheme 1 needs a -z wall, phi > 0, drho >= 0 (per region) and no fixed densities."""
    kw = dict(kw)
    p = G.lbm_params_default()
    p.nx = p.ny = p.nz = 8
    if kw.pop("bottom", 1):
        p.bc[4] = p.bc[5] = G.LBM_BC_WALL
    for k, v in kw.items():
        setattr(p, k, v)
    with pytest.raises(G.LbmError) as ei:
        G.lbm_create(p)
    assert ei.value.status == G.LBM_EINVAL


def test_setup_fields_reach_both_parameter_structs():
    """Every wetting and option field of a LatticeSetup arrives unchanged in lbm_params and in the
    oracle's parameter struct (the two sides map the record independently)."""
    import oracle
    import workloads as W
    kw = dict(wall_rho=0.0, wall_scheme=1, wall_phi=1.23, wall_drho=0.045, wall_phi_patch=1.01,
              wall_drho_patch=0.287, wall_patch_half=27.5, thermal_bgk=1, divu_mode=1)
    s = W.LatticeSetup(20, 18, 16, bc=(0, 0, 0, 0, 1, 2), **kw)
    p = G.params_from_setup(s)
    q = oracle.params_from_setup(s)
    for k, v in kw.items():
        assert getattr(p, k) == v and getattr(q, k) == v, k
    assert list(p.bc) == list(s.bc) and list(q.bc) == list(s.bc)


def test_set_wall_map_needs_a_context():
    lib = G.lib()
    assert lib.lbm_set_wall_map(None, None, None) == G.LBM_EINVAL


def test_batch_has_no_wetting_wall():
    q = G.lbm_params_default()
    q.bc[4] = q.bc[5] = G.LBM_BC_WALL
    q.wall_rho = 2.5
    with pytest.raises(G.LbmError) as ei:
        G.lbm_batch_create(q, [(8, 8, 8)])
    assert ei.value.status == G.LBM_EINVAL and "wetting" in str(ei.value)


def test_one_sided_periodic_axis_rejected():
    p = G.lbm_params_default()
    p.nx = p.ny = p.nz = 8
    p.bc[4] = G.LBM_BC_WALL
    with pytest.raises(G.LbmError) as ei:
        G.lbm_create(p)
    assert ei.value.status == G.LBM_EINVAL


def test_status_strings():
    L = lbm.lib()
    assert L.lbm_status_str(G.LBM_ENONFINITE).decode().startswith("non-finite")
    assert L.lbm_status_str(12345).decode() == "unknown status"


def test_thermo_coexistence_agrees_with_paper():
    Tc = G.thermo.critical_temperature(2 / 49, 2 / 21, 1.0)
    rl, rv, _ = G.thermo.coexistence(0.86 * Tc)
    assert abs(rl - 6.5) < 0.05 and abs(rv - 0.38) < 0.005


def test_batch_create_rejects_bad_instances_on_host():
    import ctypes as C
    p = G.lbm_params_default()
    L = G.lib()
    out = C.c_void_p()
    dims = (C.c_int * 6)(24, 24, 24, 0, 5, 5)
    assert L.lbm_batch_create(C.byref(p), 2, dims, C.byref(out)) == G.LBM_EINVAL
    assert b"instance 1" in L.lbm_last_error()
    assert L.lbm_batch_create(C.byref(p), 0, dims, C.byref(out)) == G.LBM_EINVAL
    assert L.lbm_batch_create(C.byref(p), 1, None, C.byref(out)) == G.LBM_EINVAL
    assert not out.value
