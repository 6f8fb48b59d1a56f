"""Shifted 16-bit population storage (BF16, FP16) with FP32 collision arithmetic, against the
FP64 oracle on the 64 x 64 x 96 downscaled pool-boiling case.

The state is stored as (f_a - w_a rho_ref) and (g_a - w_a T_ref) in 16 bits, with rho_ref the
initial mean density and T_ref the liquid saturation temperature 0.86 Tc; every step decodes,
collides in FP32 and re-encodes (round to nearest even).  The errors are reported per field
(rho, T, u as in tests/_parity.py, plus the liquid-vapour interface height on the centre line)
beside those of FP32 storage on the same inputs.  16-bit storage cannot meet the FP32 parity bar;
the bars below are the error budgets stated for each format.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests._parity import inputs, rel_errors, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

STEPS = 300
PREC = {"bf16": 1, "fp16": 2}
# error budgets per field after STEPS steps (relative max-norm; interface height in lattice units).
# FP32 storage sits at the FP32 rounding floor.  16-bit storage keeps ~3 (BF16) or ~4 (FP16)
# significant digits of each shifted population; rho and the interface follow to that order,
# while u (spurious currents of order 1e-3 and below) is not resolved by 16-bit storage at all.
BUDGET = {
    "fp32": dict(rho=1e-4, T=1e-5, u=1e-2, interface=0.01),
    "fp16": dict(rho=1e-2, T=3e-2, u=2.0, interface=0.1),
    "bf16": dict(rho=5e-2, T=1e-1, u=5.0, interface=1.0),
}


def interface_height(rho, rho_mid):
    """Height of the liquid-vapour interface on the vertical centre line: first downward-to-up
    crossing of rho_mid, linearly interpolated between nodes."""
    nz, ny, nx = rho.shape
    line = rho[:, ny // 2, nx // 2].astype(np.float64)
    for z in range(nz - 1):
        if line[z] >= rho_mid > line[z + 1]:
            return z + (line[z] - rho_mid) / (line[z] - line[z + 1])
    return float("nan")


@pytest.fixture(scope="module")
def downscaled():
    case = W.pool_boiling_downscaled()
    s = case["setup"]
    rho, T, u = inputs(case)
    ref = run_oracle(s, rho, T, u, STEPS)
    Tc = oracle.Tc_of(s)
    rl, rv, _ = oracle.maxwell(s, 0.86 * Tc)
    return dict(case=case, rho=rho, T=T, u=u, ref=ref, Tc=Tc, mid=0.5 * (rl + rv))


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_shifted_storage_field_errors_vs_fp64_oracle(downscaled, storage):
    d = downscaled
    s = d["case"]["setup"]
    over = {}
    if storage != "fp32":
        over = dict(precision=PREC[storage], rho_ref=float(np.mean(d["rho"])), T_ref=0.86 * d["Tc"])
    gpu, tot = run_gpu(s, d["rho"], d["T"], d["u"], STEPS, **over)
    err = rel_errors(gpu, d["ref"])
    zi_ref = interface_height(d["ref"]["rho"], d["mid"])
    zi = interface_height(gpu["rho"], d["mid"])
    err["interface"] = abs(zi - zi_ref)
    print(f"storage {storage} steps {STEPS} errors {err} interface_ref {zi_ref:.4f} mass {tot[0]:.9e}")
    for k, v in err.items():
        assert np.isfinite(v) and v <= BUDGET[storage][k], (storage, k, v, err)



@pytest.mark.parametrize("storage", ["bf16", "fp16"])
@pytest.mark.parametrize("dims", [(72, 40, 30), (41, 15, 20), (200, 22, 9)])
def test_16bit_tma_kernel_bit_identical_to_generic(storage, dims):
    """The TMA kernel with shifted 16-bit stages, output tiles and ghost stores (in-kernel ghosts
    for nx % 8 == 0, the refresh kernel otherwise) computes exactly what the generic fused and
    the two-pass kernels compute on the same 16-bit storage."""
    from paper_2201_06039_gb300 import lbm
    from tests._parity import run_gpu
    nx, ny, nz = dims
    case = W.pool_boiling(nx, ny, nz, height=nz / 2.5, hot_sigma=3.0)
    rho, T, u = inputs(case)
    s = case["setup"]
    Tc = oracle.Tc_of(s)
    over = dict(precision=PREC[storage], rho_ref=float(np.mean(rho)), T_ref=0.86 * Tc)
    lat = lbm.Lattice(lbm.params_from_setup(s, kernel=2, use_tma=1, **over))
    assert lat.kernel == lbm.LBM_KERNEL_FUSED_TMA
    lat.close()
    tma, _ = run_gpu(s, rho, T, u, 11, kernel=2, use_tma=1, **over)
    gen, _ = run_gpu(s, rho, T, u, 11, kernel=2, use_tma=0, **over)
    two, _ = run_gpu(s, rho, T, u, 11, kernel=1, **over)
    for k in tma:
        assert np.array_equal(tma[k], gen[k]), (storage, dims, k)
        assert np.array_equal(tma[k], two[k]), (storage, dims, k)


STEPS_LONG = 2000
# budgets after STEPS_LONG steps, about twice the errors measured on a GB300 (FP32: rho 4.1e-6,
# T 8.0e-7, u 2.6e-4 of the flow's 1.7e-3 scale; FP16: 0.030, 0.019, 1.7; BF16: 0.027, 0.099,
# 4.9).  Each step re-rounds every shifted population, so the 16-bit errors grow with the step
# count, and 16-bit storage does not conserve mass exactly; u is also bounded in lattice units,
# where BF16 / FP16 resolve it only to a few 1e-3 (the population quantum, 2^-9 / 2^-11 of the
# largest shifted population, over rho): above the spurious currents of this case.
BUDGET_LONG = {
    "fp32": dict(rho=2e-5, T=4e-6, u=1e-3, u_abs=2e-6, interface=1e-3, mass=1e-5),
    "fp16": dict(rho=6e-2, T=4e-2, u=3.5, u_abs=6e-3, interface=0.15, mass=3e-3),
    "bf16": dict(rho=6e-2, T=0.2, u=10.0, u_abs=1.7e-2, interface=0.1, mass=2e-3),
}


def bubble_nodes(rho, rho_mid, z_interface):
    """Vapour nodes (rho < rho_mid) below the interface height, away from the heater's first
    two layers: a nucleated bubble."""
    zi = int(np.floor(z_interface)) if np.isfinite(z_interface) else rho.shape[0]
    return int((rho[2:max(2, zi - 2)] < rho_mid).sum())


@pytest.fixture(scope="module")
def downscaled_long():
    case = W.pool_boiling_downscaled()
    s = case["setup"]
    rho, T, u = inputs(case)
    ref = run_oracle(s, rho, T, u, STEPS_LONG)
    Tc = oracle.Tc_of(s)
    rl, rv, _ = oracle.maxwell(s, 0.86 * Tc)
    return dict(case=case, rho=rho, T=T, u=u, ref=ref, Tc=Tc, mid=0.5 * (rl + rv))


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_shifted_storage_long_horizon_vs_fp64_oracle(downscaled_long, storage):
    """Config-4 error study at a long horizon: per-field error of each storage format against the
    FP64 oracle after 2000 steps of the 64 x 64 x 96 downscaled pool (rho, T, u relative, u in
    lattice units, interface height, mass drift), and the bubble-departure step, which this copy does not
    have: no bubble nucleates in the oracle within the horizon, and none may appear in the GPU
    run (16-bit noise must not nucleate one)."""
    d = downscaled_long
    s = d["case"]["setup"]
    over = {}
    if storage != "fp32":
        over = dict(precision=PREC[storage], rho_ref=float(np.mean(d["rho"])), T_ref=0.86 * d["Tc"])
    gpu, tot = run_gpu(s, d["rho"], d["T"], d["u"], STEPS_LONG, **over)
    err = rel_errors(gpu, d["ref"])
    err["u_abs"] = max(float(np.max(np.abs(gpu[k].astype(np.float64) - d["ref"][k]))) for k in ("ux", "uy", "uz"))
    u_scale = max(float(np.max(np.abs(d["ref"][k]))) for k in ("ux", "uy", "uz"))
    zi_ref = interface_height(d["ref"]["rho"], d["mid"])
    zi = interface_height(gpu["rho"], d["mid"])
    err["interface"] = abs(zi - zi_ref)
    m_ref = float(np.sum(d["ref"]["rho"]))   # the top face is an outflow: compare with the oracle's mass
    err["mass"] = abs(tot[0] - m_ref) / m_ref
    b_ref = bubble_nodes(d["ref"]["rho"], d["mid"], zi_ref)
    b_gpu = bubble_nodes(gpu["rho"], d["mid"], zi)
    print(f"storage {storage} steps {STEPS_LONG} errors {err} u_scale {u_scale:.3e} interface_ref {zi_ref:.4f} "
          f"bubble nodes oracle {b_ref} gpu {b_gpu} mass {tot[0]:.9e}")
    assert b_ref == 0 and b_gpu == 0, (b_ref, b_gpu)
    for k, v in err.items():
        assert np.isfinite(v) and v <= BUDGET_LONG[storage][k], (storage, k, v, err)
