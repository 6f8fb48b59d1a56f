"""The temperature LB on the D3Q19 lattice (thermal_q 19: Eq. 19 BGK, Sec. III.B) on the GPU
against the FP64 oracle, through the C-ABI.

It runs on the generic fused and two-pass kernels (FP32 storage, 38 population slots a node);
the same bar as the D3Q7 parity tests: 1e-5 on short horizons, max(1e-5, 4 x the FP32 floor of
the case) on longer ones.  The two kernel variants must agree bit for bit.
"""
import numpy as np
import pytest

import workloads as W
from tests._parity import BAR, bars, fp32_floor, inputs, rel_errors, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

VARIANTS = {"two_pass": dict(kernel=1), "fused": dict(kernel=2, use_tma=0)}


def _q19(case):
    return dict(case, setup=W.LatticeSetup(**{**case["setup"].__dict__, "thermal_q": 19}))


def _compare(case, steps, fixed_bar=False):
    rho, T, u = inputs(case)
    s = case["setup"]
    orc = run_oracle(s, rho, T, u, steps)
    got = {}
    for name, ov in VARIANTS.items():
        got[name], _ = run_gpu(s, rho, T, u, steps, **ov)
    for k in got["fused"]:
        assert np.array_equal(got["fused"][k], got["two_pass"][k]), k
    err = rel_errors(got["fused"], orc)
    bar = {k: BAR for k in err} if fixed_bar else bars(fp32_floor(s, rho, T, u, steps, ref=orc))
    print(case.get("name", ""), "D3Q19 thermal, steps", steps, "gpu", err, "bar", bar)
    for k, v in err.items():
        assert v <= bar[k], (k, v, bar[k])


def test_d3q19_thermal_short_horizon_fixed_bar():
    _compare(_q19(W.static_droplet(24)), 10, fixed_bar=True)
    _compare(_q19(W.pool_boiling(40, 36, 48, height=16.0, hot_sigma=4.0)), 10, fixed_bar=True)


def test_d3q19_thermal_evaporating_droplet_thermal_faces():
    _compare(_q19(W.evaporation(24, R0=7.0)), 300)


def test_d3q19_thermal_pool_walls_outflow_hot_spot():
    s = W.LatticeSetup(37, 11, 19, bc=(W.BC_WALL, W.BC_WALL, 0, 0, W.BC_WALL, W.BC_OUTFLOW),
                       T_wall_over_Tc=(0.86, 0.88, 0.86, 0.86, 0.86, 0.86), hot_dT_over_Tc=0.10,
                       hot_sigma=3.0, sigma=W.SIGMA_STAR, gravity=(0, 0, -3e-5), thermal_q=19)
    _compare(dict(name="ragged pool", setup=s, kind="pool", height=8.0, W=4.0, Tr_liquid=0.86), 300)


def test_d3q19_thermal_conduction_in_a_static_fluid():
    s = W.LatticeSetup(20, 18, 9, sigma=W.SIGMA_STAR, flow_off=1, thermal_q=19,
                       bc=(0, 0, 0, 0, W.BC_THERMAL_ONLY, W.BC_THERMAL_ONLY),
                       T_wall_over_Tc=(0.86, 0.86, 0.86, 0.86, 0.92, 0.84))
    _compare(dict(name="conduction", setup=s, kind="droplet", R0=5.0, W=4.0, Tr_drop=0.86, Tr_gas=0.86), 200)


def test_d3q19_thermal_rejected_where_unsupported():
    from paper_2201_06039_gb300 import lbm
    s = W.LatticeSetup(16, 16, 16, sigma=W.SIGMA_STAR, thermal_q=19)
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(lbm.params_from_setup(s, precision=lbm.LBM_BF16_SHIFTED))
    with pytest.raises(lbm.LbmError):
        lbm.Batch(lbm.params_from_setup(s), [(16, 16, 16)])
    lat = lbm.Lattice(lbm.params_from_setup(s))          # runs, on the generic fused kernel
    assert lat.kernel == lbm.LBM_KERNEL_FUSED
    lat.close()


def _d2_series(setup, rho, T, mid, every=500, n=16):
    from paper_2201_06039_gb300 import lbm
    lat = lbm.Lattice(lbm.params_from_setup(setup))
    lat.init(rho.astype(np.float32), T.astype(np.float32))
    d2 = []
    for _ in range(n):
        lat.step(every)
        r = lat.moments()["rho"]
        d2.append((6.0 * float((r > mid).sum()) / np.pi) ** (2.0 / 3.0))
    lat.close()
    t = every * (np.arange(n) + 1.0)
    y = np.array(d2) / d2[0]
    A = np.vstack([t[6:], np.ones(n - 6)]).T
    coef, res, _, _ = np.linalg.lstsq(A, y[6:], rcond=None)
    r2 = 1.0 - float(res[0]) / float(((y[6:] - y[6:].mean()) ** 2).sum())
    return coef[0], r2, y


def test_d3q19_and_d3q7_evaporation_follow_the_same_d2_law():
    """Sec. III.B / Sec. V: the D3Q7 lattice is enough for the temperature field.  The evaporating
    droplet of Sec. IV.A (64^3, diameter 32 at 0.86 Tc, faces at 0.95 Tc) on both lattices: each
    follows the D^2 law (R^2 >= 0.98 after the start-up transient) and the two slopes agree."""
    import oracle
    case = W.evaporation(64, R0=16.0)
    rho, T, u = inputs(case)
    s7 = case["setup"]
    Tc = oracle.Tc_of(s7)
    rl, rv, _ = oracle.maxwell(s7, 0.86 * Tc)
    mid = 0.5 * (rl + rv)
    k7, r7, y7 = _d2_series(s7, rho, T, mid)
    k19, r19, y19 = _d2_series(W.LatticeSetup(**{**s7.__dict__, "thermal_q": 19}), rho, T, mid)
    print("D3Q7  slope", k7, "R2", r7, "(D/D0)^2", np.round(y7, 4).tolist())
    print("D3Q19 slope", k19, "R2", r19, "(D/D0)^2", np.round(y19, 4).tolist())
    assert k7 < 0 and k19 < 0
    assert r7 >= 0.98 and r19 >= 0.98, (r7, r19)
    assert abs(k19 / k7 - 1) < 0.05, (k7, k19)
