"""Shared helpers of the GPU-vs-oracle parity tests: build identical seeded inputs for
both sides and compare the macroscopic fields."""
import numpy as np

import oracle
import workloads as W


def inputs(case, f32=True):
    """(rho, T, u) of a workload case with coexistence densities from the oracle's EOS,
    rounded to float32 so that both sides start from the same values."""
    s = case["setup"]
    Tc = oracle.Tc_of(s)
    Tr = case.get("Tr_drop", case.get("Tr_liquid", 0.86))
    rl, rv, _ = oracle.maxwell(s, Tr * Tc)
    rho, T, u = W.build_fields(case, Tc, rl, rv)
    if f32:
        rho = rho.astype(np.float32).astype(np.float64)
        T = T.astype(np.float32).astype(np.float64)
    return rho, T, u


def run_oracle(setup, rho, T, u, steps):
    o = oracle.Oracle(setup)
    o.init(rho, T, u)
    if steps:
        o.step(steps)
    return o.moments()


def run_gpu(setup, rho, T, u, steps, **overrides):
    from paper_2201_06039_gb300 import lbm
    p = lbm.params_from_setup(setup, **overrides)
    lat = lbm.Lattice(p)
    lat.init(rho.astype(np.float32), T.astype(np.float32),
             None if u is None else np.ascontiguousarray(u, dtype=np.float32))
    if steps:
        lat.step(steps)
    m = lat.moments()
    tot = lat.totals()
    lat.close()
    return m, tot


def rel_errors(gpu, orc):
    """max |x_gpu - x_oracle| / max |x_oracle| per field."""
    out = {}
    for k in ("rho", "ux", "uy", "uz", "T"):
        den = float(np.max(np.abs(orc[k])))
        num = float(np.max(np.abs(gpu[k].astype(np.float64) - orc[k])))
        out[k] = num / den if den > 0 else num
    return out
