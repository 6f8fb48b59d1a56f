"""Shared helpers of the GPU-vs-oracle parity tests.

Error measure (per field, element by element over the whole lattice):
    rho, T : max |x_gpu - x_oracle| / max |x_oracle|
    u      : max_k max |u_k,gpu - u_k,oracle| / max_k max |u_k,oracle|   (vector velocity scale)

Bar: the fixed 1e-5 on short horizons; on long horizons max(1e-5, FLOOR_FACTOR x floor), where
floor is the same error measure between the FP32 build of the oracle (same source, every
per-node operation and the state in float) and the FP64 oracle on the same inputs and step
count: the rounding floor of FP32 arithmetic on that case.  The GPU computes in FP32, so it
cannot be held to a bar below that floor.
"""
import numpy as np

import oracle
import workloads as W

BAR = 1e-5
FLOOR_FACTOR = 4.0


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


def run_oracle(setup, rho, T, u, steps, precision="f64"):
    o = oracle.Oracle(setup, precision=precision)
    o.init(rho, T, u)
    if steps:
        o.step(steps)
    m = o.moments()
    o.close()
    return m


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


def rel_errors(test, ref):
    out = {}
    for k in ("rho", "T"):
        den = float(np.max(np.abs(ref[k])))
        out[k] = float(np.max(np.abs(test[k].astype(np.float64) - ref[k]))) / den
    uk = ("ux", "uy", "uz")
    den = max(float(np.max(np.abs(ref[k]))) for k in uk)
    num = max(float(np.max(np.abs(test[k].astype(np.float64) - ref[k]))) for k in uk)
    out["u"] = num / den if den > 0 else num
    return out


def fp32_floor(setup, rho, T, u, steps, ref=None):
    """Error of the FP32 build of the oracle against the FP64 oracle (same inputs, same steps)."""
    ref = ref if ref is not None else run_oracle(setup, rho, T, u, steps)
    o32 = run_oracle(setup, rho, T, u, steps, precision="f32")
    return rel_errors(o32, ref)


def bars(floor):
    return {k: max(BAR, FLOOR_FACTOR * v) for k, v in floor.items()}
