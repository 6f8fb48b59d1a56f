"""Calibrate the thermodynamic-consistency constant sigma of Eq. 9 with the FP64 oracle.

The paper uses sigma (Eq. 9) to bring the pseudopotential model's coexistence densities
onto the Maxwell construction of the equation of state, but does not print its value.
This script runs the oracle (and nothing else) on a quasi-1D periodic flat interface
(1 x 1 x 128, liquid slab of half-thickness 32, isothermal at 0.86 Tc, a = 2/49, b = 2/21,
R = 1, acentric factor 0.344, tau_e = 1.25, tau_v = 0.8, other rates 1) until steady
state, for sigma on a grid, and picks the sigma* that minimises
max(|rho_l/rho_l^Maxwell - 1|, |rho_v/rho_v^Maxwell - 1|).

Output: tests/golden/sigma_calibration.json (sigma*, the sweep, Maxwell densities).
Run:    python -m oracle.calibrate_sigma           (a = 2/49)
        python -m oracle.calibrate_sigma a1_49     (a = 1/49, the paper's droplet tests; output
                                                    tests/golden/sigma_calibration_a1_49.json)
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

import oracle
import workloads as W

GRID = [round(0.09 + 0.0025 * k, 4) for k in range(17)]   # 0.0900 .. 0.1300
STEPS = 30000
GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")
VARIANTS = {"a2_49": (2.0 / 49.0, "sigma_calibration.json"), "a1_49": (1.0 / 49.0, "sigma_calibration_a1_49.json")}


def flat_interface(sigma: float, steps: int = STEPS, Tr: float = 0.86, a: float = 2.0 / 49.0):
    s = W.LatticeSetup(1, 1, 128, sigma=sigma, thermal_off=1, a=a)
    Tc = oracle.Tc_of(s)
    rl, rv, ps = oracle.maxwell(s, Tr * Tc)
    rho = W.slab(s.shape, 32.0, 2.0, rl, rv, axis=2)
    T = np.full(s.shape, Tr * Tc)
    o = oracle.Oracle(s)
    o.init(rho, T)
    o.step(steps)
    r = o.moments()["rho"].reshape(-1)
    return dict(sigma=sigma, rho_l=float(r[64]), rho_v=float(r[0]),
                err_l=float(r[64] / rl - 1.0), err_v=float(r[0] / rv - 1.0),
                maxwell_l=rl, maxwell_v=rv, p_sat=ps)


def main():
    variant = sys.argv[1] if len(sys.argv) > 1 else "a2_49"
    a, name = VARIANTS[variant]
    out_path = os.path.join(GOLDEN, name)
    rows = []
    for sg in GRID:
        try:
            r = flat_interface(sg, a=a)
        except FloatingPointError:
            r = dict(sigma=sg, unstable=True)
        rows.append(r)
        print(r, flush=True)
    ok = [r for r in rows if not r.get("unstable")]
    best = min(ok, key=lambda r: max(abs(r["err_l"]), abs(r["err_v"])))
    out = dict(
        what=f"sigma* of Eq. 9 from a flat interface (1x1x128, 0.86 Tc, a={'2' if variant == 'a2_49' else '1'}/49) "
             "run by the FP64 oracle",
        script="oracle/calibrate_sigma.py", a=a, steps=STEPS, sigma_star=best["sigma"],
        maxwell=dict(rho_l=best["maxwell_l"], rho_v=best["maxwell_v"], p_sat=best["p_sat"]),
        best=best, sweep=rows)
    with open(out_path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("sigma* =", best["sigma"], "->", out_path)
    return 0


if __name__ == "__main__":
    sys.exit(main())
