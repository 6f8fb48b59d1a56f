"""Wetting studies on the GPU behind the tables of the design notes (not collected by pytest):

  python -m tests.study_wetting angles p1.0,p1.4,d0.284,f0.35   contact angles (scheme 1: pPHI or
                                                                dDRHO; scheme 0: fFRACTION of the way
                                                                from rho_v to rho_l)
  python -m tests.study_wetting nucleation                      bubble growth and departure, Sec. IV.C
  python -m tests.study_wetting departure 3e-5,1.5e-5           departure diameter against gravity
  python -m tests.study_wetting heated pinned|free              heated-surface droplet, Sec. IV.B

Each prints one line per measurement.  The GPU tests in test_gpu_wetting.py check a subset.
"""
import math
import sys
import time

import numpy as np

import oracle
import workloads as W
from tests.test_gpu_wetting import _cap_angle, _segments


def angles(specs):
    from paper_2201_06039_gb300 import lbm
    n, nz = 120, 70
    for spec in specs.split(","):
        kind, val = spec[0], float(spec[1:])
        base = W.LatticeSetup(n, n, nz, bc=(0, 0, 0, 0, 1, 1), sigma=W.SIGMA_STAR, thermal_off=1,
                              T_wall_over_Tc=(0.86,) * 6)
        Tc = oracle.Tc_of(base)
        rl, rv, _ = oracle.maxwell(base, 0.86 * Tc)
        if kind == "f":
            kw = {"wall_rho": rv + val * (rl - rv)}
        else:
            kw = {"wall_scheme": 1, "wall_phi": val if kind == "p" else 1.0, "wall_drho": val if kind == "d" else 0.0}
        s = W.LatticeSetup(**{**base.__dict__, **kw})
        rho = W.droplet((nz, n, n), 30.0, 4.0, rl, rv, periodic=(True, True, False), center=(n / 2, n / 2, -0.5))
        lat = lbm.Lattice(lbm.params_from_setup(s))
        lat.init(rho.astype(np.float32), np.full(rho.shape, 0.86 * Tc, np.float32))
        lat.step(20000)
        r = lat.moments()["rho"].astype(np.float64)
        lat.close()
        print(f"{spec}: contact angle {_cap_angle(r, 0.5 * (rl + rv)):.1f} degrees", flush=True)


def _nucleate(g):
    from paper_2201_06039_gb300 import lbm
    case = W.nucleate_boiling(g=g)
    s = case["setup"]
    Tc = oracle.Tc_of(s)
    rl, rv, _ = oracle.maxwell(s, 0.86 * Tc)
    rho, T, _ = W.build_fields(case, Tc, rl, rv)
    lat = lbm.Lattice(lbm.params_from_setup(s))
    lat.init(rho.astype(np.float32), T.astype(np.float32))
    return s, lat, 0.5 * (rl + rv)


def nucleation():
    s, lat, mid = _nucleate(1.5e-5)
    for k in range(1000, 20001, 1000):
        lat.step(1000)
        r = lat.moments()["rho"]
        seg = _segments(r[:, s.ny // 2, s.nx // 2], mid)
        print(f"step {k}: centre column vapour {seg}", flush=True)
        if len(seg) >= 3 and seg[0][0] == 0 and seg[1][0] > seg[0][1] + 1 and seg[1][1] < seg[-1][0] - 1:
            break
    lat.close()


def departure(gs):
    from scipy import ndimage
    for g in [float(v) for v in gs.split(",")]:
        s, lat, mid = _nucleate(g)
        for k in range(1000, 30001, 1000):
            lat.step(1000)
            lab, n = ndimage.label(lat.moments()["rho"] < mid)
            attached = (set(np.unique(lab[0])) | set(np.unique(lab[-1]))) - {0}
            free = [(int((lab == i).sum()), i) for i in range(1, n + 1) if i not in attached]
            if free and max(free)[0] > 500:
                vol = max(free)[0]
                print(f"g {g:.2e}: departed by step {k}, volume {vol} nodes, D_d {(6.0 * vol / math.pi) ** (1 / 3):.1f}, "
                      f"0.253 g^-1/2 = {0.253 / math.sqrt(g):.1f}", flush=True)
                break
        else:
            print(f"g {g:.2e}: no departure within 30000 steps", flush=True)
        lat.close()


def heated(mode):
    from paper_2201_06039_gb300 import lbm
    case = W.heated_surface_droplet()
    s = case["setup"]
    Tc = oracle.Tc_of(s)
    rl, rv, _ = oracle.maxwell(s, 0.86 * Tc)
    mid = 0.5 * (rl + rv)
    rho, T, _ = W.build_fields(case, Tc, rl, rv)

    def measure(r):
        col = r[:, s.ny // 2, s.nx // 2]
        h = int(np.argmax(col < mid)) if col[0] > mid else 0
        return float(r[r > mid].sum()), math.sqrt(float((r[0] > mid).sum()) / math.pi), h

    iso = W.LatticeSetup(**{**s.__dict__, "thermal_off": 1, "bc": (0, 0, 0, 0, 1, 1)})
    a = lbm.Lattice(lbm.params_from_setup(iso))
    a.init(rho.astype(np.float32), T.astype(np.float32))
    a.step(10000)
    r = a.moments()["rho"]
    m0, R0, h0 = measure(r)
    ck = a.save_state()
    a.close()
    b = lbm.Lattice(lbm.params_from_setup(s))
    b.load_state(ck)
    if mode == "pinned":
        foot = r[0] > mid
        b.set_wall_map(np.where(foot, 1.4, 1.0).astype(np.float32), np.where(foot, 0.0, 0.3).astype(np.float32))
    print(f"settled: radius {R0:.2f} height {h0}", flush=True)
    t0 = time.time()
    for k in range(10000, 170001, 10000):
        b.step(10000)
        m, R, h = measure(b.moments()["rho"])
        print(f"{k} steps after settling: m/m0 {m / m0:.4f} radius {R:.2f} height {h} ({time.time() - t0:.0f} s)", flush=True)
    b.close()


if __name__ == "__main__":
    what = sys.argv[1]
    {"angles": lambda: angles(sys.argv[2]), "nucleation": nucleation,
     "departure": lambda: departure(sys.argv[2]), "heated": lambda: heated(sys.argv[2])}[what]()
