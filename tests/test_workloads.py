"""The synthetic workloads carry the geometry and parameters the paper states for its tests
(Sec. IV), and the nucleate-boiling patch covers exactly the 55 x 55 square of Sec. IV.C."""
import numpy as np

import oracle
import workloads as W


def test_nucleate_boiling_preset_is_the_papers_geometry():
    """Sec. IV.C: 200 x 200 x 280, saturated liquid for 0 <= z <= 200 under its vapour at
    0.86 Tc, bottom wall at 0.96 Tc, bounce-back top and bottom, periodic x and y, chi = 0.08,
    a = 2/49, b = 2/21, R = 1, buoyancy against the domain mean with g = 1.5e-5, a 55-node
    hydrophobic square at the centre of the bottom."""
    case = W.nucleate_boiling()
    s = case["setup"]
    assert (s.nx, s.ny, s.nz) == (200, 200, 280)
    assert s.bc == (W.BC_PERIODIC,) * 4 + (W.BC_WALL, W.BC_WALL)
    assert s.T_wall_over_Tc[4] == 0.96 and s.hot_dT_over_Tc == 0.0
    assert (s.a, s.b, s.R) == (2.0 / 49.0, 2.0 / 21.0, 1.0)
    assert s.lambda_mode == 0 and s.chi_or_lambda == 0.08
    assert s.gravity == (0.0, 0.0, -1.5e-5) and s.rho_buoy == 0.0
    assert s.wall_scheme == 1 and 2 * s.wall_patch_half == 55.0
    Tc = oracle.Tc_of(s)
    rl, rv, _ = oracle.maxwell(s, 0.86 * Tc)
    rho, T, _ = W.build_fields(case, Tc, rl, rv)
    mid = 0.5 * (rl + rv)
    col = rho[:, 100, 100]
    assert col[199] > mid > col[201] and abs(col[200] - mid) < 1e-9 * mid
    assert np.allclose(T, 0.86 * Tc)


def test_nucleate_boiling_patch_is_a_55_node_square():
    """One step of a uniform liquid over the preset's wall (lattice cut to 4 layers): the solid
    layer takes phi rho - drho, so a bottom-layer node whose five solid neighbours all lie on the
    patch feels one F_m,z and a node whose five lie off it another.  Those two sets are exactly
    the nodes inside (resp. away from) a 55 x 55 square of solid nodes x, y = 73..127."""
    s = W.LatticeSetup(**{**W.nucleate_boiling()["setup"].__dict__, "nz": 4, "gravity": (0.0, 0.0, 0.0)})
    Tc = oracle.Tc_of(s)
    o = oracle.Oracle(s)
    o.init(np.full(s.shape, 6.4), np.full(s.shape, 0.86 * Tc))
    o.step(1)
    fz = o.diag()["Fm"][0, :, :, 2]
    o.close()
    sq = np.zeros((200, 200), bool)
    sq[73:128, 73:128] = True

    def all5(m):   # the node and its four in-plane neighbours (periodic) all in m
        return m & np.roll(m, 1, 0) & np.roll(m, -1, 0) & np.roll(m, 1, 1) & np.roll(m, -1, 1)

    on = np.isclose(fz, fz[100, 100], rtol=0, atol=1e-12)
    off = np.isclose(fz, fz[0, 0], rtol=0, atol=1e-12)
    assert fz[100, 100] != fz[0, 0]
    assert np.array_equal(on, all5(sq)) and np.array_equal(off, all5(~sq))


def test_heated_surface_droplet_preset_is_the_papers_geometry():
    """Sec. IV.B: 200 x 200 x 100, a hemisphere of radius 30 at the centre of the bottom wall,
    wall at 0.87 Tc, open top at T_sat = 0.86 Tc, periodic x and y, chi = 0.02."""
    case = W.heated_surface_droplet()
    s = case["setup"]
    assert (s.nx, s.ny, s.nz) == (200, 200, 100)
    assert s.bc == (W.BC_PERIODIC,) * 4 + (W.BC_WALL, W.BC_OUTFLOW)
    assert s.T_wall_over_Tc[4] == 0.87 and s.T_wall_over_Tc[5] == 0.86
    assert s.lambda_mode == 0 and s.chi_or_lambda == 0.02 and s.gravity == (0.0, 0.0, 0.0)
    Tc = oracle.Tc_of(s)
    rl, rv, _ = oracle.maxwell(s, 0.86 * Tc)
    rho, _, _ = W.build_fields(case, Tc, rl, rv)
    mid = 0.5 * (rl + rv)
    # the mid-density surface crosses the centre column at z ~ 29.5 and the bottom row at r ~ 30
    col = rho[:, 100, 100]
    z = int(np.nonzero(col < mid)[0][0])
    assert 29 <= z <= 31
    row = rho[0, 100, 100:]
    x = int(np.nonzero(row < mid)[0][0])
    assert 29 <= x <= 31


def test_cpu_baseline_sample_of_the_wetting_workloads():
    """bench.py's CPU-baseline leg runs the oracle on a z-slab of the nucleate-boiling and the
    heated-surface workloads (wetting wall, patch, open top) and reports a positive rate."""
    import bench
    for case in (W.nucleate_boiling(), W.heated_surface_droplet()):
        out = bench.cpu_baseline_run(case, steps=1, warm=0)
        assert out["value"] > 0 and out["kind"] == "oracle", case["name"]
