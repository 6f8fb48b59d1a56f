"""Batched ensemble (lbm_batch_*): independent lattices of uneven sizes in one persistent launch
per step, against the FP64 oracle run on each instance alone, against single-lattice contexts,
and for the autotuner's state restoration."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests._parity import bars, fp32_floor, inputs, rel_errors, run_oracle

pytestmark = pytest.mark.gpu


def _cases():
    """Droplets and slabs of ragged sizes and different temperatures (periodic boxes)."""
    out = []
    for k, (dims, kind, Tr, R) in enumerate([((24, 24, 24), "droplet", 0.86, 7.0),
                                              ((29, 26, 31), "slab", 0.82, 6.0),
                                              ((40, 33, 36), "droplet", 0.88, 9.0),
                                              ((5, 3, 2), "slab", 0.86, 1.0),
                                              ((33, 9, 17), "droplet", 0.84, 4.0)]):
        s = W.LatticeSetup(*dims, sigma=W.SIGMA_STAR)
        out.append(dict(name=f"inst{k}", setup=s, kind=kind, R0=R, W=4.0, Tr_drop=Tr, Tr_gas=Tr,
                        noise=1e-3, noise_seed=W.MASTER_SEED + 77 + k))
    return out


def _batch(cases, **over):
    from paper_2201_06039_gb300 import lbm
    common = lbm.params_from_setup(cases[0]["setup"], **over)
    return lbm.Batch(common, [(c["setup"].nx, c["setup"].ny, c["setup"].nz) for c in cases])


def _fields(cases):
    """Seeded fields of each case; boxes thinner than 4 nodes hold uniform vapour (+ noise)."""
    rho, T = [], []
    for c in cases:
        r, t, _ = inputs(c)
        s = c["setup"]
        if min(s.nx, s.ny, s.nz) < 4:
            rv = oracle.maxwell(s, c["Tr_drop"] * oracle.Tc_of(s))[1]
            r = W.add_noise(np.full(s.shape, rv), c["noise_seed"], 1e-3).astype(np.float32).astype(np.float64)
        rho.append(r)
        T.append(t)
    return rho, T


def test_batch_matches_oracle_per_instance():
    cases = _cases()
    rho, T = _fields(cases)
    steps = 200
    b = _batch(cases)
    b.init(rho, T)
    b.step(steps)
    got = b.moments()
    b.close()
    for c, r, t, g in zip(cases, rho, T, got):
        ref = run_oracle(c["setup"], r, t, None, steps)
        err = rel_errors(g, ref)
        bar = bars(fp32_floor(c["setup"], r, t, None, steps, ref=ref))
        print(c["name"], c["setup"].shape, err, bar)
        for k, v in err.items():
            assert v <= bar[k], (c["name"], k, v, bar[k])


def test_batch_matches_single_lattices():
    from paper_2201_06039_gb300 import lbm
    cases = _cases()
    rho, T = _fields(cases)
    steps = 57
    b = _batch(cases)
    b.init(rho, T)
    b.step(steps)
    got = b.moments()
    b.close()
    for c, r, t, g in zip(cases, rho, T, got):
        p = lbm.params_from_setup(c["setup"], kernel=2, use_tma=0)
        lat = lbm.Lattice(p)
        lat.init(r.astype(np.float32), t.astype(np.float32))
        lat.step(steps)
        m = lat.moments()
        lat.close()
        err = rel_errors(g, {k: v.astype(np.float64) for k, v in m.items()})
        for k, v in err.items():
            assert v <= 1e-6, (c["name"], k, v)


@pytest.mark.parametrize("plan", [(8, 1), (4, 2), (8, 4), (0, 0)])
def test_batch_plans_bit_identical_to_single_lattices(plan):
    """Every work plan gives each instance exactly the state of its own single-lattice context
    (the TMA kernel where the instance qualifies, the generic fused kernel otherwise).  Plan
    (0, 0) is the TMA mode: a TMA launch per instance (with the ghost refresh where its tiles do
    not write their ghost cells), the generic fused kernel for the 5 x 3 x 2 box, on 48 streams."""
    from paper_2201_06039_gb300 import lbm
    cases = _cases()
    rho, T = _fields(cases)
    b = _batch(cases)
    b.select_plan(*plan)
    assert (b.plan["tile_rows"], b.plan["z_split"]) == plan
    b.init(rho, T)
    b.step(1)
    b.step(30)
    got = b.moments()
    b.close()
    for c, r, t, g in zip(cases, rho, T, got):
        lat = lbm.Lattice(lbm.params_from_setup(c["setup"]))
        lat.init(r.astype(np.float32), t.astype(np.float32))
        lat.step(31)
        m = lat.moments()
        lat.close()
        for k in m:
            assert np.array_equal(g[k], m[k]), (plan, c["name"], k)


def test_autotune_restores_state_and_keeps_results():
    cases = _cases()
    rho, T = _fields(cases)
    b = _batch(cases)
    b.init(rho, T)
    b.step(5)
    before = b.moments()
    ms = b.autotune(2)
    plan = b.plan
    assert ms > 0 and (plan["tile_rows"], plan["z_split"]) in [(4, 1), (4, 2), (4, 4), (8, 1), (8, 2), (8, 4), (0, 0)]
    assert plan["items"] >= len(cases) and plan["ctas"] >= 1
    after = b.moments()
    for x, y in zip(before, after):
        for k in x:
            assert np.array_equal(x[k], y[k]), k
    b.step(20)
    tuned = b.moments()
    b.close()
    ref = _batch(cases)
    ref.init(rho, T)
    ref.step(25)
    plain = ref.moments()
    ref.close()
    for x, y in zip(tuned, plain):
        err = rel_errors(x, {k: v.astype(np.float64) for k, v in y.items()})
        for k, v in err.items():
            assert v <= 1e-6, (k, v)


def test_batch_conserves_mass_per_instance():
    cases = _cases()
    rho, T = _fields(cases)
    b = _batch(cases)
    b.init(rho, T)
    m0 = b.totals()[:, 0].copy()
    b.step(300)
    m1 = b.totals()[:, 0]
    b.close()
    rel = np.abs(m1 / m0 - 1.0)
    assert np.all(rel < 1e-6), rel


def test_batch_of_256_ensemble_instances_steps_finite():
    """The 256-instance ensemble (edges 24..96) runs a few steps with finite totals and the
    expected total node count."""
    cases = W.batch_instances()
    dims = [(c["setup"].nx, c["setup"].ny, c["setup"].nz) for c in cases]
    total = sum(x * y * z for x, y, z in dims)
    from paper_2201_06039_gb300 import lbm
    b = lbm.Batch(lbm.params_from_setup(cases[0]["setup"]), dims)
    assert b.N == total
    Tc = oracle.Tc_of(cases[0]["setup"])
    rho, T = [], []
    for c in cases:
        rl, rv, _ = oracle.maxwell(c["setup"], c["Tr_drop"] * Tc)
        r, t, _ = W.build_fields(c, Tc, rl, rv)
        rho.append(r)
        T.append(t)
    b.init(rho, T)
    b.step(10)
    tot = b.totals()
    b.close()
    assert np.all(np.isfinite(tot))


def test_batch_tma_mode_graph_replay_and_switching():
    """The TMA mode under CUDA-graph replay, entered from a state the persistent batched kernel
    wrote (its ghost cells refreshed first) and left again, matches one plan run throughout."""
    from paper_2201_06039_gb300 import lbm
    cases = _cases()
    rho, T = _fields(cases)
    b = _batch(cases)
    b.select_plan(8, 1)
    b.init(rho, T)
    b.step(7)
    b.select_plan(0, 0)
    assert lbm.lbm_batch_launches_per_step(b.b) >= len(cases)
    b.step(12)                 # graph of 12 TMA-mode steps
    b.step(12)                 # replayed
    b.select_plan(4, 2)
    b.step(5)
    got = b.moments()
    b.close()
    ref = _batch(cases)
    ref.select_plan(8, 1)
    assert lbm.lbm_batch_launches_per_step(ref.b) == 1
    ref.init(rho, T)
    ref.step(36)
    want = ref.moments()
    ref.close()
    for x, y in zip(got, want):
        for k in x:
            assert np.array_equal(x[k], y[k]), k
