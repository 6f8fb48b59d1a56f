"""The TMA kernel's plan API (lbm_plan_shapes, lbm_get_plan, lbm_select_plan, lbm_autotune) and the
autotuner's JSON cache (Lattice.autotune): every tile shape and z-chunk computes the same bits as
the generic fused kernel, bad plans are refused, the autotuner leaves the state exactly as it found
it, and a cached plan is reused without timing."""
import json

import numpy as np
import pytest

import workloads as W
from tests._parity import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(32, 8), (40, 7), (32, 12), (24, 16), (40, 8), (40, 10)]


def _case():
    # walled bottom with a hot spot, outflow top; 88 columns: a partial 40-wide tile column
    return W.pool_boiling(88, 48, 40, height=16.0, hot_sigma=4.0)


def _lattice(s, **kw):
    from paper_2201_06039_gb300 import lbm
    return lbm.Lattice(lbm.params_from_setup(s, kernel=2, **kw))


def _run(lat, rho, T, steps):
    lat.init(rho.astype(np.float32), T.astype(np.float32))
    lat.step(steps)
    m = lat.moments()
    lat.close()
    return m


def test_every_plan_computes_the_same_bits():
    from paper_2201_06039_gb300 import lbm
    assert lbm.lbm_plan_shapes() == SHAPES
    case = _case()
    s = case["setup"]
    rho, T, _ = inputs(case)
    ref = _run(_lattice(s, use_tma=0), rho, T, 9)
    for sh, (tx, ty) in enumerate(SHAPES):
        for zc in (0, 7, s.nz):
            lat = _lattice(s, use_tma=1)
            lat.select_plan(sh, zc)
            shape, zchunk, items, ctas = lat.plan
            assert shape == sh and zchunk >= 1 and (zc == 0 or zchunk == zc), (sh, zc, lat.plan)
            tiles = -(-s.nx // tx) * -(-s.ny // ty)
            assert items == tiles * -(-s.nz // zchunk) and 1 <= ctas <= items, (sh, zc, lat.plan)
            m = _run(lat, rho, T, 9)
            for k in m:
                assert np.array_equal(m[k], ref[k]), (sh, zc, k)


def test_bad_plans_are_refused():
    from paper_2201_06039_gb300 import lbm
    s = _case()["setup"]
    lat = _lattice(s, use_tma=1)
    before = lat.plan
    with pytest.raises(lbm.LbmError):
        lat.select_plan(len(SHAPES), 0)
    with pytest.raises(lbm.LbmError):
        lat.select_plan(0, -1)
    assert lat.plan == before
    lat.close()
    two = lbm.Lattice(lbm.params_from_setup(s, kernel=1))      # the two-pass kernels: no plan
    assert two.plan[0] == -1
    with pytest.raises(lbm.LbmError):
        two.select_plan(0, 0)
    two.close()


def test_autotune_restores_the_state_and_caches_its_choice(tmp_path):
    case = _case()
    s = case["setup"]
    rho, T, _ = inputs(case)
    cache = str(tmp_path / "plans.json")
    lat = _lattice(s, use_tma=1)
    lat.init(rho.astype(np.float32), T.astype(np.float32))
    lat.step(5)
    before = lat.moments()
    res = lat.autotune(steps=3, cache=cache)
    assert not res["cached"] and res["ms_per_step"] > 0
    assert lat.plan[:2] == (res["shape"], res["zchunk"])
    after = lat.moments()
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    lat.step(7)
    tuned = lat.moments()
    key = lat.plan_key()
    lat.close()
    # the tuned run equals an untuned one, step for step
    plain = _run(_lattice(s, use_tma=1), rho, T, 12)
    for k in plain:
        assert np.array_equal(tuned[k], plain[k]), k
    # the cache holds the choice and a second context takes it without timing
    with open(cache) as fh:
        table = json.load(fh)
    assert table[key]["shape"] == res["shape"] and table[key]["zchunk"] == res["zchunk"]
    again = _lattice(s, use_tma=1)
    res2 = again.autotune(steps=3, cache=cache)
    assert res2["cached"] and res2["ms_per_step"] is None
    assert again.plan[:2] == (res["shape"], res["zchunk"])
    again.close()
