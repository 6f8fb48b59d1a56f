"""Ghost cells of the TMA kernel on FP32 lattices whose x extent is no multiple of the 16-byte
ghost band or that have a single tile across an axis: the edge nodes store their periodic images
straight into the ghost columns and rows (no refresh kernel).  The TMA kernel must then compute
exactly what the generic fused and two-pass kernels compute, step after step."""
import numpy as np
import pytest

import workloads as W
from tests._parity import inputs, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(41, 15, 20), (33, 9, 17), (37, 29, 11), (24, 24, 24), (5, 6, 7), (203, 13, 9)])
def test_fp32_tma_direct_ghosts_bit_identical(dims):
    from paper_2201_06039_gb300 import lbm
    nx, ny, nz = dims
    s = W.LatticeSetup(nx, ny, nz, sigma=W.SIGMA_STAR)
    case = dict(name=f"droplet {dims}", setup=s, kind="droplet", R0=min(dims) / 3.0, W=4.0, Tr_drop=0.86,
                Tr_gas=0.86, noise=1e-3, noise_seed=W.MASTER_SEED + 5 + nx)
    rho, T, u = inputs(case)
    lat = lbm.Lattice(lbm.params_from_setup(s, kernel=2, use_tma=1))
    assert lat.kernel == lbm.LBM_KERNEL_FUSED_TMA
    lat.close()
    tma, _ = run_gpu(s, rho, T, u, 13, kernel=2, use_tma=1)
    gen, _ = run_gpu(s, rho, T, u, 13, kernel=2, use_tma=0)
    two, _ = run_gpu(s, rho, T, u, 13, kernel=1)
    for k in tma:
        assert np.array_equal(tma[k], gen[k]), (dims, k)
        assert np.array_equal(tma[k], two[k]), (dims, k)
