"""FP32 parity on mid-size meshes (section "Demagnetization Field"), between the small meshes of the
other parity tests and the full-size sampled checks: x transforms of 64 to 256 points, z lines of 16 to
64 (N3 from 5 to 32), odd and even N1 (a ragged last cell pair), N2 = 1 (no y transform), vacuum cells
and cell maps.  The field against the FP64 oracle's direct demag sum on the FP32-rounded input
(rel-L2 <= 1e-5, as for the other meshes); the transpose product (cell inputs through the demag passes)
and one Dormand-Prince step against the FP64 path, which is pinned to the oracle on its own meshes."""
import numpy as np
import pytest

import nm_inputs as inp
from helpers import gpu_mesh, oracle_mesh, rel_l2, rounded

pytestmark = pytest.mark.gpu

SHAPES = [(40, 7, 5), (33, 3, 9), (64, 5, 17), (41, 6, 32), (128, 2, 8), (70, 1, 12), (96, 4, 31)]


@pytest.fixture(scope="module")
def nmgb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_11725_gb300 as nmgb
    nmgb.load()
    return nmgb


@pytest.mark.parametrize("shape", SHAPES)
def test_midsize_field_matches_oracle(oracle_mod, nmgb, shape):
    import torch
    rng = np.random.default_rng(sum(shape))
    p = inp.random_problem(rng, shape, vacuum=True)
    m = rounded(p.m0, 0)
    ref = oracle_mesh(oracle_mod, p)
    me = gpu_mesh(nmgb, p, 0)
    mt = torch.tensor(m, dtype=torch.float32, device="cuda")
    for terms in (oracle_mod.DEMAG, oracle_mod.ALL):
        h = me.h_eff(mt, terms, 2e-10).double().cpu().numpy()
        r = ref.h_eff(m, terms, 2e-10)
        assert rel_l2(h, r) <= 1e-5, (shape, terms, rel_l2(h, r))
    me.close()


@pytest.mark.parametrize("shape", [(40, 7, 5), (41, 6, 32), (70, 1, 12)])
def test_midsize_transpose_product_matches_fp64_path(nmgb, shape):
    import torch
    rng = np.random.default_rng(7 + sum(shape))
    p = inp.random_problem(rng, shape, vacuum=False)
    m = rounded(p.m0, 0)
    v = rounded(rng.standard_normal(p.nodes + (3,)), 0)
    out = {}
    for prec in (1, 0):
        me = gpu_mesh(nmgb, p, prec)
        gm, gMs = me.h_eff_vjp(torch.tensor(m, dtype=me.dtype, device="cuda"),
                               torch.tensor(v, dtype=me.dtype, device="cuda"), nmgb.ALL, 1e-10)
        out[prec] = (gm.double().cpu().numpy(), gMs.double().cpu().numpy())
        me.close()
    assert rel_l2(out[0][0], out[1][0]) <= 1e-5
    assert rel_l2(out[0][1], out[1][1]) <= 1e-4


def test_midsize_dp5_step_matches_fp64_path(nmgb):
    p = inp.random_problem(np.random.default_rng(77), (48, 9, 12), vacuum=True)
    p.h_freq = 0.0
    out = {}
    for prec in (1, 0):
        me = gpu_mesh(nmgb, p, prec)
        me.set_state(p.m0, 0.0, 1e-14)
        me.run_steps(2, nmgb.DP54, 1e3, 1e3)  # every attempt accepted: the same steps in both precisions
        out[prec] = me.get_state()
        me.close()
    assert out[0][1] == out[1][1] and out[0][1] > 0
    d0 = out[0][0] - p.m0
    d1 = out[1][0] - p.m0
    assert rel_l2(d0, d1) <= 1e-4
