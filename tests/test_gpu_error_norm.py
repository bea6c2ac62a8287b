"""FP32 meshes form the per-node terms of the Dormand-Prince error norm in FP32 and sum them in FP64
(the Dormand-Prince integrator of the time-integration section).  With every operation of those terms
in FP64 instead (nm_set_error_norm), the thin film run to 1 ns and the 256x256x8 throughput cuboid over
200 steps take the same accept/reject decisions step by step.  Over the first 20 attempts, where both
runs still hold the same state to rounding, the step sizes agree within 1e-5 and the error norms within
5e-5 (relative, or of 1e-2 for smaller norms); over the whole run, where the two trajectories drift
apart by the rounding of their step sizes, within 1e-4 and 5e-4.
"""
import numpy as np
import pytest

import nm_inputs as inp
from helpers import gpu_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nmgb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_11725_gb300 as nmgb
    nmgb.load()
    return nmgb


def _sequence(nmgb, p, f64_terms, t_end=None, n_steps=None, rtol=1e-5, atol=1e-5, dt0=1e-14):
    me = gpu_mesh(nmgb, p, 0)
    me.set_error_norm(f64_terms)
    me.set_state(p.m0, 0.0, dt0)
    t, dt = 0.0, dt0
    acc_seq, dts, errs = [], [], []
    while (t_end is not None and t < t_end * (1 - 1e-12)) or (n_steps is not None and len(acc_seq) < n_steps):
        if t_end is not None:
            dt = min(dt, t_end - t)
        acc, t, dt = me.llg_step(nmgb.DP54, t, dt, rtol, atol)
        acc_seq.append(acc)
        dts.append(dt)
        errs.append(me.counters()[2])
    me.close()
    return np.array(acc_seq), np.array(dts), np.array(errs)


@pytest.mark.parametrize("case", ["thin_film_1ns", "cuboid_256x256x8"])
def test_fp32_error_terms_take_the_fp64_terms_decisions(nmgb, case):
    if case == "thin_film_1ns":
        p = inp.thin_film(0)
        kw = dict(t_end=p.extra["t_end"], dt0=p.extra["dt0"])
    else:
        p = inp.throughput((256, 256, 8), seed=0)
        kw = dict(n_steps=200, dt0=1e-14)
    a32, dt32, e32 = _sequence(nmgb, p, False, **kw)
    a64, dt64, e64 = _sequence(nmgb, p, True, **kw)
    assert len(a32) == len(a64) and np.array_equal(a32, a64)
    if case == "thin_film_1ns":
        # the last step is clipped to t_end: its error norm is tiny and its proposal is not used
        dt32, dt64, e32, e64 = dt32[:-1], dt64[:-1], e32[:-1], e64[:-1]
    rdt = np.abs(dt32 / dt64 - 1)
    # error norms relative to their size, or to 1e-2 for smaller ones (the decisions are taken at 1)
    rerr = np.abs(e32 - e64) / np.maximum(e64, 1e-2)
    assert rdt[:20].max() <= 1e-5 and rerr[:20].max() <= 5e-5, (rdt[:20].max(), rerr[:20].max())
    assert rdt.max() <= 1e-4 and rerr.max() <= 5e-4, (rdt.max(), rerr.max())
    assert a32.sum() >= 100
