"""Failure paths of the integrators and the state, all returned as status codes on the host; nothing
here faults, traps or hangs the GPU.

* A non-finite state is refused by nm_set_state (NM_ERR_NONFINITE), from host and device memory, and
  the mesh then has no state until a valid one is set.
* A step whose error norm is not finite is rejected and shrinks the step by the controller's lower
  clamp, 0.2 (reading R11): a step far too large for the exchange stiffness overflows the stage values.
* Too many consecutive rejections, or a step below dt_min, end the integration with
  NM_ERR_STEP_UNDERFLOW (set through nm_set_integrator).
* nm_h_eff does not check values (it is asynchronous): a non-finite m gives a non-finite field, and the
  mesh stays usable.
"""
import numpy as np
import pytest

import nm_inputs as inp
from helpers import gpu_mesh, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nmgb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_11725_gb300 as nmgb
    nmgb.load()
    return nmgb


def _mesh(nmgb, precision, seed=70):
    p = inp.random_problem(np.random.default_rng(seed), (8, 6, 3), vacuum=True)
    p.h_freq = 0.0
    return p, gpu_mesh(nmgb, p, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_set_state_refuses_non_finite(nmgb, precision):
    import torch
    p, me = _mesh(nmgb, precision)
    me.set_state(p.m0, 0.0, 1e-14)
    for bad_value, where in ((np.nan, "host"), (np.inf, "device"), (-np.inf, "host")):
        m = p.m0.copy()
        m[3, 2, 1, 2] = bad_value
        m[0, 0, 0, 0] = bad_value
        arg = torch.tensor(m, device="cuda") if where == "device" else m
        with pytest.raises(nmgb.NMError) as e:
            me.set_state(arg, 0.0, 1e-14)
        assert e.value.code == nmgb.ERR_NONFINITE and "non-finite values at 2 nodes" in str(e.value)
        with pytest.raises(nmgb.NMError) as e:
            me.llg_step(nmgb.DP54, 0.0, 1e-14)
        assert e.value.code == nmgb.ERR_STATE
    # a valid state brings the mesh back
    me.set_state(p.m0, 0.0, 1e-14)
    acc, t, _ = me.llg_step(nmgb.DP54, 0.0, 1e-14)
    assert acc and t == 1e-14
    me.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_non_finite_error_norm_rejects_with_factor_0p2(nmgb, precision):
    p, me = _mesh(nmgb, precision)
    me.set_state(p.m0, 0.0, 1e-3)
    m_before, _, _ = me.get_state()
    acc, t, dt = me.llg_step(nmgb.DP54, 0.0, 1e-3)
    assert not acc and t == 0.0 and dt == 1e-3 * 0.2
    assert not np.isfinite(me.counters()[2])  # the error norm itself is inf or NaN
    m_after, _, _ = me.get_state()
    assert np.array_equal(m_before, m_after)
    # the state is untouched, so a sensible step goes through afterwards
    acc, t, dt = me.llg_step(nmgb.DP54, 0.0, 1e-15)
    assert acc and t == 1e-15 and np.isfinite(me.get_state()[0]).all()
    me.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_too_many_rejections_is_step_underflow(nmgb, precision):
    p, me = _mesh(nmgb, precision)
    me.set_integrator(True, 1e-22, 2)
    me.set_state(p.m0, 0.0, 1e-2)
    with pytest.raises(nmgb.NMError) as e:
        me.run_until(1.0, nmgb.DP54, 1e-5, 1e-5, dt0=1e-2)
    assert e.value.code == nmgb.ERR_STEP_UNDERFLOW
    # the third consecutive rejection exceeds max_rejections = 2
    assert me.counters()[:2] == (0, 3)
    me.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_step_below_dt_min_is_step_underflow(nmgb, precision):
    p, me = _mesh(nmgb, precision)
    me.set_integrator(True, 1e-4, 50)
    me.set_state(p.m0, 0.0, 1e-2)
    with pytest.raises(nmgb.NMError) as e:
        me.run_until(1.0, nmgb.DP54, 1e-5, 1e-5, dt0=1e-2)
    assert e.value.code == nmgb.ERR_STEP_UNDERFLOW
    # proposals 2e-3 and 4e-4 are allowed, 8e-5 is below dt_min
    assert me.counters()[:2] == (0, 3)
    me.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_h_eff_of_non_finite_m_is_non_finite_and_mesh_stays_usable(nmgb, precision):
    import torch
    p, me = _mesh(nmgb, precision)
    m = torch.tensor(p.m0, dtype=me.dtype, device="cuda")
    good = me.h_eff(m, nmgb.ALL, 0.0).double().cpu().numpy()
    bad = m.clone()
    bad[4, 3, 1, 0] = float("nan")
    h = me.h_eff(bad, nmgb.ALL, 0.0).double().cpu().numpy()
    assert np.isnan(h).any()
    again = me.h_eff(m, nmgb.ALL, 0.0).double().cpu().numpy()
    assert np.isfinite(again).all() and rel_l2(again, good) == 0.0
    me.close()
