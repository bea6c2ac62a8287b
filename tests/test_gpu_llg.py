"""Parity of the GPU LLG integration (RK4 and Dormand-Prince 5(4), device-side step control, CUDA-graph
replay) with the FP64 oracle, plus closed-form and invariant checks on the GPU path."""
import numpy as np
import pytest

import nm_inputs as inp
from helpers import gpu_mesh, oracle_mesh, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nmgb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_11725_gb300 as nmgb
    nmgb.load()
    return nmgb


def test_rk4_cuboid_matches_oracle(oracle_mod, nmgb):
    p = inp.cuboid_rk4(0)
    steps, dt = 40, 1e-14
    ref = oracle_mesh(oracle_mod, p)
    m = p.m0.copy()
    for s in range(steps):
        m = ref.rk4_step(m, s * dt, dt, p.terms, renorm=True)
    for prec, tol in ((1, 1e-12), (0, 1e-5)):
        me = gpu_mesh(nmgb, p, prec)
        me.set_state(p.m0, 0.0, dt)
        t = 0.0
        for _ in range(steps):
            acc, t, _ = me.llg_step(nmgb.RK4, t, dt)
            assert acc
        mg, tg, _ = me.get_state()
        assert abs(tg - steps * dt) < 1e-25
        assert rel_l2(mg, m) < tol, prec
        me.close()


def test_dp5_step_sequence_matches_oracle(oracle_mod, nmgb):
    """Same accepted/rejected decisions, times and states as the oracle, step by step (FP64 path)."""
    rng = np.random.default_rng(4)
    p = inp.random_problem(rng, (7, 5, 3), heterogeneous=True)
    p.h_freq = 0.0
    ref = oracle_mesh(oracle_mod, p).dp5_stepper(p.m0, 0.0, 2e-13, oracle_mod.ALL, rtol=1e-5, atol=1e-5)
    me = gpu_mesh(nmgb, p, 1)
    me.set_state(p.m0, 0.0, 2e-13)
    t, dt = 0.0, 2e-13
    n_rej = 0
    for _ in range(25):
        acc_ref = ref.step()
        acc, t, dt = me.llg_step(nmgb.DP54, t, dt, 1e-5, 1e-5)
        assert acc == acc_ref
        n_rej += not acc
        assert abs(t - ref.t.value) <= 1e-12 * abs(ref.t.value) + 1e-30
        assert abs(dt - ref.dt.value) <= 1e-9 * ref.dt.value
    mg, _, _ = me.get_state()
    assert rel_l2(mg, ref.m) < 1e-12
    me.close()


def test_dp5_fp32_trajectory_close(oracle_mod, nmgb):
    p = inp.cuboid_rk4(2)
    p.terms = 15
    ref = oracle_mesh(oracle_mod, p).dp5_stepper(p.m0, 0.0, 1e-14, oracle_mod.ALL, rtol=1e-5, atol=1e-5)
    for _ in range(20):
        ref.step()
    me = gpu_mesh(nmgb, p, 0)
    me.set_state(p.m0, 0.0, 1e-14)
    _, _, _ = me.run_until(ref.t.value, nmgb.DP54, 1e-5, 1e-5, dt0=1e-14)
    mg, tg, _ = me.get_state()
    assert abs(tg - ref.t.value) < 1e-24
    assert rel_l2(mg, ref.m) < 1e-4
    me.close()


def test_run_steps_equals_llg_steps(nmgb):
    """The graph-replayed batch of steps is bitwise the same as stepping one call at a time."""
    p = inp.cuboid_rk4(3)
    a = gpu_mesh(nmgb, p, 0)
    a.set_state(p.m0, 0.0, 1e-14)
    a.run_steps(12, nmgb.DP54, 1e-5, 1e-5)
    ma, ta, dta = a.get_state()
    b = gpu_mesh(nmgb, p, 0)
    b.set_state(p.m0, 0.0, 1e-14)
    t, dt = 0.0, 1e-14
    for _ in range(12):
        _, t, dt = b.llg_step(nmgb.DP54, t, dt, 1e-5, 1e-5)
    mb, tb, dtb = b.get_state()
    assert np.array_equal(ma, mb) and ta == tb and dta == dtb
    a.close()
    b.close()


def test_macrospin_closed_form_gpu(nmgb):
    alpha, H, Ms = 0.1, 8e4, 8e5
    p = inp.Problem("macrospin", (1, 1, 1), (3e-9, 3e-9, 3e-9), Ms, 0.0, 0.0, (0, 0, 1), alpha,
                    h_uniform=(0.0, 0.0, H), terms=15)
    th0, ph0 = 2.5, 0.3
    m0 = np.array([np.sin(th0) * np.cos(ph0), np.sin(th0) * np.sin(ph0), np.cos(th0)])
    me = gpu_mesh(nmgb, p, 1)
    me.set_state(np.broadcast_to(m0, (2, 2, 2, 3)).copy(), 0.0, 1e-13)
    T = 1e-10
    me.run_until(T, nmgb.DP54, 1e-10, 1e-10, dt0=1e-13)
    m, t, _ = me.get_state()
    g = inp.GAMMA / (1 + alpha ** 2)
    th = 2 * np.arctan(np.tan(th0 / 2) * np.exp(-alpha * g * H * T))
    ph = ph0 + g * H * T
    ref = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    assert abs(t - T) < 1e-22
    assert np.abs(m[0, 0, 0] - ref).max() < 1e-7
    me.close()


def test_run_until_samples_and_fp32_vs_fp64(nmgb):
    """Time-averaged <m> of the FP32 path within 1e-3 of the FP64 path on the thin film (short run)."""
    p = inp.thin_film(0)
    out = {}
    for prec in (1, 0):
        me = gpu_mesh(nmgb, p, prec)
        me.set_state(p.m0, 0.0, 1e-14)
        s, na, nr = me.run_until(50e-12, nmgb.DP54, 1e-5, 1e-5, dt0=1e-14, sample_dt=1e-12)
        assert s.shape == (51, 3) and na > 10
        out[prec] = s
        me.close()
    avg = {k: np.trapezoid(v, dx=1e-12, axis=0) / 50e-12 for k, v in out.items()}
    assert np.abs(avg[0] - avg[1]).max() < 1e-3
    assert np.abs(out[1][0] - p.m0.reshape(-1, 3).mean(0)).max() < 0.05


def test_norm_preserved_with_renormalisation(nmgb):
    p = inp.cuboid_rk4(5)
    me = gpu_mesh(nmgb, p, 0)
    me.set_state(p.m0, 0.0, 1e-14)
    me.run_steps(30, nmgb.DP54, 1e-5, 1e-5)
    m, t, _ = me.get_state()
    assert t > 0
    assert np.abs(np.linalg.norm(m, axis=-1) - 1).max() < 1e-12
    me.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_mean_m_is_volume_weighted_mean(nmgb, precision):
    """nm_mean_m against the weighted mean of the read-back state, weights Σ_{c∋n} V/8 over magnetic
    cells (computed here from the cell map), on a problem with vacuum cells."""
    rng = np.random.default_rng(71)
    p = inp.random_problem(rng, (9, 7, 3), vacuum=True)
    me = gpu_mesh(nmgb, p, precision)
    me.set_state(p.m0, 0.0, 1e-14)
    me.run_steps(3, nmgb.DP54, 1e-5, 1e-5)
    m, _, _ = me.get_state()
    mag = (p.Ms_cells() > 0).astype(float)
    w = np.zeros(p.nodes)
    for i in range(2):
        for j in range(2):
            for k in range(2):
                w[i:i + p.n[0], j:j + p.n[1], k:k + p.n[2]] += mag
    ref = (w[..., None] * m).sum((0, 1, 2)) / w.sum()
    got = me.mean_m()
    me.close()
    # FP32 meshes keep the volume weights in FP32 (relative rounding 6e-8)
    assert np.abs(got - ref).max() < (1e-12 if precision == 1 else 1e-7)


def test_state_round_trip_through_page_locked_memory(nmgb):
    """Page-locked host buffers are read and written by the layout kernels directly; pageable ones go
    through a device copy.  Both give the same state, bit for bit."""
    import torch
    rng = np.random.default_rng(72)
    p = inp.random_problem(rng, (33, 9, 34), vacuum=False)
    me = gpu_mesh(nmgb, p, 0)
    pinned_in = torch.from_numpy(p.m0.copy()).pin_memory()
    me.set_state_host_ptr(pinned_in, 0.0, 1e-14)
    m_pageable, _, _ = me.get_state()
    assert np.array_equal(m_pageable, p.m0)
    me.run_steps(2, nmgb.DP54, 1e-5, 1e-5)
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    me.get_state_host_ptr(pinned_out)
    m_pageable, _, _ = me.get_state()
    assert np.array_equal(pinned_out.numpy(), m_pageable)
    me.close()
