"""The small workloads at the horizons they are defined with (Eq. llg, the Runge-Kutta and
Dormand-Prince integrators of the time-integration section, the inverse problem of Eq. inverse_min):

* cuboid 16x16x4, 1000 fixed RK4 steps of 1e-14 s: the GPU FP64 trajectory against the oracle's; the
  time-averaged volume-weighted mean of m (1 ps samples, trapezoid over [0, 10 ps]) of the FP32 and
  FP64 paths within 1e-3 of each other and of the oracle's;
* thin film 200x50x1, Dormand-Prince to 1 ns: FP32 against FP64 on the time-averaged mean of m
  (1 ps samples over [0, 1 ns]) within 1e-3; the FP64 path against the oracle step by step over the
  first 20 steps (the oracle's direct demag sum on 10 000 cells takes about a second per step);
* waveguide 256x64x1 over 0-2 ns with the loss on the right 16 cells' nodes and checkpoints every
  ceil(sqrt(n)) steps: the discrete-adjoint gradient of the cell Ms map against central differences
  along seeded directions within 1e-4.  RK4 steps of 0.25 ps (the steps are fixed, so the differences
  are of the same discrete map; 0.25 ps keeps the stiffest exchange mode, about 4.7e12 rad/s, inside
  the RK4 stability region).
"""
import math

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


def _time_average(samples, dt_sample):
    """Trapezoid rule over equally spaced samples, divided by the interval length."""
    s = np.asarray(samples)
    T = dt_sample * (len(s) - 1)
    return (0.5 * (s[0] + s[-1]) + s[1:-1].sum(axis=0)) * dt_sample / T


def test_cuboid_rk4_1000_steps(oracle_mod, nmgb):
    p = inp.cuboid_rk4(0)
    steps, dt, every = 1000, 1e-14, 100
    ref = oracle_mesh(oracle_mod, p)
    w = ref.mass()[..., None]  # uniform Ms: proportional to the nodal volume weights
    m = p.m0.copy()
    means = [np.sum(w * m, axis=(0, 1, 2)) / w.sum()]
    for s in range(steps):
        m = ref.rk4_step(m, s * dt, dt, p.terms, renorm=True)
        if (s + 1) % every == 0:
            means.append(np.sum(w * m, axis=(0, 1, 2)) / w.sum())
    avg_ref = _time_average(means, every * dt)
    avg = {}
    for prec, tol in ((1, 1e-10), (0, 1e-4)):
        me = gpu_mesh(nmgb, p, prec)
        me.set_state(p.m0, 0.0, dt)
        samples, na, nr = me.run_until(steps * dt, nmgb.RK4, dt0=dt, sample_dt=every * dt)
        assert na == steps and nr == 0 and samples.shape == (steps // every + 1, 3)
        mg, tg, _ = me.get_state()
        assert abs(tg - steps * dt) < 1e-24
        assert rel_l2(mg, m) < tol, (prec, rel_l2(mg, m))
        avg[prec] = _time_average(samples, every * dt)
        assert np.abs(avg[prec] - avg_ref).max() <= (1e-12 if prec == 1 else 1e-3)
        me.close()
    assert np.abs(avg[0] - avg[1]).max() <= 1e-3


def test_thin_film_dp5_to_1ns_fp32_vs_fp64(nmgb):
    p = inp.thin_film(0)
    x = p.extra
    avg, counts = {}, {}
    for prec in (1, 0):
        me = gpu_mesh(nmgb, p, prec)
        me.set_state(p.m0, 0.0, x["dt0"])
        samples, na, nr = me.run_until(x["t_end"], nmgb.DP54, x["rtol"], x["atol"], dt0=x["dt0"],
                                       sample_dt=x["sample_dt"])
        n_s = int(round(x["t_end"] / x["sample_dt"])) + 1
        assert samples.shape == (n_s, 3) and np.isfinite(samples).all()
        assert abs(me.get_state()[1] - x["t_end"]) <= 1e-12 * x["t_end"]
        avg[prec] = _time_average(samples, x["sample_dt"])
        counts[prec] = (na, nr)
        me.close()
    assert np.abs(avg[0] - avg[1]).max() <= 1e-3, (avg[0], avg[1])
    # both precisions take about the same number of steps (the controller sees the same dynamics)
    assert abs(counts[0][0] - counts[1][0]) <= 0.05 * counts[1][0]


def test_thin_film_fp64_matches_oracle_first_steps(oracle_mod, nmgb):
    p = inp.thin_film(0)
    x = p.extra
    st = oracle_mesh(oracle_mod, p).dp5_stepper(p.m0, 0.0, x["dt0"], p.terms, x["rtol"], x["atol"])
    me = gpu_mesh(nmgb, p, 1)
    me.set_state(p.m0, 0.0, x["dt0"])
    t, dt = 0.0, x["dt0"]
    for _ in range(20):
        acc_ref = st.step()
        acc, t, dt = me.llg_step(nmgb.DP54, t, dt, x["rtol"], x["atol"])
        assert acc == acc_ref
        assert abs(t - st.t.value) <= 1e-12 * st.t.value
        assert abs(dt - st.dt.value) <= 1e-9 * st.dt.value
    assert rel_l2(me.get_state()[0], st.m) < 1e-11
    me.close()


def test_waveguide_gradient_over_2ns(nmgb):
    import torch
    from paper_2411_11725_gb300.autograd import LossSpec, llg_loss
    p = inp.waveguide(0)
    T, sample_dt, dt = p.extra["t_end"], p.extra["sample_dt"], 2.5e-13
    n_steps = int(round(T / dt))
    me = nmgb.Mesh(p.n, p.dx, nmgb.F64)
    me.set_zeeman((0, 0, 0), h_cell=p.h_cell, cell_freq=p.cell_freq, cell_phase=p.cell_phase)
    me.set_terms(p.terms)
    # mean of m_y^2 over the 1 ps samples in (0, 2 ns] and over the nodes of the right 16 cells
    W = np.zeros(p.nodes + (3,))
    W[p.n[0] - 16:, :, :, 1] = 1.0
    W /= W[..., 1].sum() * int(round(T / sample_dt))
    spec = LossSpec(t_end=T, A=p.A, alpha=p.alpha, gamma=p.gamma, method=nmgb.RK4, dt0=dt,
                    sample_dt=sample_dt, checkpoint_every=math.ceil(math.sqrt(n_steps)))
    Ms = torch.tensor(p.Ms_cells(), dtype=torch.float64, requires_grad=True)
    m0 = torch.tensor(p.m0, dtype=torch.float64)
    L = llg_loss(me, Ms, m0, W, spec)
    L.backward()
    g = Ms.grad.numpy()
    assert spec.stats["accepted_steps"] == n_steps
    assert L.item() > 0 and np.abs(g[-16:]).max() > 0
    rng = np.random.default_rng(51)

    def loss_of(Ms_map):
        # the forward run alone, with the same steps (RK4 of dt0 clipped to the samples)
        me.set_material(Ms_map, p.A, 0.0, p.axis, p.alpha, p.gamma)
        me.set_state(p.m0, 0.0, dt)
        return me.adjoint_run(T, W, None, nmgb.RK4, dt0=dt, sample_dt=sample_dt,
                              checkpoint_every=spec.checkpoint_every, loss_only=True)[0]
    assert loss_of(p.Ms_cells()) == L.item()
    for _ in range(2):
        d = rng.standard_normal(p.n) * p.Ms_cells() * 1e-4
        fd = (loss_of(p.Ms_cells() + d) - loss_of(p.Ms_cells() - d)) / 2
        ad = float(np.sum(g * d))
        assert abs(fd - ad) <= 1e-4 * abs(fd), (fd, ad)
    me.close()
