"""The inverse problem of the waveguide workload through torch.autograd: the gradient of a mean m_y^2
loss with respect to the cell Ms map, against central finite differences (step sizes
frozen), and the FP32 path against the FP64 path."""
import numpy as np
import pytest

import nm_inputs as inp
from helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nmgb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_11725_gb300 as nmgb
    nmgb.load()
    return nmgb


def _setup(nmgb, precision, T=6e-12, sample_dt=1e-13):
    from paper_2411_11725_gb300.autograd import LossSpec
    p = inp.waveguide(0)
    me = nmgb.Mesh(p.n, p.dx, precision)
    me.set_material(p.Ms_cells(), p.A, 0.0, p.axis, p.alpha, p.gamma)
    me.set_zeeman((0, 0, 0), h_cell=p.h_cell, cell_freq=p.cell_freq, cell_phase=p.cell_phase)
    me.set_terms(p.terms)
    # the workload's loss region is the right end (reached after ~1 ns); over the short horizons of these
    # tests the same form of loss is taken on the 16 node columns next to the driven region instead
    W = np.zeros(p.nodes + (3,))
    W[8:24, :, :, 1] = 1.0
    n_samples = int(round(T / sample_dt))
    W /= W[..., 1].sum() * n_samples
    # loose tolerances: every attempt accepted, the steps are fixed by the clipping to the samples
    spec = LossSpec(t_end=T, A=p.A, alpha=p.alpha, gamma=p.gamma, rtol=1e3, atol=1e3, dt0=5e-14,
                    sample_dt=sample_dt, checkpoint_every=8)
    return p, me, W, spec


def test_waveguide_gradient_matches_finite_differences(nmgb):
    import torch
    from paper_2411_11725_gb300.autograd import llg_loss
    p, me, W, spec = _setup(nmgb, nmgb.F64)
    Ms = torch.tensor(p.Ms_cells(), dtype=torch.float64, requires_grad=True)
    m0 = torch.tensor(p.m0, dtype=torch.float64)
    L = llg_loss(me, Ms, m0, W, spec)
    L.backward()
    g = Ms.grad.numpy()
    assert L.item() > 0 and np.abs(g).max() > 0
    rng = np.random.default_rng(50)
    for _ in range(2):
        d = rng.standard_normal(p.n) * p.Ms_cells() * 1e-4
        with torch.no_grad():
            lp = llg_loss(me, torch.tensor(p.Ms_cells() + d), m0, W, spec).item()
            lm = llg_loss(me, torch.tensor(p.Ms_cells() - d), m0, W, spec).item()
        fd = (lp - lm) / 2
        ad = float(np.sum(g * d))
        assert abs(fd - ad) <= 1e-4 * abs(fd), (fd, ad)
    me.close()


def test_waveguide_gradient_fp32_close_to_fp64(nmgb):
    import torch
    from paper_2411_11725_gb300.autograd import llg_loss
    grads = {}
    for prec in (nmgb.F64, nmgb.F32):
        p, me, W, spec = _setup(nmgb, prec, T=3e-12)
        Ms = torch.tensor(p.Ms_cells(), dtype=torch.float64, requires_grad=True)
        llg_loss(me, Ms, torch.tensor(p.m0), W, spec).backward()
        grads[prec] = Ms.grad.numpy().copy()
        me.close()
    assert rel_l2(grads[nmgb.F32], grads[nmgb.F64]) < 1e-2
