"""Parity at the full throughput size, 1024x1024x32 cells of 3 nm (35M nodes), with the kernels the
benchmark times (x lines of 1024, y lines of 2048, register z convolution of 64, 32x4 node tiles), and at
the largest supported mesh, 1024x1024x64 (z lines of 128 through shared memory): sampled outputs the
oracle computes one node at a time (``oracle.sampled``), and a property that holds at any size.  FP32
bars rel-L2 <= 1e-5, FP64 <= 1e-12, as for the small meshes.

- Local terms (exchange + anisotropy) of a random state at corners, edges, faces and random nodes.
- Demag of a sparse source (a 2x2x2 node block at a corner, one interior node), sampled next to the
  sources, at mid range and at the far corners, where a wrong padding would put a periodic image.
- One Dormand-Prince 5(4) step (every attempt accepted) with local terms, through the replayed step
  graph: the increment of m at sampled nodes.
- Uniform m: the mass-weighted mean of the nodal demag field is -Ms D m, D the prism's demagnetising
  factors (Aharoni's closed form).
"""
import numpy as np
import pytest

import nm_inputs as inp
from helpers import aharoni_factors, gpu_mesh, rel_l2, rounded

pytestmark = pytest.mark.gpu

N = (1024, 1024, 32)      # the benchmark's mesh
N_MAX = (1024, 1024, 64)  # the largest supported mesh
TOL = {0: 1e-5, 1: 1e-12}
_problems = {}


def _problem(n):
    """The throughput material on n cells with its seeded random state (one at a time: 0.8-1.6 GB)."""
    if n not in _problems:
        _problems.clear()
        _problems[n] = inp.throughput(n, seed=0)
    return _problems[n]


@pytest.fixture(scope="module")
def nmgb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_11725_gb300 as nmgb
    nmgb.load()
    return nmgb


@pytest.fixture(scope="module")
def sampled():
    from oracle import sampled as s
    return s


def _material(p):
    return (p.Ms, p.A, p.Ku, p.axis, p.alpha, p.gamma)


def _sample_nodes(seed, M=N, n_random=24):
    rng = np.random.default_rng(seed)
    nodes = [(a, b, c) for a in (0, M[0]) for b in (0, M[1]) for c in (0, M[2])]
    nodes += [(M[0] // 2, 0, 0), (0, M[1] // 2, M[2]), (M[0], M[1], M[2] // 2), (M[0] // 2, M[1] // 2, 0),
              (M[0] // 2, M[1], M[2] // 2), (1, 1, 1), (M[0] - 1, M[1] - 1, M[2] - 1), (31, 32, 16),
              (32, 3, 1), (993, 1000, 31)]
    nodes += [tuple(int(rng.integers(0, v + 1)) for v in M) for _ in range(n_random)]
    return nodes


def _gather(h, nodes):
    import torch
    idx = torch.tensor(nodes, dtype=torch.long, device=h.device)
    return h[idx[:, 0], idx[:, 1], idx[:, 2]].double().cpu().numpy()


@pytest.mark.parametrize("n", [N, N_MAX])
@pytest.mark.parametrize("precision", [0, 1])
def test_local_terms_at_sampled_nodes(nmgb, sampled, precision, n):
    import torch
    p = _problem(n)
    terms = inp.EXCH | inp.ANIS
    m = rounded(p.m0, precision)
    me = gpu_mesh(nmgb, p, precision)
    h = me.h_eff(torch.from_numpy(m).cuda(), terms, 0.0)
    nodes = _sample_nodes(1, n)
    got = _gather(h, nodes)
    me.close()
    del h
    ref = np.array([sampled.local_field_at(n, p.dx, _material(p), m, nd, terms) for nd in nodes])
    assert rel_l2(got, ref) < TOL[precision]
    assert np.abs(got - ref).max() <= 10 * TOL[precision] * np.abs(ref).max()


@pytest.mark.parametrize("n", [N, N_MAX])
@pytest.mark.parametrize("precision", [0, 1])
def test_sparse_demag_at_sampled_nodes(nmgb, sampled, precision, n):
    import torch
    p = _problem(n)
    z = n[2]
    rng = np.random.default_rng(2)
    m = np.zeros(p.nodes + (3,))
    for nd in [(1, 1, 1), (2, 1, 1), (1, 2, 1), (2, 2, 1), (1, 1, 2), (2, 1, 2), (1, 2, 2), (2, 2, 2),
               (700, 300, 20)]:
        m[nd] = inp.unit_vector(rng)
    m = rounded(m, precision)
    near = [(a, b, c) for a in (0, 2, 4) for b in (0, 2, 3) for c in (0, 1, 3)]
    near += [(700 + a, 300 + b, 20 + c) for a in (-1, 0, 2) for b in (-2, 0, 1) for c in (-1, 0, 1)]
    far = [(40, 30, 10), (300, 200, 16), (1024, 1024, z), (1024, 0, 0), (0, 1024, z), (512, 512, 0),
           (1020, 3, 2), (3, 1021, z - 2), (500, 600, z)]
    nodes = near + far
    me = gpu_mesh(nmgb, p, precision)
    h = me.h_eff(torch.from_numpy(m).cuda(), inp.DEMAG, 0.0)
    got = _gather(h, nodes)
    me.close()
    del h
    ref = sampled.demag_at_nodes(n, p.dx, p.Ms, m, nodes)
    assert rel_l2(got, ref) < TOL[precision]
    # every sample, the far ones included, is right to the global accuracy: a periodic image of the
    # corner source (a padding error) would put a field of the near-source size at the far corners
    assert np.abs(got - ref).max() <= TOL[precision] * np.abs(ref).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_dp5_step_at_sampled_nodes(nmgb, sampled, precision):
    p = _problem(N)
    terms = inp.EXCH | inp.ANIS
    dt = 2e-14
    me = gpu_mesh(nmgb, p, precision)
    me.set_terms(terms)
    me.set_state(p.m0, 0.0, dt)
    me.run_steps(1, nmgb.DP54, 1e3, 1e3)
    m1, t1, _ = me.get_state()
    acc, rej, _ = me.counters()
    me.close()
    assert acc == 1 and rej == 0 and abs(t1 - dt) <= 1e-12 * dt
    assert np.abs(np.linalg.norm(m1, axis=-1) - 1).max() < 1e-12
    nodes = _sample_nodes(3, N, n_random=12)
    ref = np.array([sampled.dp5_step_at(N, p.dx, _material(p), p.m0, nd, terms, dt) for nd in nodes])
    got = np.array([m1[nd] for nd in nodes])
    m0 = np.array([p.m0[nd] for nd in nodes])
    assert np.abs(ref - m0).max() > 1e-3  # the step moves m
    assert rel_l2(got - m0, ref - m0) < TOL[precision]


@pytest.mark.parametrize("n", [N, N_MAX])
@pytest.mark.parametrize("precision", [0, 1])
def test_uniform_m_mean_demag_is_prism_factor(nmgb, precision, n):
    import torch
    p = inp.throughput(n, seed=0, with_m0=False)
    mu = np.array([0.3, -0.5, 0.8])
    mu /= np.linalg.norm(mu)
    me = gpu_mesh(nmgb, p, precision)
    dtype = torch.float32 if precision == 0 else torch.float64
    m = torch.tensor(mu, dtype=dtype, device="cuda").expand(p.nodes + (3,)).contiguous()
    h = me.h_eff(m, inp.DEMAG, 0.0)
    # lumped mass of a uniform material: proportional to the number of cells around the node
    cnt = [torch.full((v + 1,), 2.0, dtype=torch.float64, device="cuda") for v in n]
    for c in cnt:
        c[0] = c[-1] = 1.0
    w = cnt[0][:, None, None] * cnt[1][None, :, None] * cnt[2][None, None, :]
    mean = ((h.double() * w[..., None]).sum(dim=(0, 1, 2)) / w.sum()).cpu().numpy()
    me.close()
    ref = -p.Ms * aharoni_factors(np.array(n) * np.array(p.dx)) * mu
    tol = {0: 1e-5, 1: 1e-11}[precision]
    assert np.abs(mean - ref).max() <= tol * p.Ms


@pytest.mark.parametrize("terms_name", ["DEMAG", "ALL"])
def test_fp32_dense_random_state_matches_fp64_path(nmgb, terms_name):
    """The state the benchmark integrates (dense random unit m on 1024x1024x32 cells): the FP32 field,
    demag alone and all terms, against the FP64 path on the same FP32-rounded input (the FP64 path
    matches the oracle at 1e-12 on the sampled outputs above and on every small mesh).  Bar: rel-L2 <=
    1e-5, as for the small meshes."""
    import torch
    p = _problem(N)
    terms = getattr(nmgb, terms_name)
    m = torch.tensor(rounded(p.m0, 0), dtype=torch.float64, device="cuda")
    out = {}
    for precision in (1, 0):
        me = gpu_mesh(nmgb, p, precision)
        h = me.h_eff(m.to(me.dtype), terms, 0.0)
        out[precision] = h.double()
        del h
        me.close()
        torch.cuda.empty_cache()
    err = (torch.linalg.vector_norm(out[0] - out[1]) / torch.linalg.vector_norm(out[1])).item()
    assert err <= 1e-5, err


@pytest.mark.parametrize("n", [(256, 256, 8), (512, 512, 16)])
@pytest.mark.parametrize("precision", [0, 1])
def test_sparse_demag_at_sweep_sizes(nmgb, sampled, precision, n):
    """The throughput sweep's smaller cuboids instantiate the y passes at 512- and 1024-point lines
    (8 or 4 kx columns per tile, padded tile rows) and the z convolution at 16 and 32 points, which the
    small meshes and the 1024x1024 meshes above do not: a sparse source (a 2x2x2 node block at a corner
    and one interior node) against the oracle's direct sum at nodes next to the sources and far away."""
    import torch
    p = _problem(n)
    z = n[2]
    src = (int(0.68 * n[0]), int(0.29 * n[1]), int(0.6 * z))
    rng = np.random.default_rng(5)
    m = np.zeros(p.nodes + (3,))
    for nd in [(1, 1, 1), (2, 1, 1), (1, 2, 1), (2, 2, 1), (1, 1, 2), (2, 1, 2), (1, 2, 2), (2, 2, 2), src]:
        m[nd] = inp.unit_vector(rng)
    m = rounded(m, precision)
    near = [(a, b, c) for a in (0, 2, 4) for b in (0, 2, 3) for c in (0, 1, 3)]
    near += [(src[0] + a, src[1] + b, src[2] + c) for a in (-1, 0, 2) for b in (-2, 0, 1) for c in (-1, 0, 1)]
    far = [(n[0], n[1], z), (n[0], 0, 0), (0, n[1], z), (n[0] // 2, n[1] // 2, 0), (n[0] - 4, 3, 2),
           (3, n[1] - 3, z - 2), (n[0] // 3, n[1] // 2 + 7, z)]
    nodes = near + far
    me = gpu_mesh(nmgb, p, precision)
    h = me.h_eff(torch.from_numpy(m).cuda(), inp.DEMAG, 0.0)
    got = _gather(h, nodes)
    me.close()
    del h
    ref = sampled.demag_at_nodes(n, p.dx, p.Ms, m, nodes)
    assert rel_l2(got, ref) < TOL[precision]
    assert np.abs(got - ref).max() <= TOL[precision] * np.abs(ref).max()
