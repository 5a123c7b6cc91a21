"""Stoichiometry-compatible species advection (Sec. 2.1.3) on the GPU against the numpy
reference (oracle/advection.py): the paper's 1-D test and random multi-line data on the
workload networks (10 and 64 species), both flux directions, with and without the
projection; element abundances to machine precision with it."""
import numpy as np
import pytest

from oracle import advection as A
from paper_2504_04941_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_04941_gb300 import build, kt as ktm
    build.build()
    return ktm


def _four_species_network():
    return I._irreversible("adv4", ["A", "A2", "AB", "B"], ["A", "B"], [1.0, 2.0, 2.0, 1.0], [0.0] * 4,
                           [1.0] * 4, [[1, 0], [2, 0], [1, 1], [0, 1]], 0, 300.0, 10.0, 1e5,
                           [((0, 0), (1,), 1.0, 0.0, 0.0, -1)])


def test_paper_advection_test_matches_reference(kt):
    import torch
    netw = _four_species_network()
    net = kt.Network(netw)
    L = 128
    dx = 1.0 / L
    x = -0.5 + (np.arange(L) + 0.5) * dx
    m, p = (x < 0).astype(float), (x > 0).astype(float)
    n0 = np.stack([0.49 * m + 0.05 * p + 0.2 * x, 0.20 * m + 0.40 * p - 0.1 * x,
                   0.01 * m + 0.05 * p, 0.09 * m + 0.05 * p])[:, None, :]
    rho, flux = np.ones((1, L)), np.ones((1, L))
    P = A.element_projector(netw.counts)
    ref = n0.copy()
    g = torch.from_numpy(n0).cuda()
    rt, ft = torch.from_numpy(rho).cuda(), torch.from_numpy(flux).cuda()
    for _ in range(256):
        ref = A.advect_ssprk2(ref, rho, flux, 0.5, dx, P)
        g = kt.advect_ssprk2(net, g, rt, ft, dx, 0.5)
    got = g.cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-14)
    elem = np.einsum("se,s...->e...", netw.counts, got)
    assert np.max(np.abs(elem[0] - 0.9) / 0.9) <= 2e-15 and np.max(np.abs(elem[1] - 0.1) / 0.1) <= 2e-15


@pytest.mark.parametrize("wid,nl,L,project", [(2, 7, 300, True), (5, 3, 257, True), (5, 2, 100, False)])
def test_random_lines_match_reference(kt, wid, nl, L, project):
    import torch
    netw = I.network(wid)
    net = kt.Network(netw)
    rng = np.random.default_rng(wid * 100 + L)
    n = 10.0 ** rng.uniform(-8, 0, (netw.ns, nl, L))
    rho = rng.uniform(0.5, 2.0, (nl, L))
    flux = rng.uniform(-1.0, 1.0, (nl, L))
    dx, dtdx = 0.37, 0.3
    P = A.element_projector(netw.counts) if project else None
    ref = A.advect_step(n, rho, flux, dtdx, dx, P)
    got = kt.advect_sweep(net, *(torch.from_numpy(a).cuda() for a in (n, rho, flux)), dx, dtdx,
                          project=project).cpu().numpy()
    scale = np.abs(n) + dtdx * np.abs(n / rho[None]).max() * 2
    assert np.all(np.abs(got - ref) <= 1e-12 * scale)
    base = 10.0 ** rng.uniform(-8, 0, n.shape)
    ref2 = 0.5 * base + 0.5 * A.advect_step(n, rho, flux, dtdx, dx, P)
    got2 = kt.advect_sweep(net, *(torch.from_numpy(a).cuda() for a in (n, rho, flux)), dx, dtdx, alpha=0.5,
                           n_base=torch.from_numpy(base).cuda(), project=project).cpu().numpy()
    assert np.all(np.abs(got2 - ref2) <= 1e-12 * (scale + base))
