"""Cartesian ray tracing with Beer-Lambert deposition (Sec. 3) on the GPU against the
FP64 reference (oracle/raytrace.py): an isotropic point source in an absorbing,
non-uniform medium with two energy bins; photon bookkeeping to rounding."""
import numpy as np
import pytest

from oracle import raytrace as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_04941_gb300 import build, kt as ktm
    build.build()
    return ktm


@pytest.mark.parametrize("shape,nrays", [((9, 7, 8), 500), ((33, 17, 24), 4000)])
def test_point_source_matches_reference(kt, shape, nrays):
    import torch
    rng = np.random.default_rng(sum(shape))
    h = (0.3, 0.45, 0.37)
    kappa = rng.uniform(0.0, 2.5, (2,) + shape)
    kappa[:, ::3] *= 0.01                       # optically thin slabs between thick ones
    src = np.array([shape[0] * h[0] * 0.43, shape[1] * h[1] * 0.51, shape[2] * h[2] * 0.47])
    lum, dt = [3.0, 0.5], 0.2
    org, dirs, n0 = R.point_source_rays(src, lum, dt, nrays)
    fo, ao, eo, _ = R.trace(shape, h, kappa, org, dirs, n0, dt)
    go, gd, gn = kt.point_source_rays(src, lum, dt, nrays)
    assert np.allclose(gd.cpu().numpy(), dirs, rtol=0, atol=1e-14)
    assert np.allclose(gn.cpu().numpy(), n0, rtol=1e-15, atol=0)
    f, a, e = kt.raytrace(h, torch.from_numpy(kappa).cuda(), go, gd, gn, dt)
    f, a, e = f.cpu().numpy(), a.cpu().numpy(), e.cpu().numpy()
    assert np.allclose(f, fo, rtol=1e-11, atol=1e-13 * fo.max())
    assert np.allclose(a, ao, rtol=1e-11, atol=1e-13 * ao.max())
    assert np.allclose(e, eo, rtol=1e-11, atol=1e-14)
    assert np.allclose(a.sum(axis=(1, 2, 3)) + e.sum(axis=0), gn.cpu().numpy().sum(axis=0), rtol=1e-13)
