"""Pins of the Cartesian ray-tracing reference (oracle/raytrace.py, Sec. 3).

* photon bookkeeping: absorbed + escaped = emitted for every ray and bin;
* geometry: the summed path lengths equal the distance from the source to the box
  boundary along the ray (closed form);
* Beer-Lambert: a ray through a uniform medium deposits N0 e^{-kappa x_i}(1 - e^{-kappa dx})
  in the cell starting at x_i, and F_eff takes the factor (1 - e^-tau)/tau;
* an isotropic source in vacuum gives F_eff ~ L / (4 pi r^2) on spherical shells, and
  the optically thin F_eff integrates to the rays' photons times their path lengths.
"""
import math

import numpy as np

from oracle import raytrace as R


def test_fibonacci_directions_unit_and_isotropic():
    d = R.fibonacci_directions(4000)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    assert np.all(np.abs(d.mean(axis=0)) < 2e-3)
    assert np.allclose((d[:, :, None] * d[:, None, :]).mean(axis=0), np.eye(3) / 3, atol=2e-3)


def test_photon_bookkeeping_and_path_length():
    rng = np.random.default_rng(0)
    shape, h = (7, 5, 6), (0.3, 0.5, 0.4)
    kappa = rng.uniform(0.0, 3.0, (2,) + shape)
    src = np.array([1.11, 1.23, 0.97])
    org, dirs, n0 = R.point_source_rays(src, [2.0, 5.0], 0.1, 300)
    feff, ab, esc, length = R.trace(shape, h, kappa, org, dirs, n0, 0.1)
    assert np.allclose(ab.sum(axis=(1, 2, 3)) + esc.sum(axis=0), n0.sum(axis=0), rtol=1e-13)
    box = np.array(shape) * np.array(h)
    for q in range(len(dirs)):
        d = dirs[q]
        t = [((box[a] if d[a] > 0 else 0.0) - src[a]) / d[a] for a in range(3) if d[a] != 0.0]
        assert abs(length[q] - min(t)) <= 1e-12 * min(t)


def test_beer_lambert_along_a_ray():
    shape, h = (10, 1, 1), (0.25, 1.0, 1.0)
    k = 1.7
    kappa = np.full((1,) + shape, k)
    org = np.array([[0.0, 0.5, 0.5]])
    d = np.array([[1.0, 0.0, 0.0]])
    n0 = np.array([[3.0]])
    dt = 2.0
    feff, ab, esc, length = R.trace(shape, h, kappa, org, d, n0, dt)
    xi = np.arange(10) * 0.25
    exact = 3.0 * np.exp(-k * xi) * (1 - math.exp(-k * 0.25))
    assert np.allclose(ab[0, :, 0, 0], exact, rtol=1e-14)
    tau = k * 0.25
    fe = 3.0 * np.exp(-k * xi) * 0.25 / (0.25 * dt) * (1 - math.exp(-tau)) / tau
    assert np.allclose(feff[0, :, 0, 0], fe, rtol=1e-14)
    assert esc[0, 0] == np.float64(3.0 * math.exp(-k * 2.5)) or abs(esc[0, 0] / (3.0 * math.exp(-k * 2.5)) - 1) < 1e-14


def test_vacuum_point_source_inverse_square_and_thin_limit():
    n, hh = 24, 1.0
    kappa = np.zeros((1, n, n, n))
    src = np.array([12.03, 11.97, 12.01])
    L, dt, nr = 1.0, 1.0, 60000
    org, dirs, n0 = R.point_source_rays(src, [L], dt, nr)
    feff, ab, esc, length = R.trace((n, n, n), (hh, hh, hh), kappa, org, dirs, n0, dt)
    assert np.all(ab == 0.0) and np.allclose(esc[:, 0], n0[:, 0])
    assert math.isclose(feff.sum() * hh ** 3 * dt, (n0[:, 0] * length).sum(), rel_tol=1e-12)
    c = (np.arange(n) + 0.5) * hh
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt((X - src[0]) ** 2 + (Y - src[1]) ** 2 + (Z - src[2]) ** 2)
    for r0 in (5.0, 8.0, 10.5):
        shell = np.abs(r - r0) < 0.5
        ratio = feff[0][shell] / (L / (4 * math.pi * r[shell] ** 2))
        assert abs(ratio.mean() - 1.0) < 0.05, (r0, ratio.mean())
