"""Pins of the species-advection reference (oracle/advection.py, Sec. 2.1).

* The paper's 1-D test (Sec. 4.1): 128 periodic zones on [-0.5, 0.5], rho = 1, v = 1,
  species A, A2, AB, B over elements A and B with the printed step-plus-linear
  profiles, advected to t = 1: the projected PLM keeps every cell's element abundances
  to machine precision, the unprojected PLM does not (the paper's ~1e-3 per ~300
  steps), donor cell does.
* Linear data are reconstructed exactly (second order); the limited slope is zero at
  extrema and never steeper than van Leer's; a smooth profile converges at second
  order; a step profile keeps its total variation; data with a sign change of the
  slope at every cell reduce to donor cell.
"""
import numpy as np
import pytest

from oracle import advection as A

COUNTS = np.array([[1, 0], [2, 0], [1, 1], [0, 1]])   # A, A2, AB, B over elements (A, B)


def _paper_profiles(L=128):
    dx = 1.0 / L
    x = -0.5 + (np.arange(L) + 0.5) * dx
    th_m, th_p = (x < 0).astype(float), (x > 0).astype(float)
    n = np.stack([0.49 * th_m + 0.05 * th_p + 0.2 * x,
                  0.20 * th_m + 0.40 * th_p - 0.1 * x,
                  0.01 * th_m + 0.05 * th_p,
                  0.09 * th_m + 0.05 * th_p])[:, None, :]
    return n, dx


def _run(n, dx, steps, P=None, donor_cell=False, cfl=0.5):
    rho = np.ones(n.shape[1:])
    flux = np.ones(n.shape[1:])          # rho v = 1 at every interface
    for _ in range(steps):
        n = A.advect_ssprk2(n, rho, flux, cfl, dx, P, donor_cell)
    return n


def test_paper_advection_conserves_elements_with_projection():
    n0, dx = _paper_profiles()
    P = A.element_projector(COUNTS)
    elem0 = np.einsum("se,s...->e...", COUNTS, n0)          # 0.9 (A) and 0.1 (B) in every cell
    assert np.allclose(elem0[0], 0.9, rtol=1e-15) and np.allclose(elem0[1], 0.1, rtol=1e-15)
    n = _run(n0, dx, 256, P)                                   # t = 1 at CFL 0.5
    elem = np.einsum("se,s...->e...", COUNTS, n)
    assert np.max(np.abs(elem[0] - 0.9) / 0.9) <= 2e-15
    assert np.max(np.abs(elem[1] - 0.1) / 0.1) <= 2e-15
    # every species' total is a telescoping sum of fluxes
    assert np.allclose(n.sum(axis=-1), n0.sum(axis=-1), rtol=1e-14, atol=0)
    # PLM beats donor cell on the same test (less diffusion), compared with the exact
    # solution (the initial profile, one period later)
    dc = _run(n0, dx, 256, donor_cell=True)
    assert np.abs(n - n0).sum() < 0.6 * np.abs(dc - n0).sum()
    dc_elem = np.einsum("se,s...->e...", COUNTS, dc)
    assert np.max(np.abs(dc_elem[0] - 0.9) / 0.9) <= 2e-15


def test_paper_advection_without_projection_violates_elements():
    n0, dx = _paper_profiles()
    n = _run(n0, dx, 256, P=None)
    elem = np.einsum("se,s...->e...", COUNTS, n)
    assert np.max(np.abs(elem[0] - 0.9) / 0.9) > 1e-4


def test_projector_is_the_null_space_projector():
    P = A.element_projector(COUNTS)
    N = COUNTS.T.astype(float)
    assert np.allclose(P @ P, P, atol=1e-15) and np.allclose(P, P.T, atol=1e-15)
    assert np.allclose(N @ P, 0.0, atol=1e-15)
    assert np.linalg.matrix_rank(P) == COUNTS.shape[0] - np.linalg.matrix_rank(N)


def test_linear_data_reconstructed_exactly():
    L, dx = 32, 0.1
    x = (2.0 + 0.3 * np.arange(L) * dx)[None, None, :]
    left, right = A.interface_states(x, dx)
    exact = 2.0 + 0.3 * (np.arange(L) - 0.5) * dx          # value at the interface j-1/2
    inner = slice(2, L - 1)
    assert np.allclose(left[0, 0, inner], exact[inner], rtol=1e-14)
    assert np.allclose(right[0, 0, inner], exact[inner], rtol=1e-14)


def test_limited_slope_properties():
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal(10000), rng.standard_normal(10000)
    s = A.limited_slope(a, b)
    assert np.all(s[a * b <= 0] == 0.0)
    same = a * b > 0
    vl = 2 * a[same] * b[same] / (a[same] + b[same])       # van Leer's harmonic slope
    assert np.all(np.abs(s[same]) <= np.abs(vl) * (1 + 1e-15))
    assert np.all(np.abs(s[same]) <= np.abs(b[same]) * (1 + 1e-15))
    assert np.all(np.sign(s[same]) == np.sign(a[same]))
    assert np.allclose(A.limited_slope(np.array([0.7]), np.array([0.7])), 0.7, rtol=1e-15)


def test_smooth_profile_second_order():
    errs = []
    for L in (64, 128, 256):
        dx = 1.0 / L
        xc = (np.arange(L) + 0.5) * dx
        n0 = (1.5 + np.sin(2 * np.pi * xc))[None, None, :]
        n = _run(n0, dx, 2 * L, cfl=0.5)                     # one period
        errs.append(np.abs(n - n0).sum() * dx)
    assert errs[0] / errs[1] > 2.8 and errs[1] / errs[2] > 2.8, errs


def test_step_profile_total_variation_does_not_grow():
    L, dx = 100, 0.01
    n = np.where(np.arange(L) < 50, 1.0, 0.2)[None, None, :].astype(float)
    rho, flux = np.ones((1, L)), np.ones((1, L))
    tv = np.abs(np.diff(n, axis=-1)).sum() + abs(n[0, 0, 0] - n[0, 0, -1])
    for _ in range(60):
        n = A.advect_ssprk2(n, rho, flux, 0.4, dx)
        tv_new = np.abs(np.diff(n, axis=-1)).sum() + abs(n[0, 0, 0] - n[0, 0, -1])
        assert tv_new <= tv * (1 + 1e-13)
        tv = tv_new


def test_alternating_data_reduce_to_donor_cell():
    L = 40
    n = (1.0 + 0.5 * (-1.0) ** np.arange(L))[None, None, :]
    rho = np.ones((1, L))
    flux = np.where(np.arange(L) % 3 == 0, -0.7, 1.3)[None, :]
    F = A.species_fluxes(n, rho, flux, 0.1)
    Fd = A.species_fluxes(n, rho, flux, 0.1, donor_cell=True)
    assert np.array_equal(F, Fd)
