"""FP64 reference of ray tracing on a Cartesian mesh with Beer-Lambert deposition (Sec. 3).

TEST INFRASTRUCTURE: only tests, the package smoke check and the benchmark's
CPU-baseline / reference legs use this module.  It shares nothing with the CUDA path.

A ray starts at x0 with direction d (|d| = 1) and photon counts N (one per energy bin).
In the cell it is in, the exit length is the smallest positive root of the face
equations of Eq. cart-dl, one per axis: d_a dl + (x_in,a - x_face,a) = 0 with the face
the ray moves towards (no root when d_a = 0).  In that cell, with tau = kappa dl (kappa
= 1/lambda_abs, the cell's inverse absorption length per bin):
    F_eff += N dl / (dV dt) (1 - e^-tau)/tau          (Eq. method-rad-equiv-flux)
    absorbed += N (1 - e^-tau)
    N <- N e^-tau                                    (Eq. method-rt-abs)
then the ray moves to the exit point and into the neighbour across that face, until it
leaves the box.  An isotropic point source of spectral luminosity L emits n_rays rays
on a Fibonacci lattice of directions, each of solid angle 4 pi / n_rays, carrying
N = L (dOmega / 4 pi) dt photons (Eq. method-rt-ph-num).
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN_ANGLE = math.pi * (3.0 - math.sqrt(5.0))


def fibonacci_directions(n: int) -> np.ndarray:
    """n unit vectors of near-equal solid angle: z_k = 1 - (2k+1)/n, azimuth k * golden angle."""
    k = np.arange(n, dtype=float)
    z = 1.0 - (2.0 * k + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ph = k * GOLDEN_ANGLE
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], axis=1)


def point_source_rays(src, lum, dt: float, n: int):
    """Origins, directions and photon counts [n, nbins] of an isotropic point source."""
    d = fibonacci_directions(n)
    n0 = np.tile(np.asarray(lum, float) * dt / n, (n, 1))
    return np.tile(np.asarray(src, float), (n, 1)), d, n0


def trace(shape, spacing, kappa: np.ndarray, origins, dirs, n0, dt: float):
    """kappa [nbins, nx, ny, nz]; returns (F_eff, absorbed) [nbins, nx, ny, nz] and the
    escaping photon counts [n_rays, nbins] and path lengths inside the box [n_rays]."""
    shape = tuple(int(v) for v in shape)
    h = np.asarray(spacing, float)
    nb = kappa.shape[0]
    dV = float(np.prod(h))
    feff = np.zeros((nb,) + shape)
    absorbed = np.zeros((nb,) + shape)
    escaped = np.zeros((len(origins), nb))
    length = np.zeros(len(origins))
    for q in range(len(origins)):
        x = np.array(origins[q], float)
        d = np.array(dirs[q], float)
        N = np.array(n0[q], float)
        cell = [int(math.floor(x[a] / h[a])) for a in range(3)]
        if any(c < 0 or c >= s for c, s in zip(cell, shape)):
            escaped[q] = N
            continue
        while all(0 <= c < s for c, s in zip(cell, shape)):
            roots = []
            for a in range(3):
                if d[a] > 0.0:
                    face = (cell[a] + 1) * h[a]
                elif d[a] < 0.0:
                    face = cell[a] * h[a]
                else:
                    continue
                dl = (face - x[a]) / d[a]
                roots.append((dl, a))
            dl, axis = min((r for r in roots if r[0] >= 0.0), key=lambda r: r[0])
            i, j, k = cell
            tau = kappa[:, i, j, k] * dl
            phi = np.where(tau > 0.0, -np.expm1(-tau) / np.where(tau > 0.0, tau, 1.0), 1.0)
            feff[:, i, j, k] += N * dl / (dV * dt) * phi
            att = np.exp(-tau)
            absorbed[:, i, j, k] += N * (1.0 - att)
            N = N * att
            length[q] += dl
            x = x + dl * d
            cell[axis] += 1 if d[axis] > 0.0 else -1
        escaped[q] = N
    return feff, absorbed, escaped, length
