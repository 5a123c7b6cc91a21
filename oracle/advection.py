"""FP64 reference of the stoichiometry-compatible species advection (Sec. 2.1).

TEST INFRASTRUCTURE: only tests, the package smoke check and the benchmark's
CPU-baseline / reference legs use this module.  It shares nothing with the CUDA path.

One directional sweep on lines of cells with uniform spacing dx and periodic ends:

* relative abundances x^s = n^s / rho per cell (Eq. method-flux-sp);
* piecewise-linear reconstruction (Eq. method-plm-general): forward and backward
  slopes a = (x_{j+1} - x_j)/dx, b = (x_j - x_{j-1})/dx of each cell j, limited by the
  modified van Leer function of Eq. method-sto-plm-def
      phi(a, b, c, d) = 0 if a b <= 0, else min(2|a|/(|a|+|b|), 2c/(c+d)) sgn(a),
  read as multiplying |b| (the printed phi is dimensionless), with the geometric
  factors c_f = c_b = 2 of a uniform grid (the printed c_f carries an index typo;
  read as (xi_{j+1} - xi_j)/(xi_{j+1/2} - xi_j)); so the limited slope is
  sgn(a) min(2|a||b|/(|a|+|b|), |b|);
* corrections chi = slope * (xi_interface - xi_cell), projected onto the null space of
  the element matrix N (Eq. method-sto-plm-proj): P = I - V_r V_r^T with V_r the right
  singular vectors of N of nonzero singular value (the paper's "V V^T" read as the
  projector onto the stoichiometric space S = null(N), in which N P chi = 0);
* upwind choice of the left or right state by the sign of the mass flux
  (Eq. method-sto-plm-recon) and species fluxes F^s = x^s F^rho;
* conservative update n^s_j -= dt/dx (F^s_{j+1/2} - F^s_{j-1/2}).
"""
from __future__ import annotations

import numpy as np


def element_projector(counts: np.ndarray) -> np.ndarray:
    """P = I - V_r V_r^T for the element matrix N = counts^T [n_elements, n_species]."""
    N = np.asarray(counts, float).T
    U, S, Vt = np.linalg.svd(N)
    r = int(np.sum(S > S.max() * 1e-12)) if S.size else 0
    Vr = Vt[:r].T
    return np.eye(N.shape[1]) - Vr @ Vr.T


def limited_slope(a: np.ndarray, b: np.ndarray, c: float = 2.0, d: float = 2.0) -> np.ndarray:
    """phi(a, b, c, d) |b| (see the module docstring)."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    out = np.zeros(np.broadcast(a, b).shape)
    ok = a * b > 0
    aa, bb = np.abs(a[ok]), np.abs(b[ok])
    phi = np.minimum(2.0 * aa / (aa + bb), 2.0 * c / (c + d)) * np.sign(a[ok])
    out[ok] = phi * bb
    return out


def interface_states(x: np.ndarray, dx: float, P=None):
    """x [n_species, n_lines, L]: left and right states at every interface j-1/2
    (index j): the left state from cell j-1, the right state from cell j."""
    fwd = (np.roll(x, -1, axis=-1) - x) / dx
    bwd = (x - np.roll(x, 1, axis=-1)) / dx
    s = limited_slope(fwd, bwd)
    chi_hi = 0.5 * dx * s                   # correction at a cell's upper interface
    chi_lo = -0.5 * dx * s                  # ... at its lower interface
    if P is not None:
        chi_hi = np.einsum("sr,r...->s...", P, chi_hi)
        chi_lo = np.einsum("sr,r...->s...", P, chi_lo)
    upper = x + chi_hi                      # state of cell j at j+1/2
    lower = x + chi_lo                      # state of cell j at j-1/2
    left = np.roll(upper, 1, axis=-1)       # at j-1/2, from cell j-1
    right = lower
    return left, right


def species_fluxes(n: np.ndarray, rho: np.ndarray, mass_flux: np.ndarray, dx: float, P=None,
                   donor_cell: bool = False) -> np.ndarray:
    """F^s at every interface j-1/2; n [n_species, n_lines, L], rho and mass_flux
    [n_lines, L] (mass_flux[j] at j-1/2)."""
    x = n / rho[None]
    if donor_cell:
        left, right = np.roll(x, 1, axis=-1), x
    else:
        left, right = interface_states(x, dx, P)
    xs = np.where(mass_flux[None] > 0, left, right)
    return xs * mass_flux[None]


def advect_step(n, rho, mass_flux, dtdx: float, dx: float, P=None, donor_cell: bool = False):
    """One forward-Euler sweep: n - dt/dx (F_{j+1/2} - F_{j-1/2})."""
    F = species_fluxes(n, rho, mass_flux, dx, P, donor_cell)
    return n - dtdx * (np.roll(F, -1, axis=-1) - F)


def advect_ssprk2(n, rho, mass_flux, dtdx: float, dx: float, P=None, donor_cell: bool = False):
    """Two-stage strong-stability-preserving Runge-Kutta step (Shu & Osher) of the
    same sweep (constant rho and mass flux)."""
    n1 = advect_step(n, rho, mass_flux, dtdx, dx, P, donor_cell)
    n2 = advect_step(n1, rho, mass_flux, dtdx, dx, P, donor_cell)
    return 0.5 * (n + n2)
