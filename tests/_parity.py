"""Comparison rule between the CUDA path and the FP64 oracle.

Per cell and species: |y_gpu - y_ora| <= 1e-6 |y_ora| when y_ora > 1e-20; below that,
|y_gpu| <= 1e-20 + 1e-6 max_s y_ora.  Temperature: 1e-8 relative.  Status codes are
integers and must match exactly.

The step-doubling accept test (err <= 1) is a discontinuous function of rounding, so a
cell whose accepted sub-step count differs from the oracle's ("flip") follows another,
equally valid, sequence of sub-steps.  Such a cell is excused from the 1e-6 rule only
if it is as accurate as the oracle itself: both are measured against a tight oracle
run of the same cell (rtol 1e-9), and the GPU's error must stay within
10 rtol + 2 e_ora, where e_ora is the oracle's own largest relative error on that cell
at the working tolerance.  (With an error proportional to rtol this is the plain
"within 10 rtol of the tight run"; the first-order scheme's global error is ~sqrt(rtol),
which the e_ora term measures per cell instead of assuming.)  Flips must also stay
rare: at most 1 % of the cells (one cell on small batches).

Species below the integration's own absolute tolerance atol (atol_cells, per cell;
only the networks whose atol scales with the cell's density set it above the 1e-20
floor) carry no relative accuracy requirement in the integration itself: there the
oracle at rtol 1e-6 differs from a tight run by up to 100 %, and a one-ulp change of
the first step moves them by ~3e-7 (measured on the radiation network).  They are
compared absolutely, |y_gpu - y_ora| <= 1e-6 atol.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np

Y_RTOL = 1e-6
Y_FLOOR = 1e-20
T_RTOL = 1e-8
TIGHT_RTOL = 1e-9


@dataclasses.dataclass
class Report:
    ncells: int
    n_flip: int
    max_rel_y: float          # over non-flipped cells, species above the floor
    max_rel_T: float
    bad_small: int            # species below the floor violating the small-value rule
    flip_max_rel_y: float     # flipped cells against the oracle at the working tolerance
    flip_bad: int             # flipped cells not excused by the tight-run check
    flip_checked: bool        # whether the flipped cells were checked against a tight run
    status_mismatch: int
    n_failed_cells: int       # non-flipped cells violating the rule

    def ok(self, max_flip_frac: float = 0.01) -> bool:
        flips_fine = self.n_flip == 0 or (self.flip_checked and self.flip_bad == 0)
        return (self.status_mismatch == 0 and self.n_failed_cells == 0 and flips_fine and
                self.n_flip <= max(1, int(max_flip_frac * self.ncells)))


def _rel(a, ref):
    big = ref > Y_FLOOR
    return np.where(big, np.abs(a - ref) / np.where(big, np.abs(ref), 1.0), 0.0)


def compare(gpu: dict, ora: dict, energy: int, rtol: float = 1e-6,
            tight: Optional[Callable[[np.ndarray], dict]] = None, atol_cells=None) -> Report:
    """gpu, ora: dicts of y [ns, ncells], T, status, nsub over the same cells.
    tight(idx) returns the oracle at rtol 1e-9 on cells idx (dict with y, T); it is
    called only when some cell flipped.  atol_cells [ncells]: the integration's absolute
    tolerance per cell, when it exceeds the 1e-20 floor."""
    yg, yo = np.asarray(gpu["y"], float), np.asarray(ora["y"], float)
    Tg, To = np.asarray(gpu["T"], float), np.asarray(ora["T"], float)
    nc = yo.shape[1]
    status_mismatch = int(np.sum(np.asarray(gpu["status"]) != np.asarray(ora["status"])))
    flip = np.asarray(gpu["nsub"]) != np.asarray(ora["nsub"])
    big = yo > Y_FLOOR
    ymax = yo.max(axis=0, initial=0.0)
    small_bad = (~big) & (np.abs(yg) > Y_FLOOR + Y_RTOL * ymax[None, :])
    if atol_cells is not None:
        at = np.maximum(np.asarray(atol_cells, float), Y_FLOOR)[None, :]
        sub = big & (yo <= at)                   # controlled absolutely by the integration
        small_bad |= sub & (np.abs(yg - yo) > Y_RTOL * at)
        big &= ~sub
    rel = np.where(big, np.abs(yg - yo) / np.where(big, np.abs(yo), 1.0), 0.0)
    relT = np.abs(Tg - To) / np.abs(To)
    cell_bad = (rel > Y_RTOL).any(axis=0) | small_bad.any(axis=0)
    if energy:
        cell_bad |= relT > T_RTOL
    keep = ~flip
    flip_bad, checked = 0, False
    idx = np.flatnonzero(flip)
    if idx.size and tight is not None:
        t = tight(idx)
        yt, Tt = np.asarray(t["y"], float), np.asarray(t["T"], float)
        e_ora = _rel(yo[:, idx], yt).max(axis=0, initial=0.0)
        e_gpu = _rel(yg[:, idx], yt).max(axis=0, initial=0.0)
        if energy:
            e_ora = np.maximum(e_ora, np.abs(To[idx] - Tt) / Tt)
            e_gpu = np.maximum(e_gpu, np.abs(Tg[idx] - Tt) / Tt)
        flip_bad = int(np.sum(e_gpu > 10.0 * rtol + 2.0 * e_ora))
        checked = True
    return Report(
        ncells=nc, n_flip=int(flip.sum()),
        max_rel_y=float(rel[:, keep].max(initial=0.0)),
        max_rel_T=float(relT[keep].max(initial=0.0)) if energy else 0.0,
        bad_small=int(small_bad[:, keep].sum()),
        flip_max_rel_y=float(rel[:, flip].max(initial=0.0)),
        flip_bad=flip_bad, flip_checked=checked,
        status_mismatch=status_mismatch,
        n_failed_cells=int((cell_bad & keep).sum()))


def atol_cells(net_py, cells, tol) -> Optional[np.ndarray]:
    """The integration's absolute tolerance of each cell: atol, or atol times the
    cell's initial element-0 total (atol_mode 1); None when it is the plain atol."""
    if tol.atol_mode != 1:
        return None
    b0 = np.asarray(net_py.counts, float)[:, 0] @ np.maximum(cells.y, 0.0)
    return tol.atol * b0


def tight_oracle(oracle_mod, net_py, cells, dt: float, tol, nthreads: int, **kw):
    """The tight-tolerance oracle run used to judge flipped cells (rtol 1e-9, the other
    options as the working run's)."""
    net = oracle_mod.OracleNetwork(net_py)

    def run(idx):
        sub = cells.subset(np.asarray(idx))
        opts = oracle_mod.options(tol, rtol=TIGHT_RTOL,
                                  max_substeps=max(400000, 40 * tol.max_substeps), **kw)
        return net.integrate(sub, dt, opts, nthreads)
    return run


def conservation_error(net, y0: np.ndarray, y1: np.ndarray) -> float:
    """max over cells and elements of |N y1 - N y0| / (|N| y0)."""
    y0c = np.maximum(y0, 0.0)
    b0 = net.counts.T @ y0c
    b1 = net.counts.T @ y1
    scale = np.abs(net.counts.T) @ y0c
    return float(np.max(np.abs(b1 - b0) / np.where(scale > 0, scale, 1.0)))
