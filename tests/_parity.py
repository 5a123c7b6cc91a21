"""Comparison rule between the CUDA path and the FP64 oracle.

Per cell and species: |y_gpu - y_ora| <= 1e-6 |y_ora| when y_ora > 1e-20; below that,
|y_gpu| <= 1e-20 + 1e-6 max_s y_ora.  Temperature: 1e-8 relative.  Status codes are
integers and must match exactly.  The step-doubling accept test (err <= 1) is a
discontinuous function of rounding, so a cell whose sub-step count differs from the
oracle's ("flip") is reported separately: it must still match the oracle within the
scheme's own accuracy (global error of step-doubling backward Euler ~ sqrt(rtol)),
and flips must stay rare.
"""
from __future__ import annotations

import dataclasses

import numpy as np

Y_RTOL = 1e-6
Y_FLOOR = 1e-20
T_RTOL = 1e-8


@dataclasses.dataclass
class Report:
    ncells: int
    n_flip: int
    max_rel_y: float          # over non-flipped cells, species above the floor
    max_rel_T: float
    bad_small: int            # species below the floor violating the small-value rule
    flip_max_rel_y: float
    status_mismatch: int
    n_failed_cells: int       # non-flipped cells violating the rule

    def ok(self, max_flip_frac: float = 0.01, rtol: float = 1e-6) -> bool:
        return (self.status_mismatch == 0 and self.n_failed_cells == 0 and
                self.n_flip <= max(1, int(max_flip_frac * self.ncells)) and
                self.flip_max_rel_y <= 10.0 * np.sqrt(rtol))


def compare(gpu: dict, ora: dict, energy: int, rtol: float = 1e-6) -> Report:
    yg, yo = np.asarray(gpu["y"], float), np.asarray(ora["y"], float)
    Tg, To = np.asarray(gpu["T"], float), np.asarray(ora["T"], float)
    nc = yo.shape[1]
    status_mismatch = int(np.sum(np.asarray(gpu["status"]) != np.asarray(ora["status"])))
    flip = np.asarray(gpu["nsub"]) != np.asarray(ora["nsub"])
    big = yo > Y_FLOOR
    rel = np.where(big, np.abs(yg - yo) / np.where(big, np.abs(yo), 1.0), 0.0)
    ymax = yo.max(axis=0, initial=0.0)
    small_bad = (~big) & (np.abs(yg) > Y_FLOOR + Y_RTOL * ymax[None, :])
    relT = np.abs(Tg - To) / np.abs(To)
    cell_bad = (rel > Y_RTOL).any(axis=0) | small_bad.any(axis=0)
    if energy:
        cell_bad |= relT > T_RTOL
    keep = ~flip
    return Report(
        ncells=nc, n_flip=int(flip.sum()),
        max_rel_y=float(rel[:, keep].max(initial=0.0)),
        max_rel_T=float(relT[keep].max(initial=0.0)) if energy else 0.0,
        bad_small=int(small_bad[:, keep].sum()),
        flip_max_rel_y=float(rel[:, flip].max(initial=0.0)),
        status_mismatch=status_mismatch,
        n_failed_cells=int((cell_bad & keep).sum()))


def conservation_error(net, y0: np.ndarray, y1: np.ndarray) -> float:
    """max over cells and elements of |N y1 - N y0| / (|N| y0)."""
    y0c = np.maximum(y0, 0.0)
    b0 = net.counts.T @ y0c
    b1 = net.counts.T @ y1
    scale = np.abs(net.counts.T) @ y0c
    return float(np.max(np.abs(b1 - b0) / np.where(scale > 0, scale, 1.0)))
