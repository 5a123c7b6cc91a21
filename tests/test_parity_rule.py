"""The comparison rule of the parity tests, exercised on the CPU.

Oracle runs stand in for the GPU side: a run that takes another sequence of sub-steps
at the same tolerance (a different first step) plays a flipped cell that must be
excused, and a run at a 100x looser tolerance plays a flipped cell that is not as
accurate as the oracle and must be rejected.
"""
import numpy as np

from paper_2504_04941_gb300 import inputs as I
from _parity import compare, tight_oracle


def _run(oracle_mod, wl, **kw):
    return oracle_mod.OracleNetwork(wl.network).integrate(
        wl.cells, wl.tol.dt, oracle_mod.options(wl.tol, **kw), 4)


def test_same_tolerance_flip_is_excused_and_looser_run_is_not(oracle_mod):
    wl = I.workload(1, 6)
    ora = _run(oracle_mod, wl)
    tight = tight_oracle(oracle_mod, wl.network, wl.cells, wl.tol.dt, wl.tol, 4)
    other = _run(oracle_mod, wl, h_init=wl.tol.h_init * 0.37)
    nflip = int(np.sum(other["nsub"] != ora["nsub"]))
    assert nflip >= 3
    rep = compare(other, ora, 0, tight=tight)
    assert rep.n_flip == nflip and rep.flip_checked and rep.flip_bad == 0
    assert not rep.ok()                      # several flips in six cells are too many
    assert rep.ok(max_flip_frac=1.0)
    loose = _run(oracle_mod, wl, rtol=wl.tol.rtol * 100)
    rep = compare(loose, ora, 0, tight=tight)
    assert rep.n_flip == 6 and rep.flip_bad == 6 and not rep.ok(max_flip_frac=1.0)


def test_flip_without_tight_run_is_not_excused(oracle_mod):
    wl = I.workload(1, 2)
    ora = _run(oracle_mod, wl)
    other = _run(oracle_mod, wl, h_init=wl.tol.h_init * 0.37)
    rep = compare(other, ora, 0)
    assert rep.n_flip > 0 and not rep.flip_checked and not rep.ok(max_flip_frac=1.0)


def test_identical_runs_pass(oracle_mod):
    wl = I.workload(2, 3)
    ora = _run(oracle_mod, wl)
    rep = compare(ora, ora, 1)
    assert rep.ok() and rep.n_flip == 0 and rep.max_rel_y == 0.0


def test_species_below_atol_compared_absolutely(oracle_mod):
    """On a density-scaled-atol network a species below the cell's atol is held to
    1e-6 atol absolutely; above it the relative 1e-6 rule applies."""
    from _parity import atol_cells
    wl = I.workload(3, 2)
    ora = _run(oracle_mod, wl)
    at = atol_cells(wl.network, wl.cells, wl.tol)
    assert at is not None and np.all(at > 1e-20)
    g = {k: np.array(v, copy=True) for k, v in ora.items()}
    s, c = np.unravel_index(np.argmin(np.where(ora["y"] > 1e-20, ora["y"], np.inf)), ora["y"].shape)
    assert ora["y"][s, c] < at[c]
    g["y"][s, c] += 0.5e-6 * at[c]                       # inside the absolute allowance
    assert compare(g, ora, 0, atol_cells=at).ok()
    assert not compare(g, ora, 0).ok()                    # the plain relative rule rejects it
    g["y"][s, c] += 2e-6 * at[c]
    assert not compare(g, ora, 0, atol_cells=at).ok()
    big = np.argmax(ora["y"][:, c])
    g = {k: np.array(v, copy=True) for k, v in ora.items()}
    g["y"][big, c] *= 1 + 2e-6
    assert not compare(g, ora, 0, atol_cells=at).ok()
