"""CUDA path vs the FP64 oracle, element by element, through the C-ABI.

Sizes: the Robertson workload at full size (1024 cells, several warps and blocks),
the combustion network on a ragged 250-cell batch (not a multiple of 32), and the
full 65,536-cell combustion workload in the benchmark's launch configuration with
the oracle on sampled cells.  Edge cases: empty and single-cell batches, non-finite
inputs, negative inputs, forced reverts, split ranges (bit-identical) and repeat
runs (bit-identical).
"""
import os

import numpy as np
import pytest

from paper_2504_04941_gb300 import inputs as I
from _parity import atol_cells, compare, conservation_error, tight_oracle

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def kt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_04941_gb300 import build, kt as ktm
    build.build()
    return ktm


def gpu_run(kt, net_py, cells, dt, opts, net=None):
    import torch
    net = net or kt.Network(net_py)
    y = torch.from_numpy(np.ascontiguousarray(cells.y)).cuda()
    T = torch.from_numpy(np.ascontiguousarray(cells.T)).cuda()
    r = kt.integrate(net, y, T, dt, opts)
    kt.check_scratch(r["scratch"])
    torch.cuda.synchronize()
    return {k: r[k].cpu().numpy() for k in ("y", "T", "status", "nsub", "nnewton")}


def ora_run(oracle_mod, net_py, cells, dt, tol, **kw):
    net = oracle_mod.OracleNetwork(net_py)
    return net.integrate(cells, dt, oracle_mod.options(tol, **kw), NTHREADS)


FORMS = [dict(form=0, persistent=0), dict(form=0, persistent=1), dict(form=1, persistent=1),
         dict(form=0, persistent=1, cells_per_warp=1), dict(form=1, persistent=0, cells_per_warp=1)]
FORM_IDS = ["fp64", "fp64-persistent", "fp32lu-persistent", "warp-fp64-persistent", "warp-fp32lu"]


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_robertson_full_parity(kt, oracle_mod, form):
    wl = I.workload(1)
    g = gpu_run(kt, wl.network, wl.cells, wl.tol.dt, kt.options(wl.tol, **form))
    o = ora_run(oracle_mod, wl.network, wl.cells, wl.tol.dt, wl.tol)
    rep = compare(g, o, wl.network.energy,
                  tight=tight_oracle(oracle_mod, wl.network, wl.cells, wl.tol.dt, wl.tol, NTHREADS))
    print(rep)
    assert rep.ok(), rep
    assert conservation_error(wl.network, wl.cells.y, g["y"]) <= 1e-12
    if form["form"] == 0:
        assert rep.n_flip == 0
        if form.get("cells_per_warp", 32) == 32:
            assert np.array_equal(g["nnewton"], o["nnewton"])


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_combustion_ragged_parity(kt, oracle_mod, form):
    wl = I.workload(2, 250)
    g = gpu_run(kt, wl.network, wl.cells, wl.tol.dt, kt.options(wl.tol, **form))
    o = ora_run(oracle_mod, wl.network, wl.cells, wl.tol.dt, wl.tol)
    rep = compare(g, o, wl.network.energy,
                  tight=tight_oracle(oracle_mod, wl.network, wl.cells, wl.tol.dt, wl.tol, NTHREADS))
    print(rep)
    assert rep.ok(), rep
    assert conservation_error(wl.network, wl.cells.y, g["y"]) <= 1e-12
    assert np.all(g["y"] >= 0)
    # energy invariant C_V T + sum h y of the pre-processed state
    net = wl.network
    y0 = np.maximum(wl.cells.y, 0)
    cv = net.cv @ y0
    E0 = cv * wl.cells.T + net.h @ y0
    E1 = cv * g["T"] + net.h @ g["y"]
    assert np.all(np.abs(E1 - E0) <= 1e-11 * (cv * wl.cells.T + np.abs(net.h) @ y0))


@pytest.mark.parametrize("form,scheme", [(0, 0), (1, 0), (1, 1)], ids=["fp64", "fp32lu", "fp32lu-trbdf2"])
def test_combustion_full_size_sampled(kt, oracle_mod, form, scheme):
    """Full 65,536-cell workload, persistent launch as benchmarked; 48 sampled cells."""
    wl = I.workload(2)
    g = gpu_run(kt, wl.network, wl.cells, wl.tol.dt,
                kt.options(wl.tol, form=form, persistent=1, scheme=scheme))
    assert np.all(g["status"] == 0)
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(wl.cells.ncells, 48, replace=False))
    sub = wl.cells.subset(idx)
    o = ora_run(oracle_mod, wl.network, sub, wl.tol.dt, wl.tol, scheme=scheme)
    gs = {k: (v[:, idx] if v.ndim == 2 else v[idx]) for k, v in g.items()}
    rep = compare(gs, o, wl.network.energy,
                  tight=tight_oracle(oracle_mod, wl.network, sub, wl.tol.dt, wl.tol, NTHREADS,
                                     scheme=scheme))
    print(rep)
    assert rep.ok(), rep
    assert conservation_error(wl.network, wl.cells.y, g["y"]) <= 1e-12


@pytest.mark.parametrize("form", [0, 1], ids=["fp64", "fp32lu"])
def test_ism_ragged_parity(kt, oracle_mod, form):
    """32-species isothermal network (warp-per-cell kernels), 97 cells."""
    wl = I.workload(3, 97)
    g = gpu_run(kt, wl.network, wl.cells, wl.tol.dt, kt.options(wl.tol, form=form, persistent=1))
    o = ora_run(oracle_mod, wl.network, wl.cells, wl.tol.dt, wl.tol)
    rep = compare(g, o, wl.network.energy, rtol=wl.tol.rtol,
                  tight=tight_oracle(oracle_mod, wl.network, wl.cells, wl.tol.dt, wl.tol, NTHREADS),
                  atol_cells=atol_cells(wl.network, wl.cells, wl.tol))
    print(rep)
    assert rep.ok(), rep
    assert conservation_error(wl.network, wl.cells.y, g["y"]) <= 1e-12
    assert np.all(g["y"] >= 0)


@pytest.mark.parametrize("form", [0, 1], ids=["fp64", "fp32lu"])
def test_combined64_ragged_parity(kt, oracle_mod, form):
    """64 species + T (65 unknowns, 1000 directed reactions; warp-per-cell), 37 cells.
    Backward Euler with step doubling over dt/1000 = 1e-9 s (~10^3 sub-steps per cell;
    the full 1e-6 s interval is covered with TR-BDF2 in test_trbdf2_parity)."""
    wl = I.workload(5, 37)
    dt = wl.tol.dt * 1e-3
    g = gpu_run(kt, wl.network, wl.cells, dt, kt.options(wl.tol, form=form, persistent=1))
    o = ora_run(oracle_mod, wl.network, wl.cells, dt, wl.tol)
    rep = compare(g, o, wl.network.energy, rtol=wl.tol.rtol,
                  tight=tight_oracle(oracle_mod, wl.network, wl.cells, dt, wl.tol, NTHREADS))
    print(rep)
    assert rep.ok(), rep
    assert conservation_error(wl.network, wl.cells.y, g["y"]) <= 1e-12
    assert np.all(g["y"] >= 0)


TR_CASES = [(1, None, dict(form=0, persistent=1)), (1, None, dict(form=1, persistent=1)),
            (1, None, dict(form=0, persistent=1, cells_per_warp=1)),
            (2, 250, dict(form=0, persistent=0)), (2, 250, dict(form=1, persistent=1)),
            (2, 250, dict(form=1, persistent=1, cells_per_warp=1)),
            (3, 97, dict(form=0, persistent=1)), (3, 97, dict(form=1, persistent=1)),
            (5, 37, dict(form=0, persistent=1)), (5, 37, dict(form=1, persistent=1)),
            (1, None, dict(form=1, persistent=1, lane_variant=1)),
            (2, 250, dict(form=1, persistent=0, lane_variant=1)),
            (2, 250, dict(form=1, persistent=0, lane_variant=2))]
TR_IDS = ["robertson-fp64", "robertson-fp32lu-lean", "robertson-warp-fp64", "combustion-fp64",
          "combustion-fp32lu-lean", "combustion-warp-fp32lu", "ism-fp64", "ism-fp32lu",
          "combined64-fp64", "combined64-fp32lu", "robertson-fp32lu-jcache", "combustion-fp32lu-jcache-onepass",
          "combustion-fp32lu-lean-onepass"]


@pytest.mark.parametrize("wid,n,form", TR_CASES, ids=TR_IDS)
def test_trbdf2_parity(kt, oracle_mod, wid, n, form):
    """TR-BDF2 sub-steps (scheme 1) on every workload network and both kernel families,
    element by element against the oracle running the same scheme."""
    wl = I.workload(wid, n) if n else I.workload(wid)
    g = gpu_run(kt, wl.network, wl.cells, wl.tol.dt, kt.options(wl.tol, scheme=1, **form))
    o = ora_run(oracle_mod, wl.network, wl.cells, wl.tol.dt, wl.tol, scheme=1)
    rep = compare(g, o, wl.network.energy, rtol=wl.tol.rtol,
                  tight=tight_oracle(oracle_mod, wl.network, wl.cells, wl.tol.dt, wl.tol, NTHREADS, scheme=1),
                  atol_cells=atol_cells(wl.network, wl.cells, wl.tol))
    print(rep)
    assert rep.ok(), rep
    assert conservation_error(wl.network, wl.cells.y, g["y"]) <= 1e-12
    assert np.all(g["y"] >= 0)
    if wl.network.energy:
        net = wl.network
        y0 = np.maximum(wl.cells.y, 0)
        cv = net.cv @ y0
        E0 = cv * wl.cells.T + net.h @ y0
        E1 = cv * g["T"] + net.h @ g["y"]
        assert np.all(np.abs(E1 - E0) <= 1e-11 * (cv * wl.cells.T + np.abs(net.h) @ y0))
    if form["form"] == 0 and wid == 1:
        assert rep.n_flip == 0


def test_edge_cases(kt, oracle_mod):
    import torch
    wl = I.workload(1, 40)
    net = kt.Network(wl.network)
    opts = kt.options(wl.tol)
    # empty batch: no-op
    y = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    T = torch.zeros(0, dtype=torch.float64, device="cuda")
    r = kt.integrate(net, y, T, 1.0, opts)
    assert r["y"].shape == (3, 0)
    # one cell
    one = wl.cells.subset([5])
    g = gpu_run(kt, wl.network, one, 10.0, opts, net)
    o = ora_run(oracle_mod, wl.network, one, 10.0, wl.tol)
    assert compare(g, o, 0, tight=tight_oracle(oracle_mod, wl.network, one, 10.0, wl.tol, 1)).ok()
    # non-finite and negative inputs, and a cell that must revert
    c = wl.cells
    c.y[0, 1] = np.nan
    c.T[2] = np.inf
    c.y[2, 3] = -1e-3
    g = gpu_run(kt, wl.network, c, 10.0, opts, net)
    o = ora_run(oracle_mod, wl.network, c, 10.0, wl.tol)
    assert list(g["status"][:4]) == [0, 3, 3, 0]
    assert np.isnan(g["y"][0, 1])
    rep = compare({k: np.delete(v, [1, 2], axis=-1) for k, v in g.items()},
                  {k: np.delete(v, [1, 2], axis=-1) for k, v in o.items()}, 0)
    assert rep.ok(), rep
    g = gpu_run(kt, wl.network, wl.cells.subset(range(3, 40)), 1e4,
                kt.options(wl.tol, max_substeps=50), net)
    assert np.all(g["status"] == 2)
    assert np.array_equal(g["y"], np.maximum(wl.cells.subset(range(3, 40)).y, 0))


@pytest.mark.parametrize("form,scheme,variant", [(0, 0, 0), (1, 0, 0), (1, 1, 1), (1, 1, 2)])
def test_split_range_bit_identical_and_deterministic(kt, form, scheme, variant):
    wl = I.workload(2, 200)
    net = kt.Network(wl.network)
    opts = kt.options(wl.tol, form=form, persistent=1, scheme=scheme, lane_variant=variant)
    a = gpu_run(kt, wl.network, wl.cells, wl.tol.dt, opts, net)
    b = gpu_run(kt, wl.network, wl.cells, wl.tol.dt, opts, net)
    lo = gpu_run(kt, wl.network, wl.cells.subset(range(0, 77)), wl.tol.dt, opts, net)
    hi = gpu_run(kt, wl.network, wl.cells.subset(range(77, 200)), wl.tol.dt, opts, net)
    for k in ("y", "T", "status", "nsub", "nnewton"):
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a[k], np.concatenate([lo[k], hi[k]], axis=-1)), k
    # persistent and one-pass launches compute the same cells bit for bit
    c = gpu_run(kt, wl.network, wl.cells, wl.tol.dt,
                kt.options(wl.tol, form=form, persistent=0, scheme=scheme, lane_variant=variant), net)
    for k in ("y", "T", "status", "nsub", "nnewton"):
        assert np.array_equal(a[k], c[k]), k
    # and so do other block shapes (2 and 8 warps per block)
    for bw in (2, 8):
        d = gpu_run(kt, wl.network, wl.cells, wl.tol.dt,
                    kt.options(wl.tol, form=form, persistent=1, scheme=scheme, lane_variant=variant,
                               block_warps=bw), net)
        for k in ("y", "T", "status", "nsub", "nnewton"):
            assert np.array_equal(a[k], d[k]), (bw, k)


def test_state_api_host_roundtrip(kt):
    wl = I.workload(1, 100)
    net = kt.Network(wl.network)
    opts = kt.options(wl.tol, persistent=1)
    st = kt.State(net, 100)
    st.upload(wl.cells.y, wl.cells.T, wl.cells.rho)
    st.integrate(wl.tol.dt, opts)
    h = st.download()
    d = gpu_run(kt, wl.network, wl.cells, wl.tol.dt, opts, net)
    for k in ("y", "T", "status", "nsub", "nnewton"):
        assert np.array_equal(h[k], d[k]), k


def test_state_upload_without_density(kt):
    """A state uploaded without densities (rho = 1 filled by the library on the caller's
    stream) integrates exactly like the device-buffer call with no density."""
    import torch
    wl = I.workload(2, 64)
    net = kt.Network(wl.network)
    opts = kt.options(wl.tol, form=1, persistent=1)
    st = kt.State(net, 64)
    stream = torch.cuda.Stream()
    st.upload(wl.cells.y, wl.cells.T, None, stream=stream)
    st.integrate(wl.tol.dt * 1e-3, opts, stream=stream)
    h = st.download(stream=stream)
    d = gpu_run(kt, wl.network, wl.cells, wl.tol.dt * 1e-3, opts, net)
    for k in ("y", "T", "status", "nsub", "nnewton"):
        assert np.array_equal(h[k], d[k]), k


NASA_CASES = [dict(form=0, persistent=0, scheme=0), dict(form=1, persistent=1, scheme=0),
              dict(form=0, persistent=1, scheme=1), dict(form=1, persistent=1, scheme=1),
              dict(form=1, persistent=1, scheme=1, cells_per_warp=1),
              dict(form=0, persistent=1, scheme=0, cells_per_warp=1)]
NASA_IDS = ["fp64-be", "fp32lu-be", "fp64-trbdf2", "fp32lu-trbdf2", "warp-fp32lu-trbdf2", "warp-fp64-be"]


@pytest.mark.parametrize("form", NASA_CASES, ids=NASA_IDS)
def test_nasa_heat_capacity_parity(kt, oracle_mod, form):
    """Temperature-dependent C_V (two-range polynomials, Sec. 4.2) on the combustion
    network, 250 ragged cells, against the oracle running the same scheme."""
    wl = I.workload(6, 250)
    g = gpu_run(kt, wl.network, wl.cells, wl.tol.dt, kt.options(wl.tol, **form))
    o = ora_run(oracle_mod, wl.network, wl.cells, wl.tol.dt, wl.tol, scheme=form["scheme"])
    rep = compare(g, o, wl.network.energy,
                  tight=tight_oracle(oracle_mod, wl.network, wl.cells, wl.tol.dt, wl.tol, NTHREADS,
                                     scheme=form["scheme"]))
    print(rep)
    assert rep.ok(), rep
    assert conservation_error(wl.network, wl.cells.y, g["y"]) <= 1e-12
    assert np.all(g["y"] >= 0)


RAD_CASES = [(7, 61, dict(form=0, persistent=1, scheme=1)), (7, 61, dict(form=1, persistent=1, scheme=1)),
             (7, 29, dict(form=0, persistent=1, scheme=0)),
             (8, 120, dict(form=0, persistent=1, scheme=1)), (8, 120, dict(form=1, persistent=1, scheme=1)),
             (8, 120, dict(form=1, persistent=0, scheme=0))]
RAD_IDS = ["ism-rad-fp64-trbdf2", "ism-rad-fp32lu-trbdf2", "ism-rad-fp64-be", "combustion-tab-fp64-trbdf2",
           "combustion-tab-fp32lu-trbdf2", "combustion-tab-fp32lu-be"]


@pytest.mark.parametrize("wid,n,form", RAD_CASES, ids=RAD_IDS)
def test_tabulated_and_photo_rates_parity(kt, oracle_mod, wid, n, form):
    """Tabulated (per-cell density slice, ln k linear in ln T) and self-shielded photo
    rates (k = F sigma (1 - e^-tau)/tau, exact Jacobian) against the oracle: the ISM
    network with radiation (warp-per-cell), the combustion network with tables (the
    warp-per-cell kernels take every network with such rates)."""
    import torch
    wl = I.workload(wid, n)
    net = kt.Network(wl.network)
    c = wl.cells
    dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    r = kt.integrate(net, dev(c.y), dev(c.T), wl.tol.dt, kt.options(wl.tol, **form), rho=dev(c.rho),
                     flux=dev(c.flux), path=dev(c.path))
    kt.check_scratch(r["scratch"])
    g = {k: r[k].cpu().numpy() for k in ("y", "T", "status", "nsub", "nnewton")}
    o = ora_run(oracle_mod, wl.network, c, wl.tol.dt, wl.tol, scheme=form["scheme"])
    rep = compare(g, o, wl.network.energy, rtol=wl.tol.rtol,
                  tight=tight_oracle(oracle_mod, wl.network, c, wl.tol.dt, wl.tol, NTHREADS, scheme=form["scheme"]),
                  atol_cells=atol_cells(wl.network, c, wl.tol))
    print(rep)
    assert rep.ok(), rep
    assert conservation_error(wl.network, c.y, g["y"]) <= 1e-12
    assert np.all(g["y"] >= 0)


def test_special_rates_refuse_the_lane_kernels(kt):
    import torch
    wl = I.workload(8, 4)
    net = kt.Network(wl.network)
    y = torch.from_numpy(wl.cells.y).cuda()
    T = torch.from_numpy(wl.cells.T).cuda()
    with pytest.raises(kt.KtError) as ei:
        kt.integrate(net, y, T, 1e-9, kt.options(wl.tol, cells_per_warp=32))
    assert ei.value.code == -1
