"""Runtime around the kernels: CUDA-graph replay, the launch autotuner, device errors."""
import json
import os

import numpy as np
import pytest

from paper_2504_04941_gb300 import inputs as I
from _parity import compare, tight_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_04941_gb300 import build, kt as ktm
    build.build()
    return ktm


def _direct(kt, net, cells, dt, opts):
    import torch
    y = torch.from_numpy(cells.y).cuda()
    T = torch.from_numpy(cells.T).cuda()
    r = kt.integrate(net, y, T, dt, opts)
    kt.check_scratch(r["scratch"])
    return {k: r[k].cpu().numpy() for k in ("y", "T", "status", "nsub", "nnewton")}


@pytest.mark.parametrize("wid,n", [(1, 300), (2, 96), (3, 40)])
def test_graph_replay_matches_direct(kt, wid, n):
    wl = I.workload(wid, n)
    net = kt.Network(wl.network)
    st = kt.State(net, n)
    for form in (0, 1):
        opts = kt.options(wl.tol, form=form, persistent=1, use_graph=1)
        ref = _direct(kt, net, wl.cells, wl.tol.dt, opts)
        for rep in range(3):          # capture once, replay twice
            st.upload(wl.cells.y, wl.cells.T, wl.cells.rho)
            st.integrate(wl.tol.dt, opts)
            out = st.download()
            for k in ref:
                assert np.array_equal(out[k], ref[k]), (form, rep, k)
        # a different dt re-captures
        st.upload(wl.cells.y, wl.cells.T, wl.cells.rho)
        st.integrate(wl.tol.dt * 0.5, opts)
        out = st.download()
        ref2 = _direct(kt, net, wl.cells, wl.tol.dt * 0.5, opts)
        for k in ref2:
            assert np.array_equal(out[k], ref2[k]), (form, "dt", k)


def test_autotune_and_cache(kt, oracle_mod, tmp_path):
    import torch
    wl = I.workload(2, 256)
    net = kt.Network(wl.network)
    y = torch.from_numpy(wl.cells.y).cuda()
    T = torch.from_numpy(wl.cells.T).cuda()
    base = kt.options(wl.tol, form=1)
    dt = wl.tol.dt * 1e-3          # tuning runs every candidate twice: keep them short
    best, sec = kt.autotune(net, y, T, dt, base)
    assert best.cells_per_warp in (1, 32) and best.block_warps in (1, 2, 4, 8) and sec > 0
    assert best.form == 1 and best.rtol == base.rtol
    # under TR-BDF2 the FP32-LU lane kernels' storage variant is a tuned dimension too
    tr = kt.options(wl.tol, form=1, scheme=1)
    best_tr, sec_tr = kt.autotune(net, y, T, dt, tr)
    assert best_tr.lane_variant in (1, 2) and best_tr.scheme == 1 and sec_tr > 0
    g = _direct(kt, net, wl.cells, dt, best_tr)
    o = oracle_mod.OracleNetwork(wl.network).integrate(wl.cells, dt, oracle_mod.options(wl.tol, scheme=1),
                                                       os.cpu_count())
    assert compare(g, o, 1, tight=tight_oracle(oracle_mod, wl.network, wl.cells, dt, wl.tol,
                                               os.cpu_count(), scheme=1)).ok()
    cache = str(tmp_path / "tuned.json")
    opts, entry = kt.tuned_options(net, y, T, dt, base, cache, sample=128)
    assert os.path.exists(cache) and len(json.load(open(cache))) == 1
    opts2, _ = kt.tuned_options(net, y, T, dt, base, cache)   # cached: no re-tune
    assert opts2.block_warps == opts.block_warps
    g = _direct(kt, net, wl.cells, dt, opts)
    o = oracle_mod.OracleNetwork(wl.network).integrate(wl.cells, dt, oracle_mod.options(wl.tol),
                                                       os.cpu_count())
    assert compare(g, o, 1, tight=tight_oracle(oracle_mod, wl.network, wl.cells, dt, wl.tol,
                                               os.cpu_count())).ok()


def test_bad_arguments_are_errors_not_faults(kt):
    import torch
    wl = I.workload(1, 8)
    net = kt.Network(wl.network)
    y = torch.from_numpy(wl.cells.y).cuda()
    T = torch.from_numpy(wl.cells.T).cuda()
    with pytest.raises(kt.KtError):
        kt.integrate(net, y, T, -1.0, kt.options(wl.tol))
    with pytest.raises(kt.KtError):
        kt.integrate(net, y, T, 1.0, kt.options(wl.tol, max_newton=0))
    big = kt.Network(I.network(5))
    with pytest.raises(kt.KtError):           # 65 unknowns cannot use one cell per lane
        kt.integrate(big, torch.zeros((64, 4), dtype=torch.float64, device="cuda"),
                     torch.full((4,), 1000.0, dtype=torch.float64, device="cuda"), 1e-9,
                     kt.options(wl.tol, cells_per_warp=32))


def test_table_exp_against_cuda_and_libm(kt):
    """The table-driven exponential (Tang 1989) is within 2 ulp of CUDA's exp and of
    the host libm over the range the rate law uses."""
    import torch
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-708.0, 709.0, 200000), rng.uniform(-1, 1, 50000),
                        np.arange(-22000, 22000) * (np.log(2) / 32),
                        [0.0, 1e-300, -1e-300, np.log(2) / 64, -np.log(2) / 64, 709.0, -708.0]])
    xd = torch.from_numpy(x).cuda()
    tang = kt.debug_exp(xd, 1).cpu().numpy()
    cuda = kt.debug_exp(xd, 0).cpu().numpy()
    host = np.exp(x)
    ulp = np.spacing(host)
    assert np.max(np.abs(tang - host) / ulp) <= 2.0
    assert np.max(np.abs(tang - cuda) / np.spacing(cuda)) <= 2.0


@pytest.mark.parametrize("wid,n,dt_scale", [(2, 300, 1e-2), (3, 40, 1e-6)])
def test_longest_first_schedule_changes_no_result(kt, wid, n, dt_scale):
    """The longest-first queue order (from the previous call's Newton counts) only moves
    cells between lanes: every output is bit-identical to the index-order launch, with
    and without graph replay, on the first call (no history) and on later ones."""
    wl = I.workload(wid, n)
    dt = wl.tol.dt * dt_scale
    net = kt.Network(wl.network)
    st = kt.State(net, n)
    for form in (0, 1):
        ref = None
        for graph in (0, 1):
            for sched in (0, 1):
                opts = kt.options(wl.tol, form=form, persistent=1, use_graph=graph, schedule=sched)
                for rep in range(2):
                    st.upload(wl.cells.y, wl.cells.T, wl.cells.rho)
                    st.integrate(dt, opts)
                    out = st.download()
                    if ref is None:
                        ref = out
                        assert np.all(out["nnewton"] > 0)
                    for k in ref:
                        assert np.array_equal(out[k], ref[k]), (form, graph, sched, rep, k)
        fresh = kt.State(net, n)            # no history: every count is zero
        fresh.upload(wl.cells.y, wl.cells.T, wl.cells.rho)
        fresh.integrate(dt, kt.options(wl.tol, form=form, persistent=1, schedule=1))
        out = fresh.download()
        for k in ref:
            assert np.array_equal(out[k], ref[k]), (form, "fresh", k)


def test_caller_cost_estimate_orders_queue_without_changing_results(kt):
    """kt_state_set_cost: any caller-given cost estimate (host or device) only reorders
    the persistent queue; with graph replay and both schemes every output equals the
    index-order launch bit for bit, and the state's counters then hold the measured
    Newton counts."""
    import torch
    n = 300
    wl = I.workload(2, n)
    dt = wl.tol.dt * 1e-2
    net = kt.Network(wl.network)
    st = kt.State(net, n)
    rng = np.random.default_rng(5)
    for scheme in (0, 1):
        ref = _direct(kt, net, wl.cells, dt, kt.options(wl.tol, form=1, persistent=1, scheme=scheme))
        costs = [np.arange(n, dtype=np.int32)[::-1].copy(),
                 torch.from_numpy(rng.integers(0, 10000, n).astype(np.int32)).cuda()]
        for cost in costs:
            opts = kt.options(wl.tol, form=1, persistent=1, use_graph=1, schedule=1, scheme=scheme)
            st.set_cost(cost)
            st.upload(wl.cells.y, wl.cells.T, wl.cells.rho)
            st.integrate(dt, opts)
            out = st.download()
            for k in ref:
                assert np.array_equal(out[k], ref[k]), (scheme, k)
