"""The entry point that allocates nothing (kt_integrate_noalloc).

It exists for callers that cannot allocate device memory where they integrate; it runs
the same kernels with its counters and network tables in a static device array.  Its
results must equal those of the allocating entry point, call after call (the array
keeps the previous call's contents), and networks too large for the array must be
refused with an error.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2504_04941_gb300 import inputs as I
from _parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_04941_gb300 import build, kt as ktm
    build.build()
    return ktm


def _outputs(y, T):
    import torch
    n = T.shape[0]
    return dict(y=torch.empty_like(y), T=torch.empty_like(T),
                status=torch.empty(n, dtype=torch.int32, device=T.device),
                nsub=torch.empty(n, dtype=torch.int32, device=T.device),
                nnewton=torch.empty(n, dtype=torch.int32, device=T.device))


@pytest.mark.parametrize("wid,n,dt_scale,form", [(1, 300, 1e-3, 0), (2, 200, 1e-2, 1), (3, 40, 1e-6, 0)])
def test_no_alloc_matches_allocating_entry_point(kt, wid, n, dt_scale, form):
    import torch
    wl = I.workload(wid, n)
    dt = wl.tol.dt * dt_scale
    net = kt.Network(wl.network)
    y = torch.from_numpy(wl.cells.y).cuda()
    T = torch.from_numpy(wl.cells.T).cuda()
    opts = kt.options(wl.tol, form=form, persistent=1)
    ref = kt.integrate(net, y, T, dt, opts)
    kt.check_scratch(ref["scratch"])
    ref = {k: ref[k].cpu().numpy() for k in ("y", "T", "status", "nsub", "nnewton")}
    for call in range(2):              # two calls in a row share the static area
        out = kt.integrate_noalloc(net, y, T, dt, opts, _outputs(y, T))
        torch.cuda.synchronize()
        got = {k: out[k].cpu().numpy() for k in ("y", "T", "status", "nsub", "nnewton")}
        assert compare(got, ref, wl.network.energy, rtol=wl.tol.rtol).ok(), (wid, call)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (wid, call, k)
        assert np.all(got["status"] == 0), (wid, call)   # every cell reached, none failed


def test_no_alloc_requires_status(kt):
    # status is the call's only report of a device-side failure, so NULL is refused
    import torch
    wl = I.workload(1, 8)
    net = kt.Network(wl.network)
    y = torch.from_numpy(wl.cells.y).cuda()
    T = torch.from_numpy(wl.cells.T).cuda()
    out = _outputs(y, T)
    del out["status"]
    with pytest.raises(kt.KtError) as ei:
        kt.integrate_noalloc(net, y, T, 1.0, kt.options(wl.tol), out)
    assert ei.value.code == -1 and "status" in str(ei.value)


def test_no_alloc_refuses_networks_beyond_its_area(kt):
    import torch
    import dataclasses
    small = I.network(2)
    rep = 25                            # 1500 directed reactions: ~84 KB of tables
    big = dataclasses.replace(small, name="big", reac_in=small.reac_in * rep, reac_out=small.reac_out * rep,
                              A=np.tile(small.A, rep), b=np.tile(small.b, rep), theta=np.tile(small.theta, rep),
                              pair=np.full(small.nr * rep, -1))
    net = kt.Network(big)
    cells = I.combustion_cells(big, 4)
    y = torch.from_numpy(cells.y).cuda()
    T = torch.from_numpy(cells.T).cuda()
    with pytest.raises(kt.KtError) as ei:
        kt.integrate_noalloc(net, y, T, 1e-12, kt.options(), _outputs(y, T))
    assert ei.value.code == -1 and "static area" in str(ei.value)
