"""Learned-guess MLP kernels against the FP64 reference (oracle/mlp_ref.py).

Forward and gradients use BF16 weights and BF16 activations with FP32 accumulation,
so they are compared with the FP64 reference evaluated on the same BF16-rounded
weights and inputs, per tensor: relative L2 error <= 3e-2 and cosine >= 0.999.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import mlp_ref as R
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


def _split(kt, flat):
    offs, _ = kt.mlp_layout()
    parts = [flat[o:o + int(np.prod(sh))].reshape(sh).astype(np.float64) for o, sh in offs]
    return [(parts[0], parts[4]), (parts[1], parts[5]), (parts[2], parts[6]), (parts[3], parts[7])]


def _ref_params(kt, mlp):
    return [(R.bf16_round(W), b) for W, b in _split(kt, mlp.params())]


def _close(a, b, rel=3e-2, cos=0.999):
    a, b = np.ravel(a), np.ravel(b)
    nb = np.linalg.norm(b)
    if nb == 0:
        return np.linalg.norm(a) == 0
    c = float(a @ b / (np.linalg.norm(a) * nb + 1e-300))
    return np.linalg.norm(a - b) <= rel * nb and c >= cos


def _data(n, nin, nout, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, 16), np.float32)
    X[:, :nin] = rng.standard_normal((n, nin))
    Tg = np.zeros((n, 16), np.float32)
    Tg[:, :nout] = rng.standard_normal((n, nout))
    return X, Tg


def test_forward_matches_reference(kt):
    import torch
    mlp = kt.Mlp(6, 3, seed=11)
    X, _ = _data(37, 6, 3, 0)
    out = mlp.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    ref, _ = R.forward(_ref_params(kt, mlp), R.bf16_round(X.astype(np.float64)))
    assert _close(out[:, :3], ref[:, :3], rel=1e-2)
    assert np.all(out[:, 3:] == 0.0)


def test_gradients_match_reference(kt):
    import torch
    mlp = kt.Mlp(6, 3, seed=5)
    X, Tg = _data(53, 6, 3, 1)
    g, loss = mlp.gradients(torch.from_numpy(X).cuda(), torch.from_numpy(Tg).cuda())
    P = _ref_params(kt, mlp)
    lref, gref = R.loss_and_grads(P, R.bf16_round(X.astype(np.float64)), Tg.astype(np.float64))
    assert abs(loss - lref) <= 1e-2 * lref
    gg = _split(kt, g)
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(gg, gref)):
        assert _close(gW, rW), (l, "W")
        assert _close(gb, rb), (l, "b")
    # padding stays exactly zero
    assert np.all(gg[0][0][:, 6:] == 0.0) and np.all(gg[3][0][3:, :] == 0.0) and np.all(gg[3][1][3:] == 0)


def test_adam_first_step(kt):
    import torch
    mlp = kt.Mlp(6, 3, seed=7)
    X, Tg = _data(64, 6, 3, 2)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(Tg).cuda()
    p0 = mlp.params().astype(np.float64)
    g, _ = mlp.gradients(Xd, Td)
    mlp.train_step(Xd, Td, 1e-3)
    p1 = mlp.params().astype(np.float64)
    g = g.astype(np.float64)
    exp = p0 - 1e-3 * g / (np.abs(g) + 1e-8)
    live = g != 0
    assert np.allclose(p1[live], exp[live], rtol=1e-5, atol=1e-7)
    assert np.array_equal(p1[~live], p0[~live])


def test_save_load_roundtrip(kt, tmp_path):
    import torch
    mlp = kt.Mlp(6, 3, seed=3)
    mlp.set_norm(np.arange(6), np.ones(6) * 2, np.arange(3), np.ones(3) * 0.5)
    path = str(tmp_path / "m.ktmlp")
    mlp.save(path)
    m2 = kt.Mlp(path=path)
    assert np.array_equal(mlp.params(), m2.params())
    X, _ = _data(20, 6, 3, 4)
    Xd = torch.from_numpy(X).cuda()
    assert torch.equal(mlp.forward(Xd), m2.forward(Xd))


def test_training_reduces_loss(kt):
    import torch
    rng = np.random.default_rng(9)
    X = np.zeros((8192, 16), np.float32)
    X[:, :6] = rng.standard_normal((8192, 6))
    Tg = np.zeros((8192, 16), np.float32)
    Tg[:, 0] = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]
    Tg[:, 1] = np.tanh(X[:, 3] - X[:, 4])
    Tg[:, 2] = X[:, 5] ** 2 / 4
    mlp = kt.Mlp(6, 3, seed=1)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(Tg).cuda()
    first = mlp.train_step(Xd[:1024], Td[:1024], 2e-3, want_loss=True)
    for k in range(600):
        s = (k * 1024) % 8192
        mlp.train_step(Xd[s:s + 1024], Td[s:s + 1024], 2e-3)
    _, last = mlp.gradients(Xd[:1024], Td[:1024])
    assert last < 0.05 * first, (first, last)


def test_untrained_guess_does_not_change_the_answer(kt, oracle_mod):
    """A random MLP gives poor starting points; the fallback keeps the solver's answer."""
    import torch
    wl = I.workload(1, 200)
    net = kt.Network(wl.network)
    mlp = kt.Mlp(net.ns + 3, net.n, seed=17)
    mlp.attach(net)
    y = torch.from_numpy(wl.cells.y).cuda()
    T = torch.from_numpy(wl.cells.T).cuda()
    for form in (0, 1):
        r = kt.integrate(net, y, T, wl.tol.dt, kt.options(wl.tol, form=form, persistent=1, guess=1))
        kt.check_scratch(r["scratch"])
        g = {k: r[k].cpu().numpy() for k in ("y", "T", "status", "nsub", "nnewton")}
        o = oracle_mod.OracleNetwork(wl.network).integrate(wl.cells, wl.tol.dt,
                                                           oracle_mod.options(wl.tol), os.cpu_count())
        rep = compare(g, o, 0, tight=tight_oracle(oracle_mod, wl.network, wl.cells, wl.tol.dt,
                                                  wl.tol, os.cpu_count()))
        assert rep.ok(), (form, rep)


def test_trained_guess_saves_newton_iterations(kt, oracle_mod):
    from paper_2504_04941_gb300 import guess
    wl = I.workload(4, 1)
    net = kt.Network(wl.network)
    st = guess.train(net, wl, n_pairs=200_000, epochs=3, val_pairs=8192, log=lambda *a: None)
    ev = guess.evaluate(net, wl, st["mlp"], 16384, seed=77)
    plain, mlp = ev["results"]["plain"], ev["results"]["mlp"]
    saved = 1.0 - mlp["nnewton"].sum() / plain["nnewton"].sum()
    print("newton iterations saved", saved, "val loss", st["val_loss"])
    assert np.all(plain["status"] == 0) and np.all(mlp["status"] == 0)
    assert saved > 0.0
    # same answer as the oracle on a sample of the test cells
    idx = np.arange(0, 16384, 257)
    cells = I.Cells(ev["y0"][:, idx].copy(), ev["T"][idx].copy(), np.ones(len(idx)))
    onet = oracle_mod.OracleNetwork(wl.network)
    for j, i in enumerate(idx):
        one = I.Cells(cells.y[:, j:j + 1].copy(), cells.T[j:j + 1].copy(), np.ones(1))
        o = onet.integrate(one, float(ev["dt"][i]), oracle_mod.options(wl.tol), 1)
        big = o["y"][:, 0] > 1e-20
        rel = np.abs(mlp["y"][:, i] - o["y"][:, 0])[big] / o["y"][big, 0]
        assert rel.max() <= 1e-6, (i, rel.max())


def test_learned_guess_on_the_combustion_network(kt, oracle_mod):
    """The learned start on the benchmark's network (10 species + T), trained by the
    library's kernels on solver-generated pairs: the answer stays the solver's, and the
    test reports what the guess does to the Newton iterations and to cells/s of the
    FP32-LU persistent form under backward Euler (a measurement: the benchmark's chosen
    form runs TR-BDF2 without it)."""
    from paper_2504_04941_gb300 import guess
    n = 8192
    out = guess.combustion_study(n_pairs=200_000, n_cells=n, epochs=2, dt_scale=0.01, log=lambda *a: None,
                                 arrays=True)
    res = out.pop("mlp_result")
    print(json.dumps(out))
    assert out["status_ok_plain"] == n and out["status_ok_mlp"] == n
    assert out["cells_changed_over_1e-6"] <= n // 100, out["cells_changed_over_1e-6"]
    assert math.isfinite(out["newton_saved_frac"]) and out["cells_per_s_mlp"] > 0 and out["cells_per_s_plain"] > 0
    # the learned start's answer against the oracle on a sample of the cells
    wl = I.workload(2, n)
    idx = np.arange(0, n, 512)
    sub = wl.cells.subset(idx)
    g = {k: (v[:, idx] if v.ndim == 2 else v[idx]) for k, v in res.items()}
    o = oracle_mod.OracleNetwork(wl.network).integrate(sub, wl.tol.dt * 0.01, oracle_mod.options(wl.tol),
                                                       os.cpu_count())
    assert compare(g, o, 1, tight=tight_oracle(oracle_mod, wl.network, sub, wl.tol.dt * 0.01, wl.tol,
                                               os.cpu_count())).ok()
