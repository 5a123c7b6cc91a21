"""Learned Newton starting point: solver-generated data, training, evaluation.

The MLP maps (log y, log T, log rho, log h) of a cell at the start of a step of size h
to the change of log y over that step; the integrator uses the prediction as the
Newton starting iterate of the step's first implicit solve and falls back to the
plain predictor when Newton does not converge from it (include/kt.h).

Data: cells of the Robertson workload are integrated along their trajectories by the
CUDA solver itself, with snapshots at log-spaced times (1e-6 .. 1e4 s); every
snapshot is paired with a step dt ~ log-uniform(1e-8, 1e-5) s and the solver's end
state after dt.  Training runs the library's own BF16/FP32 forward, backward and
Adam kernels (kt_mlp_train_step); this module only assembles tensors.
"""
from __future__ import annotations

import math
import time
from typing import Dict, Optional

import numpy as np

from . import inputs as I
from . import kt

FLOOR = 1e-30


def _features(y, T, rho, h):
    """[n, 16] float64 features: log max(y, floor), log T, log rho, log h (padded)."""
    import torch
    ns, n = y.shape
    X = torch.zeros((n, kt.MLP_IN), dtype=torch.float64, device=y.device)
    X[:, :ns] = torch.log(torch.clamp(y, min=FLOOR)).T
    X[:, ns] = torch.log(T)
    X[:, ns + 1] = torch.log(rho)
    X[:, ns + 2] = torch.log(h)
    return X


def _targets(y0, y1, T0=None, T1=None):
    """[n, 16] change of log max(y, floor) over the step (and of log T with the energy
    equation)."""
    import torch
    ns, n = y0.shape
    D = torch.zeros((n, kt.MLP_OUT), dtype=torch.float64, device=y0.device)
    D[:, :ns] = (torch.log(torch.clamp(y1, min=FLOOR)) - torch.log(torch.clamp(y0, min=FLOOR))).T
    if T0 is not None:
        D[:, ns] = torch.log(T1) - torch.log(T0)
    return D


def trajectory_states(net: kt.Network, wl: I.Workload, n_traj: int, n_snap: int, seed: int,
                      t0: float = 1e-6, t1: float = 1e4, opts=None):
    """Snapshots of n_traj cells at n_snap log-spaced times in [t0, t1] (device tensors)."""
    import torch
    cells = I.robertson_cells(n_traj, seed)
    y = torch.from_numpy(cells.y).cuda()
    T = torch.from_numpy(cells.T).cuda()
    times = np.geomspace(t0, t1, n_snap)
    prev = 0.0
    snaps = []
    opts = opts or kt.options(wl.tol, persistent=1)
    scratch = torch.empty(kt.scratch_bytes(), dtype=torch.uint8, device="cuda")
    for tk in times:
        r = kt.integrate(net, y, T, float(tk - prev), opts, scratch=scratch)
        y = r["y"]
        snaps.append(y.clone())
        prev = tk
    kt.check_scratch(scratch)
    return torch.cat(snaps, dim=1), T.repeat(n_snap)


def make_pairs(net: kt.Network, wl: I.Workload, n_pairs: int, seed: int,
               dt_range=(1e-8, 1e-5), n_snap: int = 80) -> Dict[str, "object"]:
    """Solver-generated (state, dt) -> end-state pairs on the GPU."""
    import torch
    n_traj = max(1, -(-n_pairs // n_snap))
    y0, T = trajectory_states(net, wl, n_traj, n_snap, seed)
    y0, T = y0[:, :n_pairs].contiguous(), T[:n_pairs].contiguous()
    g = torch.Generator(device="cpu").manual_seed(seed + 1)
    u = torch.rand(n_pairs, generator=g, dtype=torch.float64)
    dt = torch.exp(math.log(dt_range[0]) + u * (math.log(dt_range[1]) - math.log(dt_range[0]))).cuda()
    opts = kt.options(wl.tol, persistent=1)
    r = kt.integrate_dt(net, y0, T, dt, opts)
    kt.check_scratch(r["scratch"])
    ok = r["status"] == 0
    rho = torch.ones_like(T)
    return dict(y0=y0[:, ok], T=T[ok], rho=rho[ok], dt=dt[ok], y1=r["y"][:, ok])


def _t_pair(pairs):
    """(T at the start, T at the end) of pairs with the energy equation, else (None, None)."""
    return (pairs["T"], pairs["T1"]) if "T1" in pairs else (None, None)


def normalisation(pairs):
    X = _features(pairs["y0"], pairs["T"], pairs["rho"], pairs["dt"])
    D = _targets(pairs["y0"], pairs["y1"], *_t_pair(pairs))
    mu_in, sd_in = X.mean(0), X.std(0)
    mu_out, sd_out = D.mean(0), D.std(0)
    sd_in = torch_where_small(sd_in)
    sd_out = torch_where_small(sd_out)
    return (mu_in.cpu().numpy(), sd_in.cpu().numpy(), mu_out.cpu().numpy(), sd_out.cpu().numpy())


def torch_where_small(sd, eps: float = 1e-6):
    import torch
    return torch.where(sd > eps, sd, torch.ones_like(sd))


def normalised_tensors(pairs, norm):
    import torch
    mu_in, sd_in, mu_out, sd_out = (torch.from_numpy(np.asarray(v, np.float64)).cuda() for v in norm)
    X = (_features(pairs["y0"], pairs["T"], pairs["rho"], pairs["dt"]) - mu_in) / sd_in
    D = (_targets(pairs["y0"], pairs["y1"], *_t_pair(pairs)) - mu_out) / sd_out
    return X.float().contiguous(), D.float().contiguous()


def combustion_pairs(net: kt.Network, wl: I.Workload, n_pairs: int, seed: int,
                     h_range=(1e-12, 1e-8), n_snap: int = 40) -> Dict[str, "object"]:
    """Solver-generated pairs on a network with the energy equation (the combustion
    workload): cells of the workload's distribution advanced along their trajectories
    (snapshots at log-spaced times from 1e-11 s to the workload's dt, T and density
    per cell), each snapshot paired with a step h ~ log-uniform(h_range) (the sub-step
    sizes of that workload) and the solver's end state after h."""
    import torch
    n_traj = max(1, -(-n_pairs // n_snap))
    cells = I.combustion_cells(wl.network, n_traj, seed)
    y = torch.from_numpy(cells.y).cuda()
    T = torch.from_numpy(cells.T).cuda()
    rho = torch.from_numpy(cells.rho).cuda()
    opts = kt.options(wl.tol, form=kt.KT_FORM_FP32LU, persistent=1, scheme=kt.KT_SCHEME_TRBDF2)
    ys, Ts, prev = [], [], 0.0
    for tk in np.geomspace(1e-11, wl.tol.dt, n_snap):
        r = kt.integrate(net, y, T, float(tk - prev), opts, rho=rho)
        kt.check_scratch(r["scratch"])
        y, T = r["y"], r["T"]
        ys.append(y.clone())
        Ts.append(T.clone())
        prev = tk
    y0 = torch.cat(ys, dim=1)[:, :n_pairs].contiguous()
    T0 = torch.cat(Ts)[:n_pairs].contiguous()
    rho0 = rho.repeat(n_snap)[:n_pairs].contiguous()
    g = torch.Generator(device="cpu").manual_seed(seed + 1)
    u = torch.rand(T0.shape[0], generator=g, dtype=torch.float64)
    h = torch.exp(math.log(h_range[0]) + u * (math.log(h_range[1]) - math.log(h_range[0]))).cuda()
    r = kt.integrate_dt(net, y0, T0, h, kt.options(wl.tol, persistent=1, scheme=kt.KT_SCHEME_TRBDF2),
                        rho=rho0)
    kt.check_scratch(r["scratch"])
    ok = r["status"] == 0
    return dict(y0=y0[:, ok], T=T0[ok], rho=rho0[ok], dt=h[ok], y1=r["y"][:, ok], T1=r["T"][ok])


def train(net: kt.Network, wl: I.Workload, n_pairs: int = 1_000_000, epochs: int = 4,
          batch: int = 4096, lr: float = 2e-3, seed: int = 2504, val_pairs: int = 65536,
          log=print, pairs_fn=None) -> Dict[str, object]:
    """Generate pairs with the solver and train a fresh MLP; returns the MLP and stats."""
    import torch
    t0 = time.perf_counter()
    pairs = (pairs_fn or make_pairs)(net, wl, n_pairs + val_pairs, seed)
    t_data = time.perf_counter() - t0
    n = pairs["T"].shape[0]
    norm = normalisation({k: v[..., :n - val_pairs] for k, v in pairs.items()})
    X, D = normalised_tensors(pairs, norm)
    Xtr, Dtr, Xva, Dva = X[:n - val_pairs], D[:n - val_pairs], X[n - val_pairs:], D[n - val_pairs:]
    mlp = kt.Mlp(net.ns + 3, net.n, seed=seed)
    mlp.set_norm(*norm)
    ntr = Xtr.shape[0]
    steps = epochs * (ntr // batch)
    g = torch.Generator(device="cuda").manual_seed(seed)
    t1 = time.perf_counter()
    losses = []
    k = 0
    for ep in range(epochs):
        perm = torch.randperm(ntr, device="cuda", generator=g)
        for b in range(ntr // batch):
            idx = perm[b * batch:(b + 1) * batch]
            lr_k = lr * 0.5 * (1 + math.cos(math.pi * k / max(1, steps)))
            want = (b == 0)
            loss = mlp.train_step(Xtr[idx].contiguous(), Dtr[idx].contiguous(), lr_k, want_loss=want)
            if want:
                losses.append(loss)
                log(f"epoch {ep} step {k} lr {lr_k:.2e} loss {loss:.4e}")
            k += 1
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    pred = mlp.forward(Xva)[:, :net.n].double()
    val = float(0.5 * ((pred - Dva[:, :net.n].double()) ** 2).sum(1).mean())
    # relative error of the predicted end state vs the solver's, on held-out pairs
    sd_out = torch.from_numpy(np.asarray(norm[3], np.float64)).cuda()[:net.n]
    mu_out = torch.from_numpy(np.asarray(norm[2], np.float64)).cuda()[:net.n]
    dlog_pred = mu_out + sd_out * pred
    dlog_true = mu_out + sd_out * Dva[:, :net.n].double()
    rel = torch.expm1((dlog_pred - dlog_true).abs()).max(dim=1).values
    y0v = pairs["y0"][:, n - val_pairs:]
    y1v = pairs["y1"][:, n - val_pairs:]
    if net.energy:
        y0v = torch.cat([y0v, pairs["T"][None, n - val_pairs:]])
        y1v = torch.cat([y1v, pairs["T1"][None, n - val_pairs:]])
    plain = ((y1v - y0v).abs() / torch.clamp(y1v.abs(), min=1e-300)).max(dim=0).values
    return dict(mlp=mlp, norm=norm, val_loss=val, losses=losses, steps=k,
                seconds_data=t_data, seconds_train=t_train, pairs=ntr,
                guess_rel_err_median=float(rel.median()), plain_rel_err_median=float(plain.median()))


def evaluate(net: kt.Network, wl: I.Workload, mlp: Optional[kt.Mlp], n_cells: int, seed: int,
             form: int = kt.KT_FORM_FP64, dt_range=(1e-8, 1e-5)):
    """Integrate fresh test cells over per-cell dt with and without the learned guess."""
    import torch
    n_snap = 80
    n_traj = max(1, -(-n_cells // n_snap))                 # enough trajectories for n_cells
    y0, T = trajectory_states(net, wl, n_traj, n_snap, seed)
    y0, T = y0[:, :n_cells].contiguous(), T[:n_cells].contiguous()
    assert T.shape[0] == n_cells, (T.shape, n_cells)
    g = torch.Generator(device="cpu").manual_seed(seed + 7)
    u = torch.rand(n_cells, generator=g, dtype=torch.float64)
    dt = torch.exp(math.log(dt_range[0]) + u * (math.log(dt_range[1]) - math.log(dt_range[0]))).cuda()
    rho = torch.ones_like(T)
    res = {}
    if mlp is not None:
        mlp.attach(net)
    for name, guess in (("plain", kt.KT_GUESS_PREV), ("mlp", kt.KT_GUESS_MLP)):
        if guess == kt.KT_GUESS_MLP and mlp is None:
            continue
        opts = kt.options(wl.tol, form=form, persistent=1, guess=guess)
        kt.integrate_dt(net, y0, T, dt, opts)                       # warm-up
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r = kt.integrate_dt(net, y0, T, dt, opts)
        b.record()
        kt.check_scratch(r["scratch"])
        res[name] = dict(ms=a.elapsed_time(b), y=r["y"].cpu().numpy(), status=r["status"].cpu().numpy(),
                         nsub=r["nsub"].cpu().numpy(), nnewton=r["nnewton"].cpu().numpy())
    return dict(results=res, y0=y0.cpu().numpy(), T=T.cpu().numpy(), dt=dt.cpu().numpy())


def study(n_pairs: int, n_cells: int, epochs: int, seed: int = 2504, log=print) -> Dict[str, object]:
    """The learned-guess study on the Robertson workload: train on solver-generated
    pairs, then integrate fresh test cells over per-cell dt in every (form, guess)
    combination and report Newton iterations, time and the largest relative change of
    the answer that the guess causes (the solver's converged result decides)."""
    import torch
    wl = I.workload(4, 1)
    net = kt.Network(wl.network)
    st = train(net, wl, n_pairs=n_pairs, epochs=epochs, seed=seed, log=log)
    out = {"workload": f"Robertson ({wl.network.ns} species), {n_cells} test cells, dt log-uniform "
                       f"1e-8..1e-5 s per cell, rtol={wl.tol.rtol:g}, atol={wl.tol.atol:g}",
           "pairs": st["pairs"], "train_steps": st["steps"], "val_loss": st["val_loss"],
           "seconds_data": st["seconds_data"], "seconds_train": st["seconds_train"],
           "guess_rel_err_median": st["guess_rel_err_median"],
           "plain_rel_err_median": st["plain_rel_err_median"], "forms": {}}
    for form in (kt.KT_FORM_FP64, kt.KT_FORM_FP32LU):
        ev = evaluate(net, wl, st["mlp"], n_cells, seed + 1, form=form)
        p, m = ev["results"]["plain"], ev["results"]["mlp"]
        big = p["y"] > 1e-20
        rel = np.abs(m["y"] - p["y"])[big] / p["y"][big]
        out["forms"]["fp64" if form == 0 else "fp32lu"] = {
            "newton_plain": int(p["nnewton"].sum()), "newton_mlp": int(m["nnewton"].sum()),
            "newton_saved_frac": float(1.0 - m["nnewton"].sum() / p["nnewton"].sum()),
            "ms_plain": p["ms"], "ms_mlp": m["ms"],
            "cells_per_s_plain": n_cells / (p["ms"] * 1e-3), "cells_per_s_mlp": n_cells / (m["ms"] * 1e-3),
            "status_ok_plain": int((p["status"] == 0).sum()), "status_ok_mlp": int((m["status"] == 0).sum()),
            "max_rel_change_of_answer": float(rel.max(initial=0.0))}
    torch.cuda.synchronize()
    return out


def combustion_study(n_pairs: int = 1_000_000, n_cells: int = 65536, epochs: int = 3,
                     dt_scale: float = 0.1, seed: int = 2504, log=print,
                     arrays: bool = False) -> Dict[str, object]:
    """The learned guess on the benchmark's combustion network (10 species + T): train on
    solver-generated pairs, then integrate the benchmark batch's first n_cells cells over
    dt_scale x its interval in the FP32-LU persistent form under backward Euler (the
    scheme the learned start serves) with the plain and the learned starting point, and
    report Newton iterations, cells/s of each and the largest relative change of the
    answer (the solver's converged result decides, so it must stay at the Newton
    tolerance's level)."""
    import torch
    wl = I.workload(2, n_cells)
    net = kt.Network(wl.network)
    st = train(net, wl, n_pairs=n_pairs, epochs=epochs, seed=seed, log=log, pairs_fn=combustion_pairs)
    dt = wl.tol.dt * dt_scale
    y = torch.from_numpy(wl.cells.y).cuda()
    T = torch.from_numpy(wl.cells.T).cuda()
    rho = torch.from_numpy(wl.cells.rho).cuda()
    st["mlp"].attach(net)
    res = {}
    for name, guess in (("plain", kt.KT_GUESS_PREV), ("mlp", kt.KT_GUESS_MLP)):
        opts = kt.options(wl.tol, form=kt.KT_FORM_FP32LU, persistent=1, scheme=kt.KT_SCHEME_BE, guess=guess)
        kt.integrate(net, y, T, dt, opts, rho=rho)                     # warm-up
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r = kt.integrate(net, y, T, dt, opts, rho=rho)
        b.record()
        kt.check_scratch(r["scratch"])
        torch.cuda.synchronize()
        res[name] = dict(ms=a.elapsed_time(b), y=r["y"].cpu().numpy(), T=r["T"].cpu().numpy(),
                         status=r["status"].cpu().numpy(), nnewton=r["nnewton"].cpu().numpy(),
                         nsub=r["nsub"].cpu().numpy())
    p, m = res["plain"], res["mlp"]
    big = p["y"] > 1e-20
    relm = np.where(big, np.abs(m["y"] - p["y"]) / np.where(big, p["y"], 1.0), 0.0)
    rel = relm[big]
    out = {"workload": f"{wl.name}: {wl.network.ns} species + T, first {n_cells} cells of the benchmark "
                        f"batch over dt={dt:g} s, backward Euler, FP32-LU, persistent",
            "pairs": st["pairs"], "train_steps": st["steps"], "val_loss": st["val_loss"],
            "seconds_data": st["seconds_data"], "seconds_train": st["seconds_train"],
            "guess_rel_err_median": st["guess_rel_err_median"],
            "plain_rel_err_median": st["plain_rel_err_median"],
            "newton_plain": int(p["nnewton"].sum()), "newton_mlp": int(m["nnewton"].sum()),
            "newton_saved_frac": float(1.0 - m["nnewton"].sum() / p["nnewton"].sum()),
            "ms_plain": p["ms"], "ms_mlp": m["ms"],
            "cells_per_s_plain": n_cells / (p["ms"] * 1e-3), "cells_per_s_mlp": n_cells / (m["ms"] * 1e-3),
            "status_ok_plain": int((p["status"] == 0).sum()), "status_ok_mlp": int((m["status"] == 0).sum()),
            "max_rel_change_of_answer": float(rel.max(initial=0.0)),
            # a different start can flip an accept decision of the step control; such
            # cells follow another valid step sequence and differ at the scheme's accuracy
            "cells_changed_over_1e-6": int((relm > 1e-6).any(axis=0).sum()),
            "max_rel_change_of_T": float((np.abs(m["T"] - p["T"]) / p["T"]).max(initial=0.0))}
    if arrays:
        out["mlp_result"] = {k: m[k] for k in ("y", "T", "status", "nsub", "nnewton")}
    return out


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description=study.__doc__)
    ap.add_argument("--pairs", type=int, default=10_000_000)
    ap.add_argument("--cells", type=int, default=262_144)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--combustion", action="store_true",
                    help="the study on the combustion network instead (combustion_study)")
    a = ap.parse_args()
    if a.combustion:
        out = combustion_study(a.pairs, a.cells, a.epochs, log=lambda *x: None)
    else:
        out = study(a.pairs, a.cells, a.epochs, log=lambda *x: None)
    print(json.dumps(out), flush=True)
