"""Plant plausible mistakes in a temporary copy of the oracle and check that the pins
catch every one of them.  The mutated sources are compiled into a temporary library;
the real oracle is not touched.
"""
import math
import os
import shutil
import subprocess
import types

import numpy as np
import pytest

from paper_2504_04941_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "kt_oracle.c")
PY = os.path.join(ROOT, "oracle", "oracle.py")

# (name, original text, mutated text): each a mistake a reimplementation could make
MUTANTS = [
    ("rhs_sign", "for (j = 0; j < n->nin[r]; j++) f[n->in[r * KO_MAXSIDE + j]] -= w;",
     "for (j = 0; j < n->nin[r]; j++) f[n->in[r * KO_MAXSIDE + j]] += w;"),
    ("jac_product_term", "if (l != j) d *= y[in[l]];", "if (l == j) d *= y[in[l]];"),
    ("jac_transposed", "J[in[a] * N + m] -= d;", "J[m * N + in[a]] -= d;"),
    ("jac_drop_thermal", "for (a = 0; a < n->nin[r]; a++) J[in[a] * N + n->ns] -= dT;", ""),
    ("dkdT_sign", "dkdT[r] = k[r] * (n->b[r] + n->theta[r] / T) / T;",
     "dkdT[r] = k[r] * (n->b[r] - n->theta[r] / T) / T;"),
    ("arrhenius_sign", "double arg = n->b[r] * lt - n->theta[r] / T;",
     "double arg = n->b[r] * lt + n->theta[r] / T;"),
    ("energy_sign", "f[n->ns] = -q / heat_capacity(n, hc, y[n->ns], &dcv);",
     "f[n->ns] = q / heat_capacity(n, hc, y[n->ns], &dcv);"),
    ("cv_poly_dT_term_sign", "J[n->ns * N + n->ns] -= f[n->ns] * dcv / cv;",
     "J[n->ns * N + n->ns] += f[n->ns] * dcv / cv;"),
    ("cv_poly_range_swapped", "const double *a = n->cvp + s * 10 + (T < n->t_mid ? 0 : 5);",
     "const double *a = n->cvp + s * 10 + (T < n->t_mid ? 5 : 0);"),
    ("cv_poly_derivative_index", "if (k < 4) dv += (k + 1) * a[k + 1] * tk;", "if (k < 4) dv += k * a[k + 1] * tk;"),
    ("lu_no_swap", "if (imax != j) {\n            for (k = 0; k < N; k++) {",
     "if (0) {\n            for (k = 0; k < N; k++) {"),
    ("lu_unscaled_pivot", [("double t = fabs(a[i * N + j]) / v[i];", "double t = fabs(a[i * N + j]);"),
                           ("double tmax = fabs(a[j * N + j]) / v[j];", "double tmax = fabs(a[j * N + j]);")], None),
    ("lu_no_l_scale", "for (i = j + 1; i < N; i++) a[i * N + j] /= a[j * N + j];", ""),
    ("solve_no_perm", "double t = x[i]; x[i] = x[perm[i]]; x[perm[i]] = t;", ""),
    ("be_sign_h", "c->G[i] = y[i] - yn[i] - h * c->f[i];", "c->G[i] = y[i] - yn[i] + h * c->f[i];"),
    ("newton_update_sign", "y[i] += c->d[i];", "y[i] -= c->d[i];"),
    ("step_full_instead_of_half", "for (i = 0; i < N; i++) y[i] = y2[i];\n            nacc++;",
     "for (i = 0; i < N; i++) y[i] = yf[i];\n            nacc++;"),
    ("half_step_from_wrong_base", "ok = be_solve(c, yh, 0.5 * h, y2) == 0;", "ok = be_solve(c, y, 0.5 * h, y2) == 0;"),
    ("projection_sign", "y[s] -= y[s] * corr;", "y[s] += y[s] * corr;"),
    ("no_projection", "y[s] -= y[s] * corr;", ""),
    ("no_clip", "if (y[s] < 0.0) y[s] = 0.0;", ""),
    ("projection_no_failure_limit", "if (!(corr < 1.0)) return -1;", ""),
    ("projection_unweighted", [("m += (double)n->counts[s * ne + e] * n->counts[s * ne + f] * y[s];",
                                "m += (double)n->counts[s * ne + e] * n->counts[s * ne + f];"),
                               ("y[s] -= y[s] * corr;", "y[s] -= corr;")], None),
    ("trbdf2_gamma", "k.g = 2.0 - sqrt(2.0);", "k.g = 2.0 - sqrt(2.1);"),
    ("trbdf2_w0_sign", "k.w0 = (1.0 - k.g) * (1.0 - k.g) / (k.g * (2.0 - k.g));",
     "k.w0 = -(1.0 - k.g) * (1.0 - k.g) / (k.g * (2.0 - k.g));"),
    ("trbdf2_stage2_base", "for (i = 0; i < N; i++) r[i] = k.w1 * yg[i] - k.w0 * yn[i];",
     "for (i = 0; i < N; i++) r[i] = k.w1 * yg[i] - k.w0 * yg[i];"),
    ("trbdf2_stage1_no_f0", "for (i = 0; i < N; i++) r[i] = yn[i] + dh * f0[i];",
     "for (i = 0; i < N; i++) r[i] = yn[i];"),
    ("trbdf2_estimate_scale", "const double ce = 2.0 * k.C * h;", "const double ce = k.C * h;"),
    ("trbdf2_estimate_fg_sign", "double fg = (yg[i] - yn[i]) * inv - f0[i];",
     "double fg = (yg[i] - yn[i]) * inv + f0[i];"),
    ("table_slope_without_T", "*dk = *k * ((L[j + 1] - L[j]) / dl) / T;", "*dk = *k * ((L[j + 1] - L[j]) / dl);"),
    ("table_rho_weights_swapped", "ltab[t * nT + j] = nR > 1 ? (1.0 - w) * row[j] + w * row[nT + j] : row[j];",
     "ltab[t * nT + j] = nR > 1 ? w * row[j] + (1.0 - w) * row[nT + j] : row[j];"),
    ("table_segment_off_by_one", "*k = exp(L[j] + fr * (L[j + 1] - L[j]));", "*k = exp(L[j + 1] + fr * (L[j + 1] - L[j]));"),
    ("photo_phi_sign", "*phi = (1.0 - e) / tau;", "*phi = (1.0 + e) / tau;"),
    ("photo_depth_without_path", "return rd->path * s;", "return s;"),
    ("photo_jacobian_dropped", "J[in[0] * N + m] -= d;", "(void)d;"),
    ("accept_wrong_norm_weight", "double sc = eatol(c, i) + c->o->rtol * fmax(fabs(y[i]), fabs(y2[i]));",
     "double sc = eatol(c, i) + c->o->rtol * fabs(y[i]) * 1e3;"),
]
# Equivalent mutants, left out on purpose: they change nothing any pin (or any user)
# can observe.  A different growth law (0.9/err instead of 0.9/sqrt(err), or err^2 in
# place of err) is another valid controller of the same order.  Inside an integration
# the element projection acts on rounding-level defects only (every Newton update of
# backward Euler conserves the linear invariants exactly, N J = 0 implies
# N delta = -N G), so its mutants are caught by the direct post-processing pin.


def _load_variant(tmpdir, name, old, new):
    src = open(SRC).read()
    edits = old if isinstance(old, list) else [(old, new)]
    for o, n_ in edits:
        assert o in src, name
        src = src.replace(o, n_, 1)
    d = os.path.join(tmpdir, name)
    os.makedirs(d, exist_ok=True)
    c = os.path.join(d, "kt_oracle.c")
    open(c, "w").write(src)
    so = os.path.join(d, "libkt_oracle.so")
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-ffp-contract=off",
                           "-fPIC", "-shared", "-o", so, c, "-lm", "-lpthread"])
    mod = types.ModuleType(f"oracle_{name}")
    code = open(PY).read()
    mod.__dict__["__file__"] = os.path.join(d, "oracle.py")
    exec(compile(code, PY, "exec"), mod.__dict__)
    mod.SRC, mod.LIB = c, so
    mod._lib = None
    return mod


def _pins(m):
    """A compact run of the pins of test_oracle_pins; returns the names that fail."""
    failed = []

    def check(name, fn):
        try:
            ok = fn()
        except Exception:
            ok = False
        if not ok:
            failed.append(name)

    def lu_exact():
        A = np.array([[2.0, 1e6, 3.0], [1.0, 1.0, -2.0], [4.0, -1.0, 5.0]])
        b = np.array([1.0, 2.0, 3.0])
        rc, fac, perm = m.lu(A)
        return rc == 0 and np.allclose(m.lu_solve(fac, perm, b), np.linalg.solve(A, b), rtol=1e-12)

    def lu_pivot():
        rc, _, perm = m.lu([[2.0, 1e6], [1.0, 1.0]])
        return rc == 0 and perm[0] == 1

    def jac_fd():
        for wid in (1, 2, 6):
            netw = I.network(wid)
            net = m.OracleNetwork(netw)
            wl = I.workload(wid, 3)
            y = wl.cells.y[:, 1].copy()
            n0 = y.copy() if netw.cv_poly is not None else None
            T = float(wl.cells.T[1])
            if wid == 6:
                T = 1400.0            # above t_mid: the high-range polynomial
            cv = float(netw.cv @ y) if netw.energy else 1.0
            if netw.energy:
                y = np.append(y, T)
            J = net.jacobian(y, T, cv, n0)
            s = np.maximum(np.abs(y), 1e-6 * np.abs(y).max())
            F = np.zeros_like(J)
            for k in range(len(y)):
                h = 1e-6 * s[k]
                yp, ym = y.copy(), y.copy()
                yp[k] += h
                ym[k] -= h
                F[:, k] = (net.rhs(yp, T, cv, n0) - net.rhs(ym, T, cv, n0)) / (2 * h)
            Js, Fs = J * s[None, :], F * s[None, :]
            sc = np.maximum(np.abs(Js), np.abs(Fs)).max(axis=1, keepdims=True) + 1e-300
            if np.any(np.abs(Js - Fs) > 1e-6 * sc):
                return False
        return True

    def rhs_robertson():
        net = m.OracleNetwork(I.robertson_network())
        y = np.array([0.7, 2e-5, 0.3])
        ref = [-0.04 * y[0] + 1e4 * y[1] * y[2], 0.04 * y[0] - 1e4 * y[1] * y[2] - 3e7 * y[1] ** 2,
               3e7 * y[1] ** 2]
        return np.allclose(net.rhs(y), ref, rtol=1e-14)

    def rates_printed():
        net = m.OracleNetwork(I.stromgren_network(1e-9))
        k, dk = net.rates(1e4)
        kb = 8.617333262e-5
        kci = 1.05e-9 * (1e4 / 300) ** 0.5 * math.exp(-13.6 / (kb * 1e4))
        a = 3.5e-12 * (1e4 / 300) ** -0.75
        h = 1e-2
        fd = (3.5e-12 * ((1e4 + h) / 300) ** -0.75 - 3.5e-12 * ((1e4 - h) / 300) ** -0.75) / (2 * h)
        return abs(k[1] / kci - 1) < 1e-12 and abs(k[2] / a - 1) < 1e-14 and abs(dk[2] / fd - 1) < 1e-6

    def fixed_step_chain():
        k1, k2 = 2.0, 50.0
        net = m.OracleNetwork(I.decay_chain_network(k1, k2))
        K = np.array([[-k1, 0, 0], [k1, -k2, 0], [0, k2, 0]])
        y0 = np.array([0.7, 0.2, 0.1])
        cells = I.Cells(y0.reshape(3, 1).copy(), np.array([300.0]), np.array([1.0]))
        r = net.integrate(cells, 1.0, m.options(atol=1e-14, h_init=0.01, adaptive=0, retry=0,
                                                newton_rtol=1e-14), 1)
        ref = np.linalg.matrix_power(np.linalg.inv(np.eye(3) - 0.01 * K), 100) @ y0
        return np.allclose(r["y"][:, 0], ref, rtol=1e-13, atol=1e-16)

    def bateman():
        net = m.OracleNetwork(I.decay_chain_network(1.0, 10.0))
        cells = I.Cells(np.array([[1.0], [0.0], [0.0]]), np.array([300.0]), np.array([1.0]))
        A = math.exp(-2.0)
        B = 1 / 9 * (math.exp(-2.0) - math.exp(-20.0))
        ref = np.array([A, B, 1 - A - B])
        errs = []
        for rtol in (1e-4, 1e-6):
            r = net.integrate(cells, 2.0, m.options(rtol=rtol, atol=1e-14, h_init=1e-6), 1)
            errs.append(np.abs(r["y"][:, 0] / ref - 1).max())
        slope = math.log10(errs[0] / errs[1]) / 2
        return errs[1] <= 2e-3 and 0.45 <= slope <= 0.55

    def single_step_two_halves():
        k1, k2 = 3.0, 40.0
        net = m.OracleNetwork(I.decay_chain_network(k1, k2))
        K = np.array([[-k1, 0, 0], [k1, -k2, 0], [0, k2, 0]])
        y0 = np.array([0.6, 0.3, 0.1])
        h = 1e-3
        cells = I.Cells(y0.reshape(3, 1).copy(), np.array([300.0]), np.array([1.0]))
        r = net.integrate(cells, h, m.options(rtol=1e-2, atol=1e-12, h_init=h, newton_rtol=1e-14,
                                              retry=0), 1)
        Mh = np.linalg.inv(np.eye(3) - 0.5 * h * K)
        return r["nsub"][0] == 1 and np.allclose(r["y"][:, 0], Mh @ Mh @ y0, rtol=1e-13, atol=1e-16)

    def conservation():
        wl = I.workload(2, 4)
        netw = wl.network
        r = m.OracleNetwork(netw).integrate(wl.cells, wl.tol.dt, m.options(wl.tol), 1)
        y0 = np.maximum(wl.cells.y, 0)
        b0, b1 = netw.counts.T @ y0, netw.counts.T @ r["y"]
        cv = netw.cv @ y0
        E0 = cv * wl.cells.T + netw.h @ y0
        E1 = cv * r["T"] + netw.h @ r["y"]
        return (np.all(r["status"] == 0) and np.all(np.abs(b1 - b0) <= 1e-12 * b0) and
                np.all(r["y"] >= 0) and np.all(np.abs(E1 - E0) <= 1e-12 * (cv * wl.cells.T + np.abs(netw.h) @ y0)))

    def negative_input_clipped():
        wl = I.workload(1, 1)
        cells = I.Cells(np.array([[0.95], [-1e-7], [0.05]]), np.array([300.0]), np.array([1.0]))
        r = m.OracleNetwork(wl.network).integrate(cells, 1e-3, m.options(wl.tol), 1)
        return np.all(r["y"] >= 0) and abs(r["y"][:, 0].sum() - 1.0) < 1e-14

    def post_process():
        # hand-solved cases of the least relative change (see test_oracle_pins)
        h2 = m.OracleNetwork(I._irreversible("h_h2", ["H", "H2"], ["H"], [1.0, 2.0], [0.0, 0.0],
                                             [1.0, 1.0], [[1], [2]], 0, 300.0, 10.0, 1e5,
                                             [((0, 0), (1,), 1.0, 0.0, 0.0, -1)]))
        rc, y = h2.post_process([0.5, 0.25], [0.999])
        ok = rc == 0 and np.allclose(y, [0.5 - 1 / 3000, 0.25 - 1 / 3000], rtol=1e-14, atol=0)
        rc, y = h2.post_process([0.5, -1e-6], [0.5])
        ok = ok and rc == 0 and y[1] == 0.0 and y[0] == 0.5
        rc, _ = h2.post_process([0.5, 0.25], [0.1])
        return ok and rc != 0

    def trbdf2():
        from scipy.linalg import expm
        k1, k2 = 3.0, 7.0
        net = m.OracleNetwork(I.decay_chain_network(k1, k2))
        K = np.array([[-k1, 0, 0], [k1, -k2, 0], [0, k2, 0]])
        y0 = np.array([0.9, 0.1, 0.0])
        errs = []
        for h in (0.02, 0.01):
            cells = I.Cells(y0.reshape(3, 1).copy(), np.array([300.0]), np.array([1.0]))
            r = net.integrate(cells, 1.0, m.options(atol=1e-16, h_init=h, adaptive=0, retry=0,
                                                   newton_rtol=1e-15, scheme=1), 1)
            errs.append(np.abs(r["y"][:, 0] - expm(K) @ y0).max())
        rc, y1, est = net.trbdf2_step(y0, 2.5e-3, m.options(atol=1e-16, newton_rtol=1e-15, scheme=1))
        true = expm(K * 2.5e-3) @ y0 - y1
        return (3.7 < errs[0] / errs[1] < 4.3 and rc == 0 and
                bool(np.all(np.abs(est / true - 1.0) < 0.04)))

    def cv_poly_energy():
        # E(T) + sum h n at the end of a long interval vs the antiderivative of C_V (both
        # ranges crossed: cells start at 900-2500 K)
        wl = I.workload(6, 3)
        netw = wl.network
        P = np.polynomial.polynomial
        r = m.OracleNetwork(netw).integrate(wl.cells, wl.tol.dt, m.options(wl.tol, scheme=1), 1)
        for c in range(3):
            y0 = np.maximum(wl.cells.y[:, c], 0)
            lo = P.polyint(np.einsum("s,sk->k", y0, netw.cv_poly[:, 0, :]))
            hi = P.polyint(np.einsum("s,sk->k", y0, netw.cv_poly[:, 1, :]))

            def E(T):
                tm = netw.t_mid
                return P.polyval(min(T, tm), lo) + (P.polyval(T, hi) - P.polyval(tm, hi) if T > tm else 0.0)
            dE = E(r["T"][c]) - E(wl.cells.T[c]) + netw.h @ (r["y"][:, c] - y0)
            if not abs(dE) <= 1e-4 * (np.abs(netw.h) @ y0):
                return False
        return True

    def tables_photo():
        import dataclasses
        # density reduction and the T slope of a tabulated rate
        base = I.robertson_network()
        Rn = np.geomspace(1e-2, 1e2, 5)
        lnk = math.log(2e-3) + 0.37 * np.log(Rn)[:, None] + 0.5 * np.sin(np.arange(7))[None, :]
        net = m.OracleNetwork(dataclasses.replace(base, tables={0: lnk}, table_grid=(7, 10.0, 1e4, 5, 1e-2, 1e2)))
        k, _ = net.rates_cell(np.ones(3), T_iso=np.geomspace(10.0, 1e4, 7)[3], rho=0.013)
        ok = abs(k[0] / (math.exp(math.log(2e-3) + 0.5 * math.sin(3)) * 0.013 ** 0.37) - 1) < 1e-12
        k, dk = net.rates_cell(np.ones(3), T_iso=123.0, rho=2.0)
        kp, _ = net.rates_cell(np.ones(3), T_iso=123.0001, rho=2.0)
        km, _ = net.rates_cell(np.ones(3), T_iso=122.9999, rho=2.0)
        ok = ok and abs(dk[0] / ((kp[0] - km[0]) / 2e-4) - 1) < 1e-6
        # photolysis closed form
        sig, F, dl = 1e-18, 1e8, 1e17
        ph = I._irreversible("photolysis", ["X", "Y"], ["E"], [1.0, 1.0], [0.0, 0.0], [1.0, 1.0],
                             [[1], [1]], 0, 300.0, 10.0, 1e5, [((0,), (1,), 1.0, 0.0, 0.0, -1)])
        pn = m.OracleNetwork(dataclasses.replace(ph, photo={0: sig}))
        a, n0, t = dl * sig, 1.0 / (dl * sig), 2.0 / (sig * F)
        cells = I.Cells(np.array([[n0], [0.0]]), np.array([300.0]), np.array([1.0]), np.array([F]), np.array([dl]))
        r = pn.integrate(cells, t, m.options(rtol=1e-9, atol=1e-12 * n0, h_init=1e-6 * t, scheme=1), 1)
        exact = math.log1p(math.expm1(a * n0) * math.exp(-sig * F * t)) / a
        ok = ok and abs(r["y"][0, 0] / exact - 1) < 1e-5
        # Jacobian of the radiation workload network by central differences
        netw = I.network(7)
        wn = m.OracleNetwork(netw)
        wl = I.workload(7, 2)
        y = wl.cells.y[:, 0].copy()
        kw = dict(rho=float(wl.cells.rho[0]), flux=float(wl.cells.flux[0]), path=float(wl.cells.path[0]))
        J = wn.jacobian(y, float(wl.cells.T[0]), 1.0, None, **kw)
        Jfd = np.zeros_like(J)
        for mm in range(len(y)):
            h = 1e-6 * max(abs(y[mm]), 1e-6 * np.abs(y).max())
            yp, ym = y.copy(), y.copy()
            yp[mm] += h
            ym[mm] -= h
            Jfd[:, mm] = (wn.rhs(yp, float(wl.cells.T[0]), 1.0, None, **kw) -
                          wn.rhs(ym, float(wl.cells.T[0]), 1.0, None, **kw)) / (2 * h)
        s_ = np.maximum(np.abs(y), 1e-6 * np.abs(y).max())
        Js, Fs = J * s_[None, :], Jfd * s_[None, :]
        sc = np.maximum(np.abs(Js), np.abs(Fs)).max(axis=1, keepdims=True) + 1e-300
        return bool(ok and np.all(np.abs(Js - Fs) <= 1e-6 * sc))

    for name, fn in (("lu_exact", lu_exact), ("post_process", post_process), ("trbdf2", trbdf2),
                     ("tables_photo", tables_photo),
                     ("cv_poly_energy", cv_poly_energy), ("lu_pivot", lu_pivot), ("jac_fd", jac_fd),
                     ("rhs_robertson", rhs_robertson), ("rates_printed", rates_printed),
                     ("fixed_step_chain", fixed_step_chain), ("bateman", bateman),
                     ("single_step_two_halves", single_step_two_halves),
                     ("conservation", conservation), ("negative_input_clipped", negative_input_clipped)):
        check(name, fn)
    return failed


def test_unmutated_copy_passes_all_pins(tmp_path):
    m = _load_variant(str(tmp_path), "identity", "#include <ctype.h>", "#include <ctype.h>")
    assert _pins(m) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    m = _load_variant(str(tmp_path), name, old, new)
    failed = _pins(m)
    assert failed, f"mutant {name} survived every pin"
