"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself.  Each pin is a closed form, a library
routine on a special case, exact rational arithmetic, a printed constant of the
paper, or an invariant of the ODE class (Sec. 2.2):

* Crout LU (Algorithm lu-decomp): exact rational solutions of integer systems,
  P A = L U to rounding, the implicit-scaled pivot choice, singular detection.
* rate law (Sec. 2.2.1): the paper's Stromgren coefficients (Eq. thermo-strom).
* right-hand side (Eq. method-ode-thermochem): Robertson's textbook equations.
* Jacobian (Eq. method-jacobian): central finite differences of the right-hand side.
* backward Euler at fixed h: (I - hK)^-n y0 for a linear decay chain.
* adaptive control: Bateman closed form, first-order error scaling (~ sqrt(rtol)).
* Robertson at t = 1e4 against scipy's Radau at rtol 1e-13.
* invariants: element totals (1e-12), energy (1e-12), non-negativity,
  detailed balance at long times, the Stromgren ionisation root (Eq. strom-equil).
* failure path (Sec. 2.2.3): non-finite input, revert, retry.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2504_04941_gb300 import inputs as I

EPS = np.finfo(float).eps


# ------------------------------------------------------------------ LU


def _exact_solve(A, b):
    """Gauss-Jordan in exact rational arithmetic (brute force, tiny systems)."""
    n = len(A)
    M = [[Fraction(int(A[i][j])) for j in range(n)] + [Fraction(int(b[i]))] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [M[r][k] - f * M[c][k] for k in range(n + 1)]
    return [M[i][n] / M[i][i] for i in range(n)]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11, 16])
def test_lu_exact_rational(oracle_mod, n):
    rng = np.random.default_rng(100 + n)
    for _ in range(5):
        A = rng.integers(-9, 10, size=(n, n)).astype(float)
        if abs(np.linalg.det(A)) < 0.5:
            A += np.eye(n) * 7
        b = rng.integers(-20, 21, size=n).astype(float)
        x_ex = np.array([float(v) for v in _exact_solve(A, b)])
        rc, fac, perm = oracle_mod.lu(A)
        assert rc == 0
        x = oracle_mod.lu_solve(fac, perm, b)
        assert np.allclose(x, x_ex, rtol=1e-11, atol=1e-11 * np.abs(x_ex).max())


def _reconstruct(fac, perm, n):
    L = np.tril(fac, -1) + np.eye(n)
    U = np.triu(fac)
    P = np.eye(n)
    for j in range(n):
        P[[j, perm[j]]] = P[[perm[j], j]]
    return P, L, U


@pytest.mark.parametrize("n", [3, 11, 33, 65])
def test_lu_pa_equals_lu_ill_scaled(oracle_mod, n):
    """Rows scaled over 16 decades: P A = L U to ~ N eps ||A|| and the solve matches LAPACK."""
    rng = np.random.default_rng(7 + n)
    A = rng.standard_normal((n, n)) * 10.0 ** rng.uniform(-8, 8, size=(n, 1))
    rc, fac, perm = oracle_mod.lu(A)
    assert rc == 0
    P, L, U = _reconstruct(fac, perm, n)
    R = P @ A - L @ U
    row_scale = np.abs(A).max(axis=1, keepdims=True)
    # residual row-wise relative to that row's scale
    assert np.all(np.abs(R) <= 20 * n * EPS * (P @ row_scale))
    b = rng.standard_normal(n)
    x = oracle_mod.lu_solve(fac, perm, b)
    x_ref = np.linalg.solve(A, b)
    cond = np.linalg.cond(A / row_scale)
    assert np.allclose(x, x_ref, rtol=100 * n * EPS * cond, atol=0)


def test_lu_scaled_pivot_choice(oracle_mod):
    # unscaled pivoting would take row 0 (|2| > |1|); implicit scaling takes row 1
    rc, fac, perm = oracle_mod.lu([[2.0, 1e6], [1.0, 1.0]])
    assert rc == 0 and perm[0] == 1
    # a tie |a_i0| / v_i = 1 for both rows goes to the smaller index
    rc, fac, perm = oracle_mod.lu([[1.0, 0.5], [2.0, 1.5]])
    assert rc == 0 and perm[0] == 0


def test_lu_singular(oracle_mod):
    assert oracle_mod.lu([[1.0, 2.0], [2.0, 4.0]])[0] == -1
    assert oracle_mod.lu([[0.0, 0.0], [1.0, 1.0]])[0] == -1


# ------------------------------------------------------------------ rates / rhs / Jacobian


def _golden_stromgren():
    path = os.path.join(os.path.dirname(__file__), "golden", "stromgren_constants.txt")
    vals = {}
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            vals[line[0]] = float(line[1])
    return vals


def test_rates_stromgren_printed_constants(oracle_mod):
    g = _golden_stromgren()
    photo = 3.3e-8
    net = oracle_mod.OracleNetwork(I.stromgren_network(photo))
    kb_ev = 8.617333262e-5
    for T in (300.0, 5000.0, 1.0e4, 2.0e4):
        k, dk = net.rates(T)
        alpha = g["alpha_coeff"] * (T / g["t_ref"]) ** g["alpha_exp"]
        kci = g["kci_coeff"] * (T / g["t_ref"]) ** g["kci_exp"] * math.exp(-g["I_H"] / (kb_ev * T))
        assert k[0] == photo
        assert k[2] == pytest.approx(alpha, rel=1e-14)
        if kci > 1e-300:
            assert k[1] == pytest.approx(kci, rel=1e-12)
        # dk/dT against central differences of the printed formulas
        hT = 1e-5 * T
        a_p = g["alpha_coeff"] * ((T + hT) / 300) ** -0.75
        a_m = g["alpha_coeff"] * ((T - hT) / 300) ** -0.75
        assert dk[2] == pytest.approx((a_p - a_m) / (2 * hT), rel=1e-8)
    k, _ = net.rates(300.0)
    assert k[2] == 3.5e-12  # alpha(300 K) is the printed coefficient itself


def test_rates_underflow_flush(oracle_mod):
    net = oracle_mod.OracleNetwork(I.stromgren_network(0.0))
    k, dk = net.rates(20.0)       # exp(-157821/20) underflows: flushed to exactly 0
    assert k[1] == 0.0 and dk[1] == 0.0


def test_rhs_robertson_textbook(oracle_mod):
    net = oracle_mod.OracleNetwork(I.robertson_network())
    rng = np.random.default_rng(3)
    for _ in range(20):
        y = rng.uniform(0, 1, 3) * np.array([1, 1e-4, 1])
        f = net.rhs(y)
        ref = np.array([-0.04 * y[0] + 1e4 * y[1] * y[2],
                        0.04 * y[0] - 1e4 * y[1] * y[2] - 3e7 * y[1] ** 2,
                        3e7 * y[1] ** 2])
        assert np.allclose(f, ref, rtol=1e-14, atol=1e-17)


def _fd_jacobian(net, y, T_iso, cvtot, n0=None):
    n = len(y)
    J = np.zeros((n, n))
    floor = 1e-6 * np.abs(y).max()
    for m in range(n):
        h = 1e-6 * max(abs(y[m]), floor)
        yp, ym = y.copy(), y.copy()
        yp[m] += h
        ym[m] -= h
        J[:, m] = (net.rhs(yp, T_iso, cvtot, n0) - net.rhs(ym, T_iso, cvtot, n0)) / (2 * h)
    return J


@pytest.mark.parametrize("wid", [1, 2, 3, 5, 6])
def test_jacobian_vs_central_differences(oracle_mod, wid):
    """Workload 6 has C_V(T): its temperature row carries the dC_V/dT term."""
    netw = I.network(wid)
    net = oracle_mod.OracleNetwork(netw)
    wl = I.workload(wid, 6)
    for c in range(3):
        y = wl.cells.y[:, c].copy()
        n0 = y.copy() if netw.cv_poly is not None else None
        T = float(wl.cells.T[c])
        cvtot = float(np.dot(netw.cv, y)) if netw.energy else 1.0
        if netw.energy:
            y = np.append(y, T)
        J = net.jacobian(y, T, cvtot, n0)
        Jfd = _fd_jacobian(net, y, T, cvtot, n0)
        # columns times their variable's scale: every entry of a row is then the response
        # of f_i to a relative change of one unknown (same units along the row), so a
        # thermal-coupling term cannot hide behind the row's species entries
        s = np.maximum(np.abs(y), 1e-6 * np.abs(y).max())
        Js, Fs = J * s[None, :], Jfd * s[None, :]
        scale = np.maximum(np.abs(Js), np.abs(Fs)).max(axis=1, keepdims=True) + 1e-300
        assert np.all(np.abs(Js - Fs) <= 1e-6 * scale), (wid, c)


def test_energy_row_is_heat_release(oracle_mod):
    """dT/dt = -sum_s h_s dn_s/dt / C_V: C_V f_T + sum h_s f_s = 0 (energy invariant)."""
    netw = I.network(2)
    net = oracle_mod.OracleNetwork(netw)
    wl = I.workload(2, 4)
    for c in range(4):
        y = np.append(wl.cells.y[:, c], wl.cells.T[c])
        cv = float(np.dot(netw.cv, wl.cells.y[:, c]))
        f = net.rhs(y, 0.0, cv)
        q = np.dot(netw.h, f[:-1])
        assert abs(cv * f[-1] + q) <= 1e-12 * np.abs(netw.h * f[:-1]).sum()


# ------------------------------------------------------------------ time stepping


def test_backward_euler_fixed_step_linear_chain(oracle_mod):
    """BE at fixed h on A -> B -> C is y_n = (I - hK)^-n y0 exactly (to rounding)."""
    k1, k2 = 2.0, 50.0
    net = oracle_mod.OracleNetwork(I.decay_chain_network(k1, k2))
    K = np.array([[-k1, 0, 0], [k1, -k2, 0], [0, k2, 0]])
    y0 = np.array([0.7, 0.2, 0.1])
    h, nsteps = 0.01, 100
    cells = I.Cells(y0.reshape(3, 1).copy(), np.array([300.0]), np.array([1.0]))
    opts = oracle_mod.options(rtol=1e-6, atol=1e-14, h_init=h, h_min=1e-30, adaptive=0,
                              retry=0, newton_rtol=1e-14)
    r = net.integrate(cells, h * nsteps, opts, nthreads=1)
    ref = np.linalg.matrix_power(np.linalg.inv(np.eye(3) - h * K), nsteps) @ y0
    assert r["status"][0] == 0 and r["nsub"][0] == nsteps
    assert np.allclose(r["y"][:, 0], ref, rtol=1e-13, atol=1e-16)


def test_accepted_step_is_two_half_steps(oracle_mod):
    """With step doubling, an accepted step of size h returns two backward-Euler half
    steps: (I - (h/2) K)^-2 y0 for a linear chain (closed form, one accepted step)."""
    k1, k2 = 3.0, 40.0
    net = oracle_mod.OracleNetwork(I.decay_chain_network(k1, k2))
    K = np.array([[-k1, 0, 0], [k1, -k2, 0], [0, k2, 0]])
    y0 = np.array([0.6, 0.3, 0.1])
    h = 1e-3
    cells = I.Cells(y0.reshape(3, 1).copy(), np.array([300.0]), np.array([1.0]))
    r = net.integrate(cells, h, oracle_mod.options(rtol=1e-2, atol=1e-12, h_init=h,
                                                   newton_rtol=1e-14, retry=0), 1)
    Mh = np.linalg.inv(np.eye(3) - 0.5 * h * K)
    assert r["nsub"][0] == 1
    assert np.allclose(r["y"][:, 0], Mh @ Mh @ y0, rtol=1e-13, atol=1e-16)


def test_bateman_adaptive_first_order_scaling(oracle_mod):
    """Step-doubling BE reaches the Bateman solution with error ~ C sqrt(rtol)."""
    k1, k2, t = 1.0, 10.0, 2.0
    net = oracle_mod.OracleNetwork(I.decay_chain_network(k1, k2))
    cells = I.Cells(np.array([[1.0], [0.0], [0.0]]), np.array([300.0]), np.array([1.0]))
    A = math.exp(-k1 * t)
    B = k1 / (k2 - k1) * (math.exp(-k1 * t) - math.exp(-k2 * t))
    ref = np.array([A, B, 1 - A - B])
    errs = []
    rtols = [1e-4, 1e-5, 1e-6, 1e-7]
    for rtol in rtols:
        r = net.integrate(cells, t, oracle_mod.options(rtol=rtol, atol=1e-14, h_init=1e-6), 1)
        errs.append(np.abs(r["y"][:, 0] / ref - 1).max())
        assert errs[-1] <= 2.0 * math.sqrt(rtol)
    slope = np.polyfit(np.log10(rtols), np.log10(errs), 1)[0]
    assert 0.45 <= slope <= 0.55, slope


def test_robertson_vs_radau(oracle_mod):
    from scipy.integrate import solve_ivp
    wl = I.workload(1, 3)
    net = oracle_mod.OracleNetwork(wl.network)

    def f(t, y):
        return [-0.04 * y[0] + 1e4 * y[1] * y[2],
                0.04 * y[0] - 1e4 * y[1] * y[2] - 3e7 * y[1] ** 2, 3e7 * y[1] ** 2]

    def jac(t, y):
        return [[-0.04, 1e4 * y[2], 1e4 * y[1]],
                [0.04, -1e4 * y[2] - 6e7 * y[1], -1e4 * y[1]], [0, 6e7 * y[1], 0]]

    errs = {}
    for rtol in (1e-6, 1e-8):
        r = net.integrate(wl.cells, 1e4, oracle_mod.options(wl.tol, rtol=rtol), 3)
        e = 0.0
        for c in range(3):
            s = solve_ivp(f, (0, 1e4), wl.cells.y[:, c], method="Radau", rtol=1e-13,
                          atol=1e-22, jac=jac)
            ref = s.y[:, -1]
            e = max(e, np.abs(r["y"][:, c] / ref - 1).max())
            # conservation y1 + y2 + y3 (one pseudo-element) to rounding
            assert abs(r["y"][:, c].sum() - wl.cells.y[:, c].sum()) <= 1e-14
        errs[rtol] = e
        assert e <= math.sqrt(rtol), (rtol, e)
    assert errs[1e-8] < errs[1e-6] / 5


@pytest.mark.parametrize("wid", [2, 3])
def test_element_and_energy_conservation(oracle_mod, wid):
    wl = I.workload(wid, 12)
    netw = wl.network
    net = oracle_mod.OracleNetwork(netw)
    r = net.integrate(wl.cells, wl.tol.dt, oracle_mod.options(wl.tol), 4)
    assert np.all(r["status"] == 0)
    y0 = np.maximum(wl.cells.y, 0)
    b0 = netw.counts.T @ y0
    b1 = netw.counts.T @ r["y"]
    # element totals to 1e-12 of the element total, for every element with atoms
    assert np.all(np.abs(b1 - b0) <= 1e-12 * (netw.counts.T.__abs__() @ y0) + 0.0)
    assert np.all(r["y"] >= 0.0)
    if netw.energy:
        cv = netw.cv @ y0
        E0 = cv * wl.cells.T + netw.h @ y0
        E1 = cv * r["T"] + netw.h @ r["y"]
        mag = cv * wl.cells.T + np.abs(netw.h) @ y0
        assert np.all(np.abs(E1 - E0) <= 1e-12 * mag)


def test_detailed_balance_long_time(oracle_mod):
    """After a long step every reversible pair balances: k_f prod(r) = k_r prod(p)."""
    netw = I.network(2)
    net = oracle_mod.OracleNetwork(netw)
    wl = I.workload(2, 2)
    r = net.integrate(wl.cells, 1.0, oracle_mod.options(wl.tol, max_substeps=400000), 2)
    assert np.all(r["status"] == 0)
    for c in range(2):
        y, T = r["y"][:, c], r["T"][c]
        k, _ = net.rates(T)
        for q in range(0, netw.nr, 2):
            wf = k[q] * np.prod([y[i] for i in netw.reac_in[q]])
            wr = k[q + 1] * np.prod([y[i] for i in netw.reac_in[q + 1]])
            assert abs(wf - wr) <= 1e-6 * max(wf, wr) + 1e-300


@pytest.mark.parametrize("T,photo", [(1.0e4, 1e-9), (8000.0, 1e-12), (2.0e4, 1e-10)])
def test_stromgren_ionisation_root(oracle_mod, T, photo):
    """Isothermal H/H+/e- at t >> 1/(alpha n): x_e solves Eq. strom-equil (ionisation line)."""
    g = _golden_stromgren()
    n = g["n_amb"]
    net = oracle_mod.OracleNetwork(I.stromgren_network(photo))
    cells = I.Cells(np.array([[n * 0.999], [n * 0.001], [n * 0.001]]), np.array([T]),
                    np.array([n]))
    r = net.integrate(cells, 1e16, oracle_mod.options(rtol=1e-8, atol=1e-20, h_init=1.0,
                                                       max_substeps=400000), 1)
    assert r["status"][0] == 0
    xe = r["y"][2, 0] / n
    kb_ev = 8.617333262e-5
    alpha = g["alpha_coeff"] * (T / g["t_ref"]) ** g["alpha_exp"]
    kci = g["kci_coeff"] * (T / g["t_ref"]) ** g["kci_exp"] * math.exp(-g["I_H"] / (kb_ev * T))
    # 0 = alpha n^2 x^2 - kci n^2 x (1-x) - photo n (1-x)   (divide by n)
    a2 = alpha * n + kci * n
    a1 = photo - kci * n
    a0 = -photo
    x_root = (-a1 + math.sqrt(a1 * a1 - 4 * a2 * a0)) / (2 * a2)
    assert xe == pytest.approx(x_root, rel=1e-8)
    assert r["y"][0, 0] + r["y"][1, 0] == pytest.approx(n, rel=1e-13)


# ------------------------------------------------------------------ failure path


def test_nonfinite_input_status(oracle_mod):
    wl = I.workload(1, 4)
    wl.cells.y[0, 1] = np.nan
    wl.cells.T[2] = np.inf
    net = oracle_mod.OracleNetwork(wl.network)
    r = net.integrate(wl.cells, 1.0, oracle_mod.options(wl.tol), 1)
    assert list(r["status"]) == [0, 3, 3, 0]
    assert np.isnan(r["y"][0, 1]) and r["nsub"][1] == 0


def test_revert_and_retry(oracle_mod):
    wl = I.workload(1, 2)
    net = oracle_mod.OracleNetwork(wl.network)
    # far too few sub-steps: both attempts fail -> revert to the input
    r = net.integrate(wl.cells, 1e4, oracle_mod.options(wl.tol, max_substeps=50), 1)
    assert np.all(r["status"] == 2)
    assert np.array_equal(r["y"], wl.cells.y)
    # a first attempt that dies on h_min (huge first step, tiny h_min) and a retry
    # from a much smaller first step that succeeds
    r = net.integrate(wl.cells, 1e4, oracle_mod.options(wl.tol, h_init=1e3, h_min=1e2,
                                                        retry_h_factor=1e-9), 1)
    assert np.all(r["status"] == 1), r["status"]


def test_negative_input_clipped_and_T_clamped(oracle_mod):
    wl = I.workload(2, 2)
    wl.cells.y[3, 0] = -1e-9
    wl.cells.T[1] = 1e7
    net = oracle_mod.OracleNetwork(wl.network)
    r = net.integrate(wl.cells, 1e-12, oracle_mod.options(wl.tol), 1)
    assert np.all(r["status"] == 0)
    assert r["y"][3, 0] >= 0.0
    assert r["T"][1] <= wl.network.t_max * 1.5


def test_network_element_imbalance_rejected(oracle_mod, tmp_path):
    net = I.robertson_network()
    net.counts = np.array([[1], [1], [2]])
    p = str(tmp_path / "bad.net")
    net.write(p)
    with pytest.raises(ValueError):
        oracle_mod.OracleNetwork(p)


# ------------------------------------------------------------------ post-processing
#
# Sec. 2.2.3: negative abundances are clipped, then the element totals b0 of the
# initial state are restored.  The correction is read as the least change of the
# abundances, measured relative to each abundance: minimise sum_s dy_s^2 / y_s
# subject to N (y + dy) = b0.  Its Lagrange condition makes dy_s / y_s a combination
# of the element columns of species s, dy_s = -y_s (N^T lambda)_s, and the constraint
# fixes lambda.  The cases below are solved by hand from that definition.


def _h_h2_network():
    """One element H; species H (1 atom) and H2 (2 atoms); H + H -> H2."""
    return I._irreversible("h_h2", ["H", "H2"], ["H"], [1.0, 2.0], [0.0, 0.0], [1.0, 1.0],
                           [[1], [2]], 0, 300.0, 10.0, 1e5, [((0, 0), (1,), 1.0, 0.0, 0.0, -1)])


def _h_o_network():
    """Elements H, O; species H, O, OH, H2O; H + O -> OH, H + OH -> H2O."""
    return I._irreversible("h_o", ["H", "O", "OH", "H2O"], ["H", "O"], [1.0, 16.0, 17.0, 18.0],
                           [0.0] * 4, [1.0] * 4, [[1, 0], [0, 1], [1, 1], [2, 1]], 0, 300.0,
                           10.0, 1e5, [((0, 1), (2,), 1.0, 0.0, 0.0, -1),
                                       ((0, 2), (3,), 1.0, 0.0, 0.0, -1)])


def test_post_process_one_element_hand_solved(oracle_mod):
    """y = (H 0.5, H2 0.25) carries 1.0 H atoms against b0 = 0.999.  Then
    lambda = (1.0 - 0.999) / (1*0.5 + 4*0.25) = 1/1500 and
    y' = (0.5 (1 - 1/1500), 0.25 (1 - 2/1500)) = (0.5 - 1/3000, 0.25 - 1/3000)."""
    net = oracle_mod.OracleNetwork(_h_h2_network())
    rc, y = net.post_process([0.5, 0.25], [0.999])
    assert rc == 0
    exact = [Fraction(1, 2) - Fraction(1, 3000), Fraction(1, 4) - Fraction(1, 3000)]
    for got, ref in zip(y, exact):
        assert abs(Fraction(got) - ref) <= 8 * EPS * ref
    assert abs(y[0] + 2 * y[1] - 0.999) <= 4 * EPS


def test_post_process_two_elements_hand_solved(oracle_mod):
    """y = (H 1/2, O 1/4, OH 1/8, H2O 1/16) and lambda = (2^-10, -2^-9) chosen first.
    N y = (3/4, 7/16); N diag(y) N^T = [[7/8, 1/4], [1/4, 7/16]], so its product with
    lambda is (3/8, -5/8)/1024 and b0 = (3/4 - 3/8192, 7/16 + 5/8192).  The answer is
    y_s (1 - (N^T lambda)_s) = (1/2 - 1/2048, 1/4 + 1/2048, 1/8 + 1/8192, 1/16): every
    number here is a short binary fraction, exact in FP64."""
    net = oracle_mod.OracleNetwork(_h_o_network())
    b0 = [0.75 - 0.375 / 1024, 0.4375 + 0.625 / 1024]
    rc, y = net.post_process([0.5, 0.25, 0.125, 0.0625], b0)
    assert rc == 0
    ref = np.array([0.5 - 0.5 / 1024, 0.25 + 0.5 / 1024, 0.125 + 0.125 / 1024, 0.0625])
    assert np.all(np.abs(y - ref) <= 8 * EPS * ref)


def test_post_process_clip_keeps_clipped_species_at_zero(oracle_mod):
    """A negative abundance is set to 0 and, being weighted by its own value, stays 0;
    the other species carry the whole correction."""
    net = oracle_mod.OracleNetwork(_h_o_network())
    y_in = np.array([0.5, -1e-6, 0.125, 0.0625])
    b0 = np.array([0.75 * (1 + 1e-3), 0.1875 * (1 - 2e-3)])
    rc, y = net.post_process(y_in, b0)
    assert rc == 0
    assert y[1] == 0.0
    counts = np.array([[1, 0], [0, 1], [1, 1], [2, 1]], float)
    assert np.all(np.abs(counts.T @ y - b0) <= 4 * EPS * b0)


@pytest.mark.parametrize("wid", [2, 3, 5])
def test_post_process_is_the_least_relative_change(oracle_mod, wid):
    """Random states of the workload networks with an O(1e-3) element defect and one
    clipped negative: the totals come back to 1e-14, and the result equals the
    minimum-norm solution of the scaled constraint (N W)(z) = b0 - N y, dy = W z with
    W = diag(sqrt(y)), computed independently through numpy's SVD pseudo-inverse."""
    netw = I.network(wid)
    net = oracle_mod.OracleNetwork(netw)
    rng = np.random.default_rng(wid)
    Nm = netw.counts.T.astype(float)
    for trial in range(5):
        y = 10.0 ** rng.uniform(-12, 0, netw.ns)
        y[rng.integers(netw.ns)] = -1e-14
        yc = np.maximum(y, 0.0)
        b0 = Nm @ yc * (1.0 + 1e-3 * rng.uniform(-1, 1, netw.ne))
        rc, got = net.post_process(y, b0)
        assert rc == 0
        assert np.all(np.abs(Nm @ got - b0) <= 1e-14 * b0)
        W = np.sqrt(yc)
        z = np.linalg.pinv(Nm * W[None, :]) @ (b0 - Nm @ yc)
        ref = yc + W * z
        # the SVD route is accurate relative to the correction it computes
        assert np.all(np.abs(got - ref) <= 1e-9 * np.abs(ref - yc) + 8 * EPS * yc + 1e-300)
        assert np.all(got >= 0.0)


def test_post_process_failure_rules(oracle_mod):
    """A correction that would remove 100 % or more of a species fails, as does a
    defect in an element that no species holds any more; a zero defect there is fine."""
    h2 = oracle_mod.OracleNetwork(_h_h2_network())
    # lambda = 0.6: H2 would lose 2*0.6 = 120 % of itself
    rc, _ = h2.post_process([0.5, 0.25], [1.0 - 0.6 * 1.5])
    assert rc != 0
    # lambda = 0.45: H keeps 55 %, H2 10 %
    rc, y = h2.post_process([0.5, 0.25], [1.0 - 0.45 * 1.5])
    assert rc == 0
    assert y == pytest.approx([0.5 * 0.55, 0.25 * 0.1], rel=1e-14)
    ho = oracle_mod.OracleNetwork(_h_o_network())
    rc, _ = ho.post_process([0.5, 0.0, 0.0, 0.0], [0.5, 1e-3])
    assert rc != 0
    rc, y = ho.post_process([0.5, 0.0, 0.0, 0.0], [0.5 * (1 - 1e-3), 0.0])
    assert rc == 0
    assert y == pytest.approx([0.5 * (1 - 1e-3), 0.0, 0.0, 0.0], rel=1e-14)


# ------------------------------------------------------------------ TR-BDF2 (second scheme)
#
# The one-step scheme with one iteration matrix per step (Bank et al. 1985): a
# trapezoidal stage to t + gamma h and a BDF2 stage to t + h, gamma = 2 - sqrt(2).  On a
# linear system y' = K y each stage is one linear solve with I - d h K, d = gamma/2.

GAMMA = 2.0 - math.sqrt(2.0)


def _chain(k1=2.0, k2=50.0):
    K = np.array([[-k1, 0, 0], [k1, -k2, 0], [0, k2, 0]])
    return I.decay_chain_network(k1, k2), K


def _trbdf2_linear(K, y, h):
    """One TR-BDF2 step on y' = K y written as two linear solves."""
    g, d = GAMMA, GAMMA / 2
    A = np.eye(len(y)) - d * h * K
    yg = np.linalg.solve(A, (np.eye(len(y)) + d * h * K) @ y)
    w1, w0 = 1 / (g * (2 - g)), (1 - g) ** 2 / (g * (2 - g))
    return np.linalg.solve(A, w1 * yg - w0 * y)


def test_trbdf2_fixed_step_linear_chain(oracle_mod):
    netw, K = _chain()
    net = oracle_mod.OracleNetwork(netw)
    y0 = np.array([0.7, 0.2, 0.1])
    cells = I.Cells(y0.reshape(3, 1).copy(), np.array([300.0]), np.array([1.0]))
    r = net.integrate(cells, 1.0, oracle_mod.options(atol=1e-14, h_init=0.01, adaptive=0, retry=0,
                                                     newton_rtol=1e-14, scheme=1), 1)
    ref = y0.copy()
    for _ in range(100):
        ref = _trbdf2_linear(K, ref, 0.01)
    assert r["nsub"][0] == 100
    assert np.allclose(r["y"][:, 0], ref, rtol=1e-13, atol=1e-16)


def test_trbdf2_is_second_order(oracle_mod):
    """Fixed steps against the exact solution expm(K t) y0: halving h divides the error
    by 4 (backward Euler would divide it by 2)."""
    from scipy.linalg import expm
    netw, K = _chain(3.0, 7.0)
    net = oracle_mod.OracleNetwork(netw)
    y0 = np.array([0.9, 0.1, 0.0])
    exact = expm(K * 1.0) @ y0
    errs = []
    for h in (0.02, 0.01, 0.005):
        cells = I.Cells(y0.reshape(3, 1).copy(), np.array([300.0]), np.array([1.0]))
        r = net.integrate(cells, 1.0, oracle_mod.options(atol=1e-16, h_init=h, adaptive=0, retry=0,
                                                         newton_rtol=1e-15, scheme=1), 1)
        errs.append(np.abs(r["y"][:, 0] - exact).max())
    assert 3.7 < errs[0] / errs[1] < 4.3 and 3.7 < errs[1] / errs[2] < 4.3, errs


def test_trbdf2_estimate_is_the_local_error(oracle_mod):
    """One step from y0: the estimate equals expm(h K) y0 - y1 to leading order, so
    its ratio to the true local error tends to 1 as h shrinks."""
    from scipy.linalg import expm
    netw, K = _chain(3.0, 7.0)
    net = oracle_mod.OracleNetwork(netw)
    y0 = np.array([0.9, 0.1, 0.0])
    opts = oracle_mod.options(atol=1e-16, newton_rtol=1e-15, scheme=1)
    for h, tol in ((1e-2, 0.15), (2.5e-3, 0.04)):
        rc, y1, est = net.trbdf2_step(y0, h, opts)
        assert rc == 0
        true = expm(K * h) @ y0 - y1
        assert np.all(np.abs(est / true - 1.0) < tol), (h, est, true)


def test_trbdf2_adaptive_bateman_accuracy(oracle_mod):
    """Adaptive TR-BDF2 on A -> B -> C against the Bateman closed form.  The control
    keeps the local error per step near rtol, so steps scale like rtol^(1/3) and a
    second-order method's global error like h^2 ~ rtol^(2/3): slope 2/3 in log-log (the
    first-order scheme's is 1/2), and the error stays below 2 rtol^(2/3)."""
    net = oracle_mod.OracleNetwork(I.decay_chain_network(1.0, 10.0))
    cells = I.Cells(np.array([[1.0], [0.0], [0.0]]), np.array([300.0]), np.array([1.0]))
    A = math.exp(-2.0)
    B = 1 / 9 * (math.exp(-2.0) - math.exp(-20.0))
    ref = np.array([A, B, 1 - A - B])
    errs, nsub = [], []
    for rtol in (1e-4, 1e-6, 1e-8):
        r = net.integrate(cells, 2.0, oracle_mod.options(rtol=rtol, atol=1e-14, h_init=1e-6, scheme=1), 1)
        errs.append(np.abs(r["y"][:, 0] / ref - 1).max())
        nsub.append(int(r["nsub"][0]))
    for e, rtol in zip(errs, (1e-4, 1e-6, 1e-8)):
        assert e <= 2.0 * rtol ** (2 / 3), errs
    for a, b in zip(errs, errs[1:]):
        assert 0.6 <= math.log10(a / b) / 2 <= 0.73, errs
    # the step count grows like rtol^(-1/3): x100 tighter -> ~4.6x the steps
    assert 3.0 < nsub[1] / nsub[0] < 7.0 and 3.0 < nsub[2] / nsub[1] < 7.0, nsub


def test_trbdf2_robertson_vs_radau(oracle_mod):
    from scipy.integrate import solve_ivp
    wl = I.workload(1, 3)
    net = oracle_mod.OracleNetwork(wl.network)
    r = net.integrate(wl.cells, 1e4, oracle_mod.options(wl.tol, scheme=1), 1)
    assert np.all(r["status"] == 0)
    for c in range(3):
        y0 = wl.cells.y[:, c]

        def f(t, y):
            return [-0.04 * y[0] + 1e4 * y[1] * y[2], 0.04 * y[0] - 1e4 * y[1] * y[2] - 3e7 * y[1] ** 2,
                    3e7 * y[1] ** 2]
        ref = solve_ivp(f, (0, 1e4), y0, method="Radau", rtol=1e-13, atol=1e-20).y[:, -1]
        assert np.abs(r["y"][:, c] / ref - 1).max() <= 1e-4
        assert abs(r["y"][:, c].sum() - y0.sum()) <= 1e-14


@pytest.mark.parametrize("wid", [2, 3])
def test_trbdf2_conservation(oracle_mod, wid):
    """Both stages are combinations of states and rates, so the element totals and the
    energy invariant are kept to rounding, as with backward Euler."""
    wl = I.workload(wid, 4)
    netw = wl.network
    net = oracle_mod.OracleNetwork(netw)
    r = net.integrate(wl.cells, wl.tol.dt, oracle_mod.options(wl.tol, scheme=1), 2)
    assert np.all(r["status"] == 0)
    y0 = np.maximum(wl.cells.y, 0.0)
    b0, b1 = netw.counts.T @ y0, netw.counts.T @ r["y"]
    assert np.all(np.abs(b1 - b0) <= 1e-12 * b0)
    assert np.all(r["y"] >= 0.0)
    if netw.energy:
        cv = netw.cv @ y0
        E0 = cv * wl.cells.T + netw.h @ y0
        E1 = cv * r["T"] + netw.h @ r["y"]
        assert np.all(np.abs(E1 - E0) <= 1e-12 * (cv * wl.cells.T + np.abs(netw.h) @ y0))



# ------------------------------------------------------------------ C_V(T) (Sec. 4.2)


def _cv_antiderivative(netw, n0, T):
    """E(T) = integral_0^T C_V(T') dT' for C_V(T) = sum_s n0_s cv_s(T), piecewise, by
    numpy's exact polynomial integration (independent of the oracle's evaluation)."""
    P = np.polynomial.polynomial
    lo = np.einsum("s,sk->k", n0, netw.cv_poly[:, 0, :])
    hi = np.einsum("s,sk->k", n0, netw.cv_poly[:, 1, :])
    Ilo, Ihi = P.polyint(lo), P.polyint(hi)
    tm = netw.t_mid
    T = np.asarray(T, float)
    below = P.polyval(np.minimum(T, tm), Ilo)
    above = np.where(T > tm, P.polyval(np.maximum(T, tm), Ihi) - P.polyval(tm, Ihi), 0.0)
    return below + above


def test_cv_poly_constant_reproduces_constant_network(oracle_mod):
    """Polynomials that are constants (a0 = cv_s) give bit for bit the constant-C_V run."""
    import dataclasses
    base = I.network(2)
    poly = np.zeros((base.ns, 2, 5))
    poly[:, 0, 0] = poly[:, 1, 0] = base.cv
    flat = dataclasses.replace(base, cv_poly=poly)
    wl = I.workload(2, 4)
    for scheme in (0, 1):
        opts = oracle_mod.options(wl.tol, scheme=scheme)
        a = oracle_mod.OracleNetwork(base).integrate(wl.cells, wl.tol.dt * 1e-2, opts, 2)
        b = oracle_mod.OracleNetwork(flat).integrate(wl.cells, wl.tol.dt * 1e-2, opts, 2)
        for k in ("y", "T", "nsub", "nnewton", "status"):
            assert np.array_equal(a[k], b[k]), (scheme, k)


def test_cv_poly_energy_balance(oracle_mod):
    """With C_V(T) the energy E(T) + sum_s h_s n_s, E the antiderivative of C_V, is
    conserved by the ODE; it is nonlinear in T, so the scheme keeps it to its
    discretisation error, which shrinks with rtol (TR-BDF2: ~rtol^(2/3))."""
    wl = I.workload(6, 6)
    netw = wl.network
    net = oracle_mod.OracleNetwork(netw)
    y0 = np.maximum(wl.cells.y, 0.0)
    res = []
    for rtol in (1e-6, 1e-9):
        r = net.integrate(wl.cells, wl.tol.dt, oracle_mod.options(wl.tol, scheme=1, rtol=rtol,
                                                                  max_substeps=2000000), 2)
        assert np.all(r["status"] == 0)
        worst = 0.0
        for c in range(wl.cells.ncells):
            dE = (_cv_antiderivative(netw, y0[:, c], r["T"][c]) - _cv_antiderivative(netw, y0[:, c], wl.cells.T[c])
                  + netw.h @ (r["y"][:, c] - y0[:, c]))
            scale = np.abs(netw.h) @ y0[:, c]
            worst = max(worst, abs(dE) / scale)
        res.append(worst)
    assert res[0] <= 1e-6 and res[1] <= 1e-8 and res[1] < res[0] / 30, res


def test_cv_poly_lowers_the_temperature_rise(oracle_mod):
    """The synthetic C_V(T) is above the constant C_V at every T, so the same heat
    release raises T less (the paper's frozen-C_V control overpredicts T by ~15 %)."""
    wl = I.workload(6, 6)
    const = I.workload(2, 6)
    a = oracle_mod.OracleNetwork(wl.network).integrate(wl.cells, wl.tol.dt, oracle_mod.options(wl.tol, scheme=1), 2)
    b = oracle_mod.OracleNetwork(const.network).integrate(const.cells, wl.tol.dt, oracle_mod.options(wl.tol, scheme=1), 2)
    assert np.array_equal(wl.cells.y, const.cells.y) and np.array_equal(wl.cells.T, const.cells.T)
    rise_poly, rise_const = a["T"] - wl.cells.T, b["T"] - wl.cells.T
    hot = rise_const > 100.0
    assert hot.any()
    assert np.all(rise_poly[hot] < rise_const[hot])


# ------------------------------------------------------------------ tabulated and photo rates


def test_table_linear_in_log_T_reproduces_arrhenius(oracle_mod):
    """ln k linear in ln T (theta = 0) is interpolated exactly, so a tabulated copy of
    such reactions integrates like the Arrhenius network (rounding only), rates, dk/dT
    and the energy equation included."""
    import dataclasses
    base = I.network(2)
    theta = base.theta.copy()
    pick = [0, 3, 7, 12, 20]
    theta[pick] = 0.0
    arr = dataclasses.replace(base, theta=theta)
    Tn = np.geomspace(5.0, 2e5, 17)
    tables = {r: np.tile(math.log(base.A[r]) + base.b[r] * np.log(Tn / base.t_ref), (3, 1)) for r in pick}
    tab = dataclasses.replace(arr, tables=tables, table_grid=(17, 5.0, 2e5, 3, 1e-6, 1e2))
    a, b = oracle_mod.OracleNetwork(arr), oracle_mod.OracleNetwork(tab)
    for T in (37.0, 950.0, 2345.6, 7777.0):
        y = np.append(np.ones(base.ns), T)           # the energy network reads T from y
        ka, dka = a.rates_cell(y, rho=0.3)
        kb, dkb = b.rates_cell(y, rho=0.3)
        assert np.allclose(kb, ka, rtol=1e-13, atol=0) and np.allclose(dkb, dka, rtol=1e-12, atol=0)
    wl = I.workload(2, 4)
    ra = a.integrate(wl.cells, wl.tol.dt, oracle_mod.options(wl.tol, scheme=1), 2)
    rb = b.integrate(wl.cells, wl.tol.dt, oracle_mod.options(wl.tol, scheme=1), 2)
    assert np.allclose(rb["y"], ra["y"], rtol=1e-9, atol=1e-30)
    assert np.allclose(rb["T"], ra["T"], rtol=1e-11)


def test_table_density_reduction_and_slope(oracle_mod):
    """Pre-processing reduces the (T, rho) table at the cell's density: ln k linear in
    ln rho comes out exactly; inside a T segment dk/dT equals the central difference
    of k, and beyond the grid k is the end value with dk/dT = 0."""
    import dataclasses
    base = I.robertson_network()
    Tn = np.geomspace(10.0, 1e4, 7)
    Rn = np.geomspace(1e-2, 1e2, 5)
    c, a0 = 0.37, math.log(2e-3)
    lnk = a0 + c * np.log(Rn)[:, None] + 0.5 * np.sin(np.arange(7))[None, :]
    net = oracle_mod.OracleNetwork(dataclasses.replace(base, tables={0: lnk},
                                                      table_grid=(7, 10.0, 1e4, 5, 1e-2, 1e2)))
    y = np.ones(3)
    for rho in (0.013, 1.0, 47.0):
        k, _ = net.rates_cell(y, T_iso=Tn[3], rho=rho)
        assert k[0] == pytest.approx(math.exp(a0 + 0.5 * math.sin(3)) * rho ** c, rel=1e-13)
    T, h = 123.0, 1e-4
    k, dk = net.rates_cell(y, T_iso=T, rho=2.0)
    kp, _ = net.rates_cell(y, T_iso=T + h, rho=2.0)
    km, _ = net.rates_cell(y, T_iso=T - h, rho=2.0)
    assert dk[0] == pytest.approx((kp[0] - km[0]) / (2 * h), rel=1e-6)
    k_lo, dk_lo = net.rates_cell(y, T_iso=3.0, rho=2.0)
    k_hi, dk_hi = net.rates_cell(y, T_iso=5e4, rho=2.0)
    k0, _ = net.rates_cell(y, T_iso=10.0, rho=2.0)
    k6, _ = net.rates_cell(y, T_iso=1e4, rho=2.0)
    assert k_lo[0] == pytest.approx(k0[0], rel=1e-14) and dk_lo[0] == 0.0
    assert k_hi[0] == pytest.approx(k6[0], rel=1e-14) and dk_hi[0] == 0.0


def _photolysis_network(sigma):
    """X -> Y by photo-dissociation (cross-section sigma), one element shared."""
    return I._irreversible("photolysis", ["X", "Y"], ["E"], [1.0, 1.0], [0.0, 0.0], [1.0, 1.0],
                           [[1], [1]], 0, 300.0, 10.0, 1e5, [((0,), (1,), 1.0, 0.0, 0.0, -1)])


def test_photo_rate_thin_limit_and_shielding(oracle_mod):
    """k = F sigma (1 - e^-tau)/tau with tau = dl sum n sigma: F sigma when dl = 0,
    F sigma / tau when tau >> 1 (Eq. photo-reaction-single)."""
    import dataclasses
    sig, F = 3e-18, 2e9
    net = oracle_mod.OracleNetwork(dataclasses.replace(_photolysis_network(sig), photo={0: sig}))
    k, dk = net.rates_cell(np.array([1e4, 0.0]), flux=F, path=0.0)
    assert k[0] == F * sig and dk[0] == 0.0
    for n, dl in ((1e4, 1e10), (1e5, 1e16), (1e8, 1e18)):
        tau = dl * n * sig
        k, _ = net.rates_cell(np.array([n, 0.0]), flux=F, path=dl)
        assert k[0] == pytest.approx(F * sig * -math.expm1(-tau) / tau, rel=1e-13)


@pytest.mark.parametrize("tau0", [1e-3, 1.0, 30.0])
def test_photolysis_closed_form(oracle_mod, tau0):
    """dn/dt = -F sigma phi(a n) n = -(F/dl)(1 - e^{-a n}), a = dl sigma, integrates to
    n(t) = ln(1 + (e^{a n0} - 1) e^{-sigma F t}) / a.  TR-BDF2 at rtol 1e-9 matches it
    to its own accuracy; X + Y stays exact."""
    import dataclasses
    sig, F, dl = 1e-18, 1e8, 1e17
    net = oracle_mod.OracleNetwork(dataclasses.replace(_photolysis_network(sig), photo={0: sig}))
    a = dl * sig
    n0 = tau0 / a
    t = 2.0 / (sig * F)
    cells = I.Cells(np.array([[n0], [0.0]]), np.array([300.0]), np.array([1.0]),
                    np.array([F]), np.array([dl]))
    r = net.integrate(cells, t, oracle_mod.options(rtol=1e-9, atol=1e-30 + 1e-12 * n0, h_init=1e-6 * t,
                                                   scheme=1), 1)
    assert r["status"][0] == 0
    exact = math.log1p(math.expm1(a * n0) * math.exp(-sig * F * t)) / a
    assert r["y"][0, 0] == pytest.approx(exact, rel=1e-5)
    assert r["y"][:, 0].sum() == pytest.approx(n0, rel=1e-14)


@pytest.mark.parametrize("wid", [7, 8])
def test_jacobian_with_tables_and_photo(oracle_mod, wid):
    """Central differences of f on the radiation (photo + tabulated) and tabulated
    workload networks, at each cell's density, flux and path length."""
    netw = I.network(wid)
    net = oracle_mod.OracleNetwork(netw)
    wl = I.workload(wid, 4)
    for c in range(3):
        y = wl.cells.y[:, c].copy()
        T = float(wl.cells.T[c])
        kw = dict(rho=float(wl.cells.rho[c]))
        if wl.cells.flux is not None:
            kw.update(flux=float(wl.cells.flux[c]), path=float(wl.cells.path[c]))
        cvtot = float(np.dot(netw.cv, y)) if netw.energy else 1.0
        if netw.energy:
            y = np.append(y, T)
        J = net.jacobian(y, T, cvtot, None, **kw)
        Jfd = np.zeros_like(J)
        floor = 1e-6 * np.abs(y).max()
        for m in range(len(y)):
            h = 1e-6 * max(abs(y[m]), floor)
            yp, ym = y.copy(), y.copy()
            yp[m] += h
            ym[m] -= h
            Jfd[:, m] = (net.rhs(yp, T, cvtot, None, **kw) - net.rhs(ym, T, cvtot, None, **kw)) / (2 * h)
        s = np.maximum(np.abs(y), 1e-6 * np.abs(y).max())
        Js, Fs = J * s[None, :], Jfd * s[None, :]
        scale = np.maximum(np.abs(Js), np.abs(Fs)).max(axis=1, keepdims=True) + 1e-300
        assert np.all(np.abs(Js - Fs) <= 1e-6 * scale), (wid, c)


@pytest.mark.parametrize("wid", [7, 8])
def test_tables_and_photo_conservation(oracle_mod, wid):
    wl = I.workload(wid, 4)
    netw = wl.network
    r = oracle_mod.OracleNetwork(netw).integrate(wl.cells, wl.tol.dt, oracle_mod.options(wl.tol, scheme=1), 2)
    assert np.all(r["status"] == 0)
    y0 = np.maximum(wl.cells.y, 0.0)
    b0, b1 = netw.counts.T @ y0, netw.counts.T @ r["y"]
    assert np.all(np.abs(b1 - b0) <= 1e-12 * b0)
    assert np.all(r["y"] >= 0.0)
