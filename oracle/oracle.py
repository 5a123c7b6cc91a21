"""ctypes front-end of the FP64 CPU oracle (``kt_oracle.c``).

TEST INFRASTRUCTURE: only tests, the package smoke check and the benchmark's
CPU-baseline / reference legs use this module.  It shares nothing with the CUDA
path beyond the seeded inputs of ``paper_2504_04941_gb300.inputs``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kt_oracle.c")
LIB = os.path.join(HERE, "libkt_oracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L",
                               "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, SRC, "-lm", "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


class Options(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("h_init", ctypes.c_double), ("h_min", ctypes.c_double),
                ("newton_rtol", ctypes.c_double), ("newton_atol_frac", ctypes.c_double),
                ("facmax", ctypes.c_double), ("retry_h_factor", ctypes.c_double),
                ("retry_facmax", ctypes.c_double),
                ("max_substeps", ctypes.c_int), ("max_newton", ctypes.c_int),
                ("adaptive", ctypes.c_int), ("retry", ctypes.c_int),
                ("atol_mode", ctypes.c_int), ("guess", ctypes.c_int), ("scheme", ctypes.c_int)]


class CellPar(ctypes.Structure):
    """Per-cell parameters of the single-state pins (ko_cellpar)."""
    _fields_ = [("T_iso", ctypes.c_double), ("cvtot", ctypes.c_double),
                ("n0", ctypes.POINTER(ctypes.c_double)), ("rho", ctypes.c_double),
                ("flux", ctypes.c_double), ("path", ctypes.c_double)]


def options(tol=None, **kw) -> Options:
    """Options from an ``inputs.Tolerances`` plus keyword overrides."""
    d = dict(rtol=1e-6, atol=1e-10, h_init=1e-6, h_min=1e-30, newton_rtol=1e-12,
             newton_atol_frac=1e-2, facmax=4.0, retry_h_factor=1e-3, retry_facmax=2.0,
             max_substeps=100000, max_newton=8, adaptive=1, retry=1, atol_mode=0, guess=0,
             scheme=0)
    if tol is not None:
        d.update(rtol=tol.rtol, atol=tol.atol, h_init=tol.h_init, h_min=tol.h_min,
                 max_substeps=tol.max_substeps, max_newton=tol.max_newton,
                 atol_mode=tol.atol_mode)
    d.update(kw)
    return Options(**d)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            vp, dp, ip, i32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), \
                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int32)
            L.ko_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp)]
            L.ko_free.argtypes = [vp]
            L.ko_info.argtypes = [vp, ip, ip, ip, ip]
            L.ko_rates.argtypes = [vp, ctypes.c_double, dp, dp]
            cp = ctypes.POINTER(CellPar)
            L.ko_rhs.argtypes = [vp, dp, cp, dp]
            L.ko_jacobian.argtypes = [vp, dp, cp, dp]
            L.ko_rates_cell.argtypes = [vp, dp, cp, dp, dp]
            L.ko_lu.argtypes = [ctypes.c_int, dp, ip]
            L.ko_lu_solve.argtypes = [ctypes.c_int, dp, ip, dp]
            L.ko_lu_solve.restype = None
            L.ko_integrate_rad.argtypes = [vp, ctypes.c_int64, dp, dp, dp, dp, dp, ctypes.c_double,
                                           ctypes.POINTER(Options), ctypes.c_int, dp, dp,
                                           i32p, i32p, i32p]
            L.ko_be_step.argtypes = [vp, ctypes.POINTER(Options), dp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, dp, ip]
            L.ko_post_process.argtypes = [vp, dp, dp]
            L.ko_trbdf2_step.argtypes = [vp, ctypes.POINTER(Options), dp, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, dp, dp]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleNetwork:
    """A network loaded by the oracle's own parser."""

    def __init__(self, net_or_path):
        L = lib()
        if isinstance(net_or_path, str):
            path = net_or_path
            self._tmp = None
        else:
            fd, path = tempfile.mkstemp(suffix=".net")
            os.close(fd)
            net_or_path.write(path)
            self._tmp = path
        self.ptr = ctypes.c_void_p()
        rc = L.ko_load(path.encode(), ctypes.byref(self.ptr))
        if rc != 0:
            raise ValueError(f"oracle failed to load network {path}: code {rc}")
        a, b, c, d = (ctypes.c_int() for _ in range(4))
        L.ko_info(self.ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d))
        self.ns, self.ne, self.nr, self.energy = a.value, b.value, c.value, d.value
        self.n = self.ns + self.energy

    def __del__(self):
        try:
            if self.ptr:
                lib().ko_free(self.ptr)
            if self._tmp and os.path.exists(self._tmp):
                os.unlink(self._tmp)
        except Exception:
            pass

    # --- building blocks (pins) ---
    def rates(self, T: float):
        k = np.zeros(max(self.nr, 1))
        dk = np.zeros(max(self.nr, 1))
        rc = lib().ko_rates(self.ptr, float(T), _dp(k), _dp(dk))
        if rc:
            raise ValueError("rates failed")
        return k[:self.nr], dk[:self.nr]

    @staticmethod
    def _par(T_iso, cvtot, n0, rho, flux, path):
        n0 = None if n0 is None else np.ascontiguousarray(n0, float)
        p = CellPar(float(T_iso), float(cvtot), None if n0 is None else _dp(n0), float(rho),
                    float(flux), float(path))
        return p, n0

    def rhs(self, y, T_iso: float = 300.0, cvtot: float = 1.0, n0=None, rho: float = 1.0,
            flux: float = 1.0, path: float = 0.0):
        """f(y); cvtot is C_V of constant-heat-capacity networks, n0 the frozen
        composition of C_V(T) on polynomial ones; rho reduces the rate tables; flux and
        path are the photo-reaction parameters of the cell."""
        y = np.ascontiguousarray(y, float)
        f = np.zeros(self.n)
        p, keep = self._par(T_iso, cvtot, n0, rho, flux, path)
        rc = lib().ko_rhs(self.ptr, _dp(y), ctypes.byref(p), _dp(f))
        if rc:
            raise ValueError("rhs failed")
        return f

    def jacobian(self, y, T_iso: float = 300.0, cvtot: float = 1.0, n0=None, rho: float = 1.0,
                 flux: float = 1.0, path: float = 0.0):
        y = np.ascontiguousarray(y, float)
        J = np.zeros((self.n, self.n))
        p, keep = self._par(T_iso, cvtot, n0, rho, flux, path)
        rc = lib().ko_jacobian(self.ptr, _dp(y), ctypes.byref(p), _dp(J))
        if rc:
            raise ValueError("jacobian failed")
        return J

    def rates_cell(self, y, T_iso: float = 300.0, rho: float = 1.0, flux: float = 1.0,
                   path: float = 0.0):
        """Every reaction's k and dk/dT for one cell (Arrhenius, tabulated, photo)."""
        y = np.ascontiguousarray(y, float)
        k = np.zeros(max(self.nr, 1))
        dk = np.zeros(max(self.nr, 1))
        p, keep = self._par(T_iso, 1.0, None, rho, flux, path)
        rc = lib().ko_rates_cell(self.ptr, _dp(y), ctypes.byref(p), _dp(k), _dp(dk))
        if rc:
            raise ValueError("rates failed")
        return k[:self.nr], dk[:self.nr]

    def be_step(self, yn, h, opts: Options, T_iso: float = 300.0, cvtot: float = 1.0):
        yn = np.ascontiguousarray(yn, float)
        y = np.zeros(self.n)
        it = ctypes.c_int()
        rc = lib().ko_be_step(self.ptr, ctypes.byref(opts), _dp(yn), float(T_iso),
                              float(cvtot), float(h), _dp(y), ctypes.byref(it))
        return rc, y, it.value

    def trbdf2_step(self, yn, h, opts: Options, T_iso: float = 300.0, cvtot: float = 1.0):
        """One TR-BDF2 step: (rc, y_{n+1}, local error estimate)."""
        yn = np.ascontiguousarray(yn, float)
        y = np.zeros(self.n)
        est = np.zeros(self.n)
        rc = lib().ko_trbdf2_step(self.ptr, ctypes.byref(opts), _dp(yn), float(T_iso),
                                  float(cvtot), float(h), _dp(y), _dp(est))
        return rc, y, est

    def post_process(self, y, b0):
        """Clip + element-total correction of one state (Sec. 2.2.3): (rc, corrected y)."""
        y = np.array(y, float)
        if y.shape[0] == self.ns:
            y = np.append(y, 0.0) if self.energy else y
        b0 = np.ascontiguousarray(b0, float)
        assert b0.shape == (self.ne,)
        rc = lib().ko_post_process(self.ptr, _dp(y), _dp(b0))
        return rc, y[:self.ns]

    def integrate(self, cells, dt: float, opts: Options, nthreads: Optional[int] = None):
        """Integrate SoA cells (``inputs.Cells``) over dt; returns a dict of arrays."""
        L = lib()
        nc = cells.T.shape[0]
        y = np.ascontiguousarray(cells.y, float)
        T = np.ascontiguousarray(cells.T, float)
        rho = np.ascontiguousarray(cells.rho, float)
        flux = None if getattr(cells, "flux", None) is None else np.ascontiguousarray(cells.flux, float)
        path = None if getattr(cells, "path", None) is None else np.ascontiguousarray(cells.path, float)
        yo = np.zeros_like(y)
        To = np.zeros_like(T)
        st = np.zeros(nc, np.int32)
        nsub = np.zeros(nc, np.int32)
        nnew = np.zeros(nc, np.int32)
        if nthreads is None:
            nthreads = os.cpu_count() or 1
        i32 = ctypes.POINTER(ctypes.c_int32)
        opt = lambda a: None if a is None else _dp(a)
        rc = L.ko_integrate_rad(self.ptr, nc, _dp(y), _dp(T), _dp(rho), opt(flux), opt(path),
                                float(dt), ctypes.byref(opts),
                                int(nthreads), _dp(yo), _dp(To), st.ctypes.data_as(i32),
                            nsub.ctypes.data_as(i32), nnew.ctypes.data_as(i32))
        if rc:
            raise ValueError(f"oracle integrate failed: code {rc}")
        return dict(y=yo, T=To, status=st, nsub=nsub, nnewton=nnew)


def lu(a):
    """Oracle Crout LU of a square matrix: returns (rc, factors, perm)."""
    a = np.array(a, float, order="C")
    n = a.shape[0]
    perm = np.zeros(n, np.intc)
    rc = lib().ko_lu(n, _dp(a), perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return rc, a, perm


def lu_solve(fac, perm, b):
    x = np.array(b, float)
    perm = np.ascontiguousarray(perm, np.intc)
    lib().ko_lu_solve(fac.shape[0], _dp(np.ascontiguousarray(fac)),
                      perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(x))
    return x
