"""Plain FP64 CPU oracle of the stage-system solve (Pazner & Persson,
arXiv 1701.07181).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference leg may import it.  It shares no code
with the library's CUDA path and imports nothing from the package.

The arithmetic lives in ``irk_oracle.c`` (serial C, FP64) and in
``tableau.py`` (Radau IIA by collocation, App. A).  This module only compiles
the C file with gcc (on first use, or via ``build()``) and marshals numpy
arrays through ctypes.

Vectors are stage-major, ``X[(k*T + i)*m + a]`` (the stacking of Sec. 4.1).

Parity pins (tests/test_oracle_*.py) fix every function here against the
paper or the mathematics; none is left unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import tableau  # noqa: F401  (re-export)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "irk_oracle.c")
_LIB = os.path.join(_HERE, "libirk_oracle.so")
_LIB_OMP = os.path.join(_HERE, "libirk_oracle_omp.so")
_lock = threading.Lock()
_libs = {}

FORM_TRANSFORMED = 0
FORM_UNTRANSFORMED = 1
PC_NONE = 0
PC_UNCOUPLED = 1
PC_STAGE_MAJOR = 2
PC_ELEMENT_MAJOR = 3

_codes = {0: "ok", 1: "not converged", -1: "invalid argument", -2: "out of memory",
          -3: "singular diagonal block", -4: "non-finite value"}


def build(force: bool = False, omp: bool = False) -> str:
    """Compile irk_oracle.c next to it (gcc, -O2): libirk_oracle.so (serial),
    or with omp=True libirk_oracle_omp.so (the same source with -fopenmp)."""
    out = _LIB_OMP if omp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + ".%d.tmp" % os.getpid()
        extra = ["-fopenmp"] if omp else []
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def threads(n: int = 0) -> int:
    """Threads of the multi-core build (n > 0 sets them); returns the count
    its parallel regions use."""
    return int(_load(True).irk_ref_threads(int(n)))


def _load(omp=False):
    with _lock:
        if omp not in _libs:
            path = build(omp=omp)
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I, L, D = ctypes.c_int, ctypes.c_long, ctypes.c_double
            lib.irk_ref_apply_transformed.argtypes = [I, P, I, I, P, P, P, L, P, D, P, P]
            lib.irk_ref_apply_untransformed.argtypes = [I, P, I, I, P, P, P, L, P, D, P, P]
            lib.irk_ref_bilu0.argtypes = [I, I, P, P, P, P, P]
            lib.irk_ref_bilu0_apply.argtypes = [I, I, P, P, P, P, P, P, P]
            lib.irk_ref_bilu0_apply.restype = None
            lib.irk_ref_ilu_alg2.argtypes = [I, I, P, P, P, P, P]
            lib.irk_ref_ilu_alg3.argtypes = [I, I, I, P, P, P, P, P, P]
            lib.irk_ref_assemble_stage_major.argtypes = [I, I, P, I, I, P, P, P, L, P, D, P, P, P]
            lib.irk_ref_assemble_stage_major.restype = L
            lib.irk_ref_assemble_element_major.argtypes = [I, I, P, I, I, P, P, P, L, P, D, P]
            lib.irk_ref_assemble_element_major.restype = None
            lib.irk_ref_assemble_shifted.argtypes = [I, I, P, P, P, P, D, D, P]
            lib.irk_ref_assemble_shifted.restype = None
            lib.irk_ref_shift_column_rule.argtypes = [I, P, P]
            lib.irk_ref_shift_column_rule.restype = None
            lib.irk_ref_solve.argtypes = [I, I, P, P, I, I, P, P, P, L, P, D, I, P, I, I, D, P, P,
                                          P, P, P, P]
            lib.irk_ref_precond_apply.argtypes = [I, I, P, P, I, I, P, P, P, L, P, D, I, P, P, P]
            lib.irk_ref_assemble_ordered.argtypes = [I, I, P, P, P, P, D, D, P, P, P, P, P]
            lib.irk_ref_assemble_ordered.restype = L
            lib.irk_ref_solve_ordered.argtypes = [I, P, I, I, P, P, P, L, P, D, P, P, P, I, I, D, P, P, P,
                                                  P, P]
            lib.irk_ref_precond_apply_ordered.argtypes = [I, P, I, I, P, P, P, L, P, D, P, P, P, P, P]
            lib.irk_ref_threads.argtypes = [I]
            _libs[omp] = lib
    return _libs[omp]


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(rc, what):
    if rc < 0:
        raise RuntimeError("oracle %s failed: %s (%d)" % (what, _codes.get(rc, "?"), rc))
    return rc


class Problem:
    """Host copy of one stage system: pattern, J (shared or per stage), M."""

    def __init__(self, s, T, m, row_ptr, col_idx, J, M, A=None, omp=False):
        """omp=True: run apply / solve / precond_apply in the multi-core build
        (same source and algorithm, independent work spread over threads)."""
        self.omp = bool(omp)
        self.s, self.T, self.m = int(s), int(T), int(m)
        self.row_ptr = _i32(row_ptr)
        self.col_idx = _i32(col_idx)
        J = _f64(J)
        nnzb = int(self.row_ptr[-1])
        per = nnzb * m * m
        if J.size == per:
            self.jstride = 0
        elif J.size == s * per:
            self.jstride = per
        else:
            raise ValueError("J must hold nnzb*m*m (shared) or s*nnzb*m*m (per stage) values")
        self.J = J.reshape(-1)
        self.M = _f64(M).reshape(-1)
        if A is None:
            A = tableau.radau_iia(s)[0]
        self.A = _f64(A)
        self.Ainv = _f64(tableau.inverse(self.A))

    @property
    def n(self):
        return self.T * self.m

    def _args(self):
        return (_p(self.row_ptr), _p(self.col_idx), _p(self.J), self.jstride, _p(self.M))

    def apply(self, X, dt, form=FORM_TRANSFORMED):
        """Y = B X (form 0, eq. big-irk) or the untransformed product (form 1)."""
        lib = _load(self.omp)
        X = _f64(X).reshape(-1)
        Y = np.empty_like(X)
        rp, ci, J, js, M = self._args()
        if form == FORM_TRANSFORMED:
            _check(lib.irk_ref_apply_transformed(self.s, _p(self.Ainv), self.T, self.m, rp, ci, J,
                                                 js, M, float(dt), _p(X), _p(Y)), "apply")
        else:
            _check(lib.irk_ref_apply_untransformed(self.s, _p(self.A), self.T, self.m, rp, ci, J,
                                                   js, M, float(dt), _p(X), _p(Y)), "apply")
        return Y

    def solve(self, R, dt, rtol=1e-8, form=FORM_TRANSFORMED, precond=PC_UNCOUPLED, shift=None,
              restart=30, max_iter=3000, x0=None, history=False):
        """FGMRES(restart) solve; returns dict(x, iters, relres, cycles, rc[, est])."""
        lib = _load(self.omp)
        R = _f64(R).reshape(-1)
        X = np.zeros_like(R) if x0 is None else _f64(x0).reshape(-1).copy()
        it = ctypes.c_int(0)
        cyc = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        est = np.zeros(max_iter + 1) if history else None
        sh = None if shift is None else _f64(shift)
        rp, ci, J, js, M = self._args()
        rc = lib.irk_ref_solve(form, self.s, _p(self.A), _p(self.Ainv), self.T, self.m, rp, ci, J,
                               js, M, float(dt), precond, _p(sh), restart, max_iter, float(rtol),
                               _p(R), _p(X), ctypes.byref(it), ctypes.byref(rr), _p(est),
                               ctypes.byref(cyc))
        _check(rc, "solve")
        out = dict(x=X, iters=it.value, relres=rr.value, cycles=cyc.value, rc=rc)
        if history:
            out["est"] = est[: it.value + 1]
        return out

    def precond_apply(self, v, dt, form=FORM_TRANSFORMED, precond=PC_UNCOUPLED, shift=None):
        """z = P^{-1} v for a freshly built preconditioner."""
        lib = _load(self.omp)
        v = _f64(v).reshape(-1)
        z = np.empty_like(v)
        sh = None if shift is None else _f64(shift)
        rp, ci, J, js, M = self._args()
        _check(lib.irk_ref_precond_apply(form, self.s, _p(self.A), _p(self.Ainv), self.T, self.m,
                                         rp, ci, J, js, M, float(dt), precond, _p(sh), _p(v),
                                         _p(z)), "precond")
        return z

    # --- reordered / partitioned uncoupled preconditioner (Sec. 4.5) -------
    def solve_ordered(self, R, dt, perm=None, part=None, rtol=1e-8, shift=None, restart=30,
                      max_iter=3000):
        lib = _load()
        R = _f64(R).reshape(-1)
        X = np.zeros_like(R)
        it, cyc, rr = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
        pm = None if perm is None else _i32(perm)
        pt = None if part is None else _i32(part)
        sh = None if shift is None else _f64(shift)
        rp, ci, J, js, M = self._args()
        rc = lib.irk_ref_solve_ordered(self.s, _p(self.Ainv), self.T, self.m, rp, ci, J, js, M,
                                       float(dt), _p(sh), _p(pm), _p(pt), restart, max_iter,
                                       float(rtol), _p(R), _p(X), ctypes.byref(it), ctypes.byref(rr),
                                       ctypes.byref(cyc))
        _check(rc, "solve_ordered")
        return dict(x=X, iters=it.value, relres=rr.value, cycles=cyc.value, rc=rc)

    def precond_apply_ordered(self, v, dt, perm=None, part=None, shift=None):
        lib = _load()
        v = _f64(v).reshape(-1)
        z = np.empty_like(v)
        pm = None if perm is None else _i32(perm)
        pt = None if part is None else _i32(part)
        sh = None if shift is None else _f64(shift)
        rp, ci, J, js, M = self._args()
        _check(lib.irk_ref_precond_apply_ordered(self.s, _p(self.Ainv), self.T, self.m, rp, ci, J, js, M,
                                                 float(dt), _p(sh), _p(pm), _p(pt), _p(v), _p(z)),
               "precond_apply_ordered")
        return z

    def assemble_ordered(self, k, d, dt, perm=None, part=None):
        lib = _load()
        mm = self.m * self.m
        nnzb = int(self.row_ptr[-1])
        Jk = self.J[k * self.jstride: k * self.jstride + nnzb * mm] if self.jstride else self.J
        Jk = np.ascontiguousarray(Jk)
        pm = None if perm is None else _i32(perm)
        pt = None if part is None else _i32(part)
        args = (self.T, self.m, _p(self.row_ptr), _p(self.col_idx), _p(Jk), _p(self.M), float(d), float(dt),
                _p(pm), _p(pt))
        nb = lib.irk_ref_assemble_ordered(*args, None, None, None)
        rp = np.zeros(self.T + 1, np.int32)
        ci = np.zeros(nb, np.int32)
        vals = np.zeros(nb * mm)
        lib.irk_ref_assemble_ordered(*args, _p(rp), _p(ci), _p(vals))
        return rp, ci, vals.reshape(nb, self.m, self.m)

    # --- assembled forms (for pins) ---------------------------------------
    def assemble_stage_major(self, dt, form=FORM_TRANSFORMED):
        lib = _load()
        C = self.Ainv if form == FORM_TRANSFORMED else self.A
        rp, ci, J, js, M = self._args()
        nb = lib.irk_ref_assemble_stage_major(form, self.s, _p(C), self.T, self.m, rp, ci, J, js,
                                              M, float(dt), None, None, None)
        orp = np.zeros(self.s * self.T + 1, np.int32)
        oci = np.zeros(nb, np.int32)
        ov = np.zeros(nb * self.m * self.m)
        lib.irk_ref_assemble_stage_major(form, self.s, _p(C), self.T, self.m, rp, ci, J, js, M,
                                         float(dt), _p(orp), _p(oci), _p(ov))
        return orp, oci, ov.reshape(nb, self.m, self.m)

    def assemble_element_major(self, dt, form=FORM_TRANSFORMED):
        lib = _load()
        C = self.Ainv if form == FORM_TRANSFORMED else self.A
        sm = self.s * self.m
        ov = np.zeros(int(self.row_ptr[-1]) * sm * sm)
        rp, ci, J, js, M = self._args()
        lib.irk_ref_assemble_element_major(form, self.s, _p(C), self.T, self.m, rp, ci, J, js, M,
                                           float(dt), _p(ov))
        return self.row_ptr.copy(), self.col_idx.copy(), ov.reshape(-1, sm, sm)

    def assemble_shifted(self, k, d, dt):
        lib = _load()
        mm = self.m * self.m
        nnzb = int(self.row_ptr[-1])
        Jk = self.J[k * self.jstride: k * self.jstride + nnzb * mm] if self.jstride else self.J
        Jk = np.ascontiguousarray(Jk)
        ov = np.zeros(nnzb * mm)
        lib.irk_ref_assemble_shifted(self.T, self.m, _p(self.row_ptr), _p(self.col_idx), _p(Jk),
                                     _p(self.M), float(d), float(dt), _p(ov))
        return ov.reshape(nnzb, self.m, self.m)


def bilu0(row_ptr, col_idx, vals):
    """Generic block ILU(0) (textbook IKJ form).  Returns (factors, dlu, dpiv)."""
    lib = _load()
    rp, ci = _i32(row_ptr), _i32(col_idx)
    v = _f64(vals).copy()
    nb = rp.size - 1
    b = v.shape[-1]
    dlu = np.zeros((nb, b, b))
    dpiv = np.zeros((nb, b), np.int32)
    _check(lib.irk_ref_bilu0(nb, b, _p(rp), _p(ci), _p(v), _p(dlu), _p(dpiv)), "bilu0")
    return v, dlu, dpiv


def bilu0_apply(row_ptr, col_idx, factors, dlu, dpiv, v):
    lib = _load()
    rp, ci = _i32(row_ptr), _i32(col_idx)
    f = _f64(factors)
    nb = rp.size - 1
    b = f.shape[-1]
    v = _f64(v).reshape(-1)
    z = np.empty_like(v)
    lib.irk_ref_bilu0_apply(nb, b, _p(rp), _p(ci), _p(f), _p(_f64(dlu)), _p(_i32(dpiv)), _p(v),
                            _p(z))
    return z


def ilu_alg2(row_ptr, col_idx, vals):
    """Alg. 2 literally (simplified block ILU(0))."""
    lib = _load()
    rp, ci = _i32(row_ptr), _i32(col_idx)
    v = _f64(vals).copy()
    T = rp.size - 1
    m = v.shape[-1]
    dlu = np.zeros((T, m, m))
    dpiv = np.zeros((T, m), np.int32)
    _check(lib.irk_ref_ilu_alg2(T, m, _p(rp), _p(ci), _p(v), _p(dlu), _p(dpiv)), "alg2")
    return v, dlu, dpiv


def ilu_alg3(s, row_ptr, col_idx, Bd, Bo):
    """Alg. 3 in the corrected reading.  Bd: (s, nnzb, m, m); Bo: (s, s, T, m, m)."""
    lib = _load()
    rp, ci = _i32(row_ptr), _i32(col_idx)
    Bd = _f64(Bd).copy()
    Bo = _f64(Bo).copy()
    T = rp.size - 1
    m = Bd.shape[-1]
    dlu = np.zeros((s * T, m, m))
    dpiv = np.zeros((s * T, m), np.int32)
    _check(lib.irk_ref_ilu_alg3(s, T, m, _p(rp), _p(ci), _p(Bd), _p(Bo), _p(dlu), _p(dpiv)),
           "alg3")
    return Bd, Bo, dlu, dpiv


def shift_column_rule(Ainv):
    lib = _load()
    Ainv = _f64(Ainv)
    s = Ainv.shape[0]
    out = np.zeros(s)
    lib.irk_ref_shift_column_rule(s, _p(Ainv), _p(out))
    return out
