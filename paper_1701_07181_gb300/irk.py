"""Thin ctypes binding of ``libirk_gb300.so`` (C ABI in ``include/irk_gb300.h``).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Arrays may be numpy arrays (host memory: IRK_HOST) or CUDA torch
tensors (device memory: IRK_DEVICE); the memory space of a call follows its
arrays.  There is no CPU fallback: if the library cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libirk_gb300.so")

IRK_OK, IRK_NOT_CONVERGED = 0, 1
IRK_HOST, IRK_DEVICE = 0, 1
PRECOND = {"none": 0, "uncoupled": 1, "coupled": 2, "element": 3}
FACTOR_PREC = {"fp64": 0, "fp32": 1, "bf16": 2}
KRYLOV = {"fp64": 0, "df64": 1, "fp64-dfop": 2}
FORM = {"transformed": 0, "untransformed": 1}

_lock = threading.Lock()
_lib = None


class IrkError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (what, strerror(code), code))


class Options(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_iter", ctypes.c_int), ("precond", ctypes.c_int),
                ("factor_prec", ctypes.c_int), ("krylov_arith", ctypes.c_int),
                ("formulation", ctypes.c_int), ("shift", ctypes.POINTER(ctypes.c_double)),
                ("stream", ctypes.c_void_p), ("timing", ctypes.c_int), ("sweep", ctypes.c_int),
                ("ordering", ctypes.c_int), ("partitions", ctypes.c_int),
                ("partition", ctypes.POINTER(ctypes.c_int32)), ("stage_jacobians", ctypes.c_int),
                ("spin_limit", ctypes.c_int), ("orthogonalization", ctypes.c_int)]


class KernelOptions(ctypes.Structure):
    _fields_ = [("matvec_variant", ctypes.c_int), ("sweep_two_colour", ctypes.c_int),
                ("sweep_compiled_levels", ctypes.c_int), ("sweep_shared_upper", ctypes.c_int), ("factor_fused", ctypes.c_int),
                ("factor_gj_rows", ctypes.c_int), ("factor_gj_threads", ctypes.c_int),
                ("factor_gj_split_min", ctypes.c_int), ("arnoldi_form", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int), ("levels_lower", ctypes.c_int),
                ("levels_upper", ctypes.c_int), ("relres", ctypes.c_double),
                ("factor_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong), ("matvec_ms", ctypes.c_double),
                ("precond_ms", ctypes.c_double), ("ortho_ms", ctypes.c_double),
                ("n_matvec", ctypes.c_int), ("n_precond", ctypes.c_int), ("n_ortho", ctypes.c_int),
                ("matvec_variant", ctypes.c_int), ("factor_assemble_ms", ctypes.c_double),
                ("factor_products_ms", ctypes.c_double), ("factor_inverse_ms", ctypes.c_double),
                ("sweep_fwd_ms", ctypes.c_double), ("sweep_bwd_ms", ctypes.c_double),
                ("factor_fused_levels", ctypes.c_int), ("sweep_two_colour", ctypes.c_int)]


EXPORTS = ["irk_default_options", "irk_setup", "irk_update_values", "irk_factor", "irk_solve",
           "irk_apply_operator", "irk_apply_precond", "irk_get_stats", "irk_destroy",
           "irk_strerror", "irk_apply_precond_noalloc", "irk_group_create", "irk_group_submit",
           "irk_group_step", "irk_group_query", "irk_group_collect", "irk_group_device_bytes",
           "irk_group_destroy", "irk_dirk_setup", "irk_dirk_step", "irk_dirk_destroy", "irk_set_timing",
           "irk_step_outputs", "irk_set_spin_limit", "irk_default_kernel_options", "irk_set_kernel_options"]


def load():
    """Load the library (raises if it is missing: build it with
    ``python -m paper_1701_07181_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libirk_gb300.so not built; run `python -m paper_1701_07181_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        lib.irk_default_options.argtypes = [ctypes.POINTER(Options)]
        lib.irk_default_options.restype = None
        lib.irk_setup.argtypes = [ctypes.POINTER(P), I, P, I, I, P, P, P, P, I, ctypes.POINTER(Options)]
        lib.irk_update_values.argtypes = [P, P, P, I]
        lib.irk_factor.argtypes = [P, D]
        lib.irk_solve.argtypes = [P, P, D, D, P, I, ctypes.POINTER(I), ctypes.POINTER(D)]
        lib.irk_apply_operator.argtypes = [P, P, P, D, I]
        lib.irk_apply_precond.argtypes = [P, P, P, I]
        lib.irk_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
        lib.irk_set_timing.argtypes = [P, I]
        lib.irk_set_spin_limit.argtypes = [P, I]
        lib.irk_default_kernel_options.argtypes = [ctypes.POINTER(KernelOptions)]
        lib.irk_default_kernel_options.restype = None
        lib.irk_set_kernel_options.argtypes = [P, ctypes.POINTER(KernelOptions)]
        lib.irk_step_outputs.argtypes = [P, P, P, P, D, P, P, I]
        lib.irk_destroy.argtypes = [P]
        lib.irk_destroy.restype = None
        lib.irk_strerror.argtypes = [I]
        lib.irk_strerror.restype = ctypes.c_char_p
        lib.irk_apply_precond_noalloc.argtypes = [P, P, P, P]
        lib.irk_group_create.argtypes = [ctypes.POINTER(P), I, P, I, I, I, I, ctypes.POINTER(Options)]
        lib.irk_group_submit.argtypes = [P, I, P, P, P, P, P, D, D, I, ctypes.POINTER(I)]
        lib.irk_group_step.argtypes = [P, ctypes.POINTER(I)]
        lib.irk_group_query.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(I)]
        lib.irk_group_collect.argtypes = [P, I, P, I]
        lib.irk_group_device_bytes.argtypes = [P]
        lib.irk_group_device_bytes.restype = ctypes.c_longlong
        lib.irk_group_destroy.argtypes = [P]
        lib.irk_group_destroy.restype = None
        lib.irk_dirk_setup.argtypes = [ctypes.POINTER(P), I, P, P, I, I, P, P, P, P, I, ctypes.POINTER(Options)]
        lib.irk_dirk_step.argtypes = [P, P, D, D, P, P, I, P, ctypes.POINTER(D)]
        lib.irk_dirk_destroy.argtypes = [P]
        lib.irk_dirk_destroy.restype = None
        _lib = lib
        return lib


def strerror(code: int) -> str:
    return load().irk_strerror(int(code)).decode()


def _is_torch_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _ptr(a, dtype):
    """(pointer, keep-alive, mem_space) of an array argument."""
    if _is_torch_cuda(a):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            a = a.to(want).contiguous()
        return ctypes.c_void_p(a.data_ptr()), a, IRK_DEVICE
    if hasattr(a, "detach"):  # CPU torch tensor
        a = a.detach().numpy()
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), arr, IRK_HOST


class Solver:
    """One stage-system context (irk_setup ... irk_destroy)."""

    def __init__(self, s, T, m, row_ptr, col_idx, J, M, A=None, precond="uncoupled",
                 factor_prec="fp64", krylov="fp64", formulation="transformed", restart=30,
                 max_iter=3000, shift=None, stream=None, timing=False, sweep="auto",
                 ordering="natural", partitions=0, partition=None, stage_jacobians=False, spin_limit=0,
                 kernel_options=None, orthogonalization="mgs"):
        lib = load()
        self._lib = lib
        self.s, self.T, self.m = int(s), int(T), int(m)
        self.N = self.s * self.T * self.m
        opt = Options()
        lib.irk_default_options(ctypes.byref(opt))
        opt.restart = int(restart)
        opt.max_iter = int(max_iter)
        opt.precond = PRECOND[precond] if isinstance(precond, str) else int(precond)
        opt.factor_prec = FACTOR_PREC[factor_prec] if isinstance(factor_prec, str) else int(factor_prec)
        opt.krylov_arith = KRYLOV[krylov] if isinstance(krylov, str) else int(krylov)
        opt.formulation = FORM[formulation] if isinstance(formulation, str) else int(formulation)
        self._shift = None
        if shift is not None:
            self._shift = np.ascontiguousarray(shift, dtype=np.float64)
            opt.shift = self._shift.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if stream is not None:
            opt.stream = ctypes.c_void_p(int(stream))
        opt.timing = int(timing) if timing in (0, 1, 2) else (1 if timing else 0)
        opt.sweep = {"auto": 0, "levels": 1}[sweep]
        opt.ordering = {"natural": 0, "multicolor": 1}[ordering]
        opt.partitions = int(partitions)
        opt.stage_jacobians = 1 if stage_jacobians else 0
        opt.spin_limit = int(spin_limit)
        opt.orthogonalization = {"mgs": 0, "cgs2": 1}[orthogonalization]
        self._part = None
        if partition is not None:
            self._part = np.ascontiguousarray(partition, dtype=np.int32)
            opt.partition = self._part.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        self._opt = opt
        rp, k1, sp1 = _ptr(row_ptr, np.int32)
        ci, k2, sp2 = _ptr(col_idx, np.int32)
        Jp, k3, sp3 = _ptr(J, np.float64)
        Mp, k4, sp4 = _ptr(M, np.float64)
        if len({sp1, sp2, sp3, sp4}) != 1:
            raise ValueError("pattern and values must all be host arrays or all CUDA tensors")
        Ap = None
        if A is not None:
            self._A = np.ascontiguousarray(A, dtype=np.float64)
            Ap = self._A.ctypes.data_as(ctypes.c_void_p)
        h = ctypes.c_void_p()
        rc = lib.irk_setup(ctypes.byref(h), self.s, Ap, self.T, self.m, rp, ci, Jp, Mp, sp1,
                           ctypes.byref(opt))
        if rc != IRK_OK:
            raise IrkError(rc, "irk_setup")
        self._h = h
        if kernel_options:
            self.set_kernel_options(**kernel_options)

    def _check(self, rc, what, allow_nc=False):
        if rc == IRK_OK or (allow_nc and rc == IRK_NOT_CONVERGED):
            return rc
        raise IrkError(rc, what)

    def update_values(self, J, M):
        Jp, k1, sp = _ptr(J, np.float64)
        Mp, k2, _ = _ptr(M, np.float64)
        self._check(self._lib.irk_update_values(self._h, Jp, Mp, sp), "irk_update_values")

    def factor(self, dt):
        self._check(self._lib.irk_factor(self._h, float(dt)), "irk_factor")

    def _out_like(self, a):
        if _is_torch_cuda(a):
            import torch
            return torch.empty(self.N, dtype=torch.float64, device=a.device)
        return np.empty(self.N, dtype=np.float64)

    def solve(self, R, dt, rtol=1e-8, out=None):
        """W with B W = R; returns (W, iters, relres, status)."""
        Rp, keep, sp = _ptr(R, np.float64)
        W = self._out_like(R) if out is None else out
        Wp, keepw, spw = _ptr(W, np.float64)
        if sp != spw:
            raise ValueError("R and W must be in the same memory space")
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        rc = self._lib.irk_solve(self._h, Rp, float(dt), float(rtol), Wp, sp, ctypes.byref(it),
                                 ctypes.byref(rr))
        self._check(rc, "irk_solve", allow_nc=True)
        return W, it.value, rr.value, rc

    def apply_operator(self, X, dt):
        Xp, keep, sp = _ptr(X, np.float64)
        Y = self._out_like(X)
        Yp, keepy, _ = _ptr(Y, np.float64)
        self._check(self._lib.irk_apply_operator(self._h, Xp, Yp, float(dt), sp), "irk_apply_operator")
        return Y

    def apply_precond(self, V):
        Vp, keep, sp = _ptr(V, np.float64)
        Z = self._out_like(V)
        Zp, keepz, _ = _ptr(Z, np.float64)
        self._check(self._lib.irk_apply_precond(self._h, Vp, Zp, sp), "irk_apply_precond")
        return Z

    def step_outputs(self, W, dt, u0=None, b=None, want_K=True):
        """irk_step_outputs: (K, u1) from the stage solution W (Sec. 4.1):
        K = (A^-1 (x) I) W and u1 = u0 + dt (b^T A^-1 (x) I) W (b = None: the
        last row of A, as for Radau IIA).  K or u1 is None when not asked for."""
        Wp, keep, sp = _ptr(W, np.float64)
        K = self._out_like(W) if want_K else None
        Kp, keepk = (_ptr(K, np.float64)[:2] if want_K else (None, None))
        u1 = None
        u0p = u1p = None
        if u0 is not None:
            u0p, keep0, sp0 = _ptr(u0, np.float64)
            if sp0 != sp:
                raise ValueError("W and u0 must be in the same memory space")
            n = self.T * self.m
            if _is_torch_cuda(u0):
                import torch
                u1 = torch.empty(n, dtype=torch.float64, device=u0.device)
            else:
                u1 = np.empty(n, dtype=np.float64)
            u1p, keep1, _ = _ptr(u1, np.float64)
        bb = None if b is None else (ctypes.c_double * self.s)(*[float(x) for x in b])
        self._check(self._lib.irk_step_outputs(self._h, Wp, bb, u0p, float(dt), Kp, u1p, sp), "irk_step_outputs")
        return K, u1

    def set_kernel_options(self, **kw):
        """irk_set_kernel_options: the library's defaults with the given fields
        (names of irk_kernel_options) changed."""
        ko = KernelOptions()
        self._lib.irk_default_kernel_options(ctypes.byref(ko))
        for k, v in kw.items():
            if k not in dict(KernelOptions._fields_):
                raise KeyError(k)
            setattr(ko, k, int(v))
        self._check(self._lib.irk_set_kernel_options(self._h, ctypes.byref(ko)), "irk_set_kernel_options")

    def set_spin_limit(self, spin_limit):
        """irk_set_spin_limit: polls of a device wait on another thread block
        before it gives up (0 = the default)."""
        self._check(self._lib.irk_set_spin_limit(self._h, int(spin_limit)), "irk_set_spin_limit")

    def set_timing(self, timing):
        """irk_set_timing: 0, 1 or 2 (see irk_options.timing) for the calls that follow."""
        self._check(self._lib.irk_set_timing(self._h, int(timing)), "irk_set_timing")

    def stats(self):
        st = Stats()
        self._check(self._lib.irk_get_stats(self._h, ctypes.byref(st)), "irk_get_stats")
        return {f: getattr(st, f) for f, _ in Stats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.irk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Group:
    """Multi-request engine (irk_group_*): many stage systems of one class
    (s, m, options) solved together, admitted and collected between steps."""

    def __init__(self, s, m, max_elements, max_blocks, max_requests, A=None, precond="uncoupled",
                 factor_prec="fp32", krylov="df64", restart=30, max_iter=3000, ordering="natural",
                 stream=None, shift=None):
        lib = load()
        self._lib = lib
        self.s, self.m = int(s), int(m)
        opt = Options()
        lib.irk_default_options(ctypes.byref(opt))
        opt.restart = int(restart)
        opt.max_iter = int(max_iter)
        opt.precond = PRECOND[precond]
        opt.factor_prec = FACTOR_PREC[factor_prec]
        opt.krylov_arith = KRYLOV[krylov]
        opt.ordering = {"natural": 0, "multicolor": 1}[ordering]
        self._shift = None
        if shift is not None:
            self._shift = np.ascontiguousarray(shift, dtype=np.float64)
            opt.shift = self._shift.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if stream is not None:
            opt.stream = ctypes.c_void_p(int(stream))
        Ap = None
        if A is not None:
            self._A = np.ascontiguousarray(A, dtype=np.float64)
            Ap = self._A.ctypes.data_as(ctypes.c_void_p)
        h = ctypes.c_void_p()
        rc = lib.irk_group_create(ctypes.byref(h), self.s, Ap, self.m, int(max_elements), int(max_blocks),
                                  int(max_requests), ctypes.byref(opt))
        if rc != IRK_OK:
            raise IrkError(rc, "irk_group_create")
        self._h = h
        self._T = {}

    def submit(self, T, row_ptr, col_idx, J, M, R, dt, rtol=1e-8):
        """Admit one request; returns its slot, or None when the pools are full."""
        rp, k1, sp = _ptr(row_ptr, np.int32)
        ci, k2, _ = _ptr(col_idx, np.int32)
        Jp, k3, _ = _ptr(J, np.float64)
        Mp, k4, _ = _ptr(M, np.float64)
        Rp, k5, _ = _ptr(R, np.float64)
        slot = ctypes.c_int(-1)
        rc = self._lib.irk_group_submit(self._h, int(T), rp, ci, Jp, Mp, Rp, float(dt), float(rtol), sp,
                                        ctypes.byref(slot))
        if rc == -2:
            return None
        if rc != IRK_OK:
            raise IrkError(rc, "irk_group_submit")
        self._T[slot.value] = int(T)
        return slot.value

    def step(self):
        """One FGMRES iteration of every active request; returns how many remain."""
        n = ctypes.c_int(0)
        rc = self._lib.irk_group_step(self._h, ctypes.byref(n))
        if rc != IRK_OK:
            raise IrkError(rc, "irk_group_step")
        return n.value

    def query(self, slot):
        """(running, iters, relres, status)."""
        it, rr, stt = ctypes.c_int(0), ctypes.c_double(0.0), ctypes.c_int(0)
        rc = self._lib.irk_group_query(self._h, int(slot), ctypes.byref(it), ctypes.byref(rr), ctypes.byref(stt))
        if rc < 0:
            raise IrkError(rc, "irk_group_query")
        return rc == 1, it.value, rr.value, stt.value

    def collect(self, slot, out=None, device=None):
        """W of a finished request (numpy, or a CUDA tensor when device is given)."""
        N = self.s * self._T[slot] * self.m
        if out is None:
            if device is not None:
                import torch
                out = torch.empty(N, dtype=torch.float64, device=device)
            else:
                out = np.empty(N, dtype=np.float64)
        Wp, keep, sp = _ptr(out, np.float64)
        rc = self._lib.irk_group_collect(self._h, int(slot), Wp, sp)
        if rc != IRK_OK:
            raise IrkError(rc, "irk_group_collect")
        del self._T[slot]
        return out

    def device_bytes(self):
        return int(self._lib.irk_group_device_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.irk_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Dirk:
    """Diagonally implicit Runge-Kutta stepper of M u' = J u
    (irk_dirk_setup ... irk_dirk_destroy): stage k solves
    (M - dt a_kk J) k_k = J (u0 + dt sum_{j<k} a_kj k_j) with FGMRES and the
    block ILU(0) of the stage matrix; u1 = u0 + dt sum_k b_k k_k."""

    def __init__(self, A, b, T, m, row_ptr, col_idx, J, M, factor_prec="fp64", krylov="fp64", restart=30,
                 max_iter=3000, stream=None, sweep="auto", ordering="natural", precond="coupled"):
        lib = load()
        self._lib = lib
        self._A = np.ascontiguousarray(A, dtype=np.float64)
        self._b = np.ascontiguousarray(b, dtype=np.float64)
        self.s = int(self._b.size)
        self.T, self.m = int(T), int(m)
        self.n = self.T * self.m
        opt = Options()
        lib.irk_default_options(ctypes.byref(opt))
        opt.restart = int(restart)
        opt.max_iter = int(max_iter)
        opt.precond = PRECOND[precond] if isinstance(precond, str) else int(precond)
        opt.factor_prec = FACTOR_PREC[factor_prec] if isinstance(factor_prec, str) else int(factor_prec)
        opt.krylov_arith = KRYLOV[krylov] if isinstance(krylov, str) else int(krylov)
        if stream is not None:
            opt.stream = ctypes.c_void_p(int(stream))
        opt.sweep = {"auto": 0, "levels": 1}[sweep]
        opt.ordering = {"natural": 0, "multicolor": 1}[ordering]
        rp, k1, sp1 = _ptr(row_ptr, np.int32)
        ci, k2, sp2 = _ptr(col_idx, np.int32)
        Jp, k3, sp3 = _ptr(J, np.float64)
        Mp, k4, sp4 = _ptr(M, np.float64)
        if len({sp1, sp2, sp3, sp4}) != 1:
            raise ValueError("pattern and values must all be host arrays or all CUDA tensors")
        h = ctypes.c_void_p()
        rc = lib.irk_dirk_setup(ctypes.byref(h), self.s, self._A.ctypes.data_as(ctypes.c_void_p),
                                self._b.ctypes.data_as(ctypes.c_void_p), self.T, self.m, rp, ci, Jp, Mp, sp1,
                                ctypes.byref(opt))
        if rc != IRK_OK:
            raise IrkError(rc, "irk_dirk_setup")
        self._h = h

    def step(self, u0, dt, rtol=1e-8, want_K=False):
        """(u1, K or None, per-stage iterations, worst relres, status)."""
        up, keep, sp = _ptr(u0, np.float64)
        if sp == IRK_DEVICE:
            import torch
            u1 = torch.empty(self.n, dtype=torch.float64, device=u0.device)
            K = torch.empty(self.s * self.n, dtype=torch.float64, device=u0.device) if want_K else None
        else:
            u1 = np.empty(self.n)
            K = np.empty(self.s * self.n) if want_K else None
        u1p, k1, _ = _ptr(u1, np.float64)
        Kp = _ptr(K, np.float64)[0] if K is not None else None
        its = np.zeros(self.s, dtype=np.int32)
        rr = ctypes.c_double(0.0)
        rc = self._lib.irk_dirk_step(self._h, up, float(dt), float(rtol), u1p, Kp, sp,
                                     its.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rr))
        if rc not in (IRK_OK, IRK_NOT_CONVERGED):
            raise IrkError(rc, "irk_dirk_step")
        return u1, K, [int(x) for x in its], rr.value, rc

    def close(self):
        if getattr(self, "_h", None):
            self._lib.irk_dirk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
