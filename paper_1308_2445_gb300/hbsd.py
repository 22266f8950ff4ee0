"""Python binding of libhbsd (include/hbsd.h): argument marshalling only.

Every computation runs in the CUDA library.  If libhbsd.so is missing or cannot be loaded
this module raises; there is no CPU fallback.  Device buffers may be torch CUDA tensors (their
data_ptr() is passed) or raw integer device addresses.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhbsd.so")

HBSD_OK = 0
HBSD_NOT_CONVERGED = 1
HBSD_BUSY = 2
HBSD_ERR_ARG = -1
HBSD_ERR_OOM = -2
HBSD_ERR_NOT_SPD = -3
HBSD_ERR_RR_RANK = -4
HBSD_ERR_TIMEOUT = -5
HBSD_ERR_CUDA = -6
HBSD_ERR_UNSUPPORTED = -7

PRECISION_FP64 = 0
PRECISION_MIXED = 1
PRECOND_HYBRID = 0
PRECOND_GLOBAL = 1
PRECOND_LOCAL = 2
LOCAL_MINRES = 0
LOCAL_ONESTEP = 1


class hbsd_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.POINTER(C.c_int64)),
                ("col_idx", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_double)), ("is_complex", C.c_int)]


class hbsd_local_blocks(C.Structure):
    _fields_ = [("dof_node", C.POINTER(C.c_int32)), ("dof_cluster", C.POINTER(C.c_int32)),
                ("grid", C.c_int32 * 3)]


class hbsd_options(C.Structure):
    _fields_ = [("sigma_bar", C.c_double), ("sigma0", C.c_double), ("m0", C.c_int), ("tau1", C.c_double),
                ("tau2", C.c_double), ("eta", C.c_double), ("max_minres", C.c_int), ("max_outer", C.c_int),
                ("precision", C.c_int), ("precond", C.c_int), ("seed", C.c_uint64), ("local_solver", C.c_int),
                ("tc_update", C.c_int), ("update_hs", C.c_int), ("minres_f32", C.c_int),
                ("spmm_df64", C.c_int)]


class hbsd_server_opts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_slots", C.c_int)]


class hbsd_request(C.Structure):
    _fields_ = [("H", C.POINTER(hbsd_csr)), ("S", C.POINTER(hbsd_csr)), ("lb", C.POINTER(hbsd_local_blocks)),
                ("opt", C.POINTER(hbsd_options)), ("session_id", C.c_int64), ("H_val", C.POINTER(C.c_double)),
                ("nev", C.c_int), ("tol", C.c_double), ("X0", C.POINTER(C.c_double)), ("warm", C.c_int),
                ("nl_k", C.c_int), ("nl_F", C.POINTER(C.c_double)), ("nl_ldf", C.c_int64),
                ("nl_G", C.POINTER(C.c_double))]


class hbsd_result(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("status", C.c_int), ("iters", C.c_int), ("session_id", C.c_int64),
                ("res_max", C.c_double), ("latency_ms", C.c_double), ("queue_ms", C.c_double),
                ("run_ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class hbsd_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("iters_fp64", C.c_int), ("minres_steps", C.c_int64),
                ("precond_cols", C.c_int64), ("local_cols", C.c_int64), ("rr_fallbacks", C.c_int),
                ("res_max", C.c_double), ("t_factor_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("nnz_L", C.c_int64), ("n_supernodes", C.c_int), ("gpu_launches", C.c_int),
                ("t_matvec_ms", C.c_double), ("t_resid_ms", C.c_double), ("t_precond_ms", C.c_double),
                ("t_local_ms", C.c_double), ("t_gram_ms", C.c_double), ("t_rr_ms", C.c_double),
                ("t_update_ms", C.c_double), ("matvec_cols", C.c_int64), ("minres_spmm_cols", C.c_int64),
                ("precond_calls", C.c_int), ("local_calls", C.c_int64), ("neg_pivots", C.c_int64),
                ("gram_fma", C.c_double), ("update_fma", C.c_double), ("fp64_from_iter", C.c_int), ("fp64_gram_from_iter", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hbsd_tune(C.Structure):
    _fields_ = [("width", C.c_int), ("spmm_lanes", C.c_int), ("minres_ctas", C.c_int), ("minres_ctas_full", C.c_int),
                ("from_table", C.c_int), ("spmm_ms", C.c_double * 4), ("minres_ms", C.c_double * 6)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["spmm_ms"] = list(self.spmm_ms)
        d["minres_ms"] = list(self.minres_ms)
        return d


class hbsd_batch_item(C.Structure):
    _fields_ = [("h", C.c_void_p), ("nev", C.c_int), ("tol", C.c_double), ("X0_dev", C.c_void_p), ("ldx0", C.c_int64),
                ("lambda_dev", C.c_void_p), ("X_dev", C.c_void_p), ("ldx", C.c_int64), ("status", C.c_int),
                ("iters", C.c_int), ("res_max", C.c_double), ("run_ms", C.c_double), ("start_ms", C.c_double)]


class hbsd_batch_opts(C.Structure):
    _fields_ = [("max_concurrent", C.c_int), ("autotune", C.c_int), ("longest_first", C.c_int)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_SIGS = {
    "hbsd_options_default": (None, [C.POINTER(hbsd_options)]),
    "hbsd_create": (C.c_int, [C.POINTER(hbsd_csr), C.POINTER(hbsd_csr), C.POINTER(hbsd_local_blocks),
                              C.POINTER(hbsd_options), _P, C.POINTER(_P)]),
    "hbsd_update_H": (C.c_int, [_P, _D]),
    "hbsd_set_nonlocal": (C.c_int, [_P, C.c_int, _D, C.c_int64, _D]),
    "hbsd_res_history": (C.c_int, [_P, _D, C.c_int]),
    "hbsd_probe_barrier_timeout": (C.c_int, [C.c_double, _P]),
    "hbsd_onestep": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int, C.c_double, C.c_int, _P, C.c_int64, _P]),
    "hbsd_solve": (C.c_int, [_P, C.c_int, C.c_double, _D, C.c_int, _D, _D, C.POINTER(C.c_int),
                             C.POINTER(hbsd_stats)]),
    "hbsd_solve_device": (C.c_int, [_P, C.c_int, C.c_double, _P, C.c_int64, _P, _P, C.c_int64,
                                    C.POINTER(C.c_int), C.POINTER(hbsd_stats)]),
    "hbsd_destroy": (None, [_P]),
    "hbsd_status_string": (C.c_char_p, [C.c_int]),
    "hbsd_last_error": (C.c_char_p, []),
    "hbsd_n": (C.c_int64, [_P]),
    "hbsd_is_complex": (C.c_int, [_P]),
    "hbsd_sigma0": (C.c_double, [_P]),
    "hbsd_get_stats": (None, [_P, C.POINTER(hbsd_stats)]),
    "hbsd_spmm_pair": (C.c_int, [_P, _P, C.c_int64, C.c_int, _P, C.c_int64, _P, C.c_int64]),
    "hbsd_spmm_shifted": (C.c_int, [_P, _P, C.c_int64, C.c_int, _P, _P, C.c_int64]),
    "hbsd_spmm_pair_f32": (C.c_int, [_P, _P, C.c_int64, C.c_int, _P, C.c_int64, _P, C.c_int64]),
    "hbsd_spmm_pair_df64": (C.c_int, [_P, _P, C.c_int64, C.c_int, _P, C.c_int64, _P, C.c_int64]),
    "hbsd_precond_apply_f32": (C.c_int, [_P, _P, C.c_int64, C.c_int, _P, C.c_int64]),
    "hbsd_dscale": (C.c_int, [_P, _D]),
    "hbsd_residual": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, _P, C.c_int, _P, C.c_int64, _P]),
    "hbsd_precond_apply": (C.c_int, [_P, _P, C.c_int64, C.c_int, _P, C.c_int64]),
    "hbsd_minres": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int, C.c_double, C.c_int, _P, C.c_int64, _P]),
    "hbsd_gram": (C.c_int, [_P, C.c_int64, _P, C.c_int64, _P, C.c_int64, C.c_int64, C.c_int, _P, _P, _P]),
    "hbsd_update_oz": (C.c_int, [_P, C.c_int64, C.c_int, _P, C.c_int64, C.c_int, C.c_int64, _P, C.c_int, _P,
                                 C.c_int64, _P]),
    "hbsd_tc_gemm_bf16": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P]),
    "hbsd_gram_noalloc": (C.c_int, [_P, C.c_int64, _P, C.c_int64, _P, C.c_int64, C.c_int64, C.c_int, _P, _P, _P]),
    "hbsd_rayleigh_ritz": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P, _P, _P]),
    "hbsd_update": (C.c_int, [_P, C.c_int64, C.c_int64, C.c_int, _P, C.c_int, _P]),
    "hbsd_gram_df64": (C.c_int, [_P, C.c_int64, _P, C.c_int64, _P, C.c_int64, C.c_int64, C.c_int, _P, _P, _P]),
    "hbsd_update_df64": (C.c_int, [_P, C.c_int64, C.c_int64, C.c_int, _P, C.c_int, _P]),
    "hbsd_server_opts_default": (None, [C.POINTER(hbsd_server_opts)]),
    "hbsd_server_create": (C.c_int, [C.POINTER(hbsd_server_opts), C.POINTER(C.c_void_p)]),
    "hbsd_submit": (C.c_int, [C.c_void_p, C.POINTER(hbsd_request), _P, _P, C.POINTER(C.c_uint64)]),
    "hbsd_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(hbsd_result)]),
    "hbsd_session_release": (C.c_int, [C.c_void_p, C.c_int64]),
    "hbsd_server_destroy": (None, [C.c_void_p]),
    "hbsd_probe_peak": (C.c_int, [C.c_int, _P, C.POINTER(C.c_double)]),
    "hbsd_seed_normals": (C.c_int, [C.c_uint64, C.c_uint64, C.c_int64, _D]),
    "hbsd_autotune": (C.c_int, [_P, C.c_int, C.POINTER(hbsd_tune)]),
    "hbsd_res_stalled": (C.c_int, [_D, C.c_int, C.c_int, C.c_int, C.c_double]),
    "hbsd_batch_opts_default": (None, [C.POINTER(hbsd_batch_opts)]),
    "hbsd_solve_batch": (C.c_int, [C.POINTER(hbsd_batch_item), C.c_int, C.POINTER(hbsd_batch_opts)]),
}

_lib = None


def lib():
    """Load libhbsd.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


class HbsdError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = lib().hbsd_last_error().decode(errors="replace")
        st = lib().hbsd_status_string(code).decode()
        super().__init__(f"{where}: {st} ({code}): {msg}")


def check(code, where):
    if code < 0:
        raise HbsdError(code, where)
    return code


def ptr(x):
    """Device address of a torch tensor (or an int)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def ld(t):
    """Leading dimension (row stride, elements) of a 2-D row-major torch tensor."""
    return int(t.stride(0))


def options_default(**kw) -> hbsd_options:
    o = hbsd_options()
    lib().hbsd_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Session:
    """A solver session (hbsd_create ... hbsd_destroy) over one (H, S) pair."""

    def __init__(self, n, row_ptr, col_idx, h_val, s_val, dof_node, grid, sigma_bar, stream=None, **opts):
        self._keep = []
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        # complex Hermitian values go in as interleaved (re, im) doubles
        self.is_complex = bool(np.iscomplexobj(h_val) or np.iscomplexobj(s_val))
        vdt = np.complex128 if self.is_complex else np.float64
        hv = np.ascontiguousarray(h_val, dtype=vdt).view(np.float64)
        sv = np.ascontiguousarray(s_val, dtype=vdt).view(np.float64)
        dn = np.ascontiguousarray(dof_node, dtype=np.int32)
        self._keep += [rp, ci, hv, sv, dn]
        self.n = int(n)
        cflag = int(self.is_complex)
        H = hbsd_csr(self.n, int(ci.size), rp.ctypes.data_as(C.POINTER(C.c_int64)),
                     ci.ctypes.data_as(C.POINTER(C.c_int32)), hv.ctypes.data_as(_D), cflag)
        S = hbsd_csr(self.n, int(ci.size), rp.ctypes.data_as(C.POINTER(C.c_int64)),
                     ci.ctypes.data_as(C.POINTER(C.c_int32)), sv.ctypes.data_as(_D), cflag)
        lb = hbsd_local_blocks(dn.ctypes.data_as(C.POINTER(C.c_int32)), None, (C.c_int32 * 3)(*grid))
        self.opts = options_default(sigma_bar=float(sigma_bar), **opts)
        h = C.c_void_p()
        check(lib().hbsd_create(C.byref(H), C.byref(S), C.byref(lb), C.byref(self.opts),
                                C.c_void_p(stream) if stream else None, C.byref(h)), "hbsd_create")
        self.h = h

    @classmethod
    def from_problem(cls, p, stream=None, **opts):
        s = cls(p.n, p.row_ptr, p.col_idx, p.h_val, p.s_val, p.dof_node, p.grid, p.eps_bar, stream=stream, **opts)
        if getattr(p, "F", None) is not None:
            s.set_nonlocal(p.F, p.G)
        return s

    def res_history(self):
        """Res_max at every convergence test of the last solve (hbsd_res_history)."""
        cnt = lib().hbsd_res_history(self.h, None, 0)
        check(cnt, "hbsd_res_history")
        out = np.empty(max(cnt, 1))
        check(lib().hbsd_res_history(self.h, out.ctypes.data_as(_D), cnt), "hbsd_res_history")
        return out[:cnt]

    def set_nonlocal(self, F, G):
        """hbsd_set_nonlocal: H := H_loc + F G F^T (F n x k, G k x k symmetric); F = None removes it."""
        if F is None:
            check(lib().hbsd_set_nonlocal(self.h, 0, None, 0, None), "hbsd_set_nonlocal")
            return
        Fc = np.ascontiguousarray(F, dtype=np.float64)
        Gc = np.ascontiguousarray(G, dtype=np.float64)
        k = Fc.shape[1]
        if Fc.shape[0] != self.n or Gc.shape != (k, k):
            raise ValueError("F must be n x k and G k x k")
        check(lib().hbsd_set_nonlocal(self.h, int(k), Fc.ctypes.data_as(_D), int(k), Gc.ctypes.data_as(_D)),
              "hbsd_set_nonlocal")

    def close(self):
        if getattr(self, "h", None):
            lib().hbsd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def sigma0(self):
        return lib().hbsd_sigma0(self.h)

    def stats(self):
        st = hbsd_stats()
        lib().hbsd_get_stats(self.h, C.byref(st))
        return st.as_dict()

    def m0(self, nev):
        return self.opts.m0 if self.opts.m0 >= 0 else max(3, -(-nev // 10))

    def update_H(self, h_val):
        hv = np.ascontiguousarray(h_val, dtype=np.complex128 if self.is_complex else np.float64).view(np.float64)
        check(lib().hbsd_update_H(self.h, hv.ctypes.data_as(_D)), "hbsd_update_H")

    def solve(self, nev, tol, X0=None, warm=False, want_vectors=True):
        """hbsd_solve with host arrays: returns (lambda, X, iters, status, stats)."""
        w = nev + self.m0(nev)
        x0p = None
        vdt = np.complex128 if self.is_complex else np.float64
        if X0 is not None:
            X0 = np.ascontiguousarray(X0, dtype=vdt)
            if X0.shape != (self.n, w):
                raise ValueError(f"X0 must be {self.n} x {w}")
            x0p = X0.view(np.float64).ctypes.data_as(_D)
        lam = np.empty(nev)
        X = np.empty((self.n, nev), dtype=vdt) if want_vectors else None
        it = C.c_int(0)
        st = hbsd_stats()
        rc = check(lib().hbsd_solve(self.h, nev, tol, x0p, int(bool(warm)), lam.ctypes.data_as(_D),
                                    X.view(np.float64).ctypes.data_as(_D) if X is not None else None, C.byref(it),
                                    C.byref(st)),
                   "hbsd_solve")
        return lam, X, it.value, rc, st.as_dict()

    def solve_device(self, nev, tol, X0, lam, X=None):
        it = C.c_int(0)
        st = hbsd_stats()
        rc = check(lib().hbsd_solve_device(self.h, nev, tol, ptr(X0), ld(X0) if X0 is not None else 0, ptr(lam),
                                           ptr(X), ld(X) if X is not None else 0, C.byref(it), C.byref(st)),
                   "hbsd_solve_device")
        return it.value, rc, st.as_dict()

    def block_width(self, nev):
        """Real columns of the block a solve of nev pairs runs on."""
        return (nev + self.m0(nev)) * (2 if self.is_complex else 1)

    def autotune(self, nev):
        """hbsd_autotune for solves of nev pairs; returns the chosen shapes and the timings."""
        t = hbsd_tune()
        check(lib().hbsd_autotune(self.h, self.block_width(nev), C.byref(t)), "hbsd_autotune")
        return t.as_dict()

    # ---- step-level calls on torch CUDA tensors (row-major, float64) ----
    def spmm_pair(self, X, HX, SX):
        check(lib().hbsd_spmm_pair(self.h, ptr(X), ld(X), X.shape[1], ptr(HX), ld(HX), ptr(SX), ld(SX)),
              "hbsd_spmm_pair")

    def spmm_shifted(self, X, e, Y):
        check(lib().hbsd_spmm_shifted(self.h, ptr(X), ld(X), X.shape[1], ptr(e), ptr(Y), ld(Y)), "hbsd_spmm_shifted")

    def residual(self, PsiH, PsiS, E, m, R, res):
        check(lib().hbsd_residual(self.h, ptr(PsiH), ld(PsiH), ptr(PsiS), ld(PsiS), ptr(E), m, ptr(R),
                                  ld(R) if R is not None else 0, ptr(res)), "hbsd_residual")

    def spmm_pair_df64(self, X, HX, SX):
        check(lib().hbsd_spmm_pair_df64(self.h, ptr(X), ld(X), X.shape[1], ptr(HX), ld(HX), ptr(SX), ld(SX)),
              "hbsd_spmm_pair_df64")

    def spmm_pair_f32(self, X, HX, SX):
        check(lib().hbsd_spmm_pair_f32(self.h, ptr(X), ld(X), X.shape[1], ptr(HX), ld(HX), ptr(SX), ld(SX)),
              "hbsd_spmm_pair_f32")

    def precond_apply_f32(self, R, P):
        check(lib().hbsd_precond_apply_f32(self.h, ptr(R), ld(R), R.shape[1], ptr(P), ld(P)), "hbsd_precond_apply_f32")

    def dscale(self):
        d = np.empty(self.n)
        check(lib().hbsd_dscale(self.h, d.ctypes.data_as(_D)), "hbsd_dscale")
        return d

    def precond_apply(self, R, P):
        check(lib().hbsd_precond_apply(self.h, ptr(R), ld(R), R.shape[1], ptr(P), ld(P)), "hbsd_precond_apply")

    def minres(self, R, e, P, eta, max_minres, steps):
        check(lib().hbsd_minres(self.h, ptr(R), ld(R), ptr(e), R.shape[1], eta, max_minres, ptr(P), ld(P),
                                ptr(steps)), "hbsd_minres")

    def onestep(self, R, e, P, eta, max_steps, steps):
        check(lib().hbsd_onestep(self.h, ptr(R), ld(R), ptr(e), R.shape[1], eta, max_steps, ptr(P), ld(P),
                                 ptr(steps)), "hbsd_onestep")


def gram(Z, ZH, ZS, HR, SR, stream=0):
    check(lib().hbsd_gram(ptr(Z), ld(Z), ptr(ZH), ld(ZH), ptr(ZS), ld(ZS), Z.shape[0], Z.shape[1], ptr(HR), ptr(SR),
                          C.c_void_p(stream) if stream else None), "hbsd_gram")


def rayleigh_ritz(HR, SR, k, theta, W, info, stream=0):
    return check(lib().hbsd_rayleigh_ritz(ptr(HR), ptr(SR), HR.shape[0], k, ptr(theta), ptr(W), ptr(info),
                                          C.c_void_p(stream) if stream else None), "hbsd_rayleigh_ritz")


def update(Z, W, k, stream=0):
    check(lib().hbsd_update(ptr(Z), ld(Z), Z.shape[0], W.shape[0], ptr(W), k, C.c_void_p(stream) if stream else None),
          "hbsd_update")


def gram_df64(Z, ZH, ZS, HR, SR, stream=0):
    """Double-float Gram of the mixed form (upper entries, mirrored)."""
    check(lib().hbsd_gram_df64(ptr(Z), ld(Z), ptr(ZH), ld(ZH), ptr(ZS), ld(ZS), Z.shape[0], Z.shape[1], ptr(HR),
                               ptr(SR), C.c_void_p(stream) if stream else None), "hbsd_gram_df64")


def update_df64(Z, W, k, stream=0):
    """Double-float block update of the mixed form: Z(:, :k) = Z W."""
    check(lib().hbsd_update_df64(ptr(Z), ld(Z), Z.shape[0], W.shape[0], ptr(W), k,
                                 C.c_void_p(stream) if stream else None), "hbsd_update_df64")


def probe_peak(which, stream=0):
    """Measured FMA FLOP/s of the FP64 (which=0) or FP32 (which=1) SIMT pipes."""
    out = C.c_double(0.0)
    check(lib().hbsd_probe_peak(which, C.c_void_p(stream) if stream else None, C.byref(out)), "hbsd_probe_peak")
    return out.value


def seed_normals(seed, stream, count):
    """The library's start-block normals (host code, no GPU needed)."""
    out = np.empty(count)
    check(lib().hbsd_seed_normals(seed, stream, count, out.ctypes.data_as(_D)), "hbsd_seed_normals")
    return out


def res_stalled(hist, mark, win, below):
    """hbsd_res_stalled on a host history of Res_max values (True when the stall test fires)."""
    h = np.ascontiguousarray(hist, dtype=np.float64)
    return bool(check(lib().hbsd_res_stalled(h.ctypes.data_as(_D) if h.size else None, int(h.size), int(mark),
                                             int(win), float(below)), "hbsd_res_stalled"))


def solve_batch(entries, max_concurrent=8, autotune=True, longest_first=True):
    """hbsd_solve_batch.  entries: (session, nev, tol, X0 or None, lam, X or None) with device tensors
    as in Session.solve_device.  Returns (status, [per-entry dict of status, iters, res_max, run_ms,
    start_ms])."""
    items = (hbsd_batch_item * max(1, len(entries)))()
    for i, (sess, nev, tol, X0, lam, X) in enumerate(entries):
        it = items[i]
        it.h = sess.h
        it.nev = nev
        it.tol = tol
        it.X0_dev = ptr(X0)
        it.ldx0 = ld(X0) if X0 is not None else 0
        it.lambda_dev = ptr(lam)
        it.X_dev = ptr(X)
        it.ldx = ld(X) if X is not None else 0
    o = hbsd_batch_opts()
    lib().hbsd_batch_opts_default(C.byref(o))
    o.max_concurrent = max_concurrent
    o.autotune = int(bool(autotune))
    o.longest_first = int(bool(longest_first))
    rc = check(lib().hbsd_solve_batch(items, len(entries), C.byref(o)), "hbsd_solve_batch")
    out = [{"status": items[i].status, "iters": items[i].iters, "res_max": items[i].res_max,
            "run_ms": items[i].run_ms, "start_ms": items[i].start_ms} for i in range(len(entries))]
    return rc, out


class Server:
    """hbsd_server_*: solve requests of several problems in flight at once on one GPU.

    submit() copies what it is given and returns a ticket at once; poll(ticket) returns None
    while the request is queued or running, then (result dict, lambda, X)."""

    def __init__(self, max_slots=4, hbm_budget_bytes=0):
        o = hbsd_server_opts()
        lib().hbsd_server_opts_default(C.byref(o))
        o.max_slots = int(max_slots)
        o.hbm_budget_bytes = int(hbm_budget_bytes)
        h = C.c_void_p()
        check(lib().hbsd_server_create(C.byref(o), C.byref(h)), "hbsd_server_create")
        self.h = h
        self._out = {}   # ticket -> (lambda, X) host buffers, kept alive until polled

    def submit(self, nev, tol, problem=None, session_id=-1, H_val=None, X0=None, warm=False, want_vectors=True,
               n=None, is_complex=None, **opts):
        """Queue a request.  A complex (Bloch) problem, or a follow-up of one, takes complex H_val
        and X0 and returns a complex X; for a follow-up without X0, pass n and is_complex to get
        the eigenvectors back."""
        keep = []
        rq = hbsd_request()
        rq.session_id = int(session_id)
        rq.nev = int(nev)
        rq.tol = float(tol)
        rq.warm = int(bool(warm))
        cplx = bool(is_complex) if is_complex is not None else False
        if problem is not None:
            cplx = bool(np.iscomplexobj(problem.h_val) or np.iscomplexobj(problem.s_val))
        elif is_complex is None:
            cplx = bool((H_val is not None and np.iscomplexobj(H_val)) or (X0 is not None and np.iscomplexobj(X0)))
        vdt = np.complex128 if cplx else np.float64
        if problem is not None:
            p = problem
            rp = np.ascontiguousarray(p.row_ptr, dtype=np.int64)
            ci = np.ascontiguousarray(p.col_idx, dtype=np.int32)
            hv = np.ascontiguousarray(p.h_val, dtype=vdt).view(np.float64)
            sv = np.ascontiguousarray(p.s_val, dtype=vdt).view(np.float64)
            dn = np.ascontiguousarray(p.dof_node, dtype=np.int32)
            H = hbsd_csr(p.n, int(ci.size), rp.ctypes.data_as(C.POINTER(C.c_int64)),
                         ci.ctypes.data_as(C.POINTER(C.c_int32)), hv.ctypes.data_as(_D), int(cplx))
            S = hbsd_csr(p.n, int(ci.size), rp.ctypes.data_as(C.POINTER(C.c_int64)),
                         ci.ctypes.data_as(C.POINTER(C.c_int32)), sv.ctypes.data_as(_D), int(cplx))
            lb = hbsd_local_blocks(dn.ctypes.data_as(C.POINTER(C.c_int32)), None, (C.c_int32 * 3)(*p.grid))
            op = options_default(sigma_bar=float(p.eps_bar), **opts)
            keep += [rp, ci, hv, sv, dn, H, S, lb, op]
            if getattr(p, "F", None) is not None:
                Fc = np.ascontiguousarray(p.F, dtype=np.float64)
                Gc = np.ascontiguousarray(p.G, dtype=np.float64)
                keep += [Fc, Gc]
                rq.nl_k, rq.nl_ldf = int(Fc.shape[1]), int(Fc.shape[1])
                rq.nl_F, rq.nl_G = Fc.ctypes.data_as(_D), Gc.ctypes.data_as(_D)
            rq.H, rq.S, rq.lb, rq.opt = C.pointer(H), C.pointer(S), C.pointer(lb), C.pointer(op)
            rq.session_id = -1
            n = p.n
        if H_val is not None:
            hvn = np.ascontiguousarray(H_val, dtype=vdt).view(np.float64)
            keep.append(hvn)
            rq.H_val = hvn.ctypes.data_as(_D)
        if X0 is not None:
            x0 = np.ascontiguousarray(X0, dtype=vdt)
            keep.append(x0)
            rq.X0 = x0.view(np.float64).ctypes.data_as(_D)
            n = x0.shape[0]
        if n is None and want_vectors:
            raise ValueError("want_vectors for a follow-up needs X0 or n; pass n through X0, problem or n=")
        lam = np.empty(nev)
        X = np.empty((n, nev), dtype=vdt) if want_vectors else None
        t = C.c_uint64(0)
        check(lib().hbsd_submit(self.h, C.byref(rq), lam.ctypes.data_as(_D),
                                X.view(np.float64).ctypes.data_as(_D) if X is not None else None, C.byref(t)),
              "hbsd_submit")
        self._out[t.value] = (lam, X)
        return t.value

    def poll(self, ticket):
        r = hbsd_result()
        rc = lib().hbsd_poll(self.h, C.c_uint64(ticket), C.byref(r))
        if rc == 2:
            return None
        check(rc, "hbsd_poll")
        lam, X = self._out.pop(ticket)
        return r.as_dict(), lam, X

    def wait(self, ticket, poll_s=0.0005):
        import time
        while True:
            out = self.poll(ticket)
            if out is not None:
                return out
            time.sleep(poll_s)

    def release(self, session_id):
        return check(lib().hbsd_session_release(self.h, C.c_int64(session_id)), "hbsd_session_release")

    def close(self):
        if getattr(self, "h", None):
            lib().hbsd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
