"""Thin Python binding of the C ABI in include/mgmlmc.h (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libmgmlmc.so``.  PyTorch provides the device memory (its caching
allocator, through the library's allocator callback) and the CUDA stream.
There is no CPU fallback: without the built library or a CUDA device the
binding raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmgmlmc.so")

MAX_LEVELS = 6
OP_D, OP_PH, OP_P, OP_G5, OP_PREC, OP_DINV_C, OP_SMOOTH = range(7)

STATUS = {0: "MGMLMC_OK", -1: "MGMLMC_EINVAL", -2: "MGMLMC_ENOMEM", -3: "MGMLMC_ENOTCONVERGED",
          -4: "MGMLMC_ETIMEOUT", -5: "MGMLMC_ECUDA", -6: "MGMLMC_ENOTIMPL", -7: "MGMLMC_ENAN",
          -8: "MGMLMC_ESTATE", -9: "MGMLMC_ECANCELLED", 1: "MGMLMC_PENDING"}
ECANCELLED, PENDING = -9, 1


class MgmlmcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("mg_precision", C.c_int), ("solve_tol", C.c_double), ("fgmres_restart", C.c_int),
                ("max_iters", C.c_int), ("nu_pre", C.c_int), ("nu_post", C.c_int),
                ("max_block_rhs", C.c_int), ("verbose", C.c_int), ("kcycle_iters", C.c_int)]


class LevelStats(C.Structure):
    _fields_ = [("nsamples", C.c_int64), ("sum_re", C.c_double), ("sum_im", C.c_double),
                ("sum_abs2", C.c_double), ("mean_re", C.c_double), ("mean_im", C.c_double),
                ("variance", C.c_double), ("seconds", C.c_double), ("iters", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TraceResult(C.Structure):
    _fields_ = [("trace_re", C.c_double), ("trace_im", C.c_double), ("rel_err", C.c_double),
                ("deflated_part", C.c_double), ("nterms", C.c_int), ("converged", C.c_int),
                ("rounds", C.c_int), ("term", LevelStats * MAX_LEVELS)]


class ServerOptions(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_active", C.c_int), ("max_bypass", C.c_int)]


class Request(C.Structure):
    _fields_ = [("Lx", C.c_int), ("Lt", C.c_int), ("theta", C.POINTER(C.c_double)), ("m0", C.c_double),
                ("nlevels", C.c_int), ("agg_x", C.c_int * MAX_LEVELS), ("agg_t", C.c_int * MAX_LEVELS),
                ("nvec", C.c_int * MAX_LEVELS), ("start_vectors", C.POINTER(C.c_double) * MAX_LEVELS),
                ("setup_iters", C.c_int), ("setup_tol", C.c_double), ("k", C.c_int), ("defl_tol", C.c_double),
                ("defl_max_iters", C.c_int), ("rel_tol", C.c_double), ("max_samples", C.c_int64),
                ("seed", C.c_uint64), ("costs", C.c_double * MAX_LEVELS), ("opt", Options),
                ("sum_levels", C.c_int)]


class RequestResult(C.Structure):
    _fields_ = [("status", C.c_int), ("result", TraceResult), ("queued_s", C.c_double), ("setup_s", C.c_double),
                ("estimate_s", C.c_double), ("total_s", C.c_double), ("reserved_bytes", C.c_size_t),
                ("peak_bytes", C.c_size_t), ("retries", C.c_int), ("error", C.c_char * 160),
                ("deflation_converged", C.c_int)]


class TuneTrial(C.Structure):
    _fields_ = [("block_rhs", C.c_int), ("fgmres_restart", C.c_int), ("nu_post", C.c_int),
                ("kcycle_iters", C.c_int), ("samples_per_s", C.c_double)]


TUNE_LOG = 16


class TuneResult(C.Structure):
    _fields_ = [("block_rhs", C.c_int), ("fgmres_restart", C.c_int), ("nu_post", C.c_int),
                ("kcycle_iters", C.c_int), ("samples_per_s", C.c_double), ("footprint", C.c_size_t),
                ("budget", C.c_size_t), ("trials", C.c_int), ("log", TuneTrial * TUNE_LOG)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "log"}
        d["log"] = [{k: getattr(t, k) for k, _ in TuneTrial._fields_} for t in self.log[:min(self.trials, TUNE_LOG)]]
        return d


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int), ("active", C.c_int), ("completed", C.c_int64), ("max_active_seen", C.c_int),
                ("budget", C.c_size_t), ("reserved", C.c_size_t), ("max_reserved", C.c_size_t)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)

# (name, restype, argtypes) of every entry point declared in include/mgmlmc.h
SIGNATURES = [
    ("mgmlmc_default_options", None, [C.POINTER(Options)]),
    ("mgmlmc_create", C.c_int, [C.POINTER(_P), C.POINTER(Options), _P, ALLOC_FN, FREE_FN, _P]),
    ("mgmlmc_create_copy", C.c_int, [C.POINTER(_P), _P, C.c_void_p, ALLOC_FN, FREE_FN, C.c_void_p]),
    ("mgmlmc_destroy", None, [_P]),
    ("mgmlmc_last_error", C.c_char_p, [_P]),
    ("mgmlmc_set_gauge", C.c_int, [_P, C.c_int, C.c_int, _D]),
    ("mgmlmc_set_mass", C.c_int, [_P, C.c_double]),
    ("mgmlmc_set_hierarchy", C.c_int, [_P, C.c_int, _I, _I, _I, C.c_int, C.c_double, C.POINTER(_D)]),
    ("mgmlmc_set_terms", C.c_int, [_P, C.c_int, _I]),
    ("mgmlmc_num_terms", C.c_int, [_P, _I, _I]),
    ("mgmlmc_compute_deflation", C.c_int, [_P, C.c_int, C.c_double, C.c_int]),
    ("mgmlmc_get_deflation", C.c_int, [_P, _D, _D, _D, _D, _D]),
    ("mgmlmc_compute_term_deflation", C.c_int, [_P, C.c_int, C.c_int, C.c_double, C.c_int]),
    ("mgmlmc_get_term_deflation", C.c_int, [_P, C.c_int, _I, _D, _D, _D, _D]),
    ("mgmlmc_term_deflated_part", C.c_int, [_P, C.c_int, _D]),
    ("mgmlmc_set_options", C.c_int, [_P, C.POINTER(Options)]),
    ("mgmlmc_autotune", C.c_int, [_P, C.c_size_t, C.c_int, C.POINTER(TuneResult)]),
    ("mgmlmc_compute_term_deflation_inexact", C.c_int, [_P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int]),
    ("mgmlmc_set_term_deflation_vectors", C.c_int, [_P, C.c_int, C.c_int, _D]),
    ("mgmlmc_estimate_level", C.c_int, [_P, C.c_int, C.c_int64, C.c_int, C.c_uint64, _D, C.POINTER(LevelStats)]),
    ("mgmlmc_estimate_level_probes", C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_int8), _D,
                                               C.POINTER(LevelStats)]),
    ("mgmlmc_estimate_concurrent", C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(C.c_int), C.c_int64, C.c_int,
                                             C.c_uint64, C.POINTER(C.POINTER(C.c_int8)), C.POINTER(_D),
                                             C.POINTER(LevelStats)]),
    ("mgmlmc_get_stats", C.c_int, [_P, C.c_int, C.POINTER(LevelStats)]),
    ("mgmlmc_reset_stats", C.c_int, [_P]),
    ("mgmlmc_estimate_trace", C.c_int, [_P, C.c_double, C.c_int64, C.c_uint64, _D, C.POINTER(TraceResult)]),
    ("mgmlmc_estimate_trace_concurrent", C.c_int, [C.POINTER(_P), C.c_int, C.c_double, C.c_int64, C.c_uint64, _D,
                                                   C.POINTER(TraceResult)]),
    ("mgmlmc_apply", C.c_int, [_P, C.c_int, C.c_int, C.c_int, _D, _D]),
    ("mgmlmc_solve", C.c_int, [_P, C.c_int, C.c_int, _D, _D, _I]),
    ("mgmlmc_noise", C.c_int, [_P, C.c_int, C.c_int64, C.c_int, C.c_uint64, _D]),
    ("mgmlmc_get_test_vectors", C.c_int, [_P, C.c_int, _D]),
    ("mgmlmc_level_info", C.c_int, [_P, C.c_int, _I, _I, _I, C.POINTER(C.c_int64)]),
    ("mgmlmc_profile", C.c_int, [_P, C.c_int, C.c_int]),
    ("mgmlmc_profile_report", C.c_int, [_P, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    ("mgmlmc_fma_peak", C.c_int, [C.c_int, _D]),
    ("mgmlmc_coarse_inverse_noalloc", C.c_int, [_P, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("mgmlmc_memory", C.c_int, [_P, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    ("mgmlmc_request_footprint", C.c_int, [C.POINTER(Request), C.POINTER(C.c_size_t)]),
    ("mgmlmc_server_create", C.c_int, [C.POINTER(_P), C.POINTER(ServerOptions)]),
    ("mgmlmc_server_destroy", None, [_P]),
    ("mgmlmc_submit", C.c_int, [_P, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    ("mgmlmc_poll", C.c_int, [_P, C.c_uint64, C.POINTER(RequestResult)]),
    ("mgmlmc_wait", C.c_int, [_P, C.c_uint64, C.c_double, C.POINTER(RequestResult)]),
    ("mgmlmc_cancel", C.c_int, [_P, C.c_uint64]),
    ("mgmlmc_get_server_stats", C.c_int, [_P, C.POINTER(ServerStats)]),
    ("mgmlmc_server_last_error", C.c_char_p, [_P]),
]

_lib = None


def load(path: str = LIB_PATH):
    """Load libmgmlmc.so and declare every entry point (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise MgmlmcError(-5, f"{path} not built: run __graft_entry__.build() (no CPU fallback exists)")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _cplx(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _trace_dict(res):
    d = {k: getattr(res, k) for k, _ in TraceResult._fields_ if k != "term"}
    d["terms"] = [res.term[t].as_dict() for t in range(res.nterms)]
    d["trace"] = complex(res.trace_re, res.trace_im)
    return d


def estimate_trace_concurrent(contexts, rel_tol: float, max_samples: int, seed: int, costs=None):
    """mgmlmc_estimate_trace_concurrent: the MLMC loop with term t drawn on contexts[t]
    (one context and CUDA stream per term), the terms of each round at once."""
    n = len(contexts)
    hs = (_P * n)(*[c.h for c in contexts])
    res = TraceResult()
    cst = None
    if costs is not None:
        arr = np.ascontiguousarray(costs, dtype=np.float64)
        cst = _dptr(arr)
    contexts[0]._check(contexts[0].lib.mgmlmc_estimate_trace_concurrent(hs, n, float(rel_tol), int(max_samples),
                                                                         C.c_uint64(seed), cst, C.byref(res)))
    return _trace_dict(res)


def estimate_concurrent(contexts, terms, first_sample: int, nsamples: int, seed: int, probes=None,
                        samples: bool = True, out=None):
    """mgmlmc_estimate_concurrent: entry i estimates term terms[i] on contexts[i] (each
    created on its own CUDA stream), all entries at once.  probes: None or a list with
    None (device noise) or an int8 array [nsamples][n_a] per entry.  Returns the list of
    sample arrays (or None) and the list of statistics dicts."""
    n = len(contexts)
    lib = contexts[0].lib
    hs = (_P * n)(*[c.h for c in contexts])
    ts = (C.c_int * n)(*terms)
    keep = []
    pp = None
    if probes is not None:
        pp = (C.POINTER(C.c_int8) * n)()
        for i, p in enumerate(probes):
            if p is not None:
                a = np.ascontiguousarray(p, dtype=np.int8)
                keep.append(a)
                pp[i] = a.ctypes.data_as(C.POINTER(C.c_int8))
    outs = None
    if samples:
        outs = out if out is not None else [np.zeros(nsamples, np.complex128) for _ in range(n)]
    op = (_D * n)(*[o.ctypes.data_as(_D) for o in outs]) if outs is not None else None
    st = (LevelStats * n)()
    code = lib.mgmlmc_estimate_concurrent(hs, n, ts, first_sample, nsamples, seed, pp, op, st)
    if code != 0:
        bad = next((c for c in contexts if lib.mgmlmc_last_error(c.h)), contexts[0])
        bad._check(code)
    return outs, [s_.as_dict() for s_ in st]


def fma_peak(precision: int) -> float:
    """Measured FMA throughput (FLOP/s) of the current device, precision 64 or 32."""
    v = C.c_double()
    code = load().mgmlmc_fma_peak(int(precision), C.byref(v))
    if code != 0:
        raise MgmlmcError(code, "fma_peak failed")
    return v.value


def default_options(**kw) -> Options:
    o = Options()
    load().mgmlmc_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Context:
    """One mgmlmc context: all device state of one trace problem.

    Methods carry the names of the C entry points without the ``mgmlmc_``
    prefix.  Host arrays use numpy; vectors of level l are complex arrays of
    shape (nvec, n_l).
    """

    def __init__(self, options: Options | None = None, torch_memory: bool = True, copy_of: "Context" = None, **kw):
        """copy_of: build this context as a device copy of another one's state
        (mgmlmc_create_copy), on the stream current now."""
        import torch
        if not torch.cuda.is_available():
            raise MgmlmcError(-5, "a CUDA device is required (this library has no CPU path)")
        self.lib = load()
        self.options = copy_of.options if copy_of is not None else (
            options if options is not None else default_options(**kw))
        self._mem = {}
        # the context works on the stream current at creation; its device memory is
        # taken on that stream too, so that a block the library gives back is reused
        # only in the order of that stream (whichever host thread calls in)
        self._stream = torch.cuda.current_stream()
        stream = C.c_void_p(self._stream.cuda_stream)
        if torch_memory:
            def _alloc(user, nbytes):
                try:
                    with torch.cuda.stream(self._stream):
                        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
                except Exception:
                    return None
                self._mem[t.data_ptr()] = t
                return t.data_ptr()

            def _free(user, ptr):
                self._mem.pop(ptr, None)

            self._alloc_cb, self._free_cb = ALLOC_FN(_alloc), FREE_FN(_free)
        else:
            self._alloc_cb, self._free_cb = ALLOC_FN(), FREE_FN()
        h = C.c_void_p()
        if copy_of is not None:
            code = self.lib.mgmlmc_create_copy(C.byref(h), copy_of.h, stream, self._alloc_cb, self._free_cb, None)
            if code != 0:
                copy_of._check(code)
        else:
            self._check(self.lib.mgmlmc_create(C.byref(h), C.byref(self.options), stream, self._alloc_cb,
                                               self._free_cb, None), h)
        self.h = h

    # ---------------------------------------------------------------- plumbing
    def _check(self, code, h=None):
        if code != 0:
            hh = h if h is not None else self.h
            msg = self.lib.mgmlmc_last_error(hh).decode() if hh else ""
            raise MgmlmcError(code, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.mgmlmc_destroy(self.h)
            self.h = None
            self._mem.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- problem
    def set_gauge(self, theta: np.ndarray):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        Lt, Lx, two = th.shape
        assert two == 2
        self._check(self.lib.mgmlmc_set_gauge(self.h, Lx, Lt, _dptr(th)))

    def set_mass(self, m0: float):
        self._check(self.lib.mgmlmc_set_mass(self.h, float(m0)))

    def set_hierarchy(self, agg, nvec, start_vectors, setup_iters: int = 4, setup_tol: float = 1e-12):
        nl = len(agg) + 1
        ax = (C.c_int * max(1, nl - 1))(*[a[0] for a in agg])
        at = (C.c_int * max(1, nl - 1))(*[a[1] for a in agg])
        nv = (C.c_int * max(1, nl - 1))(*list(nvec))
        keep = [_cplx(v) for v in start_vectors]
        ptrs = (_D * max(1, nl - 1))(*[k.ctypes.data_as(_D) for k in keep])
        self._check(self.lib.mgmlmc_set_hierarchy(self.h, nl, ax, at, nv, int(setup_iters), float(setup_tol), ptrs))

    def set_terms(self, skip=()):
        arr = (C.c_int * max(1, len(skip)))(*skip)
        self._check(self.lib.mgmlmc_set_terms(self.h, len(skip), arr))

    def num_terms(self):
        n = C.c_int()
        lv = (C.c_int * MAX_LEVELS)()
        self._check(self.lib.mgmlmc_num_terms(self.h, C.byref(n), lv))
        return n.value, list(lv)[: n.value]

    def level_info(self, level: int):
        lx, lt, d, n = C.c_int(), C.c_int(), C.c_int(), C.c_int64()
        self._check(self.lib.mgmlmc_level_info(self.h, level, C.byref(lx), C.byref(lt), C.byref(d), C.byref(n)))
        return lx.value, lt.value, d.value, n.value

    # ---------------------------------------------------------------- deflation
    def compute_deflation(self, k: int, tol: float = 1e-9, max_iters: int = 200):
        self._check(self.lib.mgmlmc_compute_deflation(self.h, int(k), float(tol), int(max_iters)))

    def get_deflation(self, k: int, L: int):
        n = self.level_info(L)[3]
        lam, sig = np.zeros(k), np.zeros(k)
        U = np.zeros((k, n), np.complex128)
        V = np.zeros((k, n), np.complex128)
        tau = np.zeros(2)
        self._check(self.lib.mgmlmc_get_deflation(self.h, _dptr(lam), _dptr(sig), U.ctypes.data_as(_D),
                                                  V.ctypes.data_as(_D), _dptr(tau)))
        return lam, sig, U, V, complex(tau[0], tau[1])

    def compute_term_deflation(self, term: int, k: int, tol: float = 1e-9, max_iters: int = 200):
        self._check(self.lib.mgmlmc_compute_term_deflation(self.h, int(term), int(k), float(tol), int(max_iters)))

    def compute_term_deflation_inexact(self, term: int, k: int, eig_tol: float = 1e-1, inner_tol: float = 1e-3,
                                       max_iters: int = 200):
        self._check(self.lib.mgmlmc_compute_term_deflation_inexact(self.h, int(term), int(k), float(eig_tol),
                                                                   float(inner_tol), int(max_iters)))

    def set_term_deflation_vectors(self, term: int, V: np.ndarray):
        v = _cplx(np.atleast_2d(V))
        self._check(self.lib.mgmlmc_set_term_deflation_vectors(self.h, int(term), v.shape[0], v.ctypes.data_as(_D)))

    def get_term_deflation(self, term: int, k: int):
        _, levels = self.num_terms()
        n = self.level_info(levels[term])[3]
        kk = C.c_int()
        lam = np.zeros(k)
        L = np.zeros((k, n), np.complex128)
        R = np.zeros((k, n), np.complex128)
        tau = np.zeros(2)
        self._check(self.lib.mgmlmc_get_term_deflation(self.h, int(term), C.byref(kk), _dptr(lam),
                                                       L.ctypes.data_as(_D), R.ctypes.data_as(_D), _dptr(tau)))
        return lam, L, R, complex(tau[0], tau[1])

    # ---------------------------------------------------------------- estimation
    def set_options(self, **kw):
        o = Options()
        C.memmove(C.byref(o), C.byref(self.options), C.sizeof(Options))
        for k, v in kw.items():
            setattr(o, k, v)
        self._check(self.lib.mgmlmc_set_options(self.h, C.byref(o)))
        self.options = o

    def autotune(self, hbm_budget: int = 0, max_trials: int = 10) -> dict:
        r = TuneResult()
        self._check(self.lib.mgmlmc_autotune(self.h, int(hbm_budget), int(max_trials), C.byref(r)))
        for k in ("fgmres_restart", "nu_post", "kcycle_iters"):
            setattr(self.options, k, getattr(r, k))
        self.options.max_block_rhs = r.block_rhs
        return r.as_dict()

    def term_deflated_part(self, term: int) -> complex:
        tau = np.zeros(2)
        self._check(self.lib.mgmlmc_term_deflated_part(self.h, term, _dptr(tau)))
        return complex(tau[0], tau[1])

    def estimate_level(self, term: int, first: int, nsamples: int, seed: int, samples: bool = True):
        out = np.zeros(nsamples, np.complex128) if samples else None
        st = LevelStats()
        ptr = out.ctypes.data_as(_D) if samples else None
        self._check(self.lib.mgmlmc_estimate_level(self.h, term, int(first), int(nsamples), C.c_uint64(seed),
                                                   ptr, C.byref(st)))
        return out, st.as_dict()

    def estimate_level_probes(self, term: int, probes: np.ndarray, samples: bool = True, out=None):
        pr = np.ascontiguousarray(probes, dtype=np.int8)
        ns = pr.shape[0]
        if out is None and samples:
            out = np.zeros(ns, np.complex128)
        st = LevelStats()
        self._check(self.lib.mgmlmc_estimate_level_probes(
            self.h, term, ns, pr.ctypes.data_as(C.POINTER(C.c_int8)),
            out.ctypes.data_as(_D) if out is not None else None, C.byref(st)))
        return out, st.as_dict()

    def get_stats(self, term: int):
        st = LevelStats()
        self._check(self.lib.mgmlmc_get_stats(self.h, term, C.byref(st)))
        return st.as_dict()

    def reset_stats(self):
        self._check(self.lib.mgmlmc_reset_stats(self.h))

    def estimate_trace(self, rel_tol: float, max_samples: int, seed: int, costs=None):
        res = TraceResult()
        cst = None
        if costs is not None:
            arr = np.ascontiguousarray(costs, dtype=np.float64)
            cst = _dptr(arr)
        self._check(self.lib.mgmlmc_estimate_trace(self.h, float(rel_tol), int(max_samples), C.c_uint64(seed),
                                                   cst, C.byref(res)))
        return _trace_dict(res)

    # ---------------------------------------------------------------- test hooks
    def apply(self, op: int, level: int, x: np.ndarray, n_out: int):
        xx = _cplx(np.atleast_2d(x))
        y = np.zeros((xx.shape[0], n_out), np.complex128)
        self._check(self.lib.mgmlmc_apply(self.h, op, level, xx.shape[0], xx.ctypes.data_as(_D),
                                          y.ctypes.data_as(_D)))
        return y

    def solve(self, level: int, b: np.ndarray):
        bb = _cplx(np.atleast_2d(b))
        x = np.zeros_like(bb)
        it = C.c_int()
        self._check(self.lib.mgmlmc_solve(self.h, level, bb.shape[0], bb.ctypes.data_as(_D),
                                          x.ctypes.data_as(_D), C.byref(it)))
        return x, it.value

    def noise(self, level: int, first: int, nsamples: int, seed: int):
        n = self.level_info(level)[3]
        x = np.zeros((nsamples, n))
        self._check(self.lib.mgmlmc_noise(self.h, level, int(first), int(nsamples), C.c_uint64(seed), _dptr(x)))
        return x

    def profile(self, enable: bool = True, reset: bool = False):
        self._check(self.lib.mgmlmc_profile(self.h, int(enable), int(reset)))

    def profile_report(self) -> dict:
        import json
        need = C.c_size_t()
        self._check(self.lib.mgmlmc_profile_report(self.h, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value + 1)
        self._check(self.lib.mgmlmc_profile_report(self.h, buf, need.value + 1, C.byref(need)))
        return json.loads(buf.value.decode())

    def coarse_inverse_noalloc(self, nrhs: int, x_ptr: int, y_ptr: int, stream: int = 0):
        """y = D_L^{-1} x for caller-owned device buffers (FP32 complex [n_L][nrhs]); allocates nothing."""
        self._check(self.lib.mgmlmc_coarse_inverse_noalloc(self.h, int(nrhs), C.c_void_p(x_ptr), C.c_void_p(y_ptr),
                                                           C.c_void_p(stream)))

    def memory(self):
        """(live, peak) device bytes held through the context's allocator."""
        live, peak = C.c_size_t(), C.c_size_t()
        self._check(self.lib.mgmlmc_memory(self.h, C.byref(live), C.byref(peak)))
        return live.value, peak.value

    def get_test_vectors(self, level: int, nvec: int):
        n = self.level_info(level)[3]
        v = np.zeros((nvec, n), np.complex128)
        self._check(self.lib.mgmlmc_get_test_vectors(self.h, level, v.ctypes.data_as(_D)))
        return v


# ------------------------------------------------------------------------- serving
def make_request(theta, m0: float, agg, nvec, start_vectors, rel_tol: float, seed: int, k: int = 0,
                 setup_iters: int = 4, setup_tol: float = 1e-12, defl_tol: float = 1e-9, defl_max_iters: int = 400,
                 max_samples: int = 1 << 40, costs=None, options: Options | None = None, sum_levels: int = 0,
                 **kw):
    """A trace request (mgmlmc_request) for Server.submit.  theta [Lt][Lx][2], agg a list
    of (ax, at) per coarse level, start_vectors one complex array (nvec, n_l) per coarse
    level; costs: fixed per-sample costs of the terms (None: measured device time).
    The arrays are kept alive on the returned object until it is submitted."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    Lt, Lx, two = th.shape
    assert two == 2
    r = Request()
    r.Lx, r.Lt, r.m0 = Lx, Lt, float(m0)
    r.theta = th.ctypes.data_as(_D)
    r.nlevels = len(agg) + 1
    keep = [th]
    for l, (a, nv, sv) in enumerate(zip(agg, nvec, start_vectors)):
        r.agg_x[l], r.agg_t[l], r.nvec[l] = int(a[0]), int(a[1]), int(nv)
        v = _cplx(sv)
        keep.append(v)
        r.start_vectors[l] = v.ctypes.data_as(_D)
    r.setup_iters, r.setup_tol = int(setup_iters), float(setup_tol)
    r.k, r.defl_tol, r.defl_max_iters = int(k), float(defl_tol), int(defl_max_iters)
    r.rel_tol, r.max_samples, r.seed = float(rel_tol), int(max_samples), int(seed)
    for t, c in enumerate(costs or []):
        r.costs[t] = float(c)
    r.opt = options if options is not None else default_options(**kw)
    r.sum_levels = int(sum_levels)
    r._keep = keep
    return r


def request_footprint(req: Request) -> int:
    """mgmlmc_request_footprint: upper estimate of the request's device bytes."""
    lib = load()
    b = C.c_size_t()
    code = lib.mgmlmc_request_footprint(C.byref(req), C.byref(b))
    if code != 0:
        raise MgmlmcError(code, lib.mgmlmc_server_last_error(None).decode())
    return b.value


def _result_dict(rr: RequestResult):
    d = {k: getattr(rr, k) for k, _ in RequestResult._fields_ if k not in ("result", "error")}
    d["error"] = rr.error.decode()
    d["result"] = _trace_dict(rr.result)
    return d


class Server:
    """A request server on the current CUDA device (mgmlmc_server_*): trace requests are
    admitted by footprint against an HBM budget and run on their own contexts and
    streams, overlapping on the device."""

    def __init__(self, hbm_budget: int = 0, max_active: int = 4, max_bypass: int = 4):
        import torch
        if not torch.cuda.is_available():
            raise MgmlmcError(-5, "a CUDA device is required (this library has no CPU path)")
        self.lib = load()
        o = ServerOptions(int(hbm_budget), int(max_active), int(max_bypass))
        h = C.c_void_p()
        self._check(self.lib.mgmlmc_server_create(C.byref(h), C.byref(o)))
        self.h = h

    def _check(self, code):
        if code != 0:
            raise MgmlmcError(code, self.lib.mgmlmc_server_last_error(None).decode())

    def submit(self, req: Request) -> int:
        i = C.c_uint64()
        self._check(self.lib.mgmlmc_submit(self.h, C.byref(req), C.byref(i)))
        return i.value

    def poll(self, rid: int):
        """The result dict once finished, else None."""
        rr = RequestResult()
        code = self.lib.mgmlmc_poll(self.h, C.c_uint64(rid), C.byref(rr))
        if code == PENDING:
            return None
        self._check(code)
        return _result_dict(rr)

    def wait(self, rid: int, timeout: float = -1.0):
        """The result dict, waiting at most timeout seconds (< 0: no limit); None on timeout."""
        rr = RequestResult()
        code = self.lib.mgmlmc_wait(self.h, C.c_uint64(rid), float(timeout), C.byref(rr))
        if code == PENDING:
            return None
        self._check(code)
        return _result_dict(rr)

    def cancel(self, rid: int):
        self._check(self.lib.mgmlmc_cancel(self.h, C.c_uint64(rid)))

    def stats(self) -> dict:
        st = ServerStats()
        self._check(self.lib.mgmlmc_get_server_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.mgmlmc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
