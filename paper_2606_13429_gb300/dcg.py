"""Thin Python binding of libdcg (include/dcg.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes
plain pointers and sizes; torch tensors are accepted for device arrays
(CUDA, float64, contiguous) and the current torch stream is used unless one
is given. There is no fallback: if libdcg.so is missing or fails to load,
every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdcg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "dcg.h")

DCG_OK = 0
DCG_ERR_INVALID_ARG = 1
DCG_ERR_NOT_CONVERGED = 2
DCG_ERR_BREAKDOWN = 3
DCG_ERR_CUDA = 4
DCG_ERR_OOM = 5
DCG_ERR_UNSUPPORTED = 6
DCG_ERR_STATE = 7

DCG_INNER_FIXED, DCG_INNER_ADAPTIVE, DCG_INNER_EXACT = 0, 1, 2
DCG_FCG1, DCG_FR, DCG_FCG_INF, DCG_GMRES = 0, 1, 2, 3
DCG_FP64, DCG_MIXED = 0, 1
DCG_INV_FP32, DCG_INV_BF16 = 0, 1
DCG_RAS_MULTIPLICITY, DCG_RAS_RESTRICTED = 0, 1
DCG_IMPLICIT_EULER, DCG_CRANK_NICOLSON, DCG_BDF2 = 0, 1, 2
PROF_CLASSES = ["spmv", "vec", "ras_solve", "ras_update", "transfer", "coarse", "inner_res"]


class dcg_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int)]


class dcg_options(C.Structure):
    _fields_ = [("max_levels", C.c_int), ("patch", C.c_int), ("overlap", C.c_int), ("m1", C.c_int),
                ("m2", C.c_int), ("inner_rule", C.c_int), ("c", C.c_double), ("inner_nmax", C.c_int),
                ("recurrence", C.c_int), ("precision", C.c_int), ("ras_inverse", C.c_int),
                ("ras_weights", C.c_int), ("deflate", C.c_int), ("max_restarts", C.c_int),
                ("fcg_max_dirs", C.c_int), ("check_every", C.c_int),
                ("stall_window", C.c_int), ("device_loop", C.c_int)]


class dcg_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_its", C.c_int), ("total_mg_cycles", C.c_int),
                ("iter_mg_cycles", C.c_int), ("restarts", C.c_int), ("avg_inner", C.c_double),
                ("true_relres", C.c_double), ("solve_ms", C.c_double), ("fcg_truncated", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DCGError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__("%s failed: %s (%d): %s" % (where, status_string(code), code, msg))
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libdcg.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libdcg.so not found at %s: build it with __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    P, VP, I, D, LL = C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_longlong
    sig = {
        "dcg_default_options": (None, [C.POINTER(dcg_options)]),
        "dcg_status_string": (C.c_char_p, [I]),
        "dcg_last_error": (C.c_char_p, []),
        "dcg_assemble": (I, [C.POINTER(dcg_mesh), D, D, C.POINTER(C.c_double), I, C.POINTER(P), VP]),
        "dcg_setup": (I, [P, C.POINTER(dcg_options), VP]),
        "dcg_solve": (I, [P, VP, VP, D, I, C.POINTER(dcg_stats), VP]),
        "dcg_solve_host": (I, [P, C.POINTER(C.c_double), C.POINTER(C.c_double), D, I, C.POINTER(dcg_stats), VP]),
        "dcg_solve_batched": (I, [I, C.POINTER(P), I, C.POINTER(VP), C.POINTER(VP), D, I, C.POINTER(dcg_stats), VP]),
        "dcg_destroy": (None, [P]),
        "dcg_problem_info": (I, [P, C.POINTER(LL), C.POINTER(LL), C.POINTER(LL), C.POINTER(I)]),
        "dcg_level_nodes": (I, [P, I, C.POINTER(LL)]),
        "dcg_export_pattern": (I, [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "dcg_export_values": (I, [P, C.POINTER(C.c_double)]),
        "dcg_spmv": (I, [P, VP, VP, VP]),
        "dcg_spmv_prec": (I, [P, VP, VP, I, VP]),
        "dcg_extract": (I, [P, VP, VP, VP]),
        "dcg_embed": (I, [P, VP, VP, VP]),
        "dcg_inner_apply": (I, [P, VP, VP, VP]),
        "dcg_mg_cycles": (I, [P, VP, VP, I, VP]),
        "dcg_mg_solve": (I, [P, VP, VP, D, I, C.POINTER(I), VP]),
        "dcg_ras_step": (I, [P, I, VP, VP, VP]),
        "dcg_coarse_solve": (I, [P, VP, VP, VP]),
        "dcg_profile_enable": (I, [P, C.c_uint, VP]),
        "dcg_profile_read": (I, [P, I, C.POINTER(D), C.POINTER(LL), C.POINTER(D), C.POINTER(D), VP]),
        "dcg_kernel_launches": (LL, []),
        "dcg_measure_fma_rate": (I, [I, C.POINTER(D), VP]),
        "dcg_scheme_alpha": (D, [I, D]),
        "dcg_apply_div": (I, [P, VP, VP, VP]),
        "dcg_time_rhs": (I, [P, I, VP, VP, VP, VP, VP, VP]),
        "dcg_pressure": (I, [P, VP, VP, VP]),
        "dcg_divergence": (I, [P, VP, VP, VP]),
        "dcg_time_integrate": (I, [P, I, D, I, VP, C.POINTER(VP), C.POINTER(VP), VP, D, I, C.POINTER(dcg_stats),
                                   VP]),
        "dcg_selftest_bounded_wait": (I, [C.c_uint, C.POINTER(I), VP]),
        "dcg_coarse_solve_static": (I, [P, VP, VP, VP]),
        "dcg_autotune": (I, [P, C.POINTER(dcg_options), VP, D, I, C.POINTER(dcg_options), C.POINTER(D), VP]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_functions(path: str = HEADER):
    """Names of the functions include/dcg.h declares."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dcg_[a-z0-9_]+)\s*\(", txt)))


def status_string(code: int) -> str:
    return load().dcg_status_string(code).decode()


def last_error() -> str:
    return load().dcg_last_error().decode()


def _check(code, where, ok=(DCG_OK,)):
    if code not in ok:
        raise DCGError(code, where, last_error())
    return code


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t, n=None, name="array"):
    """Device pointer of a CUDA float64 contiguous tensor (or an int address)."""
    if isinstance(t, int):
        return C.c_void_p(t)
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("%s must be a contiguous CUDA float64 tensor" % name)
    if n is not None and t.numel() != n:
        raise ValueError("%s has %d entries, expected %d" % (name, t.numel(), n))
    return C.c_void_p(t.data_ptr())


def options(**kw) -> dcg_options:
    o = dcg_options()
    load().dcg_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError("unknown option %r" % k)
        setattr(o, k, v)
    return o


class Problem:
    """Owns a dcg_problem*; freed with dcg_destroy."""

    def __init__(self, ptr, dim, n):
        self.ptr = C.c_void_p(ptr)
        self.dim, self.n = dim, n
        N, nn, nb, lv = C.c_longlong(), C.c_longlong(), C.c_longlong(), C.c_int()
        _check(load().dcg_problem_info(self.ptr, C.byref(N), C.byref(nn), C.byref(nb), C.byref(lv)), "dcg_problem_info")
        self.N, self.n_nodes, self.nnzb = N.value, nn.value, nb.value

    @property
    def levels(self) -> int:
        lv = C.c_int()
        _check(load().dcg_problem_info(self.ptr, None, None, None, C.byref(lv)), "dcg_problem_info")
        return lv.value

    def level_nodes(self, level: int) -> int:
        """Interior nodes of multigrid level `level` (1 = coarsest)."""
        nn = C.c_longlong()
        _check(load().dcg_level_nodes(self.ptr, level, C.byref(nn)), "dcg_level_nodes")
        return nn.value

    def close(self):
        if self.ptr and self.ptr.value:
            load().dcg_destroy(self.ptr)
            self.ptr = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dcg_assemble(dim, n, dt, nu=1.0, nu_elem=None, matrix_free=False, stream=None) -> Problem:
    lib = load()
    mesh = dcg_mesh(dim, n)
    out = C.c_void_p()
    nu_ptr = None
    keep = None
    if nu_elem is not None:
        import numpy as np
        keep = np.ascontiguousarray(nu_elem, dtype=np.float64)
        if keep.size != n ** dim:
            raise ValueError("nu_elem needs n**dim entries")
        nu_ptr = keep.ctypes.data_as(C.POINTER(C.c_double))
    _check(lib.dcg_assemble(C.byref(mesh), dt, nu, nu_ptr, int(matrix_free), C.byref(out), _stream(stream)),
           "dcg_assemble")
    return Problem(out.value, dim, n)


def dcg_setup(prob: Problem, opts: dcg_options | None = None, stream=None, **kw):
    o = opts if opts is not None else options(**kw)
    _check(load().dcg_setup(prob.ptr, C.byref(o), _stream(stream)), "dcg_setup")
    prob.opts = o
    return o


def dcg_solve(prob: Problem, f, x, tol=1e-8, max_it=100000, stream=None) -> dict:
    st = dcg_stats()
    code = load().dcg_solve(prob.ptr, _dptr(f, prob.N, "f"), _dptr(x, prob.N, "x"), tol, max_it, C.byref(st),
                            _stream(stream))
    _check(code, "dcg_solve", ok=(DCG_OK, DCG_ERR_NOT_CONVERGED, DCG_ERR_BREAKDOWN))
    d = st.as_dict()
    d["status"] = code
    return d


def dcg_solve_host(prob: Problem, f_host, x_host, tol=1e-8, max_it=100000, stream=None) -> dict:
    """f_host, x_host: numpy float64 arrays (x_host in/out) or CPU tensors."""
    import numpy as np

    def ptr(a):
        if hasattr(a, "data_ptr"):
            if a.is_cuda or not a.is_contiguous():
                raise ValueError("host arrays must be contiguous CPU tensors")
            return C.cast(C.c_void_p(a.data_ptr()), C.POINTER(C.c_double))
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.size == prob.N):
            raise ValueError("host arrays must be contiguous float64 of size N")
        return a.ctypes.data_as(C.POINTER(C.c_double))

    st = dcg_stats()
    code = load().dcg_solve_host(prob.ptr, ptr(f_host), ptr(x_host), tol, max_it, C.byref(st), _stream(stream))
    _check(code, "dcg_solve_host", ok=(DCG_OK, DCG_ERR_NOT_CONVERGED, DCG_ERR_BREAKDOWN))
    d = st.as_dict()
    d["status"] = code
    return d


def dcg_solve_batched(probs, nrhs, fs, xs, tol=1e-8, max_it=100000, stream=None):
    k = len(probs) * nrhs
    if len(fs) != k or len(xs) != k:
        raise ValueError("need len(probs)*nrhs right-hand sides and solutions")
    P = (C.c_void_p * len(probs))(*[p.ptr.value for p in probs])
    F = (C.c_void_p * k)(*[_dptr(f).value for f in fs])
    X = (C.c_void_p * k)(*[_dptr(x).value for x in xs])
    stats = (dcg_stats * k)()
    code = load().dcg_solve_batched(len(probs), P, nrhs, F, X, tol, max_it, stats, _stream(stream))
    _check(code, "dcg_solve_batched", ok=(DCG_OK, DCG_ERR_NOT_CONVERGED, DCG_ERR_BREAKDOWN))
    return code, [s.as_dict() for s in stats]


def dcg_autotune(prob: Problem, f, base: dcg_options | None = None, inner_tol=1e-6, reps=3, stream=None, **kw):
    """Measure the W-cycle candidates on right-hand side f; the problem is left
    set up with the fastest. Returns (options, ms per inner solve)."""
    b = base if base is not None else options(**kw)
    best, ms = dcg_options(), C.c_double()
    _check(load().dcg_autotune(prob.ptr, C.byref(b), _dptr(f, prob.N, "f"), inner_tol, reps, C.byref(best),
                               C.byref(ms), _stream(stream)), "dcg_autotune")
    prob.opts = best
    return best, ms.value


def dcg_export_pattern(prob: Problem):
    import numpy as np
    rp = np.empty(prob.n_nodes + 1, dtype=np.int32)
    ci = np.empty(prob.nnzb, dtype=np.int32)
    _check(load().dcg_export_pattern(prob.ptr, rp.ctypes.data_as(C.POINTER(C.c_int)),
                                     ci.ctypes.data_as(C.POINTER(C.c_int))), "dcg_export_pattern")
    return rp, ci


def dcg_export_values(prob: Problem):
    import numpy as np
    b = prob.dim * prob.dim
    v = np.empty((prob.nnzb, b, b), dtype=np.float64)
    _check(load().dcg_export_values(prob.ptr, v.ctypes.data_as(C.POINTER(C.c_double))), "dcg_export_values")
    return v


def dcg_spmv(prob: Problem, x, y, stream=None):
    _check(load().dcg_spmv(prob.ptr, _dptr(x, prob.N, "x"), _dptr(y, prob.N, "y"), _stream(stream)), "dcg_spmv")


def dcg_spmv_prec(prob: Problem, x, y, precision, stream=None):
    _check(load().dcg_spmv_prec(prob.ptr, _dptr(x, prob.N, "x"), _dptr(y, prob.N, "y"), precision, _stream(stream)),
           "dcg_spmv_prec")


def dcg_extract(prob: Problem, y, q, stream=None):
    _check(load().dcg_extract(prob.ptr, _dptr(y, prob.N, "y"), _dptr(q, prob.n_nodes, "q"), _stream(stream)),
           "dcg_extract")


def dcg_embed(prob: Problem, q, y, stream=None):
    _check(load().dcg_embed(prob.ptr, _dptr(q, prob.n_nodes, "q"), _dptr(y, prob.N, "y"), _stream(stream)),
           "dcg_embed")


def dcg_inner_apply(prob: Problem, z, y, stream=None):
    _check(load().dcg_inner_apply(prob.ptr, _dptr(z, prob.n_nodes, "z"), _dptr(y, prob.n_nodes, "y"),
                                  _stream(stream)), "dcg_inner_apply")


def dcg_mg_cycles(prob: Problem, g, z, ncycles, stream=None):
    _check(load().dcg_mg_cycles(prob.ptr, _dptr(g, prob.n_nodes, "g"), _dptr(z, prob.n_nodes, "z"), ncycles,
                                _stream(stream)), "dcg_mg_cycles")


def dcg_mg_solve(prob: Problem, g, z, tol, nmax=100, stream=None) -> int:
    n = C.c_int()
    _check(load().dcg_mg_solve(prob.ptr, _dptr(g, prob.n_nodes, "g"), _dptr(z, prob.n_nodes, "z"), tol, nmax,
                               C.byref(n), _stream(stream)), "dcg_mg_solve")
    return n.value


def dcg_ras_step(prob: Problem, level, f, z, stream=None):
    nn = prob.level_nodes(level) if 1 <= level <= prob.levels else None
    _check(load().dcg_ras_step(prob.ptr, level, _dptr(f, nn, "f"), _dptr(z, nn, "z"), _stream(stream)),
           "dcg_ras_step")


def dcg_coarse_solve(prob: Problem, f, z, stream=None):
    nn = prob.level_nodes(1)
    _check(load().dcg_coarse_solve(prob.ptr, _dptr(f, nn, "f"), _dptr(z, nn, "z"), _stream(stream)),
           "dcg_coarse_solve")


def dcg_profile_enable(prob: Problem, classes=(), stream=None):
    """Time the named kernel classes (see PROF_CLASSES) with CUDA events."""
    mask = 0
    for c in classes:
        mask |= 1 << PROF_CLASSES.index(c)
    _check(load().dcg_profile_enable(prob.ptr, mask, _stream(stream)), "dcg_profile_enable")


def dcg_profile_read(prob: Problem, stream=None) -> dict:
    out = {}
    for i, name in enumerate(PROF_CLASSES):
        ms, n, fl, by = C.c_double(), C.c_longlong(), C.c_double(), C.c_double()
        _check(load().dcg_profile_read(prob.ptr, i, C.byref(ms), C.byref(n), C.byref(fl), C.byref(by),
                                       _stream(stream)), "dcg_profile_read")
        out[name] = {"ms": ms.value, "launches": n.value, "flops": fl.value, "bytes": by.value}
    return out


def dcg_coarse_solve_static(prob: Problem, f, z, stream=None):
    """Allocation-free coarsest solve (fixed device scratch inside the library)."""
    nn = prob.level_nodes(1)
    _check(load().dcg_coarse_solve_static(prob.ptr, _dptr(f, nn, "f"), _dptr(z, nn, "z"), _stream(stream)),
           "dcg_coarse_solve_static")


def dcg_measure_fma_rate(precision, stream=None) -> float:
    """Measured FMA rate (TFLOP/s) of the FP64 (DCG_FP64) or FP32 (DCG_MIXED) pipes."""
    t = C.c_double()
    _check(load().dcg_measure_fma_rate(precision, C.byref(t), _stream(stream)), "dcg_measure_fma_rate")
    return t.value


def dcg_selftest_bounded_wait(max_polls, stream=None) -> bool:
    """True when the bounded mbarrier wait gave up after max_polls polls."""
    g = C.c_int()
    _check(load().dcg_selftest_bounded_wait(max_polls, C.byref(g), _stream(stream)), "dcg_selftest_bounded_wait")
    return bool(g.value)


def dcg_scheme_alpha(scheme, dt) -> float:
    return float(load().dcg_scheme_alpha(scheme, dt))


def dcg_apply_div(prob: Problem, x, y, stream=None):
    _check(load().dcg_apply_div(prob.ptr, _dptr(x, prob.N, "x"), _dptr(y, prob.N, "y"), _stream(stream)),
           "dcg_apply_div")


def dcg_time_rhs(prob: Problem, scheme, s1, F1, rhs, s2=None, F0=None, stream=None):
    _check(load().dcg_time_rhs(prob.ptr, scheme, _dptr(s1, prob.N, "s1"),
                               _dptr(s2, prob.N, "s2") if s2 is not None else None, _dptr(F1, prob.N, "F1"),
                               _dptr(F0, prob.N, "F0") if F0 is not None else None, _dptr(rhs, prob.N, "rhs"),
                               _stream(stream)), "dcg_time_rhs")


def dcg_pressure(prob: Problem, sigma, pres, stream=None):
    _check(load().dcg_pressure(prob.ptr, _dptr(sigma, prob.N, "sigma"), _dptr(pres, prob.n_nodes, "pres"),
                               _stream(stream)), "dcg_pressure")


def dcg_divergence(prob: Problem, sigma, div_elem, stream=None):
    ne = prob.n ** prob.dim
    _check(load().dcg_divergence(prob.ptr, _dptr(sigma, prob.N, "sigma"), _dptr(div_elem, ne * prob.dim, "div"),
                                 _stream(stream)), "dcg_divergence")


def dcg_time_integrate(prob: Problem, scheme, dt, sigma0, loads, sigma_out, u_elem=None, tol=1e-8, max_it=100000,
                       stream=None):
    """loads: nsteps+1 device arrays F^0..F^nsteps; sigma_out: nsteps arrays."""
    nsteps = len(sigma_out)
    if len(loads) != nsteps + 1:
        raise ValueError("need nsteps + 1 load vectors")
    Fp = (C.c_void_p * (nsteps + 1))(*[_dptr(f, prob.N, "F").value for f in loads])
    Sp = (C.c_void_p * nsteps)(*[_dptr(x, prob.N, "sigma_out").value for x in sigma_out])
    stats = (dcg_stats * nsteps)()
    ne = prob.n ** prob.dim
    code = load().dcg_time_integrate(prob.ptr, scheme, dt, nsteps, _dptr(sigma0, prob.N, "sigma0"), Fp, Sp,
                                     _dptr(u_elem, ne * prob.dim, "u") if u_elem is not None else None, tol, max_it,
                                     stats, _stream(stream))
    _check(code, "dcg_time_integrate", ok=(DCG_OK, DCG_ERR_NOT_CONVERGED, DCG_ERR_BREAKDOWN))
    return code, [st.as_dict() for st in stats]


def dcg_kernel_launches() -> int:
    return int(load().dcg_kernel_launches())
