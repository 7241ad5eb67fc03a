"""Host-side checks of the C ABI (no GPU): the library builds for sm_103a,
loads, and exports every function include/dcg.h declares; default options
match the header; the binding refuses bad arguments before any CUDA call."""
import ctypes as C
import os
import re

import pytest

from paper_2606_13429_gb300 import build as B
from paper_2606_13429_gb300 import dcg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return dcg.load()


def test_exports_every_declared_symbol(lib):
    names = dcg.header_functions()
    assert len(names) >= 20
    raw = C.CDLL(dcg.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_header_cites_paper_passages():
    txt = open(os.path.join(ROOT, "include", "dcg.h")).read()
    for ref in ["Algorithm 2", "Algorithm 3", "Eq. Vmatrix", "Section 4.2", "Corollary 1", "Eq. fixed_tol", "Eq. tol"]:
        assert ref in txt, ref


def test_every_declaration_has_its_own_comment():
    """Each function declared in include/dcg.h is preceded by a comment of its
    own (the passage it implements, or that it has no counterpart), not only
    by a comment somewhere in the file."""
    txt = open(os.path.join(ROOT, "include", "dcg.h")).read()
    lines = txt.splitlines()
    for name in dcg.header_functions():
        i = next(k for k, ln in enumerate(lines) if re.search(r"\b%s\s*\(" % name, ln) and not ln.strip().startswith(("*", "/*")))
        # walk back over other declarations of the same group to the comment
        j = i - 1
        while j >= 0 and not lines[j].strip().endswith("*/"):
            assert lines[j].strip() == "" or re.match(r"^(int|void|double|const|long|#define)\b", lines[j].strip()) or \
                lines[j].startswith(" "), (name, lines[j])
            j -= 1
        assert j >= 0 and i - j <= 6, name


def test_default_options(lib):
    o = dcg.options()
    assert (o.max_levels, o.patch, o.overlap, o.m1, o.m2) == (4, 4, 1, 2, 2)
    assert o.inner_rule == dcg.DCG_INNER_FIXED and abs(o.c - 0.01) < 1e-15
    assert o.recurrence == dcg.DCG_FCG1 and o.precision == dcg.DCG_FP64 and o.deflate == 1
    assert o.inner_nmax == 100 and o.max_restarts == 3 and o.check_every == 1 and o.stall_window == 200


def test_status_strings(lib):
    for code in range(8):
        assert dcg.status_string(code)
    assert dcg.status_string(2) == "not converged"


def test_invalid_arguments_rejected_without_gpu(lib):
    out = C.c_void_p()
    for dim, n, dt, nu in [(1, 8, 1e-3, 1.0), (2, 1, 1e-3, 1.0), (2, 8, 0.0, 1.0), (3, 8, 1e-3, -1.0),
                           (2, 8, float("nan"), 1.0)]:
        mesh = dcg.dcg_mesh(dim, n)
        code = lib.dcg_assemble(C.byref(mesh), dt, nu, None, 0, C.byref(out), None)
        assert code == dcg.DCG_ERR_INVALID_ARG
        assert "dcg_assemble" in dcg.last_error()
    assert lib.dcg_setup(None, None, None) == dcg.DCG_ERR_INVALID_ARG
    st = dcg.dcg_stats()
    assert lib.dcg_solve(None, None, None, 1e-8, 10, C.byref(st), None) == dcg.DCG_ERR_INVALID_ARG


def test_built_for_sm103a():
    assert "compute_103a" in B.GENCODE and "sm_103a" in B.GENCODE
    assert all(f.endswith(".cu") for f in os.listdir(B.CSRC) if not f.endswith(".cuh"))


def test_binding_is_marshalling_only():
    """The binding and package never import the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_2606_13429_gb300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg, fn)).read()
            assert not re.search(r"^\s*(from|import)\s+oracle", src, re.M), fn


def test_batched_and_autotune_reject_bad_arguments_without_gpu(lib):
    st = (dcg.dcg_stats * 1)()
    assert lib.dcg_solve_batched(-1, None, 1, None, None, 1e-8, 10, st, None) == dcg.DCG_ERR_INVALID_ARG
    assert lib.dcg_solve_batched(1, None, 1, None, None, 1e-8, 10, st, None) == dcg.DCG_ERR_INVALID_ARG
    assert lib.dcg_solve_batched(0, None, 0, None, None, 1e-8, 10, st, None) == dcg.DCG_ERR_INVALID_ARG
    # an empty batch is a no-op that touches no device
    assert lib.dcg_solve_batched(0, None, 1, None, None, 1e-8, 10, st, None) == dcg.DCG_OK
    best, ms = dcg.dcg_options(), C.c_double()
    base = dcg.options()
    assert lib.dcg_autotune(None, C.byref(base), None, 1e-6, 3, C.byref(best), C.byref(ms), None) == \
        dcg.DCG_ERR_INVALID_ARG
    assert "dcg_autotune" in dcg.last_error()


def test_matrix_free_limits_rejected_without_gpu(lib):
    out = C.c_void_p()
    for dim, n in [(2, 16), (3, 3)]:
        mesh = dcg.dcg_mesh(dim, n)
        assert lib.dcg_assemble(C.byref(mesh), 1e-3, 1.0, None, 1, C.byref(out), None) == dcg.DCG_ERR_UNSUPPORTED
        assert "matrix-free" in dcg.last_error()
    assert lib.dcg_spmv_prec(None, None, None, dcg.DCG_MIXED, None) == dcg.DCG_ERR_INVALID_ARG
