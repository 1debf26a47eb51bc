"""C ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every symbol include/semax.h declares, and rejects bad arguments on
the host before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1503_07659_gb300._lib as L
    return L.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "semax.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"^\s*(?:int|const char \*|size_t)\s*\**\s*([a-z_0-9]+)\s*\(", text, flags=re.M))


def test_every_declared_symbol_is_exported(lib):
    import paper_1503_07659_gb300._lib as L
    declared = _declared()
    assert declared == set(L.EXPORTS), declared ^ set(L.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_strerror_covers_every_status(lib):
    for st in range(0, -10, -1):
        assert lib.semax_strerror(st) not in (None, b"unknown status")


# fake device addresses: argument checks run before any CUDA call
A = 1 << 40


@pytest.mark.parametrize("fn", ["sem_ax", "sem_ax_f64x", "sem_ax_f64tc", "sem_ax_f32", "sem_ax_bf16x3",
                                "sem_ax_f16x3"])
def test_argument_validation(lib, fn):
    f = getattr(lib, fn)

    def call(E, N, u=A, G=A + (1 << 32), D=A + (2 << 32), w=A + (3 << 32)):
        extra = {"sem_ax": (), "sem_ax_f64x": (), "sem_ax_f64tc": (), "sem_ax_f32": (None,),
                 "sem_ax_bf16x3": (None, 3), "sem_ax_f16x3": (None,)}[fn]
        return f(E, N, u, G, D, w, *extra, None)

    assert call(0, 7) == 0                      # empty: no-op, nothing inspected
    assert call(0, 7, None, None, None, None) == 0
    assert call(-1, 7) == -1                    # EINVAL
    assert call(4, 0) == -2 and call(4, 16) == -2   # EUNSUPPORTED_N
    assert call(4, 7, u=None) == -1
    assert call(4, 7, w=None) == -1
    assert call(4, 7, u=A + 8) == -3            # EALIGN
    assert call(4, 7, G=A + (1 << 32) + 4) == -3
    assert call(4, 7, w=A + 256) == -4          # EALIAS: w overlaps u
    assert call(4, 7, D=A + (3 << 32) + 64) == -4   # w overlaps D


def test_prepared_f64tc_validation(lib):
    size = ctypes.c_size_t(0)
    assert lib.sem_ax_f64tc_prepare_size(10, 7, ctypes.byref(size)) == 0 and size.value == 10 * 24592
    assert lib.sem_ax_f64tc_prepare_size(10, 15, ctypes.byref(size)) == 0 and size.value == 10 * 196624
    assert lib.sem_ax_f64tc_prepare_size(10, 5, ctypes.byref(size)) == -2      # orders 7 and 15 only
    assert lib.sem_ax_f64tc_prepare_size(-1, 7, ctypes.byref(size)) == -1
    assert lib.sem_ax_f64tc_prepare_size(10, 7, None) == -1
    G, Gp = A, A + (1 << 32)
    assert lib.sem_ax_f64tc_prepare(0, 7, None, None, None) == 0
    assert lib.sem_ax_f64tc_prepare(4, 5, G, Gp, None) == -2
    assert lib.sem_ax_f64tc_prepare(4, 7, None, Gp, None) == -1
    assert lib.sem_ax_f64tc_prepare(4, 7, G, Gp + 8, None) == -3             # EALIGN
    assert lib.sem_ax_f64tc_prepare(4, 7, G, G + 4096, None) == -4           # EALIAS
    u, D, w = A + (2 << 32), A + (3 << 32), A + (4 << 32)
    f = lib.sem_ax_f64tc_prepared
    assert f(0, 7, None, None, None, None, None) == 0
    assert f(4, 5, u, Gp, D, w, None) == -2
    assert f(-1, 7, u, Gp, D, w, None) == -1
    assert f(4, 7, u, None, D, w, None) == -1
    assert f(4, 7, u, Gp + 8, D, w, None) == -3
    assert f(4, 7, u, Gp, D, Gp + 1024, None) == -4                         # w overlaps Gp
    assert f(4, 7, u, Gp, D, u + 1024, None) == -4                          # w overlaps u


def test_bf16_rejects_bad_terms(lib):
    assert lib.sem_ax_bf16x3(4, 15, A, A + (1 << 32), A + (2 << 32), A + (3 << 32), None, 4, None) == -1


def test_batched_validation_and_workspace_size(lib):
    import paper_1503_07659_gb300._lib as L
    g = (L.semax_group * 2)()
    g[0] = L.semax_group(7, 10, A, A + (1 << 32), A + (2 << 32), A + (3 << 32))
    g[1] = L.semax_group(3, 10, A + (4 << 32), A + (5 << 32), A + (6 << 32), A + (7 << 32))
    size = ctypes.c_size_t(0)
    assert lib.sem_ax_batched_workspace_size(g, 2, ctypes.byref(size)) == 0 and size.value >= 8
    assert lib.sem_ax_batched(g, 2, None, 0, None) == -8          # EWORKSPACE
    g[1].w = A + (3 << 32) + 64                                   # two outputs overlap
    assert lib.sem_ax_batched_workspace_size(g, 2, ctypes.byref(size)) == -4
    g[1].w = A + (7 << 32)
    g[1].N = 20
    assert lib.sem_ax_batched(g, 2, A + (9 << 32), 4096, None) == -2
    assert lib.sem_ax_batched_workspace_size(g, 40, ctypes.byref(size)) == -1   # too many groups
    plan = ctypes.c_void_p()
    assert lib.sem_ax_plan_create(ctypes.byref(plan), g, 2, 0, None, 0) == -2
    assert lib.sem_ax_plan_create(ctypes.byref(plan), g, 2, 0, None, 4) == -1       # unknown flag
    assert lib.sem_ax_plan_exec(None, None) == -7 and lib.sem_ax_plan_destroy(None) == -7


def test_reduce_validation(lib):
    size = ctypes.c_size_t(0)
    assert lib.semax_reduce_workspace_size(10 ** 9, ctypes.byref(size)) == 0 and size.value >= 24
    assert lib.semax_reduce_workspace_size(-1, ctypes.byref(size)) == -1
    assert lib.semax_reduce(100, A, 0, A + 4096, 2, A + 8192, A + 16384, 1 << 20, None) == -1  # bad prec
    assert lib.semax_reduce(100, A, 0, A + 4096, 0, A + 8192, None, 0, None) == -8


@pytest.mark.parametrize("fn", ["sem_ax_helmholtz", "sem_ax_helmholtz_f64tc"])
def test_helmholtz_validation(lib, fn):
    import ctypes as C
    f = getattr(lib, fn)
    u, G, B, D, w = A, A + (1 << 32), A + (4 << 32), A + (2 << 32), A + (3 << 32)
    assert f(0, 7, None, None, None, None, C.c_double(1.0), C.c_double(0.0), None, None) == 0
    assert f(4, 7, u, G, None, D, C.c_double(1.0), C.c_double(0.0), w, None) == -1       # B missing
    assert f(4, 7, u, G, B + 8, D, C.c_double(1.0), C.c_double(0.0), w, None) == -3      # B misaligned
    assert f(4, 7, u, G, w + 64, D, C.c_double(1.0), C.c_double(0.0), w, None) == -4     # w overlaps B
    assert f(4, 16, u, G, B, D, C.c_double(1.0), C.c_double(0.0), w, None) == -2


def test_bf16_geo_validation(lib):
    f = lib.sem_ax_bf16x3_geo
    u, X, xq, D, w = A, A + (1 << 32), A + (5 << 32), A + (2 << 32), A + (3 << 32)
    assert f(0, 15, None, None, None, None, None, 3, None) == 0
    assert f(4, 15, u, X, xq, D, w, 4, None) == -1
    assert f(4, 7, u, X, xq, D, w, 3, None) == -2
    assert f(4, 15, u, None, xq, D, w, 3, None) == -1
    assert f(4, 15, u + 4, X, xq, D, w, 3, None) == -3
    assert f(4, 15, u, X, xq, D, u + 64, 3, None) == -4


def test_binding_constants_match_the_header():
    """The flag and enum values the Python binding passes are the header's."""
    import paper_1503_07659_gb300._lib as L
    text = open(os.path.join(ROOT, "include", "semax.h")).read()
    vals = dict((k, int(v)) for k, v in re.findall(r"\b(SEMAX_[A-Z0-9_]+)\s*=\s*(-?\d+)", text))
    for name in ("SEMAX_F64", "SEMAX_F32", "SEMAX_PLAN_F64X", "SEMAX_PLAN_F64TC", "SEMAX_PLAN_F64TC_PREPARED", "SEMAX_PCG_F64X",
                 "SEMAX_PCG_F64TC", "SEMAX_PCG_MIXED"):
        assert getattr(L, name) == vals[name], name
    for code, name in L.STATUS_NAMES.items():
        assert vals[name] == code, name


def test_plan_rejects_unknown_flags(lib):
    h = ctypes.c_void_p()
    assert lib.sem_ax_plan_create(ctypes.byref(h), None, 0, 0, None, 8) == -1   # SEMAX_EINVAL
    assert lib.sem_ax_plan_create(ctypes.byref(h), None, 0, 0, None, 4) == -1   # F64TC_PREPARED needs F64TC


def test_status_variants_validation(lib):
    """The _status entry points check their arguments like the plain ones
    (the status pointer must be int-aligned; NULL reports nothing)."""
    u, G, D, w = A, A + (1 << 32), A + (2 << 32), A + (3 << 32)
    f = lib.sem_ax_f64tc_status
    assert f(0, 7, None, None, None, None, None, None) == 0
    assert f(-1, 7, u, G, D, w, None, None) == -1
    assert f(4, 16, u, G, D, w, None, None) == -2
    assert f(4, 7, u, G, D, w, A + (5 << 32) + 2, None) == -3     # misaligned status
    assert f(4, 7, u + 8, G, D, w, A + (5 << 32), None) == -3
    assert f(4, 7, u, G, D, u + 64, A + (5 << 32), None) == -4
    fp = lib.sem_ax_f64tc_prepared_status
    Gp = A + (6 << 32)
    assert fp(0, 7, None, None, None, None, None, None) == 0
    assert fp(4, 5, u, Gp, D, w, None, None) == -2
    assert fp(4, 7, u, Gp, D, w, A + (5 << 32) + 1, None) == -3
    assert fp(4, 7, u, Gp, D, Gp + 1024, None, None) == -4
    assert lib.sem_ax_plan_status(None, None) == -7
    assert lib.semax_set_wait_polls(-1) == 0


def test_fma_probe_validation(lib):
    fl = ctypes.c_double(0.0)
    assert lib.semax_fma_probe(2, 1, 4, A, ctypes.byref(fl), None) == -1      # bad precision
    assert lib.semax_fma_probe(0, 0, 4, A, ctypes.byref(fl), None) == -1
    assert lib.semax_fma_probe(0, 1, 4, None, ctypes.byref(fl), None) == -1
    assert lib.semax_fma_probe(0, 1, 3, A, ctypes.byref(fl), None) == -1       # iters not a multiple of 4
    assert lib.semax_fma_probe(0, 1, 4, A + 4, ctypes.byref(fl), None) == -3
