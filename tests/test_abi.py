"""The C-ABI library builds, loads and exports every function declared in
include/asm.h; argument checks that need no device return INVALID_ARG."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_03915_gb300 import build
    path = build.build()
    import paper_2401_03915_gb300 as P
    return P, P.load(path)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "asm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(asm_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("asm_setup", "asm_apply", "asm_solve", "asm_get_info", "asm_destroy", "asm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    _, L = lib
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_option_defaults(lib):
    P, _ = lib
    o = P.default_options()
    assert o.spd == 1 and o.oversample == 8 and o.coarse == 1
    s = P.default_solve_opts()
    # restart 0: chosen at solve time (512 for the restricted or deflated apply, else 30)
    assert s.rtol == 1e-8 and s.restart == 0 and s.max_it == 1000
    assert o.one_level == 0 and o.coarse_mode == 0 and o.tau == 0.0


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    P, L = lib
    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([0, 1], dtype=np.int32)
    va = np.array([1.0, 1.0])
    part = np.zeros(2, dtype=np.int32)
    cases = [dict(N=0, overlap=1, nev=1), dict(N=3, overlap=1, nev=1), dict(N=1, overlap=0, nev=1),
             dict(N=1, overlap=1, nev=-1), dict(N=1, overlap=1, nev=1000)]
    for c in cases:
        with pytest.raises(P.AsmError) as e:
            P.asm_setup(rp, ci, va, part, c["N"], c["overlap"], c["nev"], on_device=False)
        assert e.value.name == "INVALID_ARG"
    with pytest.raises(P.AsmError) as e:
        P.asm_setup(rp, ci, va, part, 1, 1, 1, P.default_options(local_precision=7), on_device=False)
    assert e.value.name == "INVALID_ARG"
    # eq. uppergevp options: its eigenvalues are >= 1, it is for SPD A, nev_lift in 0..120
    for kw in (dict(nu=0.5), dict(nu=2.0, spd=0), dict(nu=2.0, nev_lift=-1), dict(nu=float("nan"))):
        with pytest.raises(P.AsmError) as e:
            P.asm_setup(rp, ci, va, part, 1, 1, 1, P.default_options(**kw), on_device=False)
        assert e.value.name == "INVALID_ARG", kw
    assert L.asm_apply(None, None, None, None) == 1
    assert b"null" in L.asm_last_error()


def test_tile_products_arguments_checked_on_the_host(lib):
    """asm_tile_products rejects a bad job list before any device work (the
    pointers below are never dereferenced)."""
    P, L = lib
    dummy = C.c_void_p(16)
    def call(**kw):
        jobs = np.zeros(1, dtype=P.TILE_JOB_DTYPE)
        jobs[0]["lda"] = jobs[0]["ldb"] = jobs[0]["ldc_out"] = jobs[0]["ldc_in"] = 64
        jobs[0]["nprod"] = 1
        for k, v in kw.items():
            jobs[0][k] = v
        cin = kw.pop("_cin", None)
        return L.asm_tile_products(jobs.ctypes.data, 1, dummy, dummy, cin, dummy, None)
    INVALID = 1
    assert call(nprod=0) == INVALID
    assert call(a0=2) == INVALID           # row starts must be 16-byte aligned
    assert call(lda=66) == INVALID
    assert call(flags=32) == INVALID       # unknown flag
    assert call(flags=4) == INVALID        # C_in asked for, none given
    assert call(lda=32) == INVALID         # row stride below the tile edge
    assert L.asm_tile_products(None, 1, dummy, dummy, None, dummy, None) == INVALID
    assert L.asm_tile_products(None, -1, dummy, dummy, None, dummy, None) == INVALID
    assert L.asm_tile_products(None, 0, None, None, None, None, None) == 0  # empty batch


def test_segmented_solve_arguments_checked_on_the_host(lib):
    """asm_solve_segments rejects null arguments and segment counts out of
    range before touching the handle's device data."""
    P, L = lib
    INVALID = 1
    infos = (P.asm_solve_info * 2)()
    off = np.array([0, 1, 2], dtype=np.int32)
    assert L.asm_solve_segments(None, C.c_void_p(16), C.c_void_p(16), 2, off.ctypes.data, None, infos, None) == INVALID
    assert L.asm_solve_segments(C.c_void_p(16), None, C.c_void_p(16), 2, off.ctypes.data, None, infos, None) == INVALID
    assert L.asm_solve_segments(C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), 0, off.ctypes.data, None, infos,
                                None) == INVALID
    assert L.asm_solve_segments(C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), 70000, off.ctypes.data, None, infos,
                                None) == INVALID
