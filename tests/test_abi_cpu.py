"""Host-side checks of the C ABI (no GPU): the library builds, loads, exports every
symbol include/lbcad.h declares, and rejects bad arguments before touching a device."""
import ctypes
import math
import os
import re

import pytest

from paper_2011_00287_gb300 import build as B
from paper_2011_00287_gb300 import lbcad as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbcad.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbcad_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_signatures():
    assert set(declared_symbols()) == set(L._SIGS), (declared_symbols(), sorted(L._SIGS))


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_lattice_table(lib):
    c, w = L.lattice()
    assert c.shape == (19, 3) and abs(w.sum() - 1.0) < 1e-15
    # isotropy: sum w c c = I/3, and the table holds each D3Q19 velocity once
    import numpy as np
    assert np.allclose((w[:, None, None] * c[:, :, None] * c[:, None, :]).sum(0), np.eye(3) / 3)
    assert len({tuple(v) for v in c}) == 19


def _create(lib, grid, **kw):
    p = L._fill_params(L.default_params(grid, **kw), None, 0, None)
    g = L.lbcad_grid(*grid)
    ctx = ctypes.c_void_p()
    code = lib.lbcad_create(ctypes.byref(g), ctypes.byref(p), 1, ctypes.byref(ctx))
    return code, lib.lbcad_last_error(None).decode()


@pytest.mark.parametrize("grid,kw,code", [
    ((3, 8, 8), {}, L.LBCAD_E_INVALID_ARG),
    ((8, 8, 8), dict(tau=0.5), L.LBCAD_E_INVALID_ARG),
    ((8, 8, 8), dict(rho0=-1.0), L.LBCAD_E_INVALID_ARG),
    ((8, 8, 8), dict(zeta=math.nan), L.LBCAD_E_INVALID_ARG),
    ((8, 8, 8), dict(precision=7), L.LBCAD_E_INVALID_ARG),
    ((8, 8, 8), dict(integrator=7), L.LBCAD_E_INVALID_ARG),
    ((8, 8, 8), dict(coupling=5), L.LBCAD_E_INVALID_ARG),
])
def test_create_rejects_bad_arguments_on_the_host(lib, grid, kw, code):
    got, msg = _create(lib, grid, **kw)
    assert got == code and msg


def test_batch_with_mixed_integrators_is_rejected_on_the_host(lib):
    grid = (8, 8, 8)
    ps = (L.lbcad_params * 2)()
    ps[0] = L._fill_params(L.default_params(grid), None, 0, None)
    ps[1] = L._fill_params(L.default_params(grid, integrator=L.HEUN), None, 0, None)
    gs = (L.lbcad_grid * 2)(L.lbcad_grid(*grid), L.lbcad_grid(*grid))
    ctx = ctypes.c_void_p()
    assert lib.lbcad_create_batch(2, gs, ps, 1, ctypes.byref(ctx)) == L.LBCAD_E_INVALID_ARG
    assert "integrator" in lib.lbcad_last_error(None).decode()


def test_null_arguments(lib):
    assert lib.lbcad_step(None, 1) == L.LBCAD_E_INVALID_ARG
    assert lib.lbcad_sync(None) == L.LBCAD_E_INVALID_ARG
    assert lib.lbcad_num_instances(None) == 0
    assert lib.lbcad_step_count(None) == -1
    lib.lbcad_destroy(None)
    assert lib.lbcad_lattice(None, None) == L.LBCAD_E_INVALID_ARG


def test_null_arguments_of_the_exchange_and_option_calls(lib):
    n = ctypes.c_size_t()
    assert lib.lbcad_state_bytes(None, 0, ctypes.byref(n)) == L.LBCAD_E_INVALID_ARG
    assert lib.lbcad_get_state(None, 0, None, 0, 0) == L.LBCAD_E_INVALID_ARG
    assert lib.lbcad_set_state(None, 0, None, 0, 0) == L.LBCAD_E_INVALID_ARG
    assert lib.lbcad_set_path(None, 0) == L.LBCAD_E_INVALID_ARG
    assert lib.lbcad_set_tiles(None, 0) == L.LBCAD_E_INVALID_ARG
    assert lib.lbcad_autotune(None, 1, None, None, 0) == L.LBCAD_E_INVALID_ARG
    assert lib.lbcad_set_observe(None, 1) == L.LBCAD_E_INVALID_ARG
    assert lib.lbcad_set_graph(None, 2) == L.LBCAD_E_INVALID_ARG


@pytest.mark.parametrize("code,q", [(L.D3Q19, 19), (L.D3Q15, 15)])
def test_velocity_sets_on_the_host(lib, code, q):
    """lbcad_velocity_set needs no GPU: the tables, their isotropy, and rejection of an
    unknown set."""
    import numpy as np
    c, w = L.lattice(code)
    assert c.shape == (q, 3) and abs(w.sum() - 1.0) < 1e-15
    cf = c.astype(float)
    assert np.allclose((w[:, None, None] * cf[:, :, None] * cf[:, None, :]).sum(0), np.eye(3) / 3)
    cc = (ctypes.c_int32 * 57)()
    ww = (ctypes.c_double * 19)()
    assert lib.lbcad_velocity_set(7, cc, ww) == L.LBCAD_E_INVALID_ARG


@pytest.mark.parametrize("kw", [dict(lattice=7), dict(lb_form=3), dict(stencil=2)])
def test_create_rejects_unknown_scheme_options_on_the_host(lib, kw):
    got, msg = _create(lib, (8, 8, 8), **kw)
    assert got == L.LBCAD_E_INVALID_ARG and msg


def _noalloc_rc(lib, grid, **kw):
    """lbcad_step_noalloc with NULL buffers: every host check except the buffer pointers runs
    first, so the message tells which check stopped the call; no device is touched."""
    p = L._fill_params(L.default_params(grid, **kw), None, 0, None)
    g = L.lbcad_grid(*grid)
    rc = lib.lbcad_step_noalloc(ctypes.byref(g), ctypes.byref(p), *([None] * 8))
    return rc, lib.lbcad_last_error(None).decode()


@pytest.mark.parametrize("prec,fits,too_big", [
    # 15 parts of round_up_256(n * element size) bytes in the 16 MiB static scratch:
    # n = 279,616 = 64 * 17 * 257 in FP32 and 139,808 = 32 * 17 * 257 in FP64 are the largest
    (L.FP32, (64, 17, 257), (4, 5, 13981)),
    (L.FP64, (32, 17, 257), (4, 4, 8739)),
])
def test_noalloc_size_limit_on_the_host(lib, prec, fits, too_big):
    rc, msg = _noalloc_rc(lib, fits, precision=prec)
    assert rc == L.LBCAD_E_INVALID_ARG and "pointer" in msg, msg  # past the size check
    rc, msg = _noalloc_rc(lib, too_big, precision=prec)
    assert rc == L.LBCAD_E_INVALID_ARG and "static limit" in msg, msg


@pytest.mark.parametrize("kw", [dict(zeta=math.nan), dict(K=math.inf), dict(tau=0.4), dict(precision=3)])
def test_noalloc_validates_parameters_like_create(lib, kw):
    rc, msg = _noalloc_rc(lib, (8, 8, 8), **kw)
    assert rc == L.LBCAD_E_INVALID_ARG and "params" in msg, msg
    rc2, msg2 = _create(lib, (8, 8, 8), **kw)
    assert rc2 == rc and msg2.endswith(msg), (msg, msg2)
