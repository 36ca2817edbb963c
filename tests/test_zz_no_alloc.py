"""lbcad_step_noalloc: one hybrid step whose scratch lives in a static device array.

It exists for callers that must not have the library allocate device memory, such as a
host framework that owns all device memory through its own pool. They pass their own
state buffers in the library's storage layout. This file checks it through the C ABI
against the context-based entry points (lbcad_create + lbcad_step) over two calls in a
row, with the tolerances of the parity tests: 1e-12 max abs in FP64, 1e-5 relative L2
in FP32.
"""
import ctypes

import numpy as np
import pytest

import paper_2011_00287_gb300 as L
from paper_2011_00287_gb300 import lbcad as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2011_00287_gb300 import build
    build.build()


def _post_to_pre(g, shape, c):
    """Stored post-collision populations of the previous step -> pre-collision f_i(x) =
    g_i(x - c_i)."""
    nx, ny, nz = shape
    g = g.reshape(19, nz, ny, nx)
    return np.stack([np.roll(g[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2)) for i in range(19)])


@pytest.mark.parametrize("prec", [L.FP64, L.FP32])
def test_noalloc_two_calls_match_context_path(prec):
    import torch
    shape = (24, 20, 16)
    nx, ny, nz = shape
    N = nx * ny * nz
    prm = L.default_params(shape, R=5.0, p0=8.0, precision=prec, zeta=0.01)
    ref = L.Simulation([shape], [prm], seed=11)
    init = ref.get_fields(0, L.FIELD_Q | L.FIELD_PSI)
    c, w = L.lattice()
    dt = torch.float64 if prec == L.FP64 else torch.float32
    dev = "cuda:0"
    if prec == L.FP64:
        g0 = torch.tensor(w, dtype=dt, device=dev)[:, None].expand(19, N).contiguous() * prm["rho0"]
    else:
        g0 = torch.zeros(19, N, dtype=dt, device=dev)  # shifted: f_i - w_i rho0 = 0 at rest
    A = dict(g=g0, q=torch.from_numpy(init["q"].reshape(5, N)).to(device=dev, dtype=dt),
             psi=torch.from_numpy(init["psi"].reshape(N)).to(device=dev, dtype=dt),
             u=torch.zeros(3, N, dtype=dt, device=dev))
    Bf = {k: torch.empty_like(v) for k, v in A.items()}
    grid = B.lbcad_grid(nx, ny, nz)
    p = B._fill_params(prm, None, 0, None)
    lib = B.library()

    def call(src, dst):
        ptrs = [ctypes.c_void_p(t.data_ptr()) for t in
                (src["g"], src["q"], src["psi"], src["u"], dst["g"], dst["q"], dst["psi"], dst["u"])]
        rc = lib.lbcad_step_noalloc(ctypes.byref(grid), ctypes.byref(p), *ptrs)
        assert rc == 0, lib.lbcad_last_error(None)

    call(A, Bf)
    call(Bf, A)
    torch.cuda.synchronize()
    ref.step(2)
    exp = ref.get_fields(0)
    got = {k: v.double().cpu().numpy() for k, v in A.items()}
    f = _post_to_pre(got["g"], shape, c)
    if prec == L.FP32:
        f = f + w.reshape(19, 1, 1, 1) * prm["rho0"]
    pairs = [("g", f, exp["g"]), ("q", got["q"].reshape(5, nz, ny, nx), exp["q"]),
             ("psi", got["psi"].reshape(nz, ny, nx), exp["psi"]), ("u", got["u"].reshape(3, nz, ny, nx), exp["u"])]
    for name, a, b in pairs:
        if prec == L.FP64:
            assert np.abs(a - b).max() <= 1e-12, name
        else:
            sh = w.reshape(19, 1, 1, 1) if name == "g" else 0.0
            assert np.linalg.norm(a - b) / max(np.linalg.norm(b - sh), 1e-300) <= 1e-5, name
    ref.close()


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    lib = B.library()
    grid = B.lbcad_grid(128, 128, 128)
    p = B._fill_params(L.default_params((128, 128, 128)), None, 0, None)
    dummy = [ctypes.c_void_p(256)] * 8  # never dereferenced: the size check comes first
    rc = lib.lbcad_step_noalloc(ctypes.byref(grid), ctypes.byref(p), *dummy)
    assert rc == B.LBCAD_E_INVALID_ARG
    assert b"static limit" in lib.lbcad_last_error(None)
