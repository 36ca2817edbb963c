"""lbcad_step_noalloc: one hybrid step whose scratch lives in a static device array.

It exists for callers that must not have the library allocate device memory, such as a
host framework that owns all device memory through its own pool. They pass their own
state buffers in the library's storage layout. This file checks it through the C ABI
against the context-based entry points (lbcad_create + lbcad_step) over two calls in a
row, with the tolerances of the parity tests: 1e-12 max abs in FP64, 1e-5 relative L2
in FP32. The boxes run from the smallest allowed edge to the largest grids that fit the
scratch, so every part of its layout is exercised; a last test checks that further calls
leave the device's free memory unchanged. The host-side size and parameter checks are
tested without a GPU in test_abi_cpu.py.
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


CASES = [
    (L.FP64, (24, 20, 16), 5.0),
    (L.FP32, (24, 20, 16), 5.0),
    (L.FP64, (4, 5, 6), 1.5),       # the smallest edges
    (L.FP32, (4, 5, 6), 1.5),
    (L.FP32, (64, 64, 64), 16.0),   # 262,144 sites of the 279,616 that fit in FP32
    (L.FP64, (48, 48, 60), 12.0),   # 138,240 of the 139,808 that fit in FP64
]


def _state(prec, shape, R, dev="cuda:0"):
    import torch
    nx, ny, nz = shape
    N = nx * ny * nz
    prm = L.default_params(shape, R=R, p0=8.0, precision=prec, zeta=0.01)
    ref = L.Simulation([shape], [prm], seed=11)
    init = ref.get_fields(0, L.FIELD_Q | L.FIELD_PSI)
    _, w = L.lattice()
    dt = torch.float64 if prec == L.FP64 else torch.float32
    if prec == L.FP64:
        g0 = torch.tensor(w, dtype=dt, device=dev)[:, None].expand(19, N).contiguous() * prm["rho0"]
    else:
        g0 = torch.zeros(19, N, dtype=dt, device=dev)  # shifted: f_i - w_i rho0 = 0 at rest
    A = dict(g=g0, q=torch.from_numpy(init["q"].reshape(5, N)).to(device=dev, dtype=dt),
             psi=torch.from_numpy(init["psi"].reshape(N)).to(device=dev, dtype=dt),
             u=torch.zeros(3, N, dtype=dt, device=dev))
    return prm, ref, A


def _caller(shape, prm):
    grid = B.lbcad_grid(*shape)
    p = B._fill_params(prm, None, 0, None)
    lib = B.library()

    def call(src, dst):
        ptrs = [ctypes.c_void_p(t.data_ptr()) for t in
                (src["g"], src["q"], src["psi"], src["u"], dst["g"], dst["q"], dst["psi"], dst["u"])]
        rc = lib.lbcad_step_noalloc(ctypes.byref(grid), ctypes.byref(p), *ptrs)
        assert rc == 0, lib.lbcad_last_error(None)
    return call


@pytest.mark.parametrize("prec,shape,R", CASES)
def test_noalloc_two_calls_match_context_path(prec, shape, R):
    import torch
    nx, ny, nz = shape
    prm, ref, A = _state(prec, shape, R)
    c, w = L.lattice()
    Bf = {k: torch.empty_like(v) for k, v in A.items()}
    call = _caller(shape, prm)
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


def test_noalloc_calls_leave_device_memory_unchanged():
    """The defining property: after a first call (which looks up the static arrays and may
    load the kernels), further calls take no device memory."""
    import torch
    shape = (24, 20, 16)
    prm, ref, A = _state(L.FP32, shape, 5.0)
    Bf = {k: torch.empty_like(v) for k, v in A.items()}
    call = _caller(shape, prm)
    call(A, Bf)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call(Bf, A)
        call(A, Bf)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    ref.close()


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    lib = B.library()
    grid = B.lbcad_grid(128, 128, 128)
    p = B._fill_params(L.default_params((128, 128, 128)), None, 0, None)
    dummy = [ctypes.c_void_p(256)] * 8  # never dereferenced: the size check comes first
    rc = lib.lbcad_step_noalloc(ctypes.byref(grid), ctypes.byref(p), *dummy)
    assert rc == B.LBCAD_E_INVALID_ARG
    assert b"static limit" in lib.lbcad_last_error(None)
