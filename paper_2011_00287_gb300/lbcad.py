"""Thin Python binding of the lbcad C ABI (include/lbcad.h): argument marshalling only.

Every computation runs in the CUDA kernels of liblbcad.so.  PyTorch provides device
memory (through the allocator callbacks) and streams.  There is no fallback: if the
shared library is missing, importing the binding's entry points raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from typing import Dict, List, Optional, Sequence, Union

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblbcad.so")

LBCAD_OK = 0
LBCAD_E_INVALID_ARG = -1
LBCAD_E_OOM = -2
LBCAD_E_CUDA = -3
LBCAD_E_TIMEOUT = -4
LBCAD_E_NAN = -5
LBCAD_E_UNSUPPORTED = -6
FP32, FP64 = 0, 1
EULER, HEUN = 0, 1
LAGGED, SYNC = 0, 1
D3Q19, D3Q15 = 0, 1
LB_BODY_FORCE, LB_STRESS_EQ = 0, 1
STENCIL_ISO, STENCIL_R2 = 0, 1
FIELD_G, FIELD_RHO, FIELD_U, FIELD_Q, FIELD_PSI = 1, 2, 4, 8, 16
PATH_FUSED, PATH_TWO_KERNEL, PATH_STAGED = 0, 1, 2
N_TILE_CONFIGS = 7  # candidates of lbcad_autotune / lbcad_set_tiles (FP32; FP64 has one)
FIELD_NCOMP = {FIELD_G: 19, FIELD_RHO: 1, FIELD_U: 3, FIELD_Q: 5, FIELD_PSI: 1}
FIELD_NAMES = {FIELD_G: "g", FIELD_RHO: "rho", FIELD_U: "u", FIELD_Q: "q", FIELD_PSI: "psi"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class LbcadError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("lbcad error %d: %s" % (code, msg))
        self.code = code


class lbcad_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class lbcad_params(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_double) for n in (
        "tau", "rho0", "A0", "chi0", "chis", "K", "q0", "gammaQ", "xi", "a", "b", "kphi", "M", "W",
        "zeta", "R")] + [("centre", ctypes.c_double * 3), ("S0", ctypes.c_double), ("noise", ctypes.c_double),
                         ("precision", ctypes.c_int32), ("integrator", ctypes.c_int32),
                         ("coupling", ctypes.c_int32), ("lattice", ctypes.c_int32), ("lb_form", ctypes.c_int32),
                         ("stencil", ctypes.c_int32),
                         ("device", ctypes.c_int32),
                         ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                         ("alloc_user", ctypes.c_void_p)])


class lbcad_obs(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("sum_psi", ctypes.c_double), ("mom", ctypes.c_double * 3),
                ("cm_cos", ctypes.c_double * 3), ("cm_sin", ctypes.c_double * 3), ("sum_phic", ctypes.c_double)]

    def as_array(self) -> np.ndarray:
        return np.array([self.mass, self.sum_psi, *self.mom, *self.cm_cos, *self.cm_sin, self.sum_phic])


# Every symbol include/lbcad.h declares, with its ctypes signature.
_P = ctypes.POINTER
_SIGS = {
    "lbcad_lattice": (ctypes.c_int, [_P(ctypes.c_int32), _P(ctypes.c_double)]),
    "lbcad_velocity_set": (ctypes.c_int, [ctypes.c_int32, _P(ctypes.c_int32), _P(ctypes.c_double)]),
    "lbcad_state_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _P(ctypes.c_size_t)]),
    "lbcad_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.c_int32]),
    "lbcad_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.c_int32]),
    "lbcad_create": (ctypes.c_int, [_P(lbcad_grid), _P(lbcad_params), ctypes.c_uint64, _P(ctypes.c_void_p)]),
    "lbcad_create_batch": (ctypes.c_int, [ctypes.c_int32, _P(lbcad_grid), _P(lbcad_params), ctypes.c_uint64,
                                          _P(ctypes.c_void_p)]),
    "lbcad_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "lbcad_set_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "lbcad_set_observe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "lbcad_set_path": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "lbcad_set_tiles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "lbcad_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _P(ctypes.c_int32), _P(ctypes.c_float),
                                      ctypes.c_int32]),
    "lbcad_get_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p,
                                        ctypes.c_size_t, ctypes.c_int32]),
    "lbcad_set_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p,
                                        ctypes.c_size_t, ctypes.c_int32]),
    "lbcad_observables": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _P(lbcad_obs)]),
    "lbcad_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, _P(ctypes.c_double),
                                     _P(ctypes.c_double), ctypes.c_void_p, _P(ctypes.c_double)]),
    "lbcad_adjoint_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t]),
    "lbcad_num_instances": (ctypes.c_int, [ctypes.c_void_p]),
    "lbcad_instance_grid": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _P(lbcad_grid)]),
    "lbcad_step_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "lbcad_stream": (ctypes.c_void_p, [ctypes.c_void_p]),
    "lbcad_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "lbcad_step_noalloc": (ctypes.c_int, [_P(lbcad_grid), _P(lbcad_params)] + [ctypes.c_void_p] * 8),
    "lbcad_destroy": (None, [ctypes.c_void_p]),
    "lbcad_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
}

_lib = None
_lock = threading.Lock()


def library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load liblbcad.so (built in-tree by paper_2011_00287_gb300.build).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError("liblbcad.so is not built (%s); run paper_2011_00287_gb300.build.build()" % p)
            L = ctypes.CDLL(p)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _check(code: int, ctx=None):
    if code != LBCAD_OK:
        msg = library().lbcad_last_error(ctx)
        raise LbcadError(code, msg.decode() if msg else "")


def lattice(velocity_set: int = D3Q19):
    """Velocities (q, 3) and weights (q,) of the population velocity set (D3Q19 or D3Q15)."""
    c = (ctypes.c_int32 * 57)()
    w = (ctypes.c_double * 19)()
    q = library().lbcad_velocity_set(int(velocity_set), c, w)
    _check(min(q, 0))
    return np.array(list(c)[:3 * q], dtype=np.int32).reshape(q, 3), np.array(list(w)[:q])


# ---------------------------------------------------------------- parameters

def default_params(shape=(32, 32, 32), R: float = 8.0, p0: float = 16.0, precision: int = FP32, **kw) -> Dict:
    """Droplet workload: A0=1, chi_in=3, K=0.04, Gamma_Q=0.3, xi=0.7, a=b=0.07, M=0.1,
    zeta=0.005, tau=1, rho0=1, q0 = 2 pi/p0, with chi0=2.5, chis=0.25, W=0.02, kphi=2a,
    S0=0.5, noise 1e-3 and the droplet at the box centre."""
    nx, ny, nz = shape
    d = dict(tau=1.0, rho0=1.0, A0=1.0, chi0=2.5, chis=0.25, K=0.04, q0=2.0 * math.pi / p0, gammaQ=0.3,
             xi=0.7, a=0.07, b=0.07, kphi=0.14, M=0.1, W=0.02, zeta=0.005, R=R,
             centre=(nx / 2.0, ny / 2.0, nz / 2.0), S0=0.5, noise=1e-3, precision=precision,
             integrator=EULER, coupling=LAGGED, lattice=D3Q19, lb_form=LB_BODY_FORCE, stencil=STENCIL_ISO)
    d.update(kw)
    return d


class _TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device
        self.live: Dict[int, object] = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda:%d" % self.device)
        except Exception:
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, user):
        self.live.pop(int(ptr) if ptr else 0, None)


def _fill_params(d: Dict, stream, device: int, allocator: Optional[_TorchAllocator]) -> lbcad_params:
    p = lbcad_params()
    for k, v in d.items():
        if k == "centre":
            for i in range(3):
                p.centre[i] = float(v[i])
        elif k in ("precision", "integrator", "coupling", "lattice", "lb_form", "stencil"):
            setattr(p, k, int(v))
        else:
            setattr(p, k, float(v))
    p.device = int(device)
    p.stream = stream
    if allocator is not None:
        p.alloc = allocator.alloc_cb
        p.free = allocator.free_cb
    return p


# ---------------------------------------------------------------- C-ABI mirrors

def lbcad_create(grid: Sequence[int], params: Dict, seed: int = 1, *, device: int = 0, stream=None,
                 torch_alloc: bool = True) -> "Simulation":
    return Simulation([grid], [params], seed, device=device, stream=stream, torch_alloc=torch_alloc)


def lbcad_create_batch(grids: Sequence[Sequence[int]], params: Sequence[Dict], seed: int = 1, *, device: int = 0,
                       stream=None, torch_alloc: bool = True) -> "Simulation":
    return Simulation(list(grids), list(params), seed, device=device, stream=stream, torch_alloc=torch_alloc)


def lbcad_step(sim: "Simulation", n: int = 1):
    sim.step(n)


def lbcad_get_fields(sim: "Simulation", inst: int = 0, mask: int = FIELD_G | FIELD_U | FIELD_Q | FIELD_PSI,
                     out=None, on_device: bool = False):
    return sim.get_fields(inst, mask, out=out, on_device=on_device)


def lbcad_set_fields(sim: "Simulation", inst: int, fields: Dict[str, np.ndarray]):
    sim.set_fields(inst, fields)


def lbcad_observables(sim: "Simulation", inst: int = 0) -> np.ndarray:
    return sim.observables(inst)


def lbcad_destroy(sim: "Simulation"):
    sim.close()


class Simulation:
    """One lbcad context: one or many droplet instances advanced by the same launches."""

    def __init__(self, grids: List[Sequence[int]], params: List[Dict], seed: int = 1, *, device: int = 0,
                 stream=None, torch_alloc: bool = True):
        L = library()
        n = len(grids)
        if len(params) != n:
            raise ValueError("one params dict per grid")
        self._alloc = _TorchAllocator(device) if torch_alloc else None
        s = None
        if stream is not None:
            s = stream if isinstance(stream, int) else int(stream.cuda_stream)
        G = (lbcad_grid * n)(*[lbcad_grid(int(g[0]), int(g[1]), int(g[2])) for g in grids])
        P = (lbcad_params * n)(*[_fill_params(p, s, device, self._alloc) for p in params])
        ctx = ctypes.c_void_p()
        code = L.lbcad_create_batch(n, G, P, int(seed), ctypes.byref(ctx))
        _check(code, None)
        self.ctx = ctx
        self.grids = [tuple(int(v) for v in g) for g in grids]
        self.params = params
        self.device = device
        self.precision = int(params[0].get("precision", FP32))
        self.q = 15 if int(params[0].get("lattice", D3Q19)) == D3Q15 else 19  # populations per site

    # -- lifecycle
    def close(self):
        if getattr(self, "ctx", None):
            library().lbcad_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- stepping
    def step(self, n: int = 1):
        _check(library().lbcad_step(self.ctx, int(n)), self.ctx)
        return self

    def set_path(self, path: int):
        _check(library().lbcad_set_path(self.ctx, int(path)), self.ctx)

    def autotune(self, reps: int = 5):
        """Time each fused tile shape without advancing the state; keep the fastest.
        Returns (chosen index, ms per launch of each candidate)."""
        chosen = ctypes.c_int32(-1)
        ms = (ctypes.c_float * 16)()
        _check(library().lbcad_autotune(self.ctx, int(reps), ctypes.byref(chosen), ms, 16), self.ctx)
        return chosen.value, [v for v in ms][:N_TILE_CONFIGS]

    def set_tiles(self, cfg: int):
        _check(library().lbcad_set_tiles(self.ctx, int(cfg)), self.ctx)

    def set_observe(self, on: bool):
        """Whether fused steps also form the FP64 mass, psi, momentum and centroid sums of
        the state they write (default on); off, observables() runs a separate pass."""
        _check(library().lbcad_set_observe(self.ctx, 1 if on else 0), self.ctx)

    def set_graph(self, steps_per_graph: int):
        _check(library().lbcad_set_graph(self.ctx, int(steps_per_graph)), self.ctx)

    def sync(self):
        _check(library().lbcad_sync(self.ctx), self.ctx)

    @property
    def stream_handle(self) -> int:
        return library().lbcad_stream(self.ctx) or 0

    def torch_stream(self):
        import torch
        return torch.cuda.ExternalStream(self.stream_handle, device="cuda:%d" % self.device)

    @property
    def step_count(self) -> int:
        return int(library().lbcad_step_count(self.ctx))

    @property
    def num_instances(self) -> int:
        return len(self.grids)

    def sites(self, inst: Optional[int] = None) -> int:
        if inst is None:
            return sum(g[0] * g[1] * g[2] for g in self.grids)
        g = self.grids[inst]
        return g[0] * g[1] * g[2]

    # -- fields
    def _inst(self, inst: int):
        if not 0 <= int(inst) < len(self.grids):
            raise LbcadError(LBCAD_E_INVALID_ARG, "instance %d out of range [0, %d)" % (inst, len(self.grids)))
        return self.grids[int(inst)]

    def _ncomp(self, b: int) -> int:
        return self.q if b == FIELD_G else FIELD_NCOMP[b]

    def get_fields(self, inst: int = 0, mask: int = FIELD_G | FIELD_U | FIELD_Q | FIELD_PSI, out=None,
                   on_device: bool = False) -> Dict[str, object]:
        nx, ny, nz = self._inst(inst)
        N = nx * ny * nz
        ncomp = sum(self._ncomp(b) for b in FIELD_NCOMP if mask & b)
        nbytes = 8 * N * ncomp
        if on_device:
            import torch
            buf = out if out is not None else torch.empty(ncomp * N, dtype=torch.float64,
                                                          device="cuda:%d" % self.device)
            _check(library().lbcad_get_fields(self.ctx, inst, mask, ctypes.c_void_p(buf.data_ptr()), nbytes, 1),
                   self.ctx)
        else:
            buf = out if out is not None else np.empty(ncomp * N, dtype=np.float64)
            ptr = buf.data_ptr() if hasattr(buf, "data_ptr") else buf.ctypes.data
            _check(library().lbcad_get_fields(self.ctx, inst, mask, ctypes.c_void_p(ptr), nbytes, 0), self.ctx)
        res, o = {}, 0
        for b in (FIELD_G, FIELD_RHO, FIELD_U, FIELD_Q, FIELD_PSI):
            if mask & b:
                c = self._ncomp(b)
                v = buf[o * N:(o + c) * N].reshape(c, nz, ny, nx)
                res[FIELD_NAMES[b]] = v[0] if b in (FIELD_RHO, FIELD_PSI) else v
                o += c
        return res

    def set_fields(self, inst: int, fields: Dict[str, np.ndarray]):
        nx, ny, nz = self._inst(inst)
        N = nx * ny * nz
        mask, parts = 0, []
        for b in (FIELD_G, FIELD_U, FIELD_Q, FIELD_PSI):
            name = FIELD_NAMES[b]
            if name in fields:
                mask |= b
                parts.append(np.asarray(fields[name], dtype=np.float64).reshape(-1))
        if not mask:
            raise ValueError("no settable field given")
        buf = np.ascontiguousarray(np.concatenate(parts))
        if buf.size != N * sum(self._ncomp(b) for b in FIELD_NCOMP if mask & b):
            raise ValueError("field sizes do not match the grid")
        _check(library().lbcad_set_fields(self.ctx, inst, mask, ctypes.c_void_p(buf.ctypes.data), buf.nbytes, 0),
               self.ctx)

    def adjoint(self, nsteps: int, ckpt_every: int = 50, want_dQ0: bool = True):
        """Run nsteps forward (the state advances) and return (J, dJ/dzeta, dJ/dq0,
        dJ/dQ0 as (5, nz, ny, nx) or None) for J = |centroid displacement|^2 / 2."""
        nx, ny, nz = self._inst(0)
        dz, dq, J = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        dQ0 = np.empty((5, nz, ny, nx)) if want_dQ0 else None
        ptr = ctypes.c_void_p(dQ0.ctypes.data) if want_dQ0 else None
        _check(library().lbcad_adjoint(self.ctx, int(nsteps), int(ckpt_every), ctypes.byref(dz), ctypes.byref(dq),
                                       ptr, ctypes.byref(J)), self.ctx)
        return J.value, dz.value, dq.value, dQ0

    def adjoint_fields(self, mask: int = FIELD_G | FIELD_U | FIELD_Q | FIELD_PSI) -> Dict[str, np.ndarray]:
        """dJ/d(initial state) of the last adjoint run, in the get_fields layout."""
        nx, ny, nz = self._inst(0)
        N = nx * ny * nz
        ncomp = sum(c for b, c in FIELD_NCOMP.items() if mask & b)
        buf = np.empty(ncomp * N)
        _check(library().lbcad_adjoint_fields(self.ctx, mask, ctypes.c_void_p(buf.ctypes.data), buf.nbytes), self.ctx)
        res, o = {}, 0
        for b in (FIELD_G, FIELD_U, FIELD_Q, FIELD_PSI):
            if mask & b:
                c = FIELD_NCOMP[b]
                v = buf[o * N:(o + c) * N].reshape(c, nz, ny, nx)
                res[FIELD_NAMES[b]] = v[0] if b == FIELD_PSI else v
                o += c
        return res

    def state_bytes(self, inst: int = 0) -> int:
        n = ctypes.c_size_t()
        _check(library().lbcad_state_bytes(self.ctx, inst, ctypes.byref(n)), self.ctx)
        return n.value

    def get_state(self, inst: int = 0, out=None):
        """Raw state in the storage precision (exact checkpoint): a uint8 numpy array, or
        `out` (a host or CUDA tensor/array of at least state_bytes bytes) filled in place."""
        n = self.state_bytes(inst)
        buf = out if out is not None else np.empty(n, dtype=np.uint8)
        on_dev = hasattr(buf, "is_cuda") and buf.is_cuda
        ptr = buf.data_ptr() if hasattr(buf, "data_ptr") else buf.ctypes.data
        _check(library().lbcad_get_state(self.ctx, inst, ctypes.c_void_p(ptr), n, 1 if on_dev else 0), self.ctx)
        return buf

    def set_state(self, inst: int, buf):
        """Restore a state returned by get_state (bit for bit)."""
        n = self.state_bytes(inst)
        on_dev = hasattr(buf, "is_cuda") and buf.is_cuda
        ptr = buf.data_ptr() if hasattr(buf, "data_ptr") else buf.ctypes.data
        size = buf.nbytes if hasattr(buf, "nbytes") else buf.numel() * buf.element_size()
        if size < n:
            raise ValueError("state buffer too small")
        _check(library().lbcad_set_state(self.ctx, inst, ctypes.c_void_p(ptr), n, 1 if on_dev else 0), self.ctx)

    def observables(self, inst: int = 0) -> np.ndarray:
        o = lbcad_obs()
        _check(library().lbcad_observables(self.ctx, inst, ctypes.byref(o)), self.ctx)
        return o.as_array()

    def centroid(self, inst: int = 0) -> np.ndarray:
        """Per-axis circular mean of phi_c = (1 + psi)/2 (periodic centroid)."""
        o = self.observables(inst)
        L = np.array(self.grids[inst], dtype=float)
        ang = np.arctan2(o[8:11], o[5:8])
        return np.mod(ang, 2 * np.pi) * L / (2 * np.pi)
