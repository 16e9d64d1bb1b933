"""Python binding of the C ABI in ``include/lbmp.h`` (argument marshalling only).

Every step of the lattice Boltzmann path runs in the CUDA kernels of
``liblbmp.so``; this module converts torch tensors or numpy arrays to
pointers and status codes to exceptions.  PyTorch supplies device memory and
the CUDA stream.  There is no CPU fallback: if the library is not built, or
no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbmp.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lbmp.h")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ENAN, ETIMEOUT = range(7)
BCX_PERIODIC, BCX_PRESSURE = 0, 1
BCY_PERIODIC, BCY_WALLS = 0, 1
STORE_FP32, STORE_FP16 = 0, 1
ROUND_STOCHASTIC, ROUND_NEAREST = 0, 1
KERNEL_AUTO, KERNEL_STAGED, KERNEL_DIRECT, KERNEL_WIDE = 0, 1, 2, 3
KN_BKC, KN_FIRST_ORDER = 0, 1
HOST, DEVICE = 0, 1

_STATUS = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ESTATE: "ESTATE",
           ENAN: "ENAN", ETIMEOUT: "ETIMEOUT"}


class LbmpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lbmp {_STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    """Mirror of ``lbmp_params``."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("tau", ctypes.c_double), ("J", ctypes.c_double),
        ("Gx", ctypes.c_double), ("Gy", ctypes.c_double),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("rho0", ctypes.c_double), ("rho_in", ctypes.c_double), ("rho_out", ctypes.c_double),
        ("forchheimer", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("fp16_log2_scale", ctypes.c_int32), ("fp16_rounding", ctypes.c_int32),
        ("kernel", ctypes.c_int32), ("kn_model", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p),
        ("kn_beta", ctypes.c_double),
    ]


class Info(ctypes.Structure):
    """Mirror of ``lbmp_info``."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("pitch", ctypes.c_int32),
        ("storage", ctypes.c_int32), ("fluid_nodes", ctypes.c_int64),
        ("steps", ctypes.c_int64), ("bytes_per_update", ctypes.c_double),
        ("fp16_scale", ctypes.c_double), ("eps_mean", ctypes.c_double),
        ("device_bytes", ctypes.c_int64), ("launches", ctypes.c_int64),
    ]


class BatchInfo(ctypes.Structure):
    """Mirror of ``lbmp_batch_info``."""
    _fields_ = [
        ("count", ctypes.c_int32), ("shape_threads", ctypes.c_int32),
        ("shape_nodes_per_thread", ctypes.c_int32), ("persistent", ctypes.c_int32),
        ("total_nodes", ctypes.c_int64), ("steps", ctypes.c_int64),
        ("launches", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
        ("bytes_per_update", ctypes.c_double),
    ]


_lib = None
_VP = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def header_functions() -> list[str]:
    """Names of the functions ``include/lbmp.h`` declares."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lbmp_\w+)\s*\(", text, re.M)))


def load(path: str = LIB_PATH):
    """Load ``liblbmp.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"liblbmp.so not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    st = ctypes.c_int32
    L.lbmp_last_error.restype = ctypes.c_char_p
    L.lbmp_last_error.argtypes = []
    L.lbmp_fc.restype = ctypes.c_double
    L.lbmp_fc.argtypes = [ctypes.c_double]
    L.lbmp_fc_model.restype = ctypes.c_double
    L.lbmp_fc_model.argtypes = [ctypes.c_int32, ctypes.c_double]
    for name, nargs in (("lbmp_kozeny_carman", 2), ("lbmp_mean_free_path", 4),
                        ("lbmp_pore_radius", 2)):
        fn = getattr(L, name)
        fn.restype = ctypes.c_double
        fn.argtypes = [ctypes.c_double] * nargs
    L.lbmp_physical_medium.restype = st
    L.lbmp_physical_medium.argtypes = [ctypes.c_int64, _VP, _VP, ctypes.c_double,
                                       ctypes.c_double, _VP, _VP]
    L.lbmp_create.restype = st
    L.lbmp_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(_VP)]
    L.lbmp_destroy.restype = st
    L.lbmp_destroy.argtypes = [_VP]
    L.lbmp_set_fields.restype = st
    L.lbmp_set_fields.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_int32]
    L.lbmp_step.restype = st
    L.lbmp_step.argtypes = [_VP, ctypes.c_int64]
    L.lbmp_synchronize.restype = st
    L.lbmp_synchronize.argtypes = [_VP]
    L.lbmp_macroscopic.restype = st
    L.lbmp_macroscopic.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_int32]
    L.lbmp_populations.restype = st
    L.lbmp_populations.argtypes = [_VP, _VP, ctypes.c_int32]
    L.lbmp_apparent_permeability.restype = st
    L.lbmp_apparent_permeability.argtypes = [_VP, _VP, ctypes.c_int32]
    L.lbmp_set_populations.restype = st
    L.lbmp_set_populations.argtypes = [_VP, _VP, ctypes.c_int32]
    L.lbmp_permeability.restype = st
    L.lbmp_permeability.argtypes = [_VP, _D, _D]
    L.lbmp_velocity_histogram.restype = st
    L.lbmp_velocity_histogram.argtypes = [_VP, ctypes.c_int32, _D, ctypes.POINTER(ctypes.c_int64)]
    L.lbmp_residual.restype = st
    L.lbmp_residual.argtypes = [_VP, _D]
    L.lbmp_mass.restype = st
    L.lbmp_mass.argtypes = [_VP, _D]
    L.lbmp_state_size.restype = st
    L.lbmp_state_size.argtypes = [_VP, ctypes.POINTER(ctypes.c_size_t)]
    L.lbmp_get_state.restype = st
    L.lbmp_get_state.argtypes = [_VP, _VP, ctypes.c_size_t, ctypes.c_int32]
    L.lbmp_set_state.restype = st
    L.lbmp_set_state.argtypes = [_VP, _VP, ctypes.c_size_t, ctypes.c_int32]
    L.lbmp_get_info.restype = st
    L.lbmp_get_info.argtypes = [_VP, ctypes.POINTER(Info)]
    L.lbmp_permeability_gradient.restype = st
    L.lbmp_permeability_gradient.argtypes = [_VP, ctypes.c_int64, ctypes.c_int64, _D, _VP, _VP,
                                             ctypes.c_int32]
    L.lbmp_permeability_noalloc.restype = st
    L.lbmp_permeability_noalloc.argtypes = [ctypes.POINTER(Params), _VP, _VP, _VP, _VP, _VP, _VP]
    I32P = ctypes.POINTER(ctypes.c_int32)
    L.lbmp_batch_create.restype = st
    L.lbmp_batch_create.argtypes = [ctypes.POINTER(Params), ctypes.c_int32, I32P, I32P,
                                    ctypes.POINTER(_VP)]
    L.lbmp_batch_destroy.restype = st
    L.lbmp_batch_destroy.argtypes = [_VP]
    L.lbmp_batch_set_fields.restype = st
    L.lbmp_batch_set_fields.argtypes = [_VP, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_int32]
    L.lbmp_batch_step.restype = st
    L.lbmp_batch_step.argtypes = [_VP, ctypes.c_int64]
    L.lbmp_batch_synchronize.restype = st
    L.lbmp_batch_synchronize.argtypes = [_VP]
    L.lbmp_batch_permeability.restype = st
    L.lbmp_batch_permeability.argtypes = [_VP, _D, _D]
    L.lbmp_batch_populations.restype = st
    L.lbmp_batch_populations.argtypes = [_VP, ctypes.c_int32, _VP, ctypes.c_int32]
    L.lbmp_batch_tune.restype = st
    L.lbmp_batch_tune.argtypes = [_VP, ctypes.c_int32, I32P, _D]
    L.lbmp_batch_tune_cached.restype = st
    L.lbmp_batch_tune_cached.argtypes = [_VP, ctypes.c_int32, I32P, _D, I32P]
    L.lbmp_batch_tune_cache_clear.restype = st
    L.lbmp_batch_tune_cache_clear.argtypes = []
    L.lbmp_batch_class.restype = st
    L.lbmp_batch_class.argtypes = [ctypes.POINTER(Params), ctypes.c_int32, I32P, I32P,
                                   ctypes.c_int32, ctypes.c_char_p, ctypes.c_int32]
    L.lbmp_batch_set_shape.restype = st
    L.lbmp_batch_set_shape.argtypes = [_VP, ctypes.c_int32]
    L.lbmp_batch_get_info.restype = st
    L.lbmp_batch_get_info.argtypes = [_VP, ctypes.POINTER(BatchInfo)]
    _lib = L
    return L


def _check(status: int):
    if status != OK:
        raise LbmpError(status, load().lbmp_last_error().decode())


def last_error() -> str:
    """``lbmp_last_error``: message of the last error raised on this thread."""
    return load().lbmp_last_error().decode()


def fc(kn: float) -> float:
    """Eq. 6-7 correction factor, evaluated by the library (host code)."""
    return float(load().lbmp_fc(float(kn)))


def fc_model(kn_model: int, kn: float) -> float:
    """f_c of Eq. 6-7 (KN_BKC) or Eq. 4-5 (KN_FIRST_ORDER), library host code."""
    return float(load().lbmp_fc_model(int(kn_model), float(kn)))


def kozeny_carman(eps: float, d: float) -> float:
    """Eq. 9: intrinsic permeability [m^2] of packed spheres of diameter d [m]."""
    return float(load().lbmp_kozeny_carman(float(eps), float(d)))


def mean_free_path(mu: float, p: float, T: float, M: float) -> float:
    """Eq. 10: mean free path [m] (mu [Pa s], p [Pa], T [K], M [kg/mol])."""
    return float(load().lbmp_mean_free_path(float(mu), float(p), float(T), float(M)))


def pore_radius(k_d: float, eps: float) -> float:
    """Eq. 11: characteristic pore radius [m] from k_d [m^2]."""
    return float(load().lbmp_pore_radius(float(k_d), float(eps)))


def physical_medium(eps, d, mean_free_path_m: float, dx: float):
    """``lbmp_physical_medium``: lattice k_i and Kn fields (for set_fields)
    of a medium given by porosity ``eps`` and grain diameter ``d`` [m] per
    node (``d`` may be a scalar), gas mean free path [m] and node spacing
    ``dx`` [m].  Returns (k_i, kn) as float64 arrays of eps's shape."""
    e = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
    dd = np.ascontiguousarray(np.broadcast_to(np.asarray(d, dtype=np.float64), e.shape))
    k_i = np.empty_like(e)
    kn = np.empty_like(e)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(load().lbmp_physical_medium(e.size, vp(e), vp(dd), float(mean_free_path_m),
                                       float(dx), vp(k_i), vp(kn)))
    return k_i, kn


def permeability_noalloc(cfg: "SimConfig", f, eps, k_i, kn, out, stream=None):
    """``lbmp_permeability_noalloc``: k_g, <u_x> and the non-finite count of
    a state held in caller device memory, written to ``out`` (3 float64 on
    the device), asynchronously on ``stream`` (a torch.cuda.Stream; default:
    the current stream).  All tensors: contiguous float64 CUDA tensors on the
    current device, f with 9 * ny * nx elements, the medium with ny * nx.
    The C entry point cannot see the sizes of the arrays it is given, so
    they are checked here, before anything is launched."""
    torch = _torch()
    named = (("f", f), ("eps", eps), ("k_i", k_i), ("kn", kn), ("out", out))
    for name, t in named:
        if not (isinstance(t, torch.Tensor) and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError(f"permeability_noalloc: {name} must be a contiguous float64 tensor")
    n = int(cfg.nx) * int(cfg.ny)
    need = {"f": 9 * n, "eps": n, "k_i": n, "kn": n}
    for name, t in named[:4]:
        if t.numel() != need[name]:
            raise ValueError(f"permeability_noalloc: {name} has {t.numel()} elements, "
                             f"a {cfg.nx} x {cfg.ny} lattice needs {need[name]}")
    if out.numel() < 3:
        raise ValueError("permeability_noalloc: out needs 3 elements")
    for name, t in named:
        if not t.is_cuda:
            raise TypeError(f"permeability_noalloc: {name} must be a CUDA tensor")
    dev = torch.cuda.current_device()
    for name, t in named:
        if t.device.index != dev:
            raise ValueError(f"permeability_noalloc: {name} is on cuda:{t.device.index}, "
                             f"the current device is cuda:{dev}")
    if stream is None:
        stream = torch.cuda.current_stream()
    params = cfg.to_params(None)
    _check(load().lbmp_permeability_noalloc(
        ctypes.byref(params), ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(eps.data_ptr()),
        ctypes.c_void_p(k_i.data_ptr()), ctypes.c_void_p(kn.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream)))


def _torch():
    import torch
    return torch


@dataclass
class SimConfig:
    nx: int
    ny: int
    tau: float = 0.8
    J: float = 1.0
    G: tuple = (0.0, 0.0)
    bc_x: int = BCX_PERIODIC
    bc_y: int = BCY_PERIODIC
    rho0: float = 1.0
    rho_in: float = 1.0
    rho_out: float = 1.0
    forchheimer: int = 0
    storage: int = STORE_FP32
    fp16_log2_scale: int = 0
    fp16_rounding: int = ROUND_STOCHASTIC
    kernel: int = KERNEL_AUTO
    seed: int = 0
    kn_model: int = KN_BKC
    kn_beta: float = 0.0

    def to_params(self, stream: int | None) -> Params:
        return Params(int(self.nx), int(self.ny), float(self.tau), float(self.J),
                      float(self.G[0]), float(self.G[1]), int(self.bc_x), int(self.bc_y),
                      float(self.rho0), float(self.rho_in), float(self.rho_out),
                      int(self.forchheimer), int(self.storage), int(self.fp16_log2_scale),
                      int(self.fp16_rounding), int(self.kernel), int(self.kn_model),
                      int(self.seed) & (2**64 - 1), stream, float(self.kn_beta))


def _context_device(stream) -> int:
    """The current CUDA device, which the library's context is created on;
    a caller's stream must belong to it."""
    torch = _torch()
    dev = torch.cuda.current_device()
    if stream is not None and stream.device.index != dev:
        raise ValueError(f"the stream is on cuda:{stream.device.index}, the current device "
                         f"(where the context is created) is cuda:{dev}")
    return dev


def _in_field(a, shape, device: int):
    """(pointer, where, keepalive) for a float64 input of ``shape``; a CUDA
    tensor must sit on ``device``, the context's: the library's kernels
    dereference the pointer there."""
    torch = _torch()
    if isinstance(a, torch.Tensor):
        t = a.detach()
        if t.is_cuda and t.device.index != device:
            raise ValueError(f"input on cuda:{t.device.index}, the lattice is on cuda:{device}")
        if t.dtype != torch.float64:
            t = t.to(torch.float64)
        t = t.contiguous()
        if tuple(t.shape) != tuple(shape):
            t = t.expand(*shape).contiguous()
        where = DEVICE if t.is_cuda else HOST
        return ctypes.c_void_p(t.data_ptr()), where, t
    arr = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shape))
    return arr.ctypes.data_as(ctypes.c_void_p), HOST, arr


def _out_field(shape, device: int | None):
    """A float64 output of ``shape``: on CUDA device ``device`` (the
    context's), or on the host for None."""
    torch = _torch()
    dev = torch.device("cuda", device) if device is not None else "cpu"
    t = torch.empty(shape, dtype=torch.float64, device=dev)
    return t, ctypes.c_void_p(t.data_ptr()), (DEVICE if device is not None else HOST)


class Sim:
    """One lattice (``lbmp_ctx``) on the current CUDA device.

    ``stream``: a ``torch.cuda.Stream`` the library queues its work on
    (default: a new stream owned by this object).
    """

    def __init__(self, cfg: SimConfig, stream=None):
        torch = _torch()
        L = load()
        if not torch.cuda.is_available():
            raise LbmpError(ECUDA, "no CUDA device available")
        self.cfg = cfg
        self.device = _context_device(stream)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._params = cfg.to_params(self.stream.cuda_stream)
        h = _VP()
        _check(L.lbmp_create(ctypes.byref(self._params), ctypes.byref(h)))
        self._h = h
        self.nx, self.ny = cfg.nx, cfg.ny

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            load().lbmp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- marshalling helpers
    def _in_field(self, a, shape):
        return _in_field(a, shape, self.device)

    def _out_field(self, shape, device: bool):
        return _out_field(shape, self.device if device else None)

    # -- C ABI calls
    def set_fields(self, eps, k_i, kn):
        shape = (self.ny, self.nx)
        pe, we, ke = self._in_field(eps, shape)
        pk, wk, kk = self._in_field(k_i, shape)
        pn, wn, kkn = self._in_field(kn, shape)
        if not (we == wk == wn):
            raise ValueError("eps, k_i and kn must all be on the host or all on the device")
        if we == DEVICE:
            _torch().cuda.current_stream(self.device).synchronize()
        _check(load().lbmp_set_fields(self._h, pe, pk, pn, we))

    def step(self, n: int = 1):
        _check(load().lbmp_step(self._h, int(n)))

    def synchronize(self):
        _check(load().lbmp_synchronize(self._h))

    def macroscopic(self, device: bool = True):
        shape = (self.ny, self.nx)
        rho, pr, w = self._out_field(shape, device)
        ux, pu, _ = self._out_field(shape, device)
        uy, pv, _ = self._out_field(shape, device)
        _check(load().lbmp_macroscopic(self._h, pr, pu, pv, w))
        return rho, ux, uy

    def apparent_permeability(self, device: bool = True):
        """``lbmp_apparent_permeability``: k_a of every node as the step uses
        it (Eq. 3), [ny, nx] float64; plate rows 0, open pores inf."""
        ka, pk, w = self._out_field((self.ny, self.nx), device)
        _check(load().lbmp_apparent_permeability(self._h, pk, w))
        return ka

    def populations(self, device: bool = True):
        f, pf, w = self._out_field((9, self.ny, self.nx), device)
        _check(load().lbmp_populations(self._h, pf, w))
        return f

    def set_populations(self, f):
        pf, w, keep = self._in_field(f, (9, self.ny, self.nx))
        if w == DEVICE:
            _torch().cuda.current_stream(self.device).synchronize()
        _check(load().lbmp_set_populations(self._h, pf, w))

    def permeability(self):
        kg, um = ctypes.c_double(), ctypes.c_double()
        _check(load().lbmp_permeability(self._h, ctypes.byref(kg), ctypes.byref(um)))
        return kg.value, um.value

    def velocity_histogram(self, nbins: int = 10):
        """``lbmp_velocity_histogram`` (Fig. 6): node counts of u0 = |u| /
        max |u| in nbins equal ranges, and max |u|."""
        counts = np.zeros(int(nbins), dtype=np.int64)
        um = ctypes.c_double()
        _check(load().lbmp_velocity_histogram(self._h, int(nbins), ctypes.byref(um),
                                              counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return counts, um.value

    def residual(self) -> float:
        r = ctypes.c_double()
        _check(load().lbmp_residual(self._h, ctypes.byref(r)))
        return r.value

    def mass(self) -> float:
        m = ctypes.c_double()
        _check(load().lbmp_mass(self._h, ctypes.byref(m)))
        return m.value

    def state_size(self) -> int:
        n = ctypes.c_size_t()
        _check(load().lbmp_state_size(self._h, ctypes.byref(n)))
        return n.value

    def get_state(self) -> np.ndarray:
        buf = np.empty(self.state_size(), dtype=np.uint8)
        _check(load().lbmp_get_state(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes, HOST))
        return buf

    def set_state(self, blob: np.ndarray):
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        _check(load().lbmp_set_state(self._h, blob.ctypes.data_as(ctypes.c_void_p), blob.nbytes, HOST))

    def info(self) -> Info:
        out = Info()
        _check(load().lbmp_get_info(self._h, ctypes.byref(out)))
        return out

    def permeability_gradient(self, nsteps: int, every: int = 0, device: bool = True):
        """``lbmp_permeability_gradient``: (k_g, dk_g/d ln k_i, dk_g/d eps)
        after ``nsteps`` steps from rest, by the discrete adjoint with
        checkpoints every ``every`` steps (0: sqrt(nsteps)).  The gradients
        are [ny, nx] float64 tensors.  Leaves the lattice at level nsteps."""
        shape = (self.ny, self.nx)
        gl, pl, w = self._out_field(shape, device)
        ge, pe, _ = self._out_field(shape, device)
        kg = ctypes.c_double()
        _check(load().lbmp_permeability_gradient(self._h, int(nsteps), int(every),
                                                 ctypes.byref(kg), pl, pe, w))
        return kg.value, gl, ge

    def run_to_steady(self, tol: float, check_every: int = 100, max_steps: int = 2_000_000):
        """Step until the relative velocity residual over ``check_every``
        steps is below ``tol`` (FP32 storage floors near 1e-7)."""
        self.residual()
        while self.info().steps < max_steps:
            self.step(check_every)
            r = self.residual()
            if r < tol:
                return r
        raise RuntimeError(f"residual did not reach {tol} in {max_steps} steps")


_KA_FN = None


def _ka_function():
    """The torch.autograd.Function behind :func:`ka_from_fields` (created on
    first use so that importing this module does not import torch)."""
    global _KA_FN
    if _KA_FN is not None:
        return _KA_FN
    torch = _torch()

    class KaFromFields(torch.autograd.Function):
        """k_g(ln k_i, eps) after a fixed number of steps from rest.  The
        forward pass runs the time loop and the adjoint in one library call
        (lbmp_permeability_gradient) when a gradient is needed, else the
        plain time loop; backward scales the stored gradient fields."""

        @staticmethod
        def forward(ctx, log_k, eps, sim, kn, nsteps, every):
            sim.set_fields(eps, torch.exp(log_k.detach()), kn)
            if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
                kg, gl, ge = sim.permeability_gradient(nsteps, every, device=True)
                ctx.save_for_backward(gl.to(log_k.device), ge.to(eps.device))
            else:
                sim.step(nsteps)
                kg, _ = sim.permeability()
            return torch.tensor(kg, dtype=torch.float64, device=log_k.device)

        @staticmethod
        def backward(ctx, grad):
            gl, ge = ctx.saved_tensors
            return grad * gl, grad * ge, None, None, None, None

    _KA_FN = KaFromFields
    return _KA_FN


def ka_from_fields(sim: "Sim", log_k, eps, kn, nsteps: int, every: int = 0):
    """Global permeability after ``nsteps`` steps from rest as a
    differentiable function of the [ny, nx] fields ``log_k`` (= ln k_i) and
    ``eps`` (float64 CUDA tensors); ``kn`` is held fixed.  Returns a 0-d
    float64 tensor; its backward pass gives dk_g/d ln k_i and dk_g/d eps
    from the discrete adjoint."""
    return _ka_function().apply(log_k, eps, sim, kn, nsteps, every)


def batch_class(cfg: SimConfig, sizes, nsm: int) -> str:
    """``lbmp_batch_class``: the key under which the batch autotuner caches
    the launch shape of a batch of ``sizes`` [(nx, ny), ...] with the physics
    of ``cfg`` on a device of ``nsm`` SMs (host only)."""
    sizes = [(int(nx), int(ny)) for nx, ny in sizes]
    nx = (ctypes.c_int32 * len(sizes))(*[s[0] for s in sizes])
    ny = (ctypes.c_int32 * len(sizes))(*[s[1] for s in sizes])
    buf = ctypes.create_string_buffer(128)
    prm = cfg.to_params(None)
    _check(load().lbmp_batch_class(ctypes.byref(prm), len(sizes), nx, ny, int(nsm), buf, 128))
    return buf.value.decode()


def batch_tune_cache_clear():
    """``lbmp_batch_tune_cache_clear``: forget this process's tuned shapes."""
    _check(load().lbmp_batch_tune_cache_clear())


class Batch:
    """Many lattices advanced together (``lbmp_batch``): ``sizes`` is a list
    of (nx, ny); the physics of ``cfg`` is shared (its nx, ny are ignored)."""

    def __init__(self, cfg: SimConfig, sizes, stream=None):
        torch = _torch()
        L = load()
        if not torch.cuda.is_available():
            raise LbmpError(ECUDA, "no CUDA device available")
        self.cfg = cfg
        self.sizes = [(int(nx), int(ny)) for nx, ny in sizes]
        self.count = len(self.sizes)
        self.device = _context_device(stream)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._params = cfg.to_params(self.stream.cuda_stream)
        nx = (ctypes.c_int32 * self.count)(*[s[0] for s in self.sizes])
        ny = (ctypes.c_int32 * self.count)(*[s[1] for s in self.sizes])
        h = _VP()
        _check(L.lbmp_batch_create(ctypes.byref(self._params), self.count, nx, ny, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().lbmp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_fields(self, i: int, eps, k_i, kn):
        nx, ny = self.sizes[i]
        pe, we, ke = _in_field(eps, (ny, nx), self.device)
        pk, wk, kk = _in_field(k_i, (ny, nx), self.device)
        pn, wn, kkn = _in_field(kn, (ny, nx), self.device)
        if not (we == wk == wn):
            raise ValueError("eps, k_i and kn must all be on the host or all on the device")
        if we == DEVICE:
            _torch().cuda.current_stream(self.device).synchronize()
        _check(load().lbmp_batch_set_fields(self._h, int(i), pe, pk, pn, we))

    def step(self, n: int = 1):
        _check(load().lbmp_batch_step(self._h, int(n)))

    def synchronize(self):
        _check(load().lbmp_batch_synchronize(self._h))

    def permeability(self):
        kg = np.zeros(self.count)
        um = np.zeros(self.count)
        _check(load().lbmp_batch_permeability(self._h, kg.ctypes.data_as(_D),
                                              um.ctypes.data_as(_D)))
        return kg, um

    def populations(self, i: int, device: bool = True):
        nx, ny = self.sizes[i]
        f, pf, w = _out_field((9, ny, nx), self.device if device else None)
        _check(load().lbmp_batch_populations(self._h, int(i), pf, w))
        return f

    def tune(self, steps: int = 10):
        chosen = ctypes.c_int32()
        ms = ctypes.c_double()
        _check(load().lbmp_batch_tune(self._h, int(steps), ctypes.byref(chosen), ctypes.byref(ms)))
        return chosen.value, ms.value

    def tune_cached(self, steps: int = 10):
        """``lbmp_batch_tune_cached``: (chosen shape, ms per step, from_cache)."""
        chosen = ctypes.c_int32()
        ms = ctypes.c_double()
        hit = ctypes.c_int32()
        _check(load().lbmp_batch_tune_cached(self._h, int(steps), ctypes.byref(chosen),
                                             ctypes.byref(ms), ctypes.byref(hit)))
        return chosen.value, ms.value, bool(hit.value)

    def set_shape(self, shape: int):
        """``lbmp_batch_set_shape``: use launch candidate ``shape``."""
        _check(load().lbmp_batch_set_shape(self._h, int(shape)))

    def info(self) -> BatchInfo:
        out = BatchInfo()
        _check(load().lbmp_batch_get_info(self._h, ctypes.byref(out)))
        return out
