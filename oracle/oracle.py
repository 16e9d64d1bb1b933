"""Python handle on the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and
by the CPU-baseline leg of the benchmark, never by the product package.  The
arithmetic lives in ``lbm_oracle.c``; this module only marshals numpy arrays
through ctypes.  It shares nothing with the CUDA library.

Paper: Chen et al., "A generalized lattice Boltzmann model for flow through
tight porous media with Klinkenberg's effect", Sections II-III (Eq. 2-17),
Section IV.A (Eq. 18-20).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")

BC_PERIODIC = 0
BC_PRESSURE = 1  # x only
BC_WALLS = 1  # y only


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("tau", ctypes.c_double), ("J", ctypes.c_double),
        ("Gx", ctypes.c_double), ("Gy", ctypes.c_double),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("rho0", ctypes.c_double),
        ("rho_in", ctypes.c_double), ("rho_out", ctypes.c_double),
        ("forchheimer", ctypes.c_int32),
        ("kn_model", ctypes.c_int32), ("kn_beta", ctypes.c_double),
    ]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _load(path: str):
    L = ctypes.CDLL(path)
    P = ctypes.POINTER(Params)
    L.orc_fc.restype = ctypes.c_double
    L.orc_fc.argtypes = [ctypes.c_double]
    for name, nargs in (("orc_fc_first_order", 1), ("orc_kozeny_carman", 2),
                        ("orc_mean_free_path", 4), ("orc_pore_radius", 2)):
        fn = getattr(L, name)
        fn.restype = ctypes.c_double
        fn.argtypes = [ctypes.c_double] * nargs
    L.orc_apparent_permeability.restype = ctypes.c_double
    L.orc_apparent_permeability.argtypes = [ctypes.c_double, ctypes.c_double]
    L.orc_node_state.argtypes = [_D, ctypes.c_double, ctypes.c_double, P, _D, _D, _D]
    L.orc_feq.argtypes = [ctypes.c_double, _D, ctypes.c_double, _D]
    L.orc_forcing.argtypes = [ctypes.c_double, _D, _D, ctypes.c_double,
                              ctypes.c_double, _D]
    L.orc_collide_node.argtypes = [_D, ctypes.c_double, ctypes.c_double, P, _D]
    L.orc_neep_node.argtypes = [_D, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, P, _D]
    L.orc_create.restype = ctypes.c_void_p
    L.orc_create.argtypes = [P]
    L.orc_destroy.argtypes = [ctypes.c_void_p]
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_max_threads.restype = ctypes.c_int
    L.orc_set_fields.argtypes = [ctypes.c_void_p, _D, _D, _D]
    L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    L.orc_steps.restype = ctypes.c_int64
    L.orc_steps.argtypes = [ctypes.c_void_p]
    L.orc_get_populations.argtypes = [ctypes.c_void_p, _D]
    L.orc_set_populations.argtypes = [ctypes.c_void_p, _D]
    L.orc_macroscopic.argtypes = [ctypes.c_void_p, _D, _D, _D]
    L.orc_driving_force.restype = ctypes.c_double
    L.orc_driving_force.argtypes = [ctypes.c_void_p]
    L.orc_permeability.restype = ctypes.c_double
    L.orc_permeability.argtypes = [ctypes.c_void_p, _D]
    L.orc_mass.restype = ctypes.c_double
    L.orc_mass.argtypes = [ctypes.c_void_p]
    L.orc_residual.restype = ctypes.c_double
    L.orc_residual.argtypes = [ctypes.c_void_p, _D, _D]
    L.orc_lattice.argtypes = [_I, _I, _D]
    L.orc_velocity_histogram.argtypes = [ctypes.c_void_p, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int64), _D]
    L.orc_kg_fd.restype = ctypes.c_int
    L.orc_kg_fd.argtypes = [P, _D, _D, _D, ctypes.c_int64, ctypes.c_double,
                            ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, ctypes.c_int, _D]
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _load(_LIB)
    return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Temporarily route every call of this module through another build of
    the oracle (used by the tests that plant mistakes in a copy of it)."""
    global _lib
    saved = lib()
    _lib = _load(path)
    try:
        yield
    finally:
        _lib = saved


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _vec(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


KN_BKC, KN_FIRST_ORDER = 0, 1


def make_params(nx, ny, tau=0.8, J=1.0, G=(0.0, 0.0), bc_x=BC_PERIODIC,
                bc_y=BC_PERIODIC, rho0=1.0, rho_in=1.0, rho_out=1.0,
                forchheimer=0, kn_model=KN_BKC, kn_beta=0.0) -> Params:
    return Params(int(nx), int(ny), float(tau), float(J), float(G[0]), float(G[1]),
                  int(bc_x), int(bc_y), float(rho0), float(rho_in), float(rho_out),
                  int(forchheimer), int(kn_model), float(kn_beta))


# ---- closed forms -------------------------------------------------------
def fc(kn: float) -> float:
    """Eq. 6-7 correction factor f_c(Kn), b = -1."""
    return lib().orc_fc(float(kn))


def fc_first_order(kn: float) -> float:
    """Eq. 4-5: f_c = 1 + 4 Kn."""
    return float(lib().orc_fc_first_order(float(kn)))


def kozeny_carman(eps: float, d: float) -> float:
    """Eq. 9: k_d [m^2] of packed spheres of diameter d [m]."""
    return float(lib().orc_kozeny_carman(float(eps), float(d)))


def mean_free_path(mu: float, p: float, T: float, M: float) -> float:
    """Eq. 10: lambda [m] (mu Pa s, p Pa, T K, M kg/mol)."""
    return float(lib().orc_mean_free_path(float(mu), float(p), float(T), float(M)))


def pore_radius(k_d: float, eps: float) -> float:
    """Eq. 11: r [m] from k_d [m^2] (Herd et al.)."""
    return float(lib().orc_pore_radius(float(k_d), float(eps)))


def apparent_permeability(k_i: float, kn: float) -> float:
    """Eq. 3: k_a = k_i f_c(Kn)."""
    return lib().orc_apparent_permeability(float(k_i), float(kn))


def lattice():
    """(e_x, e_y, w) of Eq. 13 and Eq. 14 as stored in the oracle."""
    ex = (ctypes.c_int * 9)()
    ey = (ctypes.c_int * 9)()
    w = (ctypes.c_double * 9)()
    lib().orc_lattice(ex, ey, w)
    return np.array(ex[:]), np.array(ey[:]), np.array(w[:])


# ---- single-node primitives --------------------------------------------
def node_state(f, eps, ka, params: Params):
    """rho, u (Eq. 16a, 17 / quadratic), F (Eq. 2 / 8) of one node."""
    f = _vec(f)
    rho = ctypes.c_double()
    u = np.zeros(2)
    F = np.zeros(2)
    lib().orc_node_state(_dp(f), float(eps), float(ka), ctypes.byref(params),
                         ctypes.byref(rho), _dp(u), _dp(F))
    return rho.value, u, F


def feq(rho, u, eps):
    """Eq. 14 for one node."""
    out = np.zeros(9)
    lib().orc_feq(float(rho), _dp(_vec(u)), float(eps), _dp(out))
    return out


def forcing(rho, u, F, eps, tau):
    """Eq. 15 (last term over eps) for one node."""
    out = np.zeros(9)
    lib().orc_forcing(float(rho), _dp(_vec(u)), _dp(_vec(F)), float(eps), float(tau),
                      _dp(out))
    return out


def collide_node(f, eps, ka, params: Params):
    """Eq. 12 right-hand side for one node."""
    out = np.zeros(9)
    lib().orc_collide_node(_dp(_vec(f)), float(eps), float(ka), ctypes.byref(params),
                           _dp(out))
    return out


def neep_node(fn, eps_n, ka_n, eps_b, rho_b, params: Params):
    """Pressure-boundary populations from the interior neighbour."""
    out = np.zeros(9)
    lib().orc_neep_node(_dp(_vec(fn)), float(eps_n), float(ka_n), float(eps_b),
                        float(rho_b), ctypes.byref(params), _dp(out))
    return out


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def permeability_gradient_fd(params: Params, eps, k_i, kn, nsteps: int, nodes,
                             which: str = "logk", h: float = 1e-4) -> np.ndarray:
    """Central differences of k_g after ``nsteps`` steps from rest with
    respect to ln k_i (``which="logk"``) or eps (``which="eps"``) of each
    node in ``nodes`` (flat row-major indices into the [ny][nx] fields).
    The definition of the derivative applied to the oracle; FP64."""
    ny, nx = params.ny, params.nx
    e = np.ascontiguousarray(np.broadcast_to(_vec(eps), (ny, nx)))
    k = np.ascontiguousarray(np.broadcast_to(_vec(k_i), (ny, nx)))
    n = np.ascontiguousarray(np.broadcast_to(_vec(kn), (ny, nx)))
    idx = np.ascontiguousarray(np.asarray(nodes, dtype=np.int64).ravel())
    out = np.zeros(idx.size)
    w = {"logk": 0, "eps": 1}[which]
    rc = lib().orc_kg_fd(ctypes.byref(params), _dp(e), _dp(k), _dp(n), int(nsteps), float(h),
                         idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), idx.size, w,
                         _dp(out))
    if rc != 0:
        raise ValueError("oracle: finite-difference gradient failed (bad node index or memory)")
    return out


# ---- whole-domain simulation ---------------------------------------------
class OracleSim:
    """FP64 oracle run of the porous LB model on an nx x ny lattice.

    Fields are row-major [ny][nx] float64 arrays.  Populations are exchanged
    in plane-major layout [9][ny][nx] (post-stream, time level ``steps``).
    """

    def __init__(self, params: Params):
        self.params = params
        self._L = lib()
        self._h = self._L.orc_create(ctypes.byref(params))
        if not self._h:
            raise ValueError("oracle: invalid lattice size for the boundary kinds")
        self.nx, self.ny = params.nx, params.ny

    def close(self):
        if self._h:
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _field(self, a):
        a = _vec(a)
        if a.shape != (self.ny, self.nx):
            a = np.broadcast_to(a, (self.ny, self.nx)).copy()
        return a

    def set_fields(self, eps, k_i, kn):
        e, k, n = self._field(eps), self._field(k_i), self._field(kn)
        self._L.orc_set_fields(self._h, _dp(e), _dp(k), _dp(n))

    def step(self, n: int = 1):
        self._L.orc_step(self._h, int(n))

    @property
    def steps(self) -> int:
        return int(self._L.orc_steps(self._h))

    def populations(self) -> np.ndarray:
        out = np.zeros((9, self.ny, self.nx))
        self._L.orc_get_populations(self._h, _dp(out))
        return out

    def set_populations(self, f: np.ndarray):
        f = _vec(f)
        assert f.shape == (9, self.ny, self.nx)
        self._L.orc_set_populations(self._h, _dp(f))

    def macroscopic(self):
        rho = np.zeros((self.ny, self.nx))
        ux = np.zeros_like(rho)
        uy = np.zeros_like(rho)
        self._L.orc_macroscopic(self._h, _dp(rho), _dp(ux), _dp(uy))
        return rho, ux, uy

    def permeability(self):
        um = ctypes.c_double()
        kg = self._L.orc_permeability(self._h, ctypes.byref(um))
        return kg, um.value

    def velocity_histogram(self, nbins: int = 10):
        """Fig. 6: counts of u0 = |u| / max |u| in nbins equal ranges over the
        nodes of the fluid rows, and max |u|."""
        counts = np.zeros(nbins, dtype=np.int64)
        umax = ctypes.c_double()
        self._L.orc_velocity_histogram(self._h, int(nbins),
                                       counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       ctypes.byref(umax))
        return counts, umax.value

    def driving_force(self) -> float:
        """Body force plus the imposed pressure gradient (Darcy's law driver)."""
        return float(self._L.orc_driving_force(self._h))

    def mass(self) -> float:
        return float(self._L.orc_mass(self._h))

    def residual(self, ux_prev, uy_prev) -> float:
        return float(self._L.orc_residual(self._h, _dp(_vec(ux_prev)), _dp(_vec(uy_prev))))

    def run_to_steady(self, tol=1e-10, check_every=100, max_steps=2_000_000):
        """Step until ||u^n - u^{n-K}|| / ||u^n|| < tol (K = check_every)."""
        _, ux, uy = self.macroscopic()
        while self.steps < max_steps:
            self.step(check_every)
            r = self.residual(ux, uy)
            _, ux, uy = self.macroscopic()
            if r < tol:
                return r
        raise RuntimeError(f"oracle did not reach residual {tol} in {max_steps} steps")


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB)
