"""Shared test plumbing: build the CUDA and the oracle simulation of the same
case from one description.  Inputs come from ``paper_1411_7051_gb300.media``
only; nothing here computes the method."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from paper_1411_7051_gb300 import media


@dataclass
class Case:
    nx: int
    ny: int
    tau: float = 0.8
    G: tuple = (0.0, 0.0)
    pressure: bool = False
    walls: bool = False
    rho_in: float = 1.0
    rho_out: float = 1.0
    forchheimer: int = 0
    medium: media.Medium | None = None
    kn_model: int = 0        # f_c: 0 Eq. 6-7, 1 Eq. 4-5
    kn_beta: float = 0.0     # dynamic Kn (0: static)


def oracle_sim(orc, case: Case):
    p = orc.make_params(case.nx, case.ny, tau=case.tau, G=case.G,
                        bc_x=orc.BC_PRESSURE if case.pressure else orc.BC_PERIODIC,
                        bc_y=orc.BC_WALLS if case.walls else orc.BC_PERIODIC,
                        rho_in=case.rho_in, rho_out=case.rho_out,
                        forchheimer=case.forchheimer, kn_model=case.kn_model,
                        kn_beta=case.kn_beta)
    s = orc.OracleSim(p)
    m = case.medium
    s.set_fields(m.eps, m.k_i, m.kn)
    return s


def gpu_sim(case: Case, storage: int = 0, fp16_log2_scale: int = 0, fp16_rounding: int = 0,
            seed: int = 0, kernel: int = 0):
    from paper_1411_7051_gb300 import lbmp
    cfg = lbmp.SimConfig(case.nx, case.ny, tau=case.tau, G=case.G,
                         bc_x=lbmp.BCX_PRESSURE if case.pressure else lbmp.BCX_PERIODIC,
                         bc_y=lbmp.BCY_WALLS if case.walls else lbmp.BCY_PERIODIC,
                         rho_in=case.rho_in, rho_out=case.rho_out,
                         forchheimer=case.forchheimer, storage=storage,
                         fp16_log2_scale=fp16_log2_scale, fp16_rounding=fp16_rounding,
                         seed=seed, kernel=kernel, kn_model=case.kn_model,
                         kn_beta=case.kn_beta)
    s = lbmp.Sim(cfg)
    m = case.medium
    s.set_fields(m.eps, m.k_i, m.kn)
    return s


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def fluid_rows(case: Case) -> slice:
    return slice(1, case.ny - 1) if case.walls else slice(0, case.ny)
