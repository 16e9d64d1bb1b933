"""Checks that pin the FP64 oracle to facts fixed by the paper or by
mathematics, not by the oracle itself.

Each pin takes the ``oracle`` module (so the mutation tests can run the same
pins against a copy of the oracle with a planted mistake) and raises
``AssertionError`` when violated.  Sources:

* Eq. 13 (velocity set) and the weights printed under Eq. 14.
* Eq. 6-7 limits: f_c -> 1 + 4 Kn as Kn -> 0 (first-order Klinkenberg,
  Eq. 4-5), f_c / Kn -> 5 * 1.358 as Kn -> inf, the f_c values quoted with
  Fig. 1(b) (about 2 at 4000 psi, as high as 60 at 100 psi).
* Moment identities of the porous equilibrium (Eq. 14) and of Guo's forcing
  term (Eq. 15), and Eq. 16b itself for the velocity solve.
* Closed forms: the Brinkman-Darcy channel profile (Eq. 20), the cubic law
  H^2/12 for an empty channel (Section IV.A, Fig. 3), the uniform Darcy /
  Forchheimer velocity of a homogeneous periodic medium (Eq. 2 with F = 0).
* Invariants: mass conservation with periodic edges and walls.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from paper_1411_7051_gb300 import media

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name: str):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------- lattice
def pin_lattice_eq13(orc):
    ex, ey, w = orc.lattice()
    for i in range(9):
        if i == 0:
            e = (0.0, 0.0)
        elif i <= 4:
            th = (i - 1) * math.pi / 2
            e = (math.cos(th), math.sin(th))
        else:
            th = (i - 5) * math.pi / 2 + math.pi / 4
            e = (math.sqrt(2) * math.cos(th), math.sqrt(2) * math.sin(th))
        assert (ex[i], ey[i]) == (round(e[0]), round(e[1])), f"e_{i} differs from Eq. 13"
    printed = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4  # weights printed under Eq. 14
    assert np.allclose(w, printed, rtol=0, atol=1e-16)
    E = np.stack([ex, ey], 1).astype(float)
    # isotropy identities of D2Q9 (c_s^2 = 1/3)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(w @ E, 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, E, E), np.eye(2) / 3, atol=1e-16)
    d = np.eye(2)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, E, E, E, E), iso4, atol=1e-16)


# ---------------------------------------------------------- Eq. 6-7 (f_c)
def pin_fc(orc):
    assert orc.fc(0.0) == 1.0
    # first-order (Klinkenberg) limit, Eq. 4-5: f_c = 1 + 4 Kn + o(Kn)
    for kn in (1e-10, 1e-9, 1e-8):
        slope = (orc.fc(kn) - 1.0) / kn
        assert abs(slope - 4.0) < 0.01, f"(f_c-1)/Kn = {slope} at Kn={kn}"
    # free-molecular asymptote: alpha -> 1.358, bracket -> 5
    for kn in (1e9, 1e10):
        assert abs(orc.fc(kn) / kn - 5 * 1.358) < 1e-3 * 5 * 1.358
    # monotone increase over the four flow regimes of Section II.B
    kns = np.logspace(-6, 3, 200)
    vals = np.array([orc.fc(k) for k in kns])
    assert np.all(np.diff(vals) > 0)
    # Fig. 1(b) discussion: r = 1.12 nm at eps = 0.02, lambda per pressure
    g = golden("paper_values.json")["correction_factor_fig1b"]
    kn_hi = g["lambda_nm"]["100psi"] / g["r_nm"]
    kn_lo = g["lambda_nm"]["4000psi"] / g["r_nm"]
    assert 50.0 < orc.fc(kn_hi) < 70.0, orc.fc(kn_hi)  # "as high as 60"
    assert 1.5 < orc.fc(kn_lo) < 3.0, orc.fc(kn_lo)  # "about 2"
    # Eq. 3
    assert orc.apparent_permeability(2.5, 0.3) == 2.5 * orc.fc(0.3)


# ------------------------------------------------- single-node identities
def _random_nodes(orc, n=60, seed=11):
    rng = np.random.default_rng(seed)
    _, _, w = orc.lattice()
    for j in range(n):
        eps = [1.0, rng.uniform(0.05, 1.0), 0.3][j % 3]
        ka = [np.inf, 10 ** rng.uniform(-4, 1), 10 ** rng.uniform(-2, 0)][j % 3]
        f = w * (1.0 + 0.05 * rng.uniform(-1, 1, 9)) * rng.uniform(0.9, 1.1)
        params = orc.make_params(4, 4, tau=rng.uniform(0.52, 2.0),
                                 G=(rng.uniform(-1e-3, 1e-3), rng.uniform(-1e-3, 1e-3)),
                                 forchheimer=j % 2)
        yield f, eps, ka, params


def pin_node_identities(orc):
    ex, ey, _ = orc.lattice()
    E = np.stack([ex, ey], 1).astype(float)
    for f, eps, ka, params in _random_nodes(orc):
        rho, u, F = orc.node_state(f, eps, ka, params)
        m = f @ E
        assert abs(rho - f.sum()) < 1e-15
        # Eq. 16b: rho u = sum f e + (dt/2) rho F, with F of Eq. 2 / Eq. 8
        assert np.allclose(rho * u, m + 0.5 * rho * F, rtol=0, atol=1e-15), "Eq. 16b"
        # Eq. 2 / 8 evaluated at the returned u (Forchheimer term if enabled)
        nu = (params.tau - 0.5) / 3.0 / params.J
        G = np.array([params.Gx, params.Gy])
        drag = eps * nu / ka
        if params.forchheimer:
            Feps = 1.75 / math.sqrt(150 * eps ** 3)
            drag += eps * Feps / math.sqrt(ka) * np.linalg.norm(u)
        assert np.allclose(F, -drag * u + eps * G, rtol=1e-12, atol=1e-18), "Eq. 2"
        # Eq. 14 moments: rho, rho u, rho/3 I + rho u u / eps
        fe = orc.feq(rho, u, eps)
        assert abs(fe.sum() - rho) < 1e-14
        assert np.allclose(fe @ E, rho * u, rtol=0, atol=1e-16)
        P = np.einsum("i,ia,ib->ab", fe, E, E)
        assert np.allclose(P, rho / 3 * np.eye(2) + rho * np.outer(u, u) / eps,
                           rtol=0, atol=1e-15), "second moment of Eq. 14"
        # Eq. 15 moments: 0, (1 - 1/2tau) rho F, (1 - 1/2tau) rho (uF + Fu) / eps
        Fi = orc.forcing(rho, u, F, eps, params.tau)
        c = rho * (1 - 0.5 / params.tau)
        assert abs(Fi.sum()) < 1e-17, "sum of Eq. 15 must vanish"
        assert np.allclose(Fi @ E, c * F, rtol=1e-13, atol=1e-19)
        scale = abs(c) * np.abs(F).max()
        assert np.allclose(np.einsum("i,ia,ib->ab", Fi, E, E),
                           c * (np.outer(u, F) + np.outer(F, u)) / eps,
                           rtol=1e-10, atol=1e-14 * scale), "second moment of Eq. 15"
        # Eq. 12: mass kept, momentum gains rho F
        fp = orc.collide_node(f, eps, ka, params)
        assert abs(fp.sum() - f.sum()) < 1e-15
        assert np.allclose(fp @ E, m + rho * F, rtol=0, atol=1e-16)


def pin_impermeable_limit(orc):
    """eps -> 0 with Kozeny-Carman k ~ eps^3 (Eq. 9) approaches the eps = 0
    node (Section III: infinite drag, zero velocity)."""
    _, _, w = orc.lattice()
    rng = np.random.default_rng(5)
    f = w * (1 + 0.01 * rng.uniform(-1, 1, 9))
    params = orc.make_params(4, 4, tau=0.8, G=(1e-5, 0.0))
    ref = orc.collide_node(f, 0.0, 1.0, params)
    rho, u, F = orc.node_state(f, 0.0, 1.0, params)
    assert np.all(u == 0.0)
    prev = None
    for eps in (1e-3, 1e-5, 1e-7):
        k = 1e-2 * eps ** 3 / (1 - eps) ** 2
        d = np.abs(orc.collide_node(f, eps, k, params) - ref).max()
        if prev is not None:
            assert d < prev
        prev = d
    assert prev < 1e-9


# ------------------------------------------------------ flow closed forms
def brinkman_profile(G, K, nu, eps, H, y):
    """Eq. 20 with J = 1 (nu_e = nu)."""
    a = math.sqrt(nu * eps / (nu * K))
    return G * K / nu * (1 - np.cosh(a * (y - H / 2)) / np.cosh(a * H / 2))


def channel_run(orc, nx=64, ny=33, eps=0.7, darcy=1e-3, kn=0.1, tau=0.8, G=1e-6,
                tol=1e-10, check_every=100, max_steps=20_000):
    med = media.channel(nx, ny, eps, darcy, kn)
    p = orc.make_params(nx, ny, tau=tau, G=(G, 0.0), bc_y=orc.BC_WALLS)
    sim = orc.OracleSim(p)
    sim.set_fields(med.eps, med.k_i, med.kn)
    sim.run_to_steady(tol=tol, check_every=check_every, max_steps=max_steps)
    return sim


def pin_channel_eq20(orc):
    """Section IV.A: Brinkman-extended Darcy flow between plates, Eq. 18-20,
    at the validation configuration 64 x 33, eps 0.7, Da 1e-3, Kn 0.1."""
    nx, ny, eps, tau, G = 64, 33, 0.7, 0.8, 1e-6
    H = ny - 2
    sim = channel_run(orc, nx, ny, eps, 1e-3, 0.1, tau, G)
    _, ux, uy = sim.macroscopic()
    nu = (tau - 0.5) / 3
    K = 1e-3 * H * H * orc.fc(0.1)
    y = np.arange(1, ny - 1) - 0.5  # halfway walls at y = 0.5, ny - 1.5
    ua = brinkman_profile(G, K, nu, eps, H, y)
    prof = ux[1:-1, :].mean(axis=1)
    assert np.abs(ux[1:-1] - prof[:, None]).max() < 1e-20, "x-invariance"
    assert np.abs(uy).max() < 1e-9 * np.abs(ux).max(), "u_y = 0 (Section IV.A)"
    rel = np.linalg.norm(prof - ua) / np.linalg.norm(ua)
    assert rel < 1e-2, f"Eq. 20 rel-L2 {rel}"
    c = len(prof) // 2
    assert abs(prof[c] / ua[c] - 1) < 1e-5, "Darcy plateau at the channel centre"


def pin_cubic_law(orc):
    """Empty channel (eps = 1, k = inf): k_g -> H^2/12 (Section IV.A, Fig. 3,
    paper: 530.68 simulated vs 533.3 at H = 80, tau = 0.9)."""
    g = golden("paper_values.json")["cubic_law_channel"]
    H, tau = g["H"], g["tau"]
    sim = channel_run(orc, nx=2, ny=H + 2, eps=1.0, darcy=np.inf, kn=0.0, tau=tau,
                      G=1e-6, tol=1e-11, check_every=200, max_steps=300_000)
    kg, _ = sim.permeability()
    assert abs(kg / (H * H / 12) - 1) < 1e-2, kg
    assert abs(kg / g["k_simulated"] - 1) < 1e-2, kg
    # the profile is the Poiseuille parabola
    _, ux, _ = sim.macroscopic()
    y = np.arange(1, H + 1) - 0.5
    nu = (tau - 0.5) / 3
    ua = 1e-6 / (2 * nu) * y * (H - y)
    prof = ux[1:-1, 0]
    assert np.linalg.norm(prof - ua) / np.linalg.norm(ua) < 1e-2


def pin_uniform_darcy(orc):
    """Homogeneous fully periodic medium: the steady state is uniform with
    F = 0 in Eq. 2, i.e. (eps nu/k_a) u + (eps F_eps/sqrt(k_a)) |u| u = eps G."""
    nx = ny = 4
    eps, k_i, kn, tau, G = 0.4, 1e-3, 1.0, 0.8, 1e-5
    for forch in (0, 1):
        p = orc.make_params(nx, ny, tau=tau, G=(G, 0.0), forchheimer=forch)
        sim = orc.OracleSim(p)
        sim.set_fields(np.full((ny, nx), eps), np.full((ny, nx), k_i),
                       np.full((ny, nx), kn))
        sim.step(400)
        _, ux, uy = sim.macroscopic()
        ka = k_i * orc.fc(kn)
        nu = (tau - 0.5) / 3
        if forch:
            a = eps * 1.75 / math.sqrt(150 * eps ** 3) / math.sqrt(ka)
            b = eps * nu / ka
            u_exact = max(np.roots([a, b, -eps * G]).real)
        else:
            u_exact = G * ka / nu
        assert np.allclose(ux, u_exact, rtol=1e-9, atol=0), (ux[0, 0], u_exact)
        assert np.abs(uy).max() < 1e-9 * abs(u_exact)
        kg, _ = sim.permeability()
        if not forch:
            assert abs(kg / ka - 1) < 1e-9  # Darcy's law recovers k_a


def pin_darcy_limit_channel(orc):
    """K -> 0: the Brinkman boundary layer vanishes and the global
    permeability of the filled channel tends to k_a."""
    nx, ny, eps, tau = 8, 33, 0.5, 0.8
    errs = []
    for da in (1e-4, 1e-6):
        sim = channel_run(orc, nx, ny, eps, da, 1.0, tau, 1e-6)
        kg, _ = sim.permeability()
        ka = da * (ny - 2) ** 2 * orc.fc(1.0)
        errs.append(abs(kg / ka - 1))
    assert errs[1] < errs[0] and errs[1] < 1e-2, errs


def pin_mass_conservation(orc):
    """Sum of rho is invariant under Eq. 12 with periodic edges and halfway
    bounce-back walls (sum_i F_i = 0 and feq keeps rho)."""
    _, _, w = orc.lattice()
    for bc_y, forch in ((orc.BC_PERIODIC, 0), (orc.BC_WALLS, 1)):
        nx, ny = 13, 11
        med = media.random_medium(nx, ny, seed=21, eps_range=(0.1, 1.0),
                                  log10_k_range=(-2, 1), p_open=0.2, p_solid=0.1)
        p = orc.make_params(nx, ny, tau=0.7, G=(2e-4, -1e-4), bc_y=bc_y,
                            forchheimer=forch)
        sim = orc.OracleSim(p)
        sim.set_fields(med.eps, med.k_i, med.kn)
        f0 = media.random_populations(nx, ny, seed=4, base=w, amp=1e-2)
        if bc_y == orc.BC_WALLS:
            f0[:, 0, :] = 0.0
            f0[:, -1, :] = 0.0
        sim.set_populations(f0)
        m0 = sim.mass()
        sim.step(300)
        m1 = sim.mass()
        assert abs(m1 / m0 - 1) < 1e-13, (m0, m1)


def pin_pressure_drive(orc):
    """The pressure inlet/outlet and the body force G = dp / (L rho)
    (Section IV.A), with dp = c_s^2 d rho / eps from eps p = c_s^2 rho
    (Eq. 1b), give the same global permeability for an empty channel and for
    a homogeneous Darcy medium, to O(d rho / rho)."""
    nx, ny, tau = 40, 14, 0.8
    drho = 1e-3
    for eps, darcy, bc_y in ((1.0, np.inf, orc.BC_WALLS), (0.5, 2e-3, orc.BC_PERIODIC)):
        med = media.channel(nx, ny, eps, darcy, 0.5)
        pp = orc.make_params(nx, ny, tau=tau, bc_x=orc.BC_PRESSURE, bc_y=bc_y,
                             rho_in=1 + drho / 2, rho_out=1 - drho / 2)
        ps = orc.OracleSim(pp)
        ps.set_fields(med.eps, med.k_i, med.kn)
        ps.run_to_steady(tol=1e-9, check_every=200, max_steps=100_000)
        kg_p, _ = ps.permeability()
        G = ps.driving_force()
        assert abs(G / (drho / 3 / eps / (nx - 1)) - 1) < 1e-12
        pb = orc.make_params(nx, ny, tau=tau, G=(G, 0.0), bc_y=bc_y)
        bs = orc.OracleSim(pb)
        bs.set_fields(med.eps, med.k_i, med.kn)
        bs.run_to_steady(tol=1e-9, check_every=200, max_steps=100_000)
        kg_b, _ = bs.permeability()
        assert abs(kg_p / kg_b - 1) < 1e-2, (eps, kg_p, kg_b)
        if bc_y == orc.BC_PERIODIC:
            ka = med.k_i[0, 0] * orc.fc(0.5)
            assert abs(kg_p / ka - 1) < 1e-2, (kg_p, ka)


ALL_PINS = [
    pin_lattice_eq13,
    pin_fc,
    pin_node_identities,
    pin_impermeable_limit,
    pin_channel_eq20,
    pin_cubic_law,
    pin_uniform_darcy,
    pin_darcy_limit_channel,
    pin_mass_conservation,
    pin_pressure_drive,
]
