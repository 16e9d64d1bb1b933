"""Pins of the oracle's FP64 reductions other than k_g: the relative velocity
residual that decides the steady state (||u^n - u^{n-K}||_2 / ||u^n||_2 over
the fluid nodes, the stopping rule of the validation channel run) and the
total mass (sum of rho over the fluid nodes).  No GPU.

Pinned against facts that do not come from the oracle's own code:
  * a state whose velocity is known by construction: open pores (eps = 1,
    k = inf), no body force and no Forchheimer term make Eq. 17 u = m / rho,
    and populations f_i = w_i rho (1 + 3 e_i.v) carry exactly that rho and
    m = rho v (the D2Q9 moments of Eq. 13-14).  Residual and mass are then
    plain norms and sums of known arrays (numpy), with garbage in the plate
    rows that the definitions exclude;
  * scale and single-node properties of the residual: R(u_prev = (1 - c) u)
    = |c|, R(u_prev = u) = 0, and a change of one node's y velocity by d
    gives R = |d| / ||u||;
  * a uniform periodic Darcy transient, where every node follows the scalar
    momentum recurrence m <- m + rho F (Eq. 2, 16b, 17), so that the
    residual between two time levels is |u^n - u^k| / |u^n| of that
    recurrence.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from test_oracle_gradient import uniform_velocity

NX, NY = 23, 17


def _known_state(seed=3):
    """Oracle on an open-pore NX x NY lattice with plates, its populations
    set to f_i = w_i rho (1 + 3 e_i.v); returns (sim, rho, vx, vy)."""
    rng = np.random.default_rng(seed)
    ex, ey, w = orc.lattice()
    p = orc.make_params(NX, NY, tau=0.8, bc_y=orc.BC_WALLS)
    sim = orc.OracleSim(p)
    sim.set_fields(1.0, np.inf, 0.0)
    rho = 1.0 + 0.02 * rng.uniform(-1, 1, (NY, NX))
    vx = 1e-3 * rng.standard_normal((NY, NX))
    vy = 1e-3 * rng.standard_normal((NY, NX))
    f = (w[:, None, None] * rho[None]
         * (1.0 + 3.0 * (ex[:, None, None] * vx[None] + ey[:, None, None] * vy[None])))
    # plate rows hold no fluid: garbage there must not enter either reduction
    f[:, 0, :] = rng.uniform(0.0, 5.0, (9, NX))
    f[:, -1, :] = rng.uniform(0.0, 5.0, (9, NX))
    sim.set_populations(f)
    return sim, rho, vx, vy


def test_known_state_velocity_is_the_constructed_one():
    sim, rho, vx, vy = _known_state()
    r, ux, uy = sim.macroscopic()
    fl = slice(1, NY - 1)
    np.testing.assert_allclose(r[fl], rho[fl], rtol=1e-15, atol=0)
    np.testing.assert_allclose(ux[fl], vx[fl], rtol=1e-10, atol=1e-15)
    np.testing.assert_allclose(uy[fl], vy[fl], rtol=1e-10, atol=1e-15)


def test_residual_is_the_relative_l2_norm_over_fluid_nodes():
    sim, _, vx, vy = _known_state()
    rng = np.random.default_rng(8)
    px = vx + 1e-3 * rng.standard_normal(vx.shape)
    py = vy + 1e-3 * rng.standard_normal(vy.shape)
    px[0], px[-1], py[0], py[-1] = 7.0, -3.0, 5.0, 11.0   # plate rows: ignored
    fl = slice(1, NY - 1)
    num = np.linalg.norm(np.stack([vx[fl] - px[fl], vy[fl] - py[fl]]))
    den = np.linalg.norm(np.stack([vx[fl], vy[fl]]))
    assert sim.residual(px, py) == pytest.approx(num / den, rel=1e-10, abs=0)


@pytest.mark.parametrize("c", [1.0, 0.5, 1e-3, -0.25])
def test_residual_scales_with_the_snapshot(c):
    sim, _, vx, vy = _known_state()
    assert sim.residual((1.0 - c) * vx, (1.0 - c) * vy) == pytest.approx(abs(c), rel=1e-9, abs=0)


def test_residual_single_node_y_change():
    sim, _, vx, vy = _known_state()
    _, ux, uy = sim.macroscopic()
    assert sim.residual(ux, uy) == 0.0
    fl = slice(1, NY - 1)
    d = 3e-4
    py = uy.copy()
    py[NY // 2, 5] += d
    norm = np.linalg.norm(np.stack([vx[fl], vy[fl]]))
    assert sim.residual(ux, py) == pytest.approx(d / norm, rel=1e-9, abs=0)


@pytest.mark.parametrize("forch", [0, 1])
def test_residual_uniform_darcy_transient(forch):
    nx, ny, k, n = 5, 4, 30, 40
    eps0, k0, G = 0.6, 2.0, (2e-4, 7e-5)
    p = orc.make_params(nx, ny, tau=0.8, G=G, forchheimer=forch)
    sim = orc.OracleSim(p)
    sim.set_fields(eps0, k0, 0.0)
    sim.step(k)
    _, ux, uy = sim.macroscopic()
    sim.step(n - k)
    uk = uniform_velocity(np.log(k0), eps0, k, G, forch).real
    un = uniform_velocity(np.log(k0), eps0, n, G, forch).real
    expect = np.linalg.norm(un - uk) / np.linalg.norm(un)
    assert 1e-3 < expect < 1.0   # still transient
    assert sim.residual(ux, uy) == pytest.approx(expect, rel=1e-9, abs=0)


def test_mass_is_the_sum_of_rho_over_fluid_nodes():
    sim, rho, _, _ = _known_state()
    assert sim.mass() == pytest.approx(rho[1:-1].sum(), rel=1e-14, abs=0)


# the pins above, for the planted-mistake tests of the oracle
RESIDUAL_PINS = [test_residual_is_the_relative_l2_norm_over_fluid_nodes,
                 lambda: test_residual_scales_with_the_snapshot(0.5),
                 test_residual_single_node_y_change,
                 lambda: test_residual_uniform_darcy_transient(1)]
MASS_PINS = [test_mass_is_the_sum_of_rho_over_fluid_nodes]
