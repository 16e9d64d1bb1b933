"""Pins of the oracle's finite-difference gradient of k_g (the reference the
GPU adjoint is checked against).

k_g after N steps from rest is differentiated by central differences of the
FP64 oracle.  Pinned here against:
  * a uniform medium in a fully periodic domain, where the flow stays uniform
    and one step of the lattice reduces to the momentum update
    m <- m + rho F (Eq. 16b, with u from Eq. 17 or its quadratic form with
    the drag of Eq. 2): the sum of the per-node derivatives equals the
    derivative of this scalar recurrence, taken by complex-step
    differentiation (exact to rounding, no differencing);
  * node indexing: the derivative reported for a node is that of a
    perturbation of that node, checked with hand-built perturbed media.
"""
import numpy as np
import pytest

from oracle import oracle as orc

TAU = 0.8
NU = (TAU - 0.5) / 3.0


def uniform_velocity(log_k, eps, nsteps, G, forch, rho0=1.0):
    """Velocity (u_x, u_y) of a uniform periodic medium after nsteps steps
    from rest.  Written directly from Eq. 2, 16a-b, 17 (rho stays rho0; the
    momentum of a node gains rho F per step); accepts complex log_k / eps."""
    k = np.exp(log_k)
    G = np.asarray(G, dtype=float)
    m = np.zeros(2, dtype=complex)

    def velocity(m):
        v = m / rho0 + 0.5 * eps * G
        c0 = 0.5 * (1.0 + 0.5 * eps * NU / k)
        if forch:
            Fe = 1.75 / np.sqrt(150.0 * eps ** 3)
            c1 = 0.5 * eps * Fe / np.sqrt(k)
            den = c0 + np.sqrt(c0 * c0 + c1 * np.sqrt(v[0] * v[0] + v[1] * v[1]))
        else:
            den = 2.0 * c0
        return v / den

    for _ in range(nsteps):
        u = velocity(m)
        drag = eps * NU / k
        if forch:
            drag = drag + eps * (1.75 / np.sqrt(150.0 * eps ** 3)) / np.sqrt(k) * np.sqrt(
                u[0] * u[0] + u[1] * u[1])
        F = eps * G - drag * u
        m = m + rho0 * F
    return velocity(m)


def uniform_kg(log_k, eps, nsteps, G, forch, rho0=1.0):
    """k_g of a uniform periodic medium after nsteps steps from rest (the
    mean velocity is the velocity of every node)."""
    return NU * uniform_velocity(log_k, eps, nsteps, G, forch, rho0)[0] / G[0]


def complex_step(f, x, h=1e-30):
    return f(x + 1j * h).imag / h


@pytest.mark.parametrize("forch", [0, 1])
def test_uniform_sum_matches_scalar_recurrence(forch):
    nx, ny, N = 5, 4, 40
    eps0, k0, G = 0.6, 2.0, (2e-4, 7e-5)   # slow Darcy relaxation: still transient at N
    p = orc.make_params(nx, ny, tau=TAU, G=G, forchheimer=forch)
    # the recurrence reproduces the oracle's own k_g
    s = orc.OracleSim(p)
    s.set_fields(eps0, k0, 0.0)
    s.step(N)
    kg, _ = s.permeability()
    assert kg == pytest.approx(uniform_kg(np.log(k0), eps0, N, G, forch).real, rel=1e-12, abs=0)
    nodes = np.arange(nx * ny)
    gk = orc.permeability_gradient_fd(p, eps0, k0, 0.0, N, nodes, "logk")
    ge = orc.permeability_gradient_fd(p, eps0, k0, 0.0, N, nodes, "eps")
    dk = complex_step(lambda z: uniform_kg(z, eps0, N, G, forch), np.log(k0))
    de = complex_step(lambda z: uniform_kg(np.log(k0), z, N, G, forch), eps0)
    assert gk.sum() == pytest.approx(dk, rel=1e-7, abs=0)
    assert ge.sum() == pytest.approx(de, rel=1e-7, abs=0)
    # uniform flow: every node has the same derivative
    assert np.ptp(gk) <= 1e-7 * abs(gk).max()
    assert np.ptp(ge) <= 1e-7 * abs(ge).max()


def test_node_indexing():
    nx, ny, N = 7, 5, 25
    rng = np.random.default_rng(4)
    eps = rng.uniform(0.3, 0.8, (ny, nx))
    k_i = 10.0 ** rng.uniform(-3, -1, (ny, nx))
    p = orc.make_params(nx, ny, tau=TAU, G=(1e-3, 0.0), bc_y=orc.BC_WALLS, forchheimer=1)
    nodes = [1 * nx + 2, 3 * nx + 6, 2 * nx + 0]
    h = 1e-4
    gk = orc.permeability_gradient_fd(p, eps, k_i, 0.0, N, nodes, "logk", h=h)
    ge = orc.permeability_gradient_fd(p, eps, k_i, 0.0, N, nodes, "eps", h=h)

    def kg(e, k):
        s = orc.OracleSim(p)
        s.set_fields(e, k, 0.0)
        s.step(N)
        return s.permeability()[0]

    for m, j in enumerate(nodes):
        y, x = divmod(j, nx)
        kp, km = k_i.copy(), k_i.copy()
        kp[y, x] *= np.exp(h)
        km[y, x] *= np.exp(-h)
        assert gk[m] == pytest.approx((kg(eps, kp) - kg(eps, km)) / (2 * h), rel=1e-12, abs=1e-18)
        ep, em = eps.copy(), eps.copy()
        ep[y, x] += h
        em[y, x] -= h
        assert ge[m] == pytest.approx((kg(ep, k_i) - kg(em, k_i)) / (2 * h), rel=1e-12, abs=1e-18)
    # plate rows carry no fluid: their derivative is exactly zero
    assert orc.permeability_gradient_fd(p, eps, k_i, 0.0, N, [2], "logk")[0] == 0.0
    with pytest.raises(ValueError):
        orc.permeability_gradient_fd(p, eps, k_i, 0.0, N, [nx * ny], "logk")
