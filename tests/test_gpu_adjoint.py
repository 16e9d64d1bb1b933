"""Discrete adjoint of the time loop (lbmp_permeability_gradient) against
the oracle's central-difference gradient of k_g (FP64, h = 1e-4).

Small lattices: every node, both parameters (ln k_i and eps), each boundary
kind, impermeable and open nodes.  Then a 64 x 64 crop of the
two-component adjoint workload (Kn = 0.1, pressure drive, plates) at 2000
steps on 64 seeded nodes, the full 1024 x 1024 workload at 20000 steps
(properties that hold at any size), checkpoint-interval invariance, the
uniform-medium sum rule, the autograd wrapper and the error paths.
"""
import numpy as np
import pytest

from paper_1411_7051_gb300 import lbmp, media
from helpers import Case, gpu_sim
from test_oracle_gradient import complex_step, uniform_kg

pytestmark = pytest.mark.gpu


def _params(orc, case):
    return orc.make_params(case.nx, case.ny, tau=case.tau, G=case.G,
                           bc_x=orc.BC_PRESSURE if case.pressure else orc.BC_PERIODIC,
                           bc_y=orc.BC_WALLS if case.walls else orc.BC_PERIODIC,
                           rho_in=case.rho_in, rho_out=case.rho_out,
                           forchheimer=case.forchheimer)


def _fd(orc, case, nsteps, nodes, which):
    m = case.medium
    return orc.permeability_gradient_fd(_params(orc, case), m.eps, m.k_i, m.kn, nsteps, nodes,
                                        which, h=1e-4)


def _gpu_grad(case, nsteps, every=0, kernel=0):
    with gpu_sim(case, kernel=kernel) as s:
        kg, gl, ge = s.permeability_gradient(nsteps, every, device=False)
    return kg, gl.numpy(), ge.numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


SMALL = {
    "pressure_walls_forch": Case(20, 12, tau=0.8, pressure=True, walls=True, rho_in=1.002,
                                 rho_out=0.999, forchheimer=1,
                                 medium=media.random_medium(20, 12, seed=31, eps_range=(0.2, 0.9),
                                                            log10_k_range=(-2.5, 0.5),
                                                            kn_range=(0.0, 1.0), p_open=0.06,
                                                            p_solid=0.06)),
    "body_force_walls_forch": Case(16, 10, tau=0.7, G=(2e-4, 4e-5), walls=True, forchheimer=1,
                                   medium=media.random_medium(16, 10, seed=32, eps_range=(0.2, 0.9),
                                                              log10_k_range=(-2.0, 1.0),
                                                              p_open=0.05, p_solid=0.05)),
    "periodic_darcy": Case(12, 12, tau=1.1, G=(1e-4, 6e-5), forchheimer=0,
                           medium=media.random_medium(12, 12, seed=33, eps_range=(0.3, 0.9),
                                                      log10_k_range=(-1.5, 1.0))),
}


@pytest.mark.parametrize("name", sorted(SMALL))
def test_gradient_every_node(orc, name):
    case = SMALL[name]
    N = 90
    kg, gl, ge = _gpu_grad(case, N, every=7)   # 13 segments, the last one ragged
    o = orc.OracleSim(_params(orc, case))
    m = case.medium
    o.set_fields(m.eps, m.k_i, m.kn)
    o.step(N)
    assert kg == pytest.approx(o.permeability()[0], rel=1e-5, abs=0)
    nodes = np.arange(case.nx * case.ny)
    fl = _fd(orc, case, N, nodes, "logk").reshape(case.ny, case.nx)
    fe = _fd(orc, case, N, nodes, "eps").reshape(case.ny, case.nx)
    assert _rel(gl, fl) <= 1e-4, _rel(gl, fl)
    assert np.abs(gl - fl).max() <= 1e-4 * np.abs(fl).max()
    porous = m.eps > 0.0          # eps = 0 is a branch point of the step
    assert _rel(ge[porous], fe[porous]) <= 1e-4, _rel(ge[porous], fe[porous])
    assert np.abs(ge - fe)[porous].max() <= 1e-4 * np.abs(fe[porous]).max()
    # impermeable and open nodes: no dependence on k_i
    assert np.all(gl[(m.eps == 0.0) | np.isinf(m.k_i)] == 0.0)
    if case.walls:
        assert np.all(gl[[0, -1]] == 0.0) and np.all(ge[[0, -1]] == 0.0)


def test_staged_forward_kernel(orc):
    """The forward and recompute passes use the kernel the context selected."""
    case = SMALL["pressure_walls_forch"]
    kg_d, gl_d, ge_d = _gpu_grad(case, 40, every=0, kernel=lbmp.KERNEL_DIRECT)
    kg_s, gl_s, ge_s = _gpu_grad(case, 40, every=0, kernel=lbmp.KERNEL_STAGED)
    assert kg_s == pytest.approx(kg_d, rel=1e-6, abs=0)
    assert _rel(gl_s, gl_d) <= 1e-5 and _rel(ge_s, ge_d) <= 1e-5


def test_checkpoint_interval_invariance():
    """Recomputation is exact: any checkpoint interval gives the same bits."""
    case = SMALL["body_force_walls_forch"]
    N = 37
    ref = _gpu_grad(case, N, every=1)
    for every in (3, 0, 10, N, 1000):
        got = _gpu_grad(case, N, every=every)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])


def test_value_and_state_match_plain_run():
    case = SMALL["pressure_walls_forch"]
    N = 70
    with gpu_sim(case) as s:
        kg, _, _ = s.permeability_gradient(N)
        kg2, _ = s.permeability()
        f_adj = s.populations(device=False).numpy()
        assert s.info().steps == N
    with gpu_sim(case) as s:
        s.step(N)
        kg3, _ = s.permeability()
        f_run = s.populations(device=False).numpy()
    assert kg == kg2 == kg3
    assert np.array_equal(f_adj, f_run)


@pytest.mark.parametrize("forch", [0, 1])
def test_uniform_sum_rule(forch):
    """Uniform periodic medium: the gradient summed over nodes is the
    derivative of the one-node momentum recurrence (complex step)."""
    nx, ny, N = 32, 24, 60
    eps0, k0, G = 0.6, 2.0, (2e-4, 7e-5)
    med = media.Medium(np.full((ny, nx), eps0), np.full((ny, nx), k0), np.zeros((ny, nx)), "uniform")
    case = Case(nx, ny, tau=0.8, G=G, forchheimer=forch, medium=med)
    kg, gl, ge = _gpu_grad(case, N)
    assert kg == pytest.approx(uniform_kg(np.log(k0), eps0, N, G, forch).real, rel=1e-5, abs=0)
    dk = complex_step(lambda z: uniform_kg(z, eps0, N, G, forch), np.log(k0))
    de = complex_step(lambda z: uniform_kg(np.log(k0), z, N, G, forch), eps0)
    assert gl.sum() == pytest.approx(dk, rel=2e-5, abs=0)
    assert ge.sum() == pytest.approx(de, rel=2e-5, abs=0)


def _adjoint_workload(n):
    return media.two_component(n, seed=2, kn=0.1)


def _adjoint_case(med):
    ny, nx = med.eps.shape
    return Case(nx, ny, tau=0.8, pressure=True, walls=True, rho_in=1.0005, rho_out=0.9995,
                forchheimer=1, medium=med)


def test_crop_64_sampled_nodes(orc):
    """64 x 64 crop of the two-component adjoint workload, 2000 steps,
    FD on 64 seeded nodes of each parameter."""
    med = _adjoint_workload(1024).crop(64, 64, 300, 500)
    case = _adjoint_case(med)
    N = 2000
    kg, gl, ge = _gpu_grad(case, N)
    rng = np.random.default_rng(64)
    ys = rng.integers(1, 63, 64)
    xs = rng.integers(0, 64, 64)
    nodes = ys * 64 + xs
    fl = _fd(orc, case, N, nodes, "logk")
    fe = _fd(orc, case, N, nodes, "eps")
    assert _rel(gl[ys, xs], fl) <= 1e-4, _rel(gl[ys, xs], fl)
    assert _rel(ge[ys, xs], fe) <= 1e-4, _rel(ge[ys, xs], fe)


def test_full_size_workload():
    """1024 x 1024 two-component medium, Kn = 0.1, 20000 steps (sqrt(N)
    checkpoints): J equals the plain run's k_g, and the gradient predicts the
    change of k_g under a smooth rescaling of k_i and of eps (FP32 forward
    differences, h = 1e-2)."""
    import torch
    med = _adjoint_workload(1024)
    case = _adjoint_case(med)
    N = 20000
    with gpu_sim(case) as s:
        kg, gl, ge = s.permeability_gradient(N, device=True)
        gl = gl.cpu().numpy()
        ge = ge.cpu().numpy()
        kg2, _ = s.permeability()
    assert kg == kg2
    assert np.all(np.isfinite(gl)) and np.all(np.isfinite(ge))
    ny, nx = med.eps.shape
    yy, xx = np.mgrid[0:ny, 0:nx]
    d = 1.0 + 0.5 * np.sin(2 * np.pi * xx / nx) * np.cos(2 * np.pi * yy / ny)
    h = 1e-2

    def kg_of(eps, k_i):
        m = media.Medium(eps, k_i, med.kn, "perturbed")
        with gpu_sim(Case(nx, ny, tau=0.8, pressure=True, walls=True, rho_in=1.0005,
                          rho_out=0.9995, forchheimer=1, medium=m)) as s:
            s.step(N)
            return s.permeability()[0]

    fd_k = (kg_of(med.eps, med.k_i * np.exp(h * d)) - kg_of(med.eps, med.k_i * np.exp(-h * d))) / (2 * h)
    assert float((gl * d).sum()) == pytest.approx(fd_k, rel=2e-3, abs=0)
    de = 0.1 * d * med.eps
    fd_e = (kg_of(med.eps + h * de, med.k_i) - kg_of(med.eps - h * de, med.k_i)) / (2 * h)
    assert float((ge * de).sum()) == pytest.approx(fd_e, rel=2e-3, abs=0)
    torch.cuda.empty_cache()


def test_autograd_function():
    import torch
    case = SMALL["periodic_darcy"]
    m = case.medium
    N = 50
    with gpu_sim(case) as s:
        kg_ref, gl_ref, ge_ref = s.permeability_gradient(N, device=False)
    dev = torch.device("cuda")
    log_k = torch.tensor(np.log(m.k_i), device=dev, requires_grad=True)
    eps = torch.tensor(m.eps, device=dev, requires_grad=True)
    kn = torch.tensor(m.kn, device=dev)
    with gpu_sim(case) as s:
        J = lbmp.ka_from_fields(s, log_k, eps, kn, N)
        (3.0 * J).backward()
        # without a gradient request: the plain run
        with torch.no_grad():
            J2 = lbmp.ka_from_fields(s, log_k, eps, kn, N)
    assert J.item() == pytest.approx(kg_ref, rel=1e-6, abs=0)
    assert J2.item() == J.item()
    assert np.allclose(log_k.grad.cpu().numpy(), 3.0 * gl_ref.numpy(), rtol=1e-5, atol=1e-14)
    assert np.allclose(eps.grad.cpu().numpy(), 3.0 * ge_ref.numpy(), rtol=1e-5, atol=1e-14)


def test_errors():
    case = SMALL["periodic_darcy"]
    with gpu_sim(case) as s:
        with pytest.raises(lbmp.LbmpError) as e:
            s.permeability_gradient(0)
        assert e.value.status == lbmp.EINVAL
        with pytest.raises(lbmp.LbmpError) as e:
            s.permeability_gradient(5, every=-1)
        assert e.value.status == lbmp.EINVAL
    with gpu_sim(case, storage=lbmp.STORE_FP16) as s:
        with pytest.raises(lbmp.LbmpError) as e:
            s.permeability_gradient(5)
        assert e.value.status == lbmp.EINVAL
    cfg = lbmp.SimConfig(case.nx, case.ny, G=case.G)
    with lbmp.Sim(cfg) as s:
        with pytest.raises(lbmp.LbmpError) as e:
            s.permeability_gradient(5)
        assert e.value.status == lbmp.ESTATE
