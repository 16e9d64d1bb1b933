"""Dynamic Knudsen number and the first-order Klinkenberg factor on the GPU
against the FP64 oracle (the tolerances of test_gpu_parity: one FP32 step
within 2e-9 absolute; FP32 rel-L2(u) <= 1e-5 and k_g <= 1e-6, steady or
transient; FP16 k_g <= 1e-3).

With a dynamic Kn a node's apparent permeability is k_i f_c(Kn0 p0 / p)
at its current pressure p / p0 = 1 + beta (rho - rho0); the GPU evaluates
f_c in FP32 every step (relative error ~1e-7), the oracle in FP64.
"""
import numpy as np
import pytest

from paper_1411_7051_gb300 import lbmp, media
from helpers import Case, fluid_rows, gpu_sim, oracle_sim, rel_l2

pytestmark = pytest.mark.gpu

FP32, FP16 = 0, 1
RHO_IN, RHO_OUT = 1.0005, 0.9995
BETA2 = 1.0 / ((RHO_IN - 1.0) - 2.0 * (RHO_OUT - 1.0))  # p_in = 2 p_out


def _np(t):
    return t.detach().cpu().numpy()


def _compare(gs, osim, case, rel_u, rel_k):
    _, gux, guy = gs.macroscopic()
    _, oux, ouy = osim.macroscopic()
    fr = fluid_rows(case)
    e_u = rel_l2(np.stack([_np(gux)[fr], _np(guy)[fr]]), np.stack([oux[fr], ouy[fr]]))
    kg_g, _ = gs.permeability()
    kg_o, _ = osim.permeability()
    e_k = abs(kg_g / kg_o - 1)
    assert e_u <= rel_u, f"rel-L2(u) = {e_u:.3e}"
    assert e_k <= rel_k, f"k_g rel err = {e_k:.3e}"
    return kg_g


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("beta", [0.0, 300.0])
@pytest.mark.parametrize("walls,pressure,forch", [(True, True, 1), (False, False, 0),
                                                  (True, False, 1)])
def test_one_step(orc, model, beta, walls, pressure, forch):
    nx, ny = 133, 21
    med = media.random_medium(nx, ny, seed=17, p_open=0.1, p_solid=0.1,
                              log10_k_range=(-3, 0), kn_range=(0.0, 5.0))
    case = Case(nx, ny, tau=0.7, G=(3e-5, -1e-5), walls=walls, pressure=pressure,
                rho_in=1.001, rho_out=0.999, forchheimer=forch, medium=med, kn_model=model,
                kn_beta=beta)
    _, _, w = orc.lattice()
    f0 = media.random_populations(nx, ny, seed=4, base=w, amp=2e-3)
    osim = oracle_sim(orc, case)
    osim.set_populations(f0)
    gs = gpu_sim(case, FP32)
    gs.set_populations(f0)
    fr = fluid_rows(case)
    for _ in range(3):
        osim.step(1)
        gs.step(1)
        np.testing.assert_allclose(_np(gs.populations())[:, fr], osim.populations()[:, fr],
                                   rtol=0, atol=2e-9)


@pytest.mark.parametrize("model", [0, 1])
def test_darcy_closed_form(orc, model):
    """Steady 1-D Darcy flow with the pressure-dependent permeability: the
    GPU's k_g equals the oracle's and the mean of k_a over the density range."""
    from scipy.integrate import quad
    nx, ny = 48, 3
    eps, k_i, kn0 = 0.5, 0.04, 0.5
    med = media.Medium(np.full((ny, nx), eps), np.full((ny, nx), k_i), np.full((ny, nx), kn0))
    case = Case(nx, ny, tau=0.8, pressure=True, rho_in=RHO_IN, rho_out=RHO_OUT, medium=med,
                kn_model=model, kn_beta=BETA2)
    osim = oracle_sim(orc, case)
    osim.run_to_steady(tol=1e-12, check_every=500)
    gs = gpu_sim(case, FP32)
    gs.step(osim.steps)
    kg = _compare(gs, osim, case, rel_u=1e-5, rel_k=1e-6)
    fc = orc.fc if model == 0 else orc.fc_first_order
    ka = lambda rho: k_i * fc(kn0 / (1.0 + BETA2 * (rho - 1.0)))  # noqa: E731
    expect = quad(ka, RHO_OUT, RHO_IN, epsrel=1e-13)[0] / (RHO_IN - RHO_OUT)
    assert kg == pytest.approx(expect, rel=5e-4, abs=0)


def _two_component(kn, model=0):
    med = media.two_component(96, seed=2, corr_len=12.0, kn=kn, ny=64)
    return Case(96, 64, tau=0.8, pressure=True, walls=True, rho_in=RHO_IN, rho_out=RHO_OUT,
                forchheimer=1, medium=med, kn_model=model, kn_beta=BETA2)


@pytest.mark.parametrize("kn", [0.1, 1.0])
def test_two_component_transient(orc, kn):
    case = _two_component(kn)
    osim = oracle_sim(orc, case)
    gs = gpu_sim(case, FP32)
    for n in (150, 850):
        osim.step(n)
        gs.step(n)
    _compare(gs, osim, case, rel_u=1e-5, rel_k=1e-6)
    # the dynamic Kn changes the answer: against the static run
    static = Case(**{**case.__dict__, "kn_beta": 0.0})
    gst = gpu_sim(static, FP32)
    gst.step(1000)
    assert abs(gst.permeability()[0] / gs.permeability()[0] - 1) > 1e-3


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("storage", [FP32, FP16])
def test_heterogeneous_steady(orc, model, storage):
    med = media.two_component(48, seed=7, corr_len=6.0, kn=0.5, ny=32, matrix=(0.4, 0.1),
                              inclusion=(0.8, 1.0))
    case = Case(48, 32, tau=0.8, pressure=True, walls=True, rho_in=RHO_IN, rho_out=RHO_OUT,
                medium=med, kn_model=model, kn_beta=BETA2)
    osim = oracle_sim(orc, case)
    osim.run_to_steady(tol=1e-10, check_every=200, max_steps=400_000)
    gs = gpu_sim(case, storage)
    gs.step(osim.steps)
    if storage == FP32:
        _compare(gs, osim, case, rel_u=1e-5, rel_k=1e-6)
    else:
        kg_g, _ = gs.permeability()
        kg_o, _ = osim.permeability()
        assert abs(kg_g / kg_o - 1) <= 1e-3, (kg_g, kg_o)


def test_first_order_static_steady(orc):
    """The first-order correlation (Eq. 4-5) with a static Kn, body force."""
    med = media.random_medium(64, 48, seed=31, eps_range=(0.3, 1.0), log10_k_range=(-1, 1),
                              kn_range=(0, 2), p_open=0.1)
    case = Case(64, 48, tau=0.8, G=(2e-6, 5e-7), walls=True, forchheimer=1, medium=med,
                kn_model=1)
    osim = oracle_sim(orc, case)
    osim.run_to_steady(tol=1e-10, check_every=200, max_steps=400_000)
    gs = gpu_sim(case, FP32)
    gs.step(osim.steps)
    _compare(gs, osim, case, rel_u=1e-5, rel_k=1e-6)


def test_batch_honours_kn_model():
    case = Case(64, 40, tau=0.8, pressure=True, walls=True, rho_in=RHO_IN, rho_out=RHO_OUT,
                forchheimer=1, medium=media.two_component(64, seed=3, corr_len=8.0, kn=1.0, ny=40),
                kn_model=1)
    gs = gpu_sim(case, FP32, kernel=lbmp.KERNEL_DIRECT)
    gs.step(300)
    kg1, _ = gs.permeability()
    cfg = lbmp.SimConfig(1, 1, tau=0.8, bc_x=lbmp.BCX_PRESSURE, bc_y=lbmp.BCY_WALLS,
                         rho_in=RHO_IN, rho_out=RHO_OUT, forchheimer=1, kn_model=1)
    with lbmp.Batch(cfg, [(64, 40)]) as b:
        m = case.medium
        b.set_fields(0, m.eps, m.k_i, m.kn)
        b.step(300)
        kgb, _ = b.permeability()
    assert kgb[0] == pytest.approx(kg1, rel=1e-6, abs=0)


def test_noalloc_dynamic(orc):
    import torch
    case = _two_component(0.5)
    gs = gpu_sim(case, FP32)
    gs.step(400)
    kg, um = gs.permeability()
    f = gs.populations(device=True)
    dev = f.device
    m = case.medium
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    cfg = lbmp.SimConfig(case.nx, case.ny, tau=0.8, bc_x=lbmp.BCX_PRESSURE, bc_y=lbmp.BCY_WALLS,
                         rho_in=RHO_IN, rho_out=RHO_OUT, forchheimer=1, kn_beta=BETA2)
    lbmp.permeability_noalloc(cfg, f, t(m.eps), t(m.k_i), t(m.kn), out)
    torch.cuda.synchronize()
    assert out[0].item() == pytest.approx(kg, rel=1e-6, abs=0)
    assert out[2].item() == 0.0


def test_unsupported_combinations():
    case = _two_component(0.5)
    cfg = lbmp.SimConfig(8, 8, bc_x=lbmp.BCX_PRESSURE, rho_in=RHO_IN, rho_out=RHO_OUT,
                         kn_beta=BETA2)
    with pytest.raises(lbmp.LbmpError) as e:
        lbmp.Batch(cfg, [(8, 8)])
    assert e.value.status == lbmp.EINVAL
    with gpu_sim(case, FP32) as s:
        with pytest.raises(lbmp.LbmpError) as e:
            s.permeability_gradient(10)
        assert e.value.status == lbmp.EINVAL
        assert s.info().bytes_per_update == 84.0
    # FP16 + dynamic Kn runs the staged kernel with the Kn plane staged
    with gpu_sim(case, FP16) as s:
        s.step(10)
        assert np.isfinite(s.permeability()[0])
        assert s.info().bytes_per_update == 48.0
