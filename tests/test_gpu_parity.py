"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances:

* one step from the same state, FP32 storage: populations within 2e-9
  absolute (FP32 rounding of O(1e-3) deviations and of rho);
* many steps, FP32: relative L2 of the velocity <= 1e-5 and global
  permeability <= 1e-6 relative;
* FP16-stored populations: global permeability <= 1e-3 relative.
"""
import numpy as np
import pytest

from paper_1411_7051_gb300 import media
from helpers import Case, fluid_rows, gpu_sim, oracle_sim, rel_l2

pytestmark = pytest.mark.gpu

FP32, FP16 = 0, 1


def _np(t):
    return t.detach().cpu().numpy()


def _compare_velocity(gs, osim, case, rel_u=1e-5, rel_k=1e-6):
    _, gux, guy = gs.macroscopic()
    _, oux, ouy = osim.macroscopic()
    fr = fluid_rows(case)
    g = np.stack([_np(gux)[fr], _np(guy)[fr]])
    o = np.stack([oux[fr], ouy[fr]])
    e_u = rel_l2(g, o)
    kg_g, _ = gs.permeability()
    kg_o, _ = osim.permeability()
    e_k = abs(kg_g / kg_o - 1)
    assert e_u <= rel_u, f"rel-L2(u) = {e_u:.3e}"
    assert e_k <= rel_k, f"k_g rel err = {e_k:.3e} ({kg_g} vs {kg_o})"
    return e_u, e_k


# ----------------------------------------------------- one step, elementwise
ONE_STEP_CASES = {
    "periodic": dict(walls=False, pressure=False, forchheimer=0),
    "walls_forch": dict(walls=True, pressure=False, forchheimer=1),
    "pressure_walls": dict(walls=True, pressure=True, forchheimer=1),
    "pressure_periodic": dict(walls=False, pressure=True, forchheimer=0),
}


@pytest.mark.parametrize("name", list(ONE_STEP_CASES))
@pytest.mark.parametrize("nx,ny", [(131, 37), (300, 9), (1, 5), (5, 1)])
def test_one_step_from_random_state(orc, name, nx, ny):
    kw = ONE_STEP_CASES[name]
    if kw["walls"] and ny < 3 or kw["pressure"] and nx < 3:
        pytest.skip("lattice too small for this boundary kind")
    med = media.random_medium(nx, ny, seed=nx * 7 + ny, p_open=0.15, p_solid=0.1,
                              log10_k_range=(-3, 0))
    case = Case(nx, ny, tau=0.7, G=(3e-5, -1e-5), rho_in=1.001, rho_out=0.999,
                medium=med, **kw)
    _, _, w = orc.lattice()
    f0 = media.random_populations(nx, ny, seed=3, base=w, amp=2e-3)
    osim = oracle_sim(orc, case)
    osim.set_populations(f0)
    gs = gpu_sim(case, FP32)
    gs.set_populations(f0)
    fr = fluid_rows(case)
    # the loaded state itself (pressure columns re-extrapolated on both sides)
    np.testing.assert_allclose(_np(gs.populations())[:, fr], osim.populations()[:, fr],
                               rtol=0, atol=2e-9)
    for _ in range(3):
        osim.step(1)
        gs.step(1)
        np.testing.assert_allclose(_np(gs.populations())[:, fr],
                                   osim.populations()[:, fr], rtol=0, atol=2e-9)


# --------------------------------------------- validation channel (config 1)
def test_channel_validation_config(orc):
    """64 x 33 channel, eps 0.7, tau 0.8, Da 1e-3, Kn 0.1, G 1e-6 (FP64 oracle
    to residual < 1e-10); FP32 GPU to a fixed step count."""
    med = media.channel(64, 33, 0.7, 1e-3, 0.1)
    case = Case(64, 33, tau=0.8, G=(1e-6, 0.0), walls=True, medium=med)
    osim = oracle_sim(orc, case)
    osim.run_to_steady(tol=1e-10, check_every=100)
    gs = gpu_sim(case, FP32)
    gs.step(max(osim.steps, 2000))
    _compare_velocity(gs, osim, case)
    # and the analytic Brinkman-Darcy profile (Eq. 20)
    import pins
    _, ux, _ = gs.macroscopic()
    prof = _np(ux)[1:-1].mean(axis=1)
    H = 31
    ua = pins.brinkman_profile(1e-6, 1e-3 * H * H * orc.fc(0.1), 0.1, 0.7, H,
                               np.arange(1, 32) - 0.5)
    assert rel_l2(prof, ua) < 1e-2


# ------------------------------------------ heterogeneous media, many steps
def _two_component_case(n=128, ny=96, kn=0.1, seed=2, walls=True):
    med = media.two_component(n, seed=seed, corr_len=16.0, kn=kn, ny=ny)
    return Case(n, ny, tau=0.8, pressure=True, walls=walls, rho_in=1.0005, rho_out=0.9995,
                medium=med)


@pytest.mark.parametrize("kn", [0.001, 1.0, 10.0])
def test_two_component_fp32(orc, kn):
    case = _two_component_case(kn=kn)
    osim = oracle_sim(orc, case)
    gs = gpu_sim(case, FP32)
    for n in (100, 900):
        osim.step(n)
        gs.step(n)
    _compare_velocity(gs, osim, case)


def test_forchheimer_shale_fp32(orc):
    med = media.shale_fractures(n=160, seed=5, n_fractures=4, length=(40, 120))
    case = Case(160, 160, tau=0.9, pressure=True, walls=False, rho_in=1.001,
                rho_out=0.999, forchheimer=1, medium=med)
    osim = oracle_sim(orc, case)
    gs = gpu_sim(case, FP32)
    osim.step(600)
    gs.step(600)
    _compare_velocity(gs, osim, case)


def test_impermeable_and_open_nodes_fp32(orc):
    med = media.random_medium(97, 45, seed=9, p_open=0.3, p_solid=0.2,
                              log10_k_range=(-2, 1))
    case = Case(97, 45, tau=1.1, G=(1e-5, 2e-6), walls=True, forchheimer=1, medium=med)
    osim = oracle_sim(orc, case)
    gs = gpu_sim(case, FP32)
    osim.step(400)
    gs.step(400)
    _compare_velocity(gs, osim, case)


# ------------------------------------------------------------- FP16 storage
def test_fp16_channel_permeability(orc):
    med = media.channel(64, 33, 0.7, 1e-3, 0.1)
    case = Case(64, 33, tau=0.8, G=(1e-6, 0.0), walls=True, medium=med)
    osim = oracle_sim(orc, case)
    osim.run_to_steady(tol=1e-10, check_every=100)
    gs = gpu_sim(case, FP16)
    gs.step(max(osim.steps, 2000))
    kg_g, _ = gs.permeability()
    kg_o, _ = osim.permeability()
    assert abs(kg_g / kg_o - 1) <= 1e-3, (kg_g, kg_o)


@pytest.mark.parametrize("kn", [0.01, 1.0])
def test_fp16_two_component_permeability(orc, kn):
    case = _two_component_case(kn=kn)
    osim = oracle_sim(orc, case)
    gs = gpu_sim(case, FP16)
    osim.step(1000)
    gs.step(1000)
    kg_g, _ = gs.permeability()
    kg_o, _ = osim.permeability()
    assert abs(kg_g / kg_o - 1) <= 1e-3, (kg_g, kg_o)


# --------------------------------------------------------- invariants, state
def test_mass_conservation_gpu(orc):
    med = media.random_medium(130, 70, seed=4, p_open=0.2, p_solid=0.1)
    case = Case(130, 70, tau=0.75, G=(2e-5, 1e-5), walls=True, forchheimer=1, medium=med)
    gs = gpu_sim(case, FP32)
    m0 = gs.mass()
    gs.step(2000)
    m1 = gs.mass()
    assert abs(m1 / m0 - 1) < 1e-9, (m0, m1)


def test_graph_replay_matches_single_launches():
    case = _two_component_case(n=200, ny=50)
    a = gpu_sim(case, FP32)
    b = gpu_sim(case, FP32)
    a.step(70)            # two graph replays + 6 single launches
    for _ in range(70):
        b.step(1)
    assert np.array_equal(_np(a.populations()), _np(b.populations()))


@pytest.mark.parametrize("storage", [FP32, FP16])
def test_checkpoint_restart_bitwise(storage):
    case = _two_component_case(n=96, ny=40)
    a = gpu_sim(case, storage)
    a.step(50)
    blob = a.get_state()
    a.step(50)
    b = gpu_sim(case, storage)
    b.set_state(blob)
    assert b.info().steps == 50
    b.step(50)
    assert np.array_equal(_np(a.populations()), _np(b.populations()))


def test_residual_semantics():
    case = _two_component_case(n=64, ny=40)
    gs = gpu_sim(case, FP32)
    gs.step(10)
    assert gs.residual() == pytest.approx(1.0)   # against the zero snapshot
    assert gs.residual() == 0.0                  # nothing moved since
    gs.step(10)
    assert 0.0 < gs.residual() < 1.0


def test_set_fields_rejects_bad_values():
    from paper_1411_7051_gb300 import lbmp
    med = media.random_medium(16, 8, seed=1)
    case = Case(16, 8, medium=med)
    gs = gpu_sim(case, FP32)
    for field, bad in (("eps", 1.5), ("eps", np.nan), ("k_i", 0.0), ("k_i", -1.0),
                       ("kn", -0.1), ("kn", np.inf)):
        e, k, n = med.eps.copy(), med.k_i.copy(), med.kn.copy()
        {"eps": e, "k_i": k, "kn": n}[field][3, 5] = bad
        with pytest.raises(lbmp.LbmpError) as ei:
            gs.set_fields(e, k, n)
        assert ei.value.status == lbmp.EINVAL
    with pytest.raises(lbmp.LbmpError) as ei:
        gs.step(1)  # the failed set_fields left no valid medium
    assert ei.value.status == lbmp.ESTATE
    gs.set_fields(med.eps, med.k_i, med.kn)
    gs.step(1)


def test_device_inputs_match_host_inputs():
    import torch
    case = _two_component_case(n=64, ny=32)
    a = gpu_sim(case, FP32)
    b = gpu_sim(case, FP32)
    m = case.medium
    b.set_fields(torch.tensor(m.eps, device="cuda"), torch.tensor(m.k_i, device="cuda"),
                 torch.tensor(m.kn, device="cuda"))
    a.step(20)
    b.step(20)
    assert np.array_equal(_np(a.populations()), _np(b.populations()))


def test_simulated_allocation_failure(monkeypatch):
    from paper_1411_7051_gb300 import lbmp
    import torch
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("LBMP_FAULT_ALLOC", "3")
    with pytest.raises(lbmp.LbmpError) as ei:
        lbmp.Sim(lbmp.SimConfig(512, 512))
    assert ei.value.status == lbmp.ENOMEM
    monkeypatch.delenv("LBMP_FAULT_ALLOC")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20)  # nothing leaked
