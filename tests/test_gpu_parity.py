"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances:

* one step from the same state, FP32 storage: populations within 2e-9
  absolute (FP32 rounding of O(1e-3) deviations and of rho);
* steady states, FP32: relative L2 of the velocity <= 1e-5 and global
  permeability <= 1e-6 relative;
* transient states of pressure-driven runs, FP32: the same bounds.  While
  the pressure wave crosses the lattice the stored deviations f_i - w_i rho0
  carry the density deviation (up to 5e-4), about 1e3 times the velocity
  signal, so one FP32 rounding (2^-24) moves the velocity of a node by
  ~1e-4 relative per step.  Exactly conserving collisions and explicitly
  rounded arithmetic keep these errors zero-mean, and the domain mean of
  the velocity (k_g) stays within 1e-6;
* FP16-stored populations (stochastic rounding, the default): global
  permeability <= 1e-3 relative; one step from the same state: each
  population within one FP16 ulp of its deviation (2^-10 relative).

Measured errors are appended to $LBMP_PARITY_LOG (JSON lines) when set.
"""
import json
import os

import numpy as np
import pytest

from paper_1411_7051_gb300 import media
from helpers import Case, fluid_rows, gpu_sim, oracle_sim, rel_l2

pytestmark = pytest.mark.gpu

FP32, FP16 = 0, 1
SR, RN = 0, 1
STAGED, DIRECT = 1, 2


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
    _log(e_u=e_u, e_k=e_k, kg=kg_g, kg_oracle=kg_o)
    assert e_u <= rel_u, f"rel-L2(u) = {e_u:.3e}"
    assert e_k <= rel_k, f"k_g rel err = {e_k:.3e} ({kg_g} vs {kg_o})"
    return e_u, e_k


def _log(**kw):
    path = os.environ.get("LBMP_PARITY_LOG")
    if path:
        kw["test"] = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
        with open(path, "a") as fh:
            fh.write(json.dumps(kw) + "\n")


# ----------------------------------------------------- one step, elementwise
ONE_STEP_CASES = {
    "periodic": dict(walls=False, pressure=False, forchheimer=0),
    "walls_forch": dict(walls=True, pressure=False, forchheimer=1),
    "pressure_walls": dict(walls=True, pressure=True, forchheimer=1),
    "pressure_periodic": dict(walls=False, pressure=True, forchheimer=0),
}


@pytest.mark.parametrize("kernel", [STAGED, DIRECT])
@pytest.mark.parametrize("name", list(ONE_STEP_CASES))
@pytest.mark.parametrize("nx,ny", [(131, 37), (300, 9), (1, 5), (5, 1), (257, 6)])
def test_one_step_from_random_state(orc, name, nx, ny, kernel):
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
    gs = gpu_sim(case, FP32, kernel=kernel)
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


@pytest.mark.parametrize("rounding", [SR, RN])
def test_one_step_fp16_within_one_ulp(orc, rounding):
    nx, ny = 130, 21
    med = media.random_medium(nx, ny, seed=5, p_open=0.1, p_solid=0.1, log10_k_range=(-3, 0))
    case = Case(nx, ny, tau=0.75, G=(2e-5, 0.0), walls=True, pressure=True, rho_in=1.001,
                rho_out=0.999, forchheimer=1, medium=med)
    _, _, w = orc.lattice()
    f0 = media.random_populations(nx, ny, seed=8, base=w, amp=2e-3)
    osim = oracle_sim(orc, case)
    gs = gpu_sim(case, FP16, fp16_rounding=rounding)
    gs.set_populations(f0)
    # start both from the FP16-rounded state the GPU holds
    osim.set_populations(_np(gs.populations()))
    fr = fluid_rows(case)
    wb = w[:, None, None]
    for _ in range(2):
        osim.step(1)
        gs.step(1)
        fo = osim.populations()[:, fr]
        dev = np.abs(fo - wb)
        err = np.abs(_np(gs.populations())[:, fr] - fo)
        # interior columns: one FP16 rounding of the node's own deviation
        inner = (slice(None), slice(None), slice(1, nx - 1))
        assert np.all(err[inner] <= dev[inner] * 2.0 ** -10 + 1e-10), err[inner].max()
        # pressure columns are extrapolated from their neighbour and inherit
        # its rounding: bound by the neighbour's deviation
        for xb, xn in ((0, 1), (nx - 1, nx - 2)):
            bound = 2.0 * dev[:, :, xn].max(axis=0) * 2.0 ** -10 + 1e-10
            assert np.all(err[:, :, xb] <= bound[None, :]), err[:, :, xb].max()
        osim.set_populations(_np(gs.populations()))


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
    _compare_velocity(gs, osim, case, rel_k=1e-6)


def test_forchheimer_shale_fp32(orc):
    """Fractured shale, transient, tau 0.9.  Matrix velocities (k_i ~ 1e-6)
    are ~1e-9 under a density deviation of ~1e-3, so FP32 carries them with
    a few significant digits only; the fracture velocities dominate the L2
    norm.  Velocity bound 1e-5 (measured 1.4e-6 with the collision's
    1 - omega and omega summing to exactly 1), permeability 1e-6."""
    med = media.shale_fractures(n=160, seed=5, n_fractures=4, length=(40, 120))
    case = Case(160, 160, tau=0.9, pressure=True, walls=False, rho_in=1.001,
                rho_out=0.999, forchheimer=1, medium=med)
    osim = oracle_sim(orc, case)
    gs = gpu_sim(case, FP32)
    osim.step(600)
    gs.step(600)
    _compare_velocity(gs, osim, case, rel_u=1e-5, rel_k=1e-6)


def test_impermeable_and_open_nodes_fp32(orc):
    med = media.random_medium(97, 45, seed=9, p_open=0.3, p_solid=0.2,
                              log10_k_range=(-2, 1))
    case = Case(97, 45, tau=1.1, G=(1e-5, 2e-6), walls=True, forchheimer=1, medium=med)
    osim = oracle_sim(orc, case)
    gs = gpu_sim(case, FP32)
    osim.step(400)
    gs.step(400)
    _compare_velocity(gs, osim, case)


# ---------------------------------------------- heterogeneous steady states
def _steady_cases():
    body = Case(64, 48, tau=0.8, G=(2e-6, 5e-7), walls=True, forchheimer=1,
                medium=media.random_medium(64, 48, seed=31, eps_range=(0.3, 1.0),
                                           log10_k_range=(-1, 1), kn_range=(0, 2),
                                           p_open=0.1))
    pres = Case(48, 32, tau=0.8, pressure=True, walls=True, rho_in=1.0005, rho_out=0.9995,
                medium=media.two_component(48, seed=7, corr_len=6.0, kn=0.5, ny=32,
                                           matrix=(0.4, 0.1), inclusion=(0.8, 1.0)))
    return {"body_force_random": body, "pressure_two_component": pres}


@pytest.mark.parametrize("name", ["body_force_random", "pressure_two_component"])
@pytest.mark.parametrize("storage", [FP32, FP16])
def test_heterogeneous_steady_state(orc, name, storage):
    case = _steady_cases()[name]
    osim = oracle_sim(orc, case)
    osim.run_to_steady(tol=1e-10, check_every=200, max_steps=400_000)
    gs = gpu_sim(case, storage)
    gs.step(osim.steps)
    if storage == FP32:
        _compare_velocity(gs, osim, case)
    else:
        kg_g, _ = gs.permeability()
        kg_o, _ = osim.permeability()
        _log(e_k=abs(kg_g / kg_o - 1), kg=kg_g, kg_oracle=kg_o, storage="fp16")
        assert abs(kg_g / kg_o - 1) <= 1e-3, (kg_g, kg_o)


# ------------------------------------------------------------- FP16 storage
@pytest.mark.parametrize("rounding", [SR, RN])
def test_fp16_channel_permeability(orc, rounding):
    """Steady channel.  Round-to-nearest repeats the same rounding error at
    every step of a steady state, which the weak damping (eps nu / k_a =
    0.05 per step) amplifies about 20-fold: measured ~3e-3.  Stochastic
    rounding makes the error zero-mean in time: ~1e-5."""
    med = media.channel(64, 33, 0.7, 1e-3, 0.1)
    case = Case(64, 33, tau=0.8, G=(1e-6, 0.0), walls=True, medium=med)
    osim = oracle_sim(orc, case)
    osim.run_to_steady(tol=1e-10, check_every=100)
    gs = gpu_sim(case, FP16, fp16_rounding=rounding)
    gs.step(max(osim.steps, 2000))
    kg_g, _ = gs.permeability()
    kg_o, _ = osim.permeability()
    _log(e_k=abs(kg_g / kg_o - 1), kg=kg_g, kg_oracle=kg_o, storage="fp16",
         rounding="SR" if rounding == SR else "RN")
    assert abs(kg_g / kg_o - 1) <= (1e-3 if rounding == SR else 1e-2), (kg_g, kg_o)


@pytest.mark.parametrize("kn", [0.01, 1.0])
def test_fp16_two_component_permeability(orc, kn):
    case = _two_component_case(kn=kn)
    osim = oracle_sim(orc, case)
    gs = gpu_sim(case, FP16, fp16_rounding=SR)
    osim.step(1000)
    gs.step(1000)
    kg_g, _ = gs.permeability()
    kg_o, _ = osim.permeability()
    _log(e_k=abs(kg_g / kg_o - 1), kg=kg_g, kg_oracle=kg_o, storage="fp16")
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


@pytest.mark.parametrize("storage", [FP32, FP16])
def test_graph_replay_matches_single_launches(storage):
    case = _two_component_case(n=200, ny=50)
    a = gpu_sim(case, storage)
    b = gpu_sim(case, storage)
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


@pytest.mark.parametrize("storage", [FP32, FP16])
@pytest.mark.parametrize("walls,pressure", [(True, True), (False, False), (True, False)])
@pytest.mark.parametrize("nx", [300, 301])
def test_staged_matches_direct(storage, walls, pressure, nx):
    """Same arithmetic in both kernels, every rounding written out: the
    staged kernel's packed node pairs give the direct kernel's one-node
    results bit for bit.  FP16 is compared with round-to-nearest (the
    stochastic streams of the two kernels differ).  An odd width leaves a
    lone last node in every row (stored as a pair with the row padding)."""
    med = media.random_medium(nx, 41, seed=12, p_open=0.1, p_solid=0.1, log10_k_range=(-3, 0))
    case = Case(nx, 41, tau=0.7, G=(1e-5, 0.0), walls=walls, pressure=pressure,
                rho_in=1.001, rho_out=0.999, forchheimer=1, medium=med)
    a = gpu_sim(case, storage, kernel=STAGED, fp16_rounding=RN)
    b = gpu_sim(case, storage, kernel=DIRECT, fp16_rounding=RN)
    a.step(50)
    b.step(50)
    fa, fb = _np(a.populations()), _np(b.populations())
    assert np.array_equal(fa, fb), f"{np.sum(fa != fb)} populations differ"
    ka, _ = a.permeability()
    kb, _ = b.permeability()
    assert ka == kb


@pytest.mark.parametrize("walls,pressure", [(True, True), (False, False)])
@pytest.mark.parametrize("nx", [300, 301])
def test_staged_matches_direct_dynamic_kn(walls, pressure, nx):
    """FP16 with a dynamic Kn: the staged kernel (which stages the Kn plane
    beside the medium) and the direct kernel form f_c(Kn0 p0 / p) node by
    node with the same operations, so the populations agree bit for bit
    (round-to-nearest)."""
    med = media.random_medium(nx, 41, seed=14, p_open=0.1, p_solid=0.1, log10_k_range=(-3, 0),
                              kn_range=(0.0, 5.0))
    case = Case(nx, 41, tau=0.7, G=(1e-5, 0.0), walls=walls, pressure=pressure,
                rho_in=1.001, rho_out=0.999, forchheimer=1, medium=med, kn_beta=100.0)
    a = gpu_sim(case, FP16, kernel=STAGED, fp16_rounding=RN)
    b = gpu_sim(case, FP16, kernel=DIRECT, fp16_rounding=RN)
    assert a.info().bytes_per_update == b.info().bytes_per_update == 48.0
    a.step(50)
    b.step(50)
    fa, fb = _np(a.populations()), _np(b.populations())
    assert np.array_equal(fa, fb), f"{np.sum(fa != fb)} populations differ"
    ka, _ = a.permeability()
    kb, _ = b.permeability()
    assert ka == kb


@pytest.mark.parametrize("storage,kn_beta", [(FP32, 0.0), (FP16, 50.0)])
def test_bounded_wait_reports_timeout(monkeypatch, storage, kn_beta):
    """The staged kernel's waits are bounded: with the copies of one tile
    withheld, the consumers give up after their limit, the host reports
    ETIMEOUT, and the context stays usable.  FP16 with a dynamic Kn runs the
    form that also stages the Kn plane."""
    from paper_1411_7051_gb300 import lbmp
    monkeypatch.setenv("LBMP_TEST_DROP_TILE", "3")
    case = _two_component_case(n=1024, ny=64)
    case.kn_beta = kn_beta
    gs = gpu_sim(case, storage, kernel=STAGED)
    monkeypatch.delenv("LBMP_TEST_DROP_TILE")
    gs.step(1)
    with pytest.raises(lbmp.LbmpError) as ei:
        gs.synchronize()
    assert ei.value.status == lbmp.ETIMEOUT
    ok = gpu_sim(case, storage, kernel=STAGED)   # a fresh context works
    ok.step(5)
    ok.synchronize()


def test_stochastic_rounding_is_seeded():
    case = _two_component_case(n=96, ny=40)
    a = gpu_sim(case, FP16, seed=7)
    b = gpu_sim(case, FP16, seed=7)
    c = gpu_sim(case, FP16, seed=8)
    for s_ in (a, b, c):
        s_.step(40)
    fa, fb, fc = (_np(s_.populations()) for s_ in (a, b, c))
    assert np.array_equal(fa, fb)
    assert not np.array_equal(fa, fc)


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
