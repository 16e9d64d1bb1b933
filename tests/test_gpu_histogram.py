"""Normalised-velocity histogram (Fig. 6) on the GPU and the trimodal medium
of Section IV.B.

The bin of a node is an integer decided in floating point: the GPU decides
it from its own FP32 velocity (in FP64, each operation rounded), so the
histogram is checked bit for bit against the same decision replayed on the
host from the velocity lbmp_macroscopic returns, and against the oracle's
histogram up to the nodes whose normalised speed lies within the velocity
tolerance of a bin edge (those may fall on either side)."""
import numpy as np
import pytest

from paper_1411_7051_gb300 import lbmp, media
from helpers import Case, fluid_rows, gpu_sim, oracle_sim, rel_l2

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _replay(gs, case, nbins):
    _, ux, uy = gs.macroscopic()
    fr = fluid_rows(case)
    ux, uy = _np(ux)[fr], _np(uy)[fr]
    sp = np.sqrt(ux * ux + uy * uy)
    um = sp.max()
    if um == 0.0:
        return np.bincount(np.zeros(sp.size, int), minlength=nbins), um
    k = np.minimum(np.floor(sp / um * nbins), nbins - 1).astype(int)
    return np.bincount(k.ravel(), minlength=nbins), um


def _against_oracle(counts, osim, case, nbins, rel_u):
    oc, oum = osim.velocity_histogram(nbins)
    _, oux, ouy = osim.macroscopic()
    fr = fluid_rows(case)
    u0 = np.sqrt(oux[fr] ** 2 + ouy[fr] ** 2) / oum * nbins
    near = np.abs(u0 - np.round(u0)) < 4 * rel_u * nbins
    slack = np.zeros(nbins, dtype=np.int64)
    for v in u0[near]:
        k = int(np.round(v))
        for b in (k - 1, k):
            if 0 <= b < nbins:
                slack[b] += 1
    assert counts.sum() == oc.sum()
    assert np.all(np.abs(counts - oc) <= slack), (counts, oc, slack)


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("nbins", [10, 1, 64])
def test_histogram_replay_and_oracle(orc, storage, nbins):
    med = media.random_medium(150, 70, seed=21, p_open=0.2, p_solid=0.2, log10_k_range=(-2, 1))
    case = Case(150, 70, tau=0.8, G=(2e-5, 4e-6), pressure=True, walls=True, rho_in=1.0005,
                rho_out=0.9995, forchheimer=1, medium=med)
    gs = gpu_sim(case, storage)
    gs.step(500)
    counts, um = gs.velocity_histogram(nbins)
    rc, rum = _replay(gs, case, nbins)
    assert um == rum
    assert np.array_equal(counts, rc)
    assert counts.sum() == case.nx * (case.ny - 2)
    if storage == 0:
        osim = oracle_sim(orc, case)
        osim.step(500)
        _against_oracle(counts, osim, case, nbins, rel_u=1e-5)


def test_histogram_edge_cases():
    med = media.random_medium(40, 20, seed=2)
    case = Case(40, 20, tau=0.8, walls=True, medium=med)  # no drive: u = 0
    with gpu_sim(case) as gs:
        gs.step(3)
        counts, um = gs.velocity_histogram(10)
        assert um == 0.0 and counts[0] == 40 * 18 and counts[1:].sum() == 0
        for bad in (0, 65):
            with pytest.raises(lbmp.LbmpError) as e:
                gs.velocity_histogram(bad)
            assert e.value.status == lbmp.EINVAL


def _trimodal_case(lib_side: bool, orc, lam: float, eps_ps: float = 0.5):
    """Section IV.B: 410 x 200 trimodal medium at 10 nm resolution, permeable
    solids with Kozeny-Carman k_d (d = 40 nm, Eq. 9) and Kn = lambda / r
    (Eq. 10-11); pressure drive in x, periodic in y, tau 0.9 (Section IV.A).
    The GPU side builds its fields with the library's host functions, the
    oracle side with the oracle's."""
    lab = media.trimodal(seed=4)
    eps = media.trimodal_medium(lab, eps_ps, 1.0, 0.0).eps
    if lib_side:
        k_i, kn = lbmp.physical_medium(eps, 40e-9, lam, 10e-9)
    else:
        kd = orc.kozeny_carman(eps_ps, 40e-9)
        k_i = kd / 1e-16
        kn = lam / orc.pore_radius(kd, eps_ps)
    med = media.trimodal_medium(lab, eps_ps, k_i, kn)
    return Case(410, 200, tau=0.9, pressure=True, rho_in=1.0005, rho_out=0.9995, medium=med)


@pytest.mark.parametrize("lam", [0.38e-9, 10.26e-9])
def test_trimodal_section_4b(orc, lam):
    gcase = _trimodal_case(True, orc, lam)
    ocase = _trimodal_case(False, orc, lam)
    np.testing.assert_allclose(gcase.medium.k_i, ocase.medium.k_i, rtol=1e-14)
    np.testing.assert_allclose(gcase.medium.kn, ocase.medium.kn, rtol=1e-14)
    gs = gpu_sim(gcase, 0)
    osim = oracle_sim(orc, ocase)
    gs.step(1500)
    osim.step(1500)
    _, gux, guy = gs.macroscopic()
    _, oux, ouy = osim.macroscopic()
    e_u = rel_l2(np.stack([_np(gux), _np(guy)]), np.stack([oux, ouy]))
    kg, _ = gs.permeability()
    ko, _ = osim.permeability()
    assert e_u <= 1e-5, e_u
    assert abs(kg / ko - 1) <= 1e-6, (kg, ko)
    counts, _ = gs.velocity_histogram(10)
    _against_oracle(counts, osim, gcase, 10, rel_u=1e-5)
