"""Host functions of the library for the physical inputs of Kn (Eq. 9-11)
and the correction factors (Eq. 4-7), against the oracle's (no GPU)."""
import math

import numpy as np
import pytest

from paper_1411_7051_gb300 import build, lbmp


@pytest.fixture(scope="module")
def L():
    build.build()
    return lbmp.load()


def test_formulas_match_oracle(L, orc):
    for eps in (0.02, 0.3, 0.75):
        for d in (40e-9, 2e-6):
            assert lbmp.kozeny_carman(eps, d) == pytest.approx(orc.kozeny_carman(eps, d), rel=1e-14, abs=0)
    for k_d in (1e-22, 5e-17, 1e-12):
        for eps in (0.05, 0.5):
            assert lbmp.pore_radius(k_d, eps) == pytest.approx(orc.pore_radius(k_d, eps), rel=1e-14, abs=0)
    for mu, p in ((1.4e-5, 689475.0), (2.0e-5, 2.76e7)):
        assert lbmp.mean_free_path(mu, p, 323.0, 16e-3) == pytest.approx(
            orc.mean_free_path(mu, p, 323.0, 16e-3), rel=1e-14, abs=0)
    for kn in (0.0, 1e-4, 0.3, 5.0):
        assert lbmp.fc_model(lbmp.KN_BKC, kn) == pytest.approx(orc.fc(kn), rel=1e-15, abs=0)
        assert lbmp.fc_model(lbmp.KN_FIRST_ORDER, kn) == pytest.approx(orc.fc_first_order(kn), rel=1e-15, abs=0)
    assert math.isnan(lbmp.fc_model(7, 0.1))
    assert math.isnan(lbmp.kozeny_carman(1.0, 1e-6))
    assert math.isnan(lbmp.mean_free_path(0.0, 1e5, 300.0, 0.016))
    assert math.isnan(lbmp.pore_radius(1e-18, 0.0))


def test_physical_medium(L, orc):
    rng = np.random.default_rng(5)
    eps = rng.uniform(0.02, 0.95, (6, 7))
    eps[0, 0] = 0.0
    eps[1, 2] = 1.0
    d = rng.uniform(20e-9, 200e-9, eps.shape)
    lam, dx = 1.09e-9, 10e-9
    k_i, kn = lbmp.physical_medium(eps, d, lam, dx)
    assert k_i[0, 0] == 1.0 and kn[0, 0] == 0.0
    assert math.isinf(k_i[1, 2]) and kn[1, 2] == 0.0
    for (y, x), e in np.ndenumerate(eps):
        if 0.0 < e < 1.0:
            kd = orc.kozeny_carman(e, d[y, x])
            assert k_i[y, x] == pytest.approx(kd / dx ** 2, rel=1e-14, abs=0)
            assert kn[y, x] == pytest.approx(lam / orc.pore_radius(kd, e), rel=1e-14, abs=0)
    # scalar grain diameter
    k2, kn2 = lbmp.physical_medium(eps, 40e-9, lam, dx)
    assert k2.shape == eps.shape
    with pytest.raises(lbmp.LbmpError):
        lbmp.physical_medium(eps + 1.0, d, lam, dx)
    with pytest.raises(lbmp.LbmpError):
        lbmp.physical_medium(eps, -d, lam, dx)
    with pytest.raises(lbmp.LbmpError):
        lbmp.physical_medium(eps, d, lam, 0.0)


def test_fig1_pipeline_trends(L):
    """Section IV.A, Fig. 1 through the library: d = 40 nm and the printed
    mean free paths at 4000 / 1000 / 100 psi; Kn falls with porosity and
    rises as the pressure drops, and so does f_c."""
    eps = np.linspace(0.02, 0.9, 30)
    prev = None
    for lam in (0.38e-9, 1.09e-9, 10.26e-9):
        _, kn = lbmp.physical_medium(eps, 40e-9, lam, 1e-8)
        fc = np.array([lbmp.fc(k) for k in kn])
        assert np.all(np.diff(kn) < 0) and np.all(np.diff(fc) < 0)
        if prev is not None:
            assert np.all(kn > prev)
        prev = kn
