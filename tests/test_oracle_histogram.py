"""Pins of the oracle's normalised-velocity histogram (Section IV.B, Fig. 6)
and properties of the trimodal medium generator."""
import numpy as np
import pytest

import pins
from oracle import oracle as orc
from paper_1411_7051_gb300 import media


def test_uniform_flow_fills_last_bin():
    p = orc.make_params(9, 7, tau=0.8, G=(1e-4, 3e-5), forchheimer=1)
    s = orc.OracleSim(p)
    s.set_fields(0.6, 0.5, 0.1)
    s.step(20)
    counts, umax = s.velocity_histogram(10)
    assert counts.sum() == 63 and counts[-1] == 63 and umax > 0


def test_no_flow_fills_first_bin():
    p = orc.make_params(9, 7, tau=0.8, bc_y=orc.BC_WALLS)
    s = orc.OracleSim(p)
    s.set_fields(0.6, 0.5, 0.1)
    s.step(5)
    counts, umax = s.velocity_histogram(7)
    assert umax == 0.0 and counts[0] == 9 * 5 and counts[1:].sum() == 0


def test_channel_histogram_follows_eq20():
    """Steady Brinkman-Darcy channel (Section IV.A): every row of nx nodes
    falls in one bin, and the counts are those of the Eq. 20 profile at the
    node rows, except for rows whose normalised speed lies within the
    profile's discretisation error (2e-2) of a bin edge."""
    nx, ny, eps, tau, G = 64, 33, 0.7, 0.8, 1e-6
    sim = pins.channel_run(orc, nx, ny, eps, 1e-3, 0.1, tau, G)
    nb = 10
    counts, umax = sim.velocity_histogram(nb)
    assert counts.sum() == nx * (ny - 2)
    assert np.all(counts % nx == 0)
    H = ny - 2
    nu = (tau - 0.5) / 3
    K = 1e-3 * H * H * orc.fc(0.1)
    ua = pins.brinkman_profile(G, K, nu, eps, H, np.arange(1, ny - 1) - 0.5)
    u0 = ua / ua.max() * nb
    exp = np.bincount(np.minimum(np.floor(u0).astype(int), nb - 1), minlength=nb) * nx
    near = np.abs(u0 - np.round(u0)) < 2e-2 * nb
    slack = np.zeros(nb, dtype=int)
    for v in u0[near]:
        k = int(np.round(v))
        for b in (k - 1, k):
            if 0 <= b < nb:
                slack[b] += nx
    assert np.all(np.abs(counts - exp) <= slack), (counts, exp)


def test_trimodal_generator():
    lab = media.trimodal(seed=4)
    assert lab.shape == (200, 410)
    frac = [np.mean(lab == k) for k in (media.PORE, media.IMPERMEABLE, media.PERMEABLE)]
    assert frac[1] == pytest.approx(0.4, abs=0.01)
    assert frac[2] == pytest.approx(0.3, abs=1e-4)
    assert np.array_equal(lab, media.trimodal(seed=4))
    assert not np.array_equal(lab, media.trimodal(seed=5))
    m = media.trimodal_medium(lab, 0.5, 0.04, 0.3)
    assert np.all(m.eps[lab == media.PORE] == 1.0) and np.all(np.isinf(m.k_i[lab == media.PORE]))
    assert np.all(m.eps[lab == media.IMPERMEABLE] == 0.0)
    assert np.all(m.kn[lab == media.PERMEABLE] == 0.3)


def test_layered_darcy_flow_bins():
    """Periodic lattice of Darcy layers: row y has k proportional to y + 1/2
    under a strong drag (eps nu / k >= 500 per step), so its steady velocity
    is G k_y / nu to ~1e-4 (the viscous coupling of the layers) and
    u0 = (y + 1/2) / (ny - 1/2).  With ny = 10 rows and 10 bins every row
    falls in a bin of its own, at least 0.05 of a bin from its edges."""
    nx, ny, nb = 4, 10, 10
    k_row = 1e-4 * (np.arange(ny) + 0.5) / ny
    p = orc.make_params(nx, ny, tau=0.8, G=(1e-5, 0.0))
    s = orc.OracleSim(p)
    s.set_fields(0.5, np.repeat(k_row[:, None], nx, axis=1), 0.0)
    s.run_to_steady(tol=1e-12, check_every=200)
    counts, umax = s.velocity_histogram(nb)
    assert list(counts) == [nx] * nb
    nu = (0.8 - 0.5) / 3.0
    assert umax == pytest.approx(1e-5 * k_row[-1] / nu, rel=1e-3, abs=0)
