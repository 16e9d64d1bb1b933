"""The medium precompute (k_a = k_i f_c(Kn), Eq. 3 with Eq. 6-7 or Eq. 4-5)
against the FP64 oracle, node by node, through lbmp_apparent_permeability.

The library stores 1/k_a as an FP32 number.  It forms 1/k_a as one fraction
of k_i and Kn in FP32-pair arithmetic (~44 significant bits), with only
t = Kn^-0.4348 taken from the hardware base-2 logarithm and power (~3e-7
relative), and t enters numerator and denominator alike: the sensitivity
d ln(1/k_a) / d ln t stays below 0.08, so the pair value is within ~2.4e-8
(0.4 FP32 ulp) of the exact one before its final rounding (0.5 ulp).
Bound: 1.3e-7 relative per node (1 ulp and a margin), over Kn = 0 and Kn
from 1e-4 to 1e2 (the regimes of Section II.B).  With a dynamic Kn the step
forms k_a itself with an FP32 f_c (a few FP32 roundings): 5e-7 there.
"""
import json
import os

import numpy as np
import pytest

from paper_1411_7051_gb300 import lbmp, media

pytestmark = pytest.mark.gpu

REL = 1.3e-7
REL_DYNAMIC = 5e-7


def _medium(nx=97, ny=40, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    m = media.random_medium(nx, ny, seed=seed, eps_range=(0.05, 1.0), log10_k_range=(-6, 1),
                            p_open=0.05, p_solid=0.05)
    kn = 10.0 ** rng.uniform(-4, 2, (ny, nx))
    kn[rng.uniform(size=(ny, nx)) < 0.05] = 0.0
    m.kn = kn
    return m


def _log(**kw):
    path = os.environ.get("LBMP_PARITY_LOG")
    if path:
        kw["test"] = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
        with open(path, "a") as fh:
            fh.write(json.dumps(kw) + "\n")


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("kn_model", [lbmp.KN_BKC, lbmp.KN_FIRST_ORDER])
def test_apparent_permeability_against_oracle(orc, kn_model, walls):
    m = _medium()
    ny, nx = m.eps.shape
    cfg = lbmp.SimConfig(nx, ny, bc_y=lbmp.BCY_WALLS if walls else lbmp.BCY_PERIODIC,
                         kn_model=kn_model)
    with lbmp.Sim(cfg) as sim:
        sim.set_fields(m.eps, m.k_i, m.kn)
        ka = sim.apparent_permeability(device=False).numpy()
    fc = orc.fc if kn_model == lbmp.KN_BKC else orc.fc_first_order
    ref = m.k_i * np.vectorize(fc)(m.kn)
    rows = slice(1, ny - 1) if walls else slice(0, ny)
    if walls:
        assert np.all(ka[0] == 0.0) and np.all(ka[-1] == 0.0)
    g, r = ka[rows], ref[rows]
    open_ = np.isinf(r)
    assert np.array_equal(np.isinf(g), open_)
    err = np.abs(g[~open_] / r[~open_] - 1.0)
    _log(max_rel=float(err.max()), rms_rel=float(np.sqrt(np.mean(err ** 2))), kn_model=kn_model)
    assert err.max() <= REL, (err.max(), np.unravel_index(np.argmax(err), err.shape))


def test_apparent_permeability_dynamic_kn_at_reference_pressure(orc):
    m = _medium(seed=5)
    ny, nx = m.eps.shape
    cfg = lbmp.SimConfig(nx, ny, kn_beta=50.0)
    with lbmp.Sim(cfg) as sim:
        sim.set_fields(m.eps, m.k_i, m.kn)
        ka = sim.apparent_permeability(device=False).numpy()
    ref = m.k_i * np.vectorize(orc.fc)(m.kn)
    open_ = np.isinf(ref)
    assert np.array_equal(np.isinf(ka), open_)
    err = np.abs(ka[~open_] / ref[~open_] - 1.0)
    assert err.max() <= REL_DYNAMIC, err.max()


def test_medium_rejects_bad_values_and_keeps_the_mean_porosity(orc):
    """The integer range checks of the precompute: eps outside [0, 1], k_i
    not > 0, Kn negative or not finite, k_a below 1e-15 -- and -0.0 passes
    as 0 -- and the mean porosity that the pressure drop uses: each thread
    sums its nodes' eps in FP32 pairs (~44 significant bits, error below
    1e-12 of the sum), the partial sums meet in FP64."""
    m = media.random_medium(40, 12, seed=2, p_solid=0.1)
    cfg = lbmp.SimConfig(40, 12, bc_x=lbmp.BCX_PRESSURE, rho_in=1.001, rho_out=0.999)
    with lbmp.Sim(cfg) as sim:
        for field, bad in (("eps", 1.0 + 1e-12), ("eps", -1e-300), ("eps", np.nan),
                           ("k_i", 0.0), ("k_i", -np.inf), ("k_i", np.nan), ("k_i", 1e-18),
                           ("kn", -1e-300), ("kn", np.inf), ("kn", np.nan)):
            e, k, n = m.eps.copy(), m.k_i.copy(), m.kn.copy()
            {"eps": e, "k_i": k, "kn": n}[field][5, 7] = bad
            with pytest.raises(lbmp.LbmpError) as ei:
                sim.set_fields(e, k, n)
            assert ei.value.status == lbmp.EINVAL, (field, bad)
        e, n = m.eps.copy(), m.kn.copy()
        e[3, 3] = -0.0
        n[4, 4] = -0.0
        sim.set_fields(e, m.k_i, n)
        assert sim.info().eps_mean == pytest.approx(e.mean(), rel=1e-12, abs=0)


def test_pinned_host_inputs_match_pageable_ones():
    """Pinned, device-mapped host arrays are read by the precompute in place;
    the medium, and the run from it, are those of pageable host arrays."""
    import torch
    m = media.random_medium(130, 40, seed=6, p_open=0.1, p_solid=0.1)
    ny, nx = m.eps.shape
    cfg = lbmp.SimConfig(nx, ny, bc_x=lbmp.BCX_PRESSURE, bc_y=lbmp.BCY_WALLS, rho_in=1.001,
                         rho_out=0.999, forchheimer=1)
    pinned = [torch.from_numpy(np.ascontiguousarray(f)).pin_memory() for f in (m.eps, m.k_i, m.kn)]
    with lbmp.Sim(cfg) as a, lbmp.Sim(cfg) as b:
        a.set_fields(m.eps, m.k_i, m.kn)
        b.set_fields(*pinned)
        assert np.array_equal(a.apparent_permeability(False).numpy(),
                              b.apparent_permeability(False).numpy())
        assert a.info().eps_mean == b.info().eps_mean
        a.step(30)
        b.step(30)
        assert np.array_equal(a.populations(False).numpy(), b.populations(False).numpy())
        bad = pinned[0].clone().pin_memory()
        bad[3, 4] = 2.0   # out of range: rejected as from pageable memory
        with pytest.raises(lbmp.LbmpError) as ei:
            b.set_fields(bad, pinned[1], pinned[2])
        assert ei.value.status == lbmp.EINVAL


@pytest.mark.parametrize("kn_model", [lbmp.KN_BKC, lbmp.KN_FIRST_ORDER])
def test_apparent_permeability_at_the_range_edges(orc, kn_model):
    """k_i and Kn at and around the edges of the FP32-pair evaluation
    (k_i in [1e-16, 1e12], Kn 0 or in [1e-12, 1e6]; outside them the
    precompute takes the FP64 fraction), one ulp either side of each edge,
    and the extremes it accepts: the same 1.3e-7 bound on both sides."""
    up, dn = (lambda v: np.nextafter(v, np.inf)), (lambda v: np.nextafter(v, 0.0))
    ks = [1e-14, dn(1e-16) * 100, 1e-16 * 100, 1e-12, 1.0, dn(1e12), 1e12, up(1e12), 1e13,
          1e15, 3.7e-9]
    kns = [0.0, 1e-14, dn(1e-12), 1e-12, up(1e-12), 1e-7, 0.5, 1.0, 3e3, dn(1e6), 1e6,
           up(1e6), 1e7, 1e9]
    # k_i = 1e-16 itself would give k_a below the 1e-15 floor; the pair path's
    # lower edge is crossed with Kn large enough that k_a stays above it
    kk = np.array([[k for k in ks] for _ in kns])
    nn = np.array([[n for _ in ks] for n in kns])
    edge = np.array([dn(1e-16), 1e-16, up(1e-16)])
    kk = np.vstack([kk, np.tile(edge, (1, len(ks)))[:, :len(ks)]])
    nn = np.vstack([nn, np.full((1, len(ks)), 1e3)])
    ny, nx = kk.shape
    eps = np.full((ny, nx), 0.4)
    fc = orc.fc if kn_model == lbmp.KN_BKC else orc.fc_first_order
    ref = kk * np.vectorize(fc)(nn)
    ok = ref >= 1e-15 * (1 + 1e-6)
    kk[~ok] = 1.0   # below the floor the medium is rejected (tested elsewhere)
    ref = kk * np.vectorize(fc)(nn)
    cfg = lbmp.SimConfig(nx, ny, kn_model=kn_model)
    with lbmp.Sim(cfg) as sim:
        sim.set_fields(eps, kk, nn)
        ka = sim.apparent_permeability(device=False).numpy()
    err = np.abs(ka / ref - 1.0)
    _log(max_rel=float(err.max()), kn_model=kn_model)
    assert err.max() <= REL, (err.max(), kk.flat[np.argmax(err)], nn.flat[np.argmax(err)])
