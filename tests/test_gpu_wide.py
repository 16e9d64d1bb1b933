"""The vectorised FP16 step kernel (LBMP_KERNEL_WIDE) against the staged and
direct kernels.  All three apply the same FP32 arithmetic (lattice.cuh) and
the wide and staged kernels draw the same stochastic-rounding word per node
pair, so their FP16 states agree bit for bit; under round-to-nearest the
direct kernel agrees too.  Shapes cover ragged row ends (nx not a multiple
of 4), rows narrower than one thread's span, every boundary kind, and the
dynamic Knudsen number."""
import numpy as np
import pytest

from paper_1411_7051_gb300 import lbmp, media
from helpers import Case, gpu_sim

pytestmark = pytest.mark.gpu

FP16 = lbmp.STORE_FP16
SR, RN = lbmp.ROUND_STOCHASTIC, lbmp.ROUND_NEAREST


def _np(t):
    return t.detach().cpu().numpy()


SHAPES = [(131, 37), (300, 9), (1, 5), (2, 3), (5, 1), (257, 6), (3, 4), (64, 64), (1030, 3),
          (4097, 2)]
BCS = {"periodic": dict(walls=False, pressure=False, forchheimer=0),
       "walls_forch": dict(walls=True, pressure=False, forchheimer=1),
       "pressure_walls": dict(walls=True, pressure=True, forchheimer=1),
       "pressure_periodic": dict(walls=False, pressure=True, forchheimer=0)}


def _run(case, kernel, rounding, f0, steps=3, seed=7):
    with gpu_sim(case, FP16, fp16_rounding=rounding, seed=seed, kernel=kernel) as s:
        s.set_populations(f0)
        out = []
        for _ in range(steps):
            s.step(1)
            out.append(_np(s.populations()))
        s.step(40)   # graph replays
        out.append(_np(s.populations()))
        return out


@pytest.mark.parametrize("rounding", [SR, RN])
@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("nx,ny", SHAPES)
def test_wide_matches_staged(orc, nx, ny, bc, rounding):
    kw = BCS[bc]
    if kw["walls"] and ny < 3 or kw["pressure"] and nx < 3:
        pytest.skip("lattice too small for this boundary kind")
    med = media.random_medium(nx, ny, seed=nx + 3 * ny, p_open=0.15, p_solid=0.1,
                              log10_k_range=(-3, 0))
    case = Case(nx, ny, tau=0.7, G=(3e-5, -1e-5), rho_in=1.001, rho_out=0.999, medium=med, **kw)
    _, _, w = orc.lattice()
    f0 = media.random_populations(nx, ny, seed=3, base=w, amp=2e-3)
    a = _run(case, lbmp.KERNEL_WIDE, rounding, f0)
    b = _run(case, lbmp.KERNEL_STAGED, rounding, f0)
    for fa, fb in zip(a, b):
        bad = np.argwhere(fa != fb)
        assert bad.size == 0, (len(bad), bad[:8].tolist())
    if rounding == RN:
        c = _run(case, lbmp.KERNEL_DIRECT, rounding, f0)
        for fa, fc in zip(a, c):
            assert np.array_equal(fa, fc)


@pytest.mark.parametrize("nx,ny", [(131, 37), (257, 6)])
def test_wide_dynamic_kn(orc, nx, ny):
    med = media.random_medium(nx, ny, seed=5, p_open=0.1, p_solid=0.1, log10_k_range=(-3, 0),
                              kn_range=(0, 5))
    case = Case(nx, ny, tau=0.7, pressure=True, walls=True, rho_in=1.001, rho_out=0.999,
                forchheimer=1, medium=med, kn_beta=300.0)
    _, _, w = orc.lattice()
    f0 = media.random_populations(nx, ny, seed=3, base=w, amp=2e-3)
    a = _run(case, lbmp.KERNEL_WIDE, RN, f0)
    c = _run(case, lbmp.KERNEL_DIRECT, RN, f0)
    for fa, fc in zip(a, c):
        assert np.array_equal(fa, fc)


def test_wide_rejects_fp32():
    cfg = lbmp.SimConfig(8, 8, kernel=lbmp.KERNEL_WIDE)
    with pytest.raises(lbmp.LbmpError) as e:
        lbmp.Sim(cfg)
    assert e.value.status == lbmp.EINVAL
