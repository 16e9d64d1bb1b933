"""Parity at full size, in the launch configuration bench.py times.

At 4096 x 4096 the oracle cannot run the lattice, so one time step is checked
on sampled nodes: from the GPU's own state at level K (downloaded exactly,
FP64), the oracle's single-node collision of the nine upstream neighbours
gives the populations of level K + 1 at each sampled node, which must match
the GPU's.  Interior columns only (the pressure columns are covered by the
small-lattice tests).  Also checked: the largest row count the API accepts,
and a lattice whose population planes lie beyond 2^31 elements.
"""
import numpy as np
import pytest

from paper_1411_7051_gb300 import lbmp, media

pytestmark = pytest.mark.gpu

EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]


def _sampled_one_step(orc, sim, cfg, med, storage, nsamp=1500, seed=0, kn_beta=0.0):
    import torch
    ny, nx = med.eps.shape
    rng = np.random.default_rng(seed)
    y0 = 1 if cfg.bc_y == lbmp.BCY_WALLS else 0
    ys = rng.integers(y0, ny - y0, nsamp)
    xs = rng.integers(2, nx - 2, nsamp)
    # the 3 x 3 neighbourhoods of the samples, from the device copy of f(K)
    fK = sim.populations(device=True)
    yy = (ys[:, None] + np.array([-1, 0, 1])[None, :]) % ny
    xx = xs[:, None] + np.array([-1, 0, 1])[None, :]
    ty = torch.as_tensor(yy, device="cuda")
    tx = torch.as_tensor(xx, device="cuda")
    patch = fK[:, ty[:, :, None], tx[:, None, :]].cpu().numpy()  # [9, n, 3, 3]
    del fK
    sim.step(1)
    f1 = sim.populations(device=True)
    got = f1[:, torch.as_tensor(ys, device="cuda"), torch.as_tensor(xs, device="cuda")].cpu().numpy().T
    del f1
    params = orc.make_params(nx, ny, tau=cfg.tau, G=cfg.G,
                             bc_x=orc.BC_PRESSURE if cfg.bc_x else orc.BC_PERIODIC,
                             bc_y=orc.BC_WALLS if cfg.bc_y else orc.BC_PERIODIC,
                             rho_in=cfg.rho_in, rho_out=cfg.rho_out,
                             forchheimer=cfg.forchheimer)

    def ka_of(f, sy, sx):
        """k_a of a source node: static, or with a dynamic Kn at the pressure
        of its own post-stream state f (p / p0 = 1 + beta (rho - rho0))."""
        if kn_beta == 0.0:
            return med.k_i[sy, sx] * orc.fc(med.kn[sy, sx])
        q = 1.0 + kn_beta * (float(np.sum(f)) - 1.0)
        return med.k_i[sy, sx] * orc.fc(med.kn[sy, sx] / q)
    exp = np.zeros_like(got)
    opp = [0, 3, 4, 1, 2, 7, 8, 5, 6]
    for n in range(nsamp):
        for i in range(9):
            sy = ys[n] - EY[i]
            if cfg.bc_y == lbmp.BCY_WALLS and sy in (0, ny - 1):
                post = orc.collide_node(patch[:, n, 1, 1], med.eps[ys[n], xs[n]],
                                        ka_of(patch[:, n, 1, 1], ys[n], xs[n]), params)
                exp[n, i] = post[opp[i]]
                continue
            sy %= ny
            sx = xs[n] - EX[i]
            src = patch[:, n, 1 - EY[i], 1 - EX[i]]
            post = orc.collide_node(src, med.eps[sy, sx], ka_of(src, sy, sx), params)
            exp[n, i] = post[i]
    _, _, w = orc.lattice()
    dev = np.abs(exp - w[None, :])
    err = np.abs(got - exp)
    if storage == lbmp.STORE_FP32:
        assert err.max() <= 2e-9, err.max()
    else:
        assert np.all(err <= dev * 2.0 ** -10 + 1e-10), (err / (dev + 1e-30)).max()


@pytest.mark.parametrize("storage,dynamic", [(lbmp.STORE_FP32, False), (lbmp.STORE_FP16, False),
                                             (lbmp.STORE_FP32, True), (lbmp.STORE_FP16, True)])
def test_bench_workload_sampled_step(orc, storage, dynamic):
    """The bench workload (4096^2 fractured shale, pressure x, periodic y,
    Forchheimer), AUTO kernel selection as timed by bench.py; also its
    dynamic-Kn variant (inlet pressure twice the outlet one)."""
    import bench
    med, c = bench.workload(4096)
    beta = bench.kn_beta_for(c) if dynamic else 0.0
    cfg = lbmp.SimConfig(c["nx"], c["ny"], tau=c["tau"], bc_x=c["bc_x"], bc_y=c["bc_y"],
                         rho_in=c["rho_in"], rho_out=c["rho_out"], forchheimer=c["forchheimer"],
                         storage=storage, kn_beta=beta)
    with lbmp.Sim(cfg) as sim:
        sim.set_fields(med.eps, med.k_i, med.kn)
        sim.step(64)   # two graph replays: the timed path
        _sampled_one_step(orc, sim, cfg, med, storage, kn_beta=beta)
        kg, _ = sim.permeability()
        assert np.isfinite(kg)


@pytest.mark.parametrize("storage", [lbmp.STORE_FP32, lbmp.STORE_FP16])
def test_largest_row_count(orc, storage):
    """ny = 65535 (the largest the C ABI accepts) with walls, body force."""
    nx, ny = 64, 65535
    med = media.random_medium(nx, ny, seed=77, log10_k_range=(-3, 0), p_open=0.1, p_solid=0.05)
    cfg = lbmp.SimConfig(nx, ny, tau=0.75, G=(1e-5, 2e-6), bc_y=lbmp.BCY_WALLS,
                         forchheimer=1, storage=storage)
    with lbmp.Sim(cfg) as sim:
        sim.set_fields(med.eps, med.k_i, med.kn)
        sim.step(40)
        _sampled_one_step(orc, sim, cfg, med, storage, nsamp=800, seed=3)


@pytest.fixture(scope="module")
def medium_16k():
    n = 16384
    return media.random_medium(n, n, seed=93, log10_k_range=(-3, 0), p_open=0.02, p_solid=0.02)


@pytest.mark.parametrize("storage", [lbmp.STORE_FP32, lbmp.STORE_FP16])
def test_offsets_beyond_int32(orc, medium_16k, storage):
    """16384 x 16384 (row pitch 16448): a population buffer's nine planes span
    2.4e9 elements, so every update reads and writes plane offsets above 2^31
    elements (above 2^32 bytes), and a staged launch walks 131 000 tiles.
    Pressure x, plates y, Forchheimer, AUTO kernel: one step on sampled nodes
    against the oracle after 8 steps, and the mean velocity of
    lbmp_permeability against the FP64 sum of the velocity field that
    lbmp_macroscopic (another kernel) reports over the fluid rows."""
    import torch
    med = medium_16k
    ny, nx = med.eps.shape
    cfg = lbmp.SimConfig(nx, ny, tau=0.8, bc_x=lbmp.BCX_PRESSURE, bc_y=lbmp.BCY_WALLS,
                         rho_in=1.002, rho_out=0.998, forchheimer=1, storage=storage)
    with lbmp.Sim(cfg) as sim:
        sim.set_fields(med.eps, med.k_i, med.kn)
        sim.step(8)
        _sampled_one_step(orc, sim, cfg, med, storage, nsamp=1500, seed=5)
        kg, um = sim.permeability()
        _, ux, _ = sim.macroscopic(device=True)
        ref = float(ux[1:ny - 1].sum(dtype=torch.float64)) / (nx * (ny - 2))
        del ux
    assert np.isfinite(kg) and kg > 0.0
    assert um == pytest.approx(ref, rel=1e-9, abs=0), (um, ref)
