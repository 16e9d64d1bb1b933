"""lbmp_permeability_noalloc, the entry point for callers that cannot call
cudaMalloc (code running while another component holds the device in a
stream capture, processes whose device memory belongs to another
framework's pool, latency-bound loops), checked through the C ABI against
lbmp_permeability on the same lattice state, on consecutive calls.

This file is collected last on purpose: when it fails, a run that stops at
the first failure has already run every other test."""
import numpy as np
import pytest

from paper_1411_7051_gb300 import lbmp, media

pytestmark = pytest.mark.gpu

REL = 1e-6  # the FP32 global-permeability tolerance of the parity tests


def _case():
    med = media.two_component(256, seed=2, corr_len=16.0, kn=0.1, ny=128)
    cfg = lbmp.SimConfig(256, 128, tau=0.8, bc_x=lbmp.BCX_PRESSURE, bc_y=lbmp.BCY_WALLS,
                         rho_in=1.0005, rho_out=0.9995, forchheimer=1)
    return med, cfg


def test_noalloc_matches_permeability_on_consecutive_calls():
    import torch
    med, cfg = _case()
    sim = lbmp.Sim(cfg)
    sim.set_fields(med.eps, med.k_i, med.kn)
    eps = torch.tensor(med.eps, device="cuda")
    k_i = torch.tensor(med.k_i, device="cuda")
    kn = torch.tensor(med.kn, device="cuda")
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    previous = None
    for call in range(2):
        sim.step(300)
        f = sim.populations(device=True)
        kg_ref, um_ref = sim.permeability()
        lbmp.permeability_noalloc(cfg, f, eps, k_i, kn, out, stream)
        stream.synchronize()
        kg, um, bad = out.cpu().tolist()
        assert bad == 0.0
        assert abs(kg / kg_ref - 1.0) <= REL, (call, kg, kg_ref)
        assert abs(um / um_ref - 1.0) <= REL, (call, um, um_ref)
        # a second call on the same state reproduces the first exactly
        lbmp.permeability_noalloc(cfg, f, eps, k_i, kn, out, stream)
        stream.synchronize()
        assert out.cpu().tolist() == [kg, um, bad]
        if previous is not None:
            assert kg != previous  # the state moved between the two calls
        previous = kg


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import torch
    cfg = lbmp.SimConfig(4096, 4097)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lbmp.LbmpError) as ei:
        lbmp.permeability_noalloc(cfg, t, t, t, t, t)
    assert ei.value.status == lbmp.EINVAL
    assert "scratch" in str(ei.value)
