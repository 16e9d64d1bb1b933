"""lbmp_permeability_noalloc, the entry point for callers that cannot call
cudaMalloc (processes whose device memory belongs to another framework's
pool, latency-bound loops that may not pay for an allocation), checked
through the C ABI against lbmp_permeability on the same lattice state, on
consecutive calls, with the device's free memory unchanged by a call.

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
        torch.cuda.synchronize()
        held, free = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
        lbmp.permeability_noalloc(cfg, f, eps, k_i, kn, out, stream)
        stream.synchronize()
        if call > 0:   # the first call may load the kernels' code on the device
            assert torch.cuda.memory_allocated() == held
            assert torch.cuda.mem_get_info()[0] == free
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


def _c_call(cfg, t):
    """The C entry point itself, every array pointing at the tensor t; only
    for calls that the entry point rejects before any launch."""
    import ctypes
    import torch
    params = cfg.to_params(None)
    p = ctypes.c_void_p(t.data_ptr())
    return lbmp.load().lbmp_permeability_noalloc(
        ctypes.byref(params), p, p, p, p, p,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import torch
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _c_call(lbmp.SimConfig(4096, 4097), t) == lbmp.EINVAL
    assert "scratch" in lbmp.last_error()


def test_noalloc_binding_checks_sizes_before_any_launch():
    import torch
    nx, ny = 64, 32
    cfg = lbmp.SimConfig(nx, ny)
    z = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda")   # noqa: E731
    with pytest.raises(ValueError):
        lbmp.permeability_noalloc(cfg, z(9 * nx * ny - 1), z(nx * ny), z(nx * ny), z(nx * ny), z(3))
    with pytest.raises(ValueError):
        lbmp.permeability_noalloc(cfg, z(9 * nx * ny), z(nx * ny), z(nx * ny - 1), z(nx * ny), z(3))
    with pytest.raises(ValueError):
        lbmp.permeability_noalloc(cfg, z(9 * nx * ny), z(nx * ny), z(nx * ny), z(nx * ny), z(2))
