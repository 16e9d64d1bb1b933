"""C ABI: the library loads, exports every function the header declares,
and validates parameters before touching a GPU (no GPU needed)."""
import ctypes
import math

import pytest

from paper_1411_7051_gb300 import build, lbmp


@pytest.fixture(scope="module")
def L():
    build.build()
    return lbmp.load()


def test_exports_every_declared_function(L):
    names = lbmp.header_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/lbmp.h but not exported"


def test_every_declaration_is_documented():
    """Each function include/lbmp.h declares is preceded by its own comment
    (what it computes, its arguments' meaning and layout, ownership, errors)."""
    import re
    with open(lbmp.HEADER) as fh:
        lines = fh.read().splitlines()
    for name in lbmp.header_functions():
        i = next(k for k, l in enumerate(lines)
                 if re.search(r"\b%s\s*\(" % name, l) and not l.lstrip().startswith(("*", "/*")))
        assert lines[i - 1].rstrip().endswith("*/"), f"{name} has no comment of its own"


def test_fc_host_function(L, orc):
    # library's host f_c against the oracle's (Eq. 6-7)
    for kn in (0.0, 1e-6, 1e-3, 0.1, 0.339, 1.0, 9.16, 10.0, 1e4):
        assert lbmp.fc(kn) == pytest.approx(orc.fc(kn), rel=1e-15, abs=0)
    assert math.isnan(lbmp.fc(-1.0))
    assert math.isnan(lbmp.fc(float("nan")))


def _create(L, **kw):
    cfg = lbmp.SimConfig(**{"nx": 8, "ny": 8, **kw})
    p = cfg.to_params(None)
    h = ctypes.c_void_p()
    st = L.lbmp_create(ctypes.byref(p), ctypes.byref(h))
    if st == lbmp.OK:
        L.lbmp_destroy(h)
    return st, L.lbmp_last_error().decode()


@pytest.mark.parametrize("kw,needle", [
    ({"nx": 0}, "nx, ny"),
    ({"ny": -3}, "nx, ny"),
    ({"ny": 70000}, "ny must be"),
    ({"tau": 0.5}, "tau"),
    ({"tau": float("nan")}, "tau"),
    ({"J": -1.0}, "J"),
    ({"G": (float("inf"), 0.0)}, "G must"),
    ({"bc_x": 7}, "bc_x"),
    ({"bc_y": 2}, "bc_y"),
    ({"bc_x": lbmp.BCX_PRESSURE, "nx": 2}, "nx >= 3"),
    ({"bc_x": lbmp.BCX_PRESSURE, "rho_in": 0.0}, "rho_in"),
    ({"bc_y": lbmp.BCY_WALLS, "ny": 2}, "ny >= 3"),
    ({"forchheimer": 2}, "forchheimer"),
    ({"storage": 5}, "storage"),
    ({"fp16_log2_scale": 100}, "fp16_log2_scale"),
    ({"fp16_rounding": 3}, "fp16_rounding"),
    ({"kn_model": 2}, "kn_model"),
    ({"kn_beta": float("nan")}, "kn_beta"),
    ({"kn_beta": 10.0, "kernel": lbmp.KERNEL_STAGED}, "direct kernel"),
    ({"kn_beta": 1000.0, "bc_x": lbmp.BCX_PRESSURE, "rho_in": 1.0, "rho_out": 0.998},
     "non-positive pressure"),
])
def test_create_rejects_bad_parameters(L, kw, needle):
    st, msg = _create(L, **kw)
    assert st == lbmp.EINVAL, (st, msg)
    assert needle in msg


def test_null_arguments(L):
    assert L.lbmp_create(None, None) == lbmp.EINVAL
    assert L.lbmp_destroy(None) == lbmp.OK
    assert L.lbmp_step(None, 1) == lbmp.EINVAL
    assert L.lbmp_get_info(None, None) == lbmp.EINVAL


@pytest.mark.parametrize("sizes,kw,needle", [
    ([], {}, "count must be"),
    ([(64, 32), (0, 16)], {}, "nx, ny"),
    ([(64, 32), (40, 70000)], {}, "ny must be"),
    ([(64, 32)], {"kn_beta": 5.0}, "dynamic Kn"),
    ([(64, 32)], {"tau": 0.4}, "tau"),
    ([(64, 32), (2, 16)], {"bc_x": lbmp.BCX_PRESSURE}, "nx >= 3"),
    ([(64, 32), (16, 2)], {"bc_y": lbmp.BCY_WALLS}, "ny >= 3"),
])
def test_batch_create_rejects_bad_parameters(L, sizes, kw, needle):
    """lbmp_batch_create checks the count and every instance under the rules
    of lbmp_create before anything is allocated (no GPU needed)."""
    p = lbmp.SimConfig(**{"nx": 1, "ny": 1, **kw}).to_params(None)
    n = len(sizes)
    nx = (ctypes.c_int32 * max(n, 1))(*[s[0] for s in sizes])
    ny = (ctypes.c_int32 * max(n, 1))(*[s[1] for s in sizes])
    h = ctypes.c_void_p()
    st = L.lbmp_batch_create(ctypes.byref(p), n, nx, ny, ctypes.byref(h))
    assert st == lbmp.EINVAL, (st, lbmp.last_error())
    assert needle in lbmp.last_error()
    assert not h.value


@pytest.mark.parametrize("kw,needle", [
    ({"kn_model": 7}, "kn_model"),
    ({"bc_x": 5}, "bc_x"),
    ({"bc_y": -1}, "bc_y"),
    ({"J": -1.0}, "J"),
    ({"tau": 0.5}, "tau"),
    ({"bc_x": lbmp.BCX_PRESSURE, "rho_in": 1.01, "rho_out": 0.99, "kn_beta": -200.0},
     "non-positive pressure"),
    ({"bc_y": lbmp.BCY_WALLS, "ny": 2}, "ny >= 3"),
])
def test_noalloc_rejects_what_create_rejects(L, kw, needle):
    """lbmp_permeability_noalloc checks the parameters it reads as
    lbmp_create does, before any CUDA call (the pointers are never used)."""
    cfg = lbmp.SimConfig(**{"nx": 64, "ny": 32, **kw})
    p = cfg.to_params(None)
    dummy = (ctypes.c_double * 4)()
    ptr = ctypes.cast(dummy, ctypes.c_void_p)
    st = L.lbmp_permeability_noalloc(ctypes.byref(p), ptr, ptr, ptr, ptr, ptr, None)
    assert st == lbmp.EINVAL
    assert needle in lbmp.last_error()


def test_noalloc_binding_checks_sizes_first():
    """The binding checks the sizes the C entry point cannot see before it
    needs a GPU: arrays one element short raise ValueError."""
    import torch
    nx, ny = 16, 8
    cfg = lbmp.SimConfig(nx, ny)
    z = lambda n: torch.zeros(n, dtype=torch.float64)   # noqa: E731
    good = [z(9 * nx * ny), z(nx * ny), z(nx * ny), z(nx * ny), z(3)]
    for k in range(5):
        args = list(good)
        args[k] = z(good[k].numel() - 1)
        with pytest.raises(ValueError):
            lbmp.permeability_noalloc(cfg, *args)
    with pytest.raises(TypeError):   # right sizes, but host tensors
        lbmp.permeability_noalloc(cfg, *good)
