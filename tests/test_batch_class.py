"""Host logic of the batch autotuner's shape cache: the class key under which
a tuned launch shape is reused (lbmp_batch_class; no GPU needed)."""
import pytest

from paper_1411_7051_gb300 import lbmp


def _cfg(**kw):
    base = dict(storage=lbmp.STORE_FP16, fp16_rounding=lbmp.ROUND_STOCHASTIC,
                bc_x=lbmp.BCX_PRESSURE, bc_y=lbmp.BCY_WALLS, forchheimer=1)
    base.update(kw)
    return lbmp.SimConfig(1, 1, **base)


SIZES = [(256, 256)] * 3 + [(1024, 1024)]


def test_key_ignores_instance_order():
    assert lbmp.batch_class(_cfg(), SIZES, 152) == lbmp.batch_class(_cfg(), SIZES[::-1], 152)


def test_key_fields():
    # 3 x 256^2 + 1024^2 = 1 245 184 nodes: floor(log2) = 20; the 1024-wide
    # instance holds most nodes, so the node-weighted median width class is
    # ceil(log2 1024) = 10
    assert lbmp.batch_class(_cfg(), SIZES, 152) == "s1-r1-x1-y1-f1-n10-t20-m152"
    # thirty 256^2 instances outweigh one 1024^2: class 8, 3 014 656 nodes
    assert lbmp.batch_class(_cfg(), [(256, 256)] * 30 + [(1024, 1024)], 152) == \
        "s1-r1-x1-y1-f1-n8-t21-m152"
    # a width between powers of two takes the next one up
    assert "-n9-" in lbmp.batch_class(_cfg(), [(300, 10)], 152)


@pytest.mark.parametrize("kw", [dict(storage=lbmp.STORE_FP32), dict(fp16_rounding=lbmp.ROUND_NEAREST),
                                dict(bc_x=lbmp.BCX_PERIODIC), dict(bc_y=lbmp.BCY_PERIODIC),
                                dict(forchheimer=0)])
def test_key_separates_physics_that_changes_the_kernel(kw):
    assert lbmp.batch_class(_cfg(**kw), SIZES, 152) != lbmp.batch_class(_cfg(), SIZES, 152)


def test_key_separates_devices_and_sizes():
    k = lbmp.batch_class(_cfg(), SIZES, 152)
    assert lbmp.batch_class(_cfg(), SIZES, 148) != k
    assert lbmp.batch_class(_cfg(), [(256, 256)] * 4, 152) != k


def test_fp32_rounding_mode_is_not_part_of_the_key():
    a = lbmp.batch_class(_cfg(storage=lbmp.STORE_FP32), SIZES, 152)
    b = lbmp.batch_class(_cfg(storage=lbmp.STORE_FP32, fp16_rounding=lbmp.ROUND_NEAREST), SIZES, 152)
    assert a == b


@pytest.mark.parametrize("sizes,nsm,needle", [([], 152, "count"), ([(0, 4)], 152, "nx, ny"),
                                              ([(4, 4)], 0, "nsm")])
def test_key_rejects_bad_arguments(sizes, nsm, needle):
    with pytest.raises(lbmp.LbmpError, match=needle):
        lbmp.batch_class(_cfg(), sizes, nsm)


def test_key_buffer_too_small():
    import ctypes
    L = lbmp.load()
    prm = _cfg().to_params(None)
    nx = (ctypes.c_int32 * 1)(64)
    ny = (ctypes.c_int32 * 1)(64)
    buf = ctypes.create_string_buffer(8)
    assert L.lbmp_batch_class(ctypes.byref(prm), 1, nx, ny, 152, buf, 8) == lbmp.EINVAL
    assert L.lbmp_batch_class(ctypes.byref(prm), 1, nx, ny, 152, None, 64) == lbmp.EINVAL
