"""Index arithmetic of the staged step kernel, replayed on the CPU (no GPU).

The staged kernel copies row tiles with cp.async.bulk, which needs 16-byte
aligned global and shared addresses and sizes, and must stay inside the
population buffer and inside its shared-memory stage.  This test walks the
producer's copy list and the consumers' shared-memory reads for many lattice
shapes and boundary kinds and checks every range and alignment.  The tile
constants are read from the kernel header so the replay cannot drift."""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1411_7051_gb300", "csrc")


def stage_cfg():
    text = open(os.path.join(CSRC, "staged.cuh")).read()
    out = {}
    for store, elem in (("StoreF32", 4), ("StoreF16", 2)):
        m = re.search(r"struct StageCfg<%s>\s*{\s*static constexpr int W = (\d+), H = (\d+), "
                      r"A = (\d+), STAGES = (\d+);" % store, text)
        assert m, store
        W, H, A, NS = map(int, m.groups())
        out[store] = dict(W=W, H=H, A=A, NS=NS, elem=elem)
    cw = int(re.search(r"kConsumerWarps = (\d+);", text).group(1))
    return out, cw


def pitch_of(nx):
    text = open(os.path.join(CSRC, "lbmp_api.cu")).read()
    align = int(re.search(r"kPitchAlign = (\d+);", text).group(1))
    return ((nx + align - 1) // align) * align


EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]


def src_row(ny, walls, i, y):
    ys = y - EY[i]
    if walls and EY[i] != 0 and ys in (0, ny - 1):
        return -1
    return ys % ny


def replay(nx, ny, walls, store):
    cfg, cw = stage_cfg()
    c = cfg[store]
    W, H, A, NS, elem = c["W"], c["H"], c["A"], c["NS"], c["elem"]
    RW = W + 2 * A
    pop_bytes = 9 * H * RW * elem
    med_bytes_stage = H * W * 8
    stage_bytes = pop_bytes + med_bytes_stage
    bar_bytes = 128
    smem_bytes = bar_bytes + NS * stage_bytes
    assert smem_bytes <= 227 * 1024
    assert 2 * NS * 8 <= bar_bytes
    pitch = pitch_of(nx)
    plane = pitch * ny
    y0, rows = (1, ny - 2) if walls else (0, ny)
    tiles_x = -(-nx // W)
    tiles_y = -(-rows // H)
    for t in range(tiles_x * tiles_y):
        ya = y0 + (t // tiles_x) * H
        xa = (t % tiles_x) * W
        nrow = min(H, y0 + rows - ya)
        assert nrow >= 1
        gx0, gx1 = max(xa - A, 0), min(xa + W + A, pitch)
        scol = gx0 - (xa - A)
        row_bytes = (gx1 - gx0) * elem
        med_bytes = (min(xa + W, pitch) - xa) * 8
        total = nrow * med_bytes
        for i in range(9):
            for r in range(nrow):
                ys = src_row(ny, walls, i, ya + r)
                if ys < 0:
                    continue
                total += row_bytes
                # shared destination inside row (i, r) of the stage, aligned
                dst = ((i * H + r) * RW + scol) * elem
                assert dst % 16 == 0 and row_bytes % 16 == 0 and row_bytes > 0
                assert scol >= 0 and scol + (gx1 - gx0) <= RW
                assert dst + row_bytes <= pop_bytes
                # global source inside the plane row, aligned
                src = (i * plane + ys * pitch + gx0) * elem
                assert src % 16 == 0
                assert 0 <= ys < ny and 0 <= gx0 < gx1 <= pitch
        for r in range(nrow):
            dst = pop_bytes + r * W * 8
            assert dst % 16 == 0 and med_bytes % 16 == 0 and med_bytes <= W * 8
            src = ((ya + r) * pitch + xa) * 8
            assert src % 16 == 0 and (ya + r) < ny
        assert total < 2 ** 20  # mbarrier tx-count range
        # consumer reads: row (i, r), column A + c - 1 .. A + c + 1 for the node
        # and its pressure-neighbour (c - 1 .. c + 1)
        for c in (-1, 0, 1, W - 2, W - 1, W):
            for sh in (-1, 0, 1):
                col = A + c + sh
                if c in (-1, W) and sh != 0:
                    continue  # neighbours are only taken at c + 1 >= 0 or c - 1 <= W - 1
                assert 0 <= col < RW
    # consumer thread mapping covers each tile node exactly once
    per = H * W // (cw * 32)
    seen = set()
    for tid in range(cw * 32):
        for j in range(per):
            q = tid + j * cw * 32
            seen.add((q // W, q % W))
    assert len(seen) == H * W


@pytest.mark.parametrize("store", ["StoreF32", "StoreF16"])
@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("nx,ny", [(1, 3), (3, 3), (5, 1), (64, 33), (131, 37), (255, 9), (256, 4),
                                   (257, 5), (513, 17), (1000, 7), (4096, 12), (4099, 6)])
def test_staged_copies_in_bounds_and_aligned(nx, ny, walls, store):
    if walls and ny < 3:
        pytest.skip("walls need ny >= 3")
    replay(nx, ny, walls, store)
