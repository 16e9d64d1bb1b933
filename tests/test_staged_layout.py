"""Index arithmetic of the staged step kernel, replayed on the CPU (no GPU).

The staged kernel copies spans of the flattened lattice with cp.async.bulk,
which needs 16-byte aligned global and shared addresses and sizes, and must
stay inside the population buffer and inside its shared-memory stage.  This
test walks the producer's copy segments (with the wrap around the plane),
the consumers' shared-memory reads and their incremental tile coordinates
for many lattice shapes, boundary kinds and grid sizes, and checks every
range and alignment.  The tile
constants are read from the kernel header so the replay cannot drift."""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1411_7051_gb300", "csrc")


def stage_cfg(kind="single"):
    """Stage constants of the single-lattice kernel (staged.cuh) or of the
    batched one (batch.cu)."""
    text = open(os.path.join(CSRC, "staged.cuh")).read()
    cw = int(re.search(r"kConsumerWarps = (\d+);", text).group(1))
    out = {}
    for store, elem in (("StoreF32", 4), ("StoreF16", 2)):
        m = re.search(r"struct StageCfg<%s>\s*{\s*static constexpr int W = (\d+), H = (\d+), "
                      r"A = (\d+), STAGES = (\d+);" % store, text)
        assert m, store
        W, H, A, NS = map(int, m.groups())
        out[store] = dict(W=W, H=H, A=A, NS=NS, elem=elem, warps=cw, head=0, kn0=False)
    if kind == "dyn":  # FP16 with a dynamic Kn: the Kn plane staged too
        m = re.search(r"struct StageCfgDyn16\s*{\s*static constexpr int W = (\d+), H = (\d+), "
                      r"A = (\d+), STAGES = (\d+);", text)
        assert m
        W, H, A, NS = map(int, m.groups())
        out = {"StoreF16": dict(W=W, H=H, A=A, NS=NS, elem=2, warps=cw, head=0, kn0=True)}
    if kind == "batch":
        btext = open(os.path.join(CSRC, "batch.cu")).read()
        head = int(re.search(r"kHeadBytes = (\d+);", btext).group(1))
        for store, elem in (("StoreF32", 4), ("StoreF16", 2)):
            m = re.search(r"struct BatchCfg<%s>\s*{\s*static constexpr int W = (\d+), H = (\d+), "
                          r"A = (\d+), STAGES = (\d+);\s*static constexpr int WARPS = (\d+);" % store,
                          btext)
            assert m, store
            W, H, A, NS, warps = map(int, m.groups())
            out[store] = dict(W=W, H=H, A=A, NS=NS, elem=elem, warps=warps, head=head, kn0=False)
    return out


def batch_pitch_of(nx):
    """Row pitch of a batched instance (batch.cu: no skew)."""
    text = open(os.path.join(CSRC, "batch.cu")).read()
    align = int(re.search(r"kBatchPitchAlign = (\d+);", text).group(1))
    return ((nx + align - 1) // align) * align


def pitch_of(nx):
    text = open(os.path.join(CSRC, "kernels.h")).read()
    align = int(re.search(r"kPitchAlign = (\d+);", text).group(1))
    every = int(re.search(r"kPitchSkewEvery = (\d+);", text).group(1))
    skew = int(re.search(r"kPitchSkew = (\d+);", text).group(1))
    p = ((nx + align - 1) // align) * align
    return p + skew if p % every == 0 else p


EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]


def replay(nx, ny, walls, store, grids=(1, 7, 152), kind="single"):
    c = stage_cfg(kind)[store]
    W, H, A, NS, elem, cw = c["W"], c["H"], c["A"], c["NS"], c["elem"], c["warps"]
    assert H == 1 and W % 64 == 0
    RW = W + 2 * A
    pop_bytes = 9 * RW * elem
    stage_bytes = pop_bytes + W * 8 + (W * 4 if c["kn0"] else 0)
    bar_bytes = 128
    assert bar_bytes + NS * stage_bytes + NS * c["head"] <= 227 * 1024
    assert (bar_bytes + NS * stage_bytes) % 16 == 0  # the batched tile headers follow
    assert 2 * NS * 8 <= bar_bytes
    pitch = batch_pitch_of(nx) if kind == "batch" else pitch_of(nx)
    NP = pitch * ny                      # nodes of a plane (the wrap length)
    stride = NP                          # plane stride
    y0, rows = (1, ny - 2) if walls else (0, ny)
    F0, Fend = y0 * pitch, (y0 + rows) * pitch
    ntiles = -(-(Fend - F0) // W)
    for t in range(ntiles):
        T0 = F0 + t * W
        assert T0 < Fend
        med_elems = min(W, Fend - T0)
        total = 9 * RW * elem + med_elems * 8 + (med_elems * 4 if c["kn0"] else 0)
        assert total < 2 ** 20  # mbarrier tx-count range
        if c["kn0"]:
            # the Kn span [T0, T0 + med_elems) of the float plane, after the medium
            assert (T0 * 4) % 16 == 0 and (med_elems * 4) % 16 == 0
            assert (pop_bytes + W * 8) % 16 == 0
        for lane in range(9):
            # producer lane `lane`: plane lane's sources, flat [T0 - e_y pitch - A, + RW) mod NP
            v = T0 - EY[lane] * pitch - A
            while v < 0:
                v += NP
            while v >= NP:
                v -= NP
            dst = lane * RW * elem
            left = RW
            virt = T0 - EY[lane] * pitch - A
            while left > 0:
                seg = min(left, NP - v)
                assert seg > 0
                src = (lane * stride + v) * elem
                assert src % 16 == 0 and (seg * elem) % 16 == 0 and dst % 16 == 0
                assert 0 <= v and v + seg <= NP
                assert dst + seg * elem <= (lane + 1) * RW * elem
                # every stage element holds plane[virtual index mod NP]
                assert (virt + (dst // elem - lane * RW)) % NP == v
                dst += seg * elem
                left -= seg
                v = 0
            assert dst == (lane + 1) * RW * elem
        # medium: [T0, T0 + med_elems) of the float2 plane, into the stage tail
        assert (T0 * 8) % 16 == 0 and (med_elems * 8) % 16 == 0 and T0 + med_elems <= NP
        assert pop_bytes % 16 == 0
        # consumer reads of an interior node at tile offset cc: stage index
        # A + cc + sh, which holds the flat source p - e_y pitch + sh
        for cc in range(0, W, max(1, W // 97)):
            p = T0 + cc
            if p >= Fend:
                break
            x, y = p % pitch, p // pitch
            if not (1 <= x <= nx - 2):
                continue
            for sh in (-1, 0, 1):
                assert 0 <= A + cc + sh < RW
                assert (p + sh) // pitch == y  # never across a row end
    # consumers track the tile start (x, y) incrementally: same as the division
    for g in grids:
        g = min(g, ntiles)
        for b in range(g):
            Tb = F0 + b * W
            yT, xT = divmod(Tb, pitch)
            dy, dx = divmod(g * W, pitch)
            for t in range(b, ntiles, g):
                assert (yT, xT) == divmod(F0 + t * W, pitch)
                xT += dx
                yT += dy
                if xT >= pitch:
                    xT -= pitch
                    yT += 1
        # launches reading buffer 1 walk the tiles from the end: block b's
        # k-th tile is ntiles - 1 - (b + k g), tracked backwards
        seen = []
        for b in range(g):
            yT, xT = divmod(F0 + (ntiles - 1 - b) * W, pitch)
            dy, dx = divmod(g * W, pitch)
            for t in range(b, ntiles, g):
                tt = ntiles - 1 - t
                assert (yT, xT) == divmod(F0 + tt * W, pitch)
                seen.append(tt)
                xT -= dx
                yT -= dy
                if xT < 0:
                    xT += pitch
                    yT -= 1
        assert sorted(seen) == list(range(ntiles))
    # the column-edge pass: consumer thread k takes row yT + k // 2, pair x = 0
    # (k even) or x = (nx - 1) & ~1 (k odd); with the consumer loop, which
    # skips those pairs, every pair of every tile is updated exactly once
    xl = (nx - 1) & ~1
    for t in range(ntiles):
        T0 = F0 + t * W
        yT, xT = divmod(T0, pitch)
        done = []
        for k in range(cw * 32):
            r, x = k >> 1, (xl if k & 1 else 0)
            if (k & 1) and xl == 0:
                continue
            y = yT + r
            if y >= y0 + rows:
                continue
            cc = r * pitch + x - xT
            if cc < 0 or cc >= W:
                continue
            assert cc % 2 == 0 and (cc * 8) % 16 == 0
            done.append((y, x))
        for cc in range(0, W, 2):
            p = T0 + cc
            y, x = divmod(p, pitch)
            if y >= y0 + rows or x >= nx:
                continue
            if x == 0 or x + 2 >= nx:
                continue  # left to the pass
            done.append((y, x))
        want = [divmod(p, pitch) for p in range(T0, min(T0 + W, Fend), 2) if p % pitch < nx]
        assert sorted(done) == sorted(want)
    # consumer thread mapping covers each tile node pair exactly once
    per = W // 2 // (cw * 32)
    seen = set()
    for tid in range(cw * 32):
        for j in range(per):
            seen.add(2 * (tid + j * cw * 32))
    assert seen == set(range(0, W, 2))


@pytest.mark.parametrize("store", ["StoreF32", "StoreF16"])
@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("nx,ny", [(1, 3), (3, 3), (5, 1), (64, 33), (131, 37), (255, 9), (256, 4),
                                   (257, 5), (513, 17), (1000, 7), (4096, 12), (4099, 6)])
@pytest.mark.parametrize("kind", ["single", "batch", "dyn"])
def test_staged_copies_in_bounds_and_aligned(nx, ny, walls, store, kind):
    if walls and ny < 3:
        pytest.skip("walls need ny >= 3")
    if kind == "dyn" and store != "StoreF16":
        pytest.skip("a dynamic Kn stages FP16 populations only")
    replay(nx, ny, walls, store, kind=kind)
