"""CPU checks of the kernels' index and culling logic (read from the kernel
source): every staged cell of a tile and its halo has its own slot inside the
staging buffer, 16-byte chunks of four x-consecutive cells stay whole and
aligned (the copies move chunks), the dense layout is the boxes the tensor
copies land, the bank-spread layout spreads the face runs' and far faces'
stencil loads over the 32 banks as its search found (a lane-by-lane model of
the kernel's access patterns), the per-cell accumulation array's slots are a
conflict-free permutation, and the initial condition's per-tile bubble culling
keeps every bubble that can be a cell's nearest."""
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_1705_04374_gb300", "csrc", "kernels.cuh")
TS, HALO, RW, XOFF = 8, 3, 16, 4
ROWS_INT, NSLAB = TS * TS * RW, HALO * TS * TS
ROWS_Y = ROWS_INT + 2 * NSLAB
NCROSS = ROWS_Y + 2 * NSLAB


def _source():
    with open(SRC) as f:
        return f.read()


def _slab_table():
    text = _source()
    body = text[text.index("c_slab[2][96] = {"):]
    body = body[:body.index("};")]
    vals = [int(v) for v in re.findall(r"-?\d+", body.split("=", 1)[1])]
    assert len(vals) == 192
    return vals[:96], vals[96:]


def _rows_xor_coefficients():
    text = _source()
    fn = text[text.index("__device__ __forceinline__ int rows_xor(int row)"):]
    fn = fn[:fn.index("}")]
    pairs = re.findall(r"\(g & (\d+)\) \? (\d+) : 0", fn)
    return {int(bit): int(v) for bit, v in pairs}


def _rows_xor(row, coef):
    g, s = row >> 1, 0
    for bit, v in coef.items():
        if g & bit:
            s ^= v
    return s << 2


def make_slot(layout):
    ytab, ztab = _slab_table()
    coef = _rows_xor_coefficients()

    def slot(x, y, z):
        yi, zi = 0 <= y < TS, 0 <= z < TS
        if yi and zi:
            row = z * TS + y
            s = row * RW + XOFF + x
            return s ^ _rows_xor(row, coef) if layout == "swz" else s
        if zi:
            side, h = (0, y + HALO) if y < 0 else (1, y - TS)
            if layout == "swz":
                return ROWS_INT + ytab[((side * HALO + h) * TS + z) * 2 + (x >> 2)] + (x & 3)
            return ROWS_INT + side * NSLAB + (z * HALO + h) * TS + x
        side, h = (0, z + HALO) if z < 0 else (1, z - TS)
        if layout == "swz":
            return ROWS_Y + ztab[((side * HALO + h) * TS + y) * 2 + (x >> 2)] + (x & 3)
        return ROWS_Y + side * NSLAB + (h * TS + y) * TS + x
    return slot


def staged_rows():
    """(y, z, x range) of every staged row (the tile's rows carry x = -4..11)."""
    for z in range(-HALO, TS + HALO):
        for y in range(-HALO, TS + HALO):
            yi, zi = 0 <= y < TS, 0 <= z < TS
            if yi and zi:
                yield y, z, range(-4, 12)
            elif yi or zi:
                yield y, z, range(0, 8)


@pytest.mark.parametrize("layout", ["dense", "swz"])
def test_every_staged_cell_has_its_own_slot_and_chunks_stay_whole(layout):
    slot = make_slot(layout)
    seen = set()
    for y, z, xs in staged_rows():
        for x0 in range(xs.start, xs.stop, 4):
            base = slot(x0, y, z)
            assert base % 4 == 0, (layout, x0, y, z)   # a chunk starts on a 16-byte boundary (FP32)
            for k in range(4):
                s = slot(x0 + k, y, z)
                assert s == base + k and 0 <= s < NCROSS
                assert s not in seen
                seen.add(s)
    assert len(seen) == NCROSS


def test_dense_layout_is_the_tensor_copy_boxes():
    slot = make_slot("dense")
    for v_off, (x0, y0, z0, bx, by, bz) in ((0, (-4, 0, 0, 16, 8, 8)), (ROWS_INT, (0, -3, 0, 8, 3, 8)),
                                            (ROWS_INT + NSLAB, (0, 8, 0, 8, 3, 8)), (ROWS_Y, (0, 0, -3, 8, 8, 3)),
                                            (ROWS_Y + NSLAB, (0, 0, 8, 8, 8, 3))):
        for k in range(bz):
            for j in range(by):
                for i in range(bx):
                    assert slot(x0 + i, y0 + j, z0 + k) == v_off + (k * by + j) * bx + i


def _warp_loads():
    """(cells per lane) of every warp-wide stencil load of one variable in a tile:
    the runs of two near faces (256 per direction) and the far faces (192)."""
    out = []
    for d in range(3):
        for w in range(8):
            for i in range(7):
                cells = []
                for lane in range(32):
                    t = 32 * w + lane
                    if d == 0:
                        j, a, b = 2 * (t & 3), (t >> 2) & 7, t >> 5
                        cells.append((j - 3 + i, a, b))
                    else:
                        a, j, b = t & 7, 2 * ((t >> 3) & 3), t >> 5
                        cells.append((a, j - 3 + i, b) if d == 1 else (a, b, j - 3 + i))
                out.append(cells)
    for w in range(6):
        for k in range(6):
            cells = []
            for lane in range(32):
                f = 32 * w + lane
                d, line = f >> 6, f & 63
                a, b = line & 7, line >> 3
                cells.append((TS - 3 + k, a, b) if d == 0 else ((a, TS - 3 + k, b) if d == 1 else (a, b, TS - 3 + k)))
            out.append(cells)
    return out


def _wavefronts(slot, loads):
    total = 0
    for cells in loads:
        per_bank = {}
        for s in {slot(*c) for c in cells}:
            per_bank[s % 32] = per_bank.get(s % 32, 0) + 1
        total += max(per_bank.values())
    return total


def test_bank_spread_layout_spreads_the_stencil_loads():
    loads = _warp_loads()
    dense, swz = _wavefronts(make_slot("dense"), loads), _wavefronts(make_slot("swz"), loads)
    assert len(loads) == 204
    assert dense == 864
    assert swz <= 327   # the x runs read one parity (two-way at best), the x far faces one x (four-way)


def _rslot():
    text = _source()
    m = re.search(r"__device__ __forceinline__ int rslot\(int c\) \{ return (.*?); \}", text)
    assert m, "rslot not found"
    expr = m.group(1)
    return lambda c: eval(expr, {"c": c})


def test_accumulation_slots_are_a_permutation_without_bank_conflicts():
    """The per-cell y + z flux-difference array: the y-run stores (lanes x, runs
    y = 0, 2, 4, 6 and y + 1), the z-run updates (lanes x, runs z = 0, 2, 4, 6 and
    z + 1) and the owners' paired reads (cells 2t, 2t + 1 of a warp) touch 32
    distinct banks, and the owners' pairs stay adjacent and 8-byte aligned."""
    rslot = _rslot()
    assert sorted(rslot(c) for c in range(512)) == list(range(512))

    def banks(slots):
        return len({s % 32 for s in slots})
    for b in range(8):
        for off in (0, 8):
            assert banks([rslot(a + 8 * 2 * g + 64 * b + off) for g in range(4) for a in range(8)]) == 32
        for off in (0, 64):
            assert banks([rslot(a + 8 * b + 64 * 2 * g + off) for g in range(4) for a in range(8)]) == 32
    for w in range(8):
        for half in range(2):
            words = []
            for lane in range(16 * half, 16 * half + 16):
                s0 = rslot(64 * w + 2 * lane)
                assert s0 % 2 == 0 and rslot(64 * w + 2 * lane + 1) == s0 + 1
                words += [s0, s0 + 1]
            assert banks(words) == 32


def test_initial_condition_candidates_keep_every_nearest_bubble():
    """The initial condition's per-tile culling (a bubble whose lower bound of the
    surface distance over the tile's cell centres exceeds the smallest upper
    bound, by the kernel's margin, is dropped): restated here in FP64 and checked
    on seeded clouds of 4 to 500 bubbles on 8^3 to 64^3 that fmin over the kept
    bubbles equals fmin over all of them, bit for bit, in every cell."""
    import numpy as np
    text = _source()
    margin = float(re.search(r"const double margin = ([0-9.e-]+);", text).group(1))
    rng = np.random.default_rng(7)
    for N, nb in ((8, 4), (16, 20), (32, 50), (64, 500)):
        h = 1.0 / N
        bub = np.column_stack([0.5 + rng.uniform(-0.3, 0.3, (nb, 3)), rng.uniform(0.05, 0.1, nb) * 0.3])
        tiles = [(x0, y0, z0) for x0 in range(0, N, 8) for y0 in range(0, N, 8) for z0 in range(0, N, 8)]
        for x0, y0, z0 in tiles[:: max(1, len(tiles) // 24)]:
            lo = np.array([(x0 + 0.5) * h, (y0 + 0.5) * h, (z0 + 0.5) * h])
            hi = np.array([(x0 + 7.5) * h, (y0 + 7.5) * h, (z0 + 7.5) * h])
            far = np.maximum(np.abs(bub[:, :3] - lo), np.abs(bub[:, :3] - hi))
            U = np.min(np.sqrt((far ** 2).sum(1)) - bub[:, 3])
            near = np.where(bub[:, :3] < lo, lo - bub[:, :3], np.where(bub[:, :3] > hi, bub[:, :3] - hi, 0.0))
            keep = np.sqrt((near ** 2).sum(1)) - bub[:, 3] <= U + margin
            assert keep.any()
            g = np.arange(8) + 0.5
            xs = np.stack(np.meshgrid((x0 + g) * h, (y0 + g) * h, (z0 + g) * h, indexing="ij"), -1).reshape(-1, 3)
            d = np.sqrt(((xs[:, None, :] - bub[None, :, :3]) ** 2).sum(-1)) - bub[None, :, 3]
            assert np.array_equal(d.min(1), d[:, keep].min(1))
