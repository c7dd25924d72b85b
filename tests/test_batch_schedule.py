"""Host-side queue of the persistent batched form (ppe_batch_schedule; no device
work).  Checked against its definition: every stage of every grid lists each of
its tiles exactly once; a grid's stage s - 1 is complete in the queue before
its stage s begins (the dependency a waiting CTA relies on, so the queue cannot
deadlock); the window / stagger order; the tile counts of each stage, worked out
here from the tilings the stage kernels use, and their grouping into runs of
about `grain` elements; refusal of lengths the kernel has no instance for."""
import math

import pytest

from paper_2103_01874_gb300 import fields, ppe

LENGTHS = (32, 48, 64, 96, 128, 192, 256)


def _tiles(nx, ny, nz, rho_given):
    """Tiles per stage, from the tilings of the stage kernels: 256-thread CTAs;
    power-of-two transform lengths n take 4096 / n lines per CTA, radix-3 ones
    the shared-memory tiles (x: the largest power of two <= min(64, 4096/nx)
    lines; z: 16 columns, y: 8 columns, fewer if 8 (2 t n + n) > 160 KiB);
    rho_0: 65536 cells per CTA; correction: 16 v faces per thread."""
    def pow2(n):
        return n & (n - 1) == 0

    def lpb(n):
        l = 1
        while 2 * l <= 4096 // n and 2 * l <= 64:
            l *= 2
        return l

    def cols(n, t):
        while t > 2 and 8 * (2 * t * n + n) > 160 * 1024:
            t //= 2
        return t
    nxh = nx // 2 + 1
    xl = 4096 // (nx // 2) if pow2(nx // 2) else lpb(nx)
    zl = 4096 // nz if pow2(nz) else cols(nz, 16)
    yl = 4096 // ny if pow2(ny) else cols(ny, 8)
    x = math.ceil(ny * nz / xl)
    z = ny * math.ceil(nxh / zl)
    y = nz * math.ceil(nxh / yl)
    tj = 256 // nx  # one line per thread stack
    rhs = math.ceil(ny / tj) * math.ceil(nz / min(nz, 8))
    first = [0 if rho_given else math.ceil(nx * ny * nz / 65536), 1, rhs, x, z, y, z, x]
    sweep = [x, z, y, z, x, math.ceil(nz * (ny + 1) * nx / 4096), 1]
    return first + sweep


def _chunk(nx, ny, nz, s, grain):
    """Tiles per item: about `grain` elements (1 to 255 tiles)."""
    def pow2(n):
        return n & (n - 1) == 0
    nxh = nx // 2 + 1
    if s in (0, 1, 14):
        return 1
    if s == 2:
        per = (256 // nx) * nx * min(nz, 8)
    elif s in (3, 7, 8, 12):
        l = 4096 // (nx // 2) if pow2(nx // 2) else max(t for t in (1, 2, 4, 8, 16, 32, 64) if t <= 4096 // nx)
        per = l * nx
    elif s in (4, 6, 9, 11):
        l = 4096 // nz if pow2(nz) else 16
        per = min(l, nxh) * nz
    elif s in (5, 10):
        l = 4096 // ny if pow2(ny) else 8
        per = min(l, nxh) * ny
    else:
        per = 16 * 256
    return max(1, min(255, grain // per))


def _check_queue(items, need, tiles, dims, rho, first, grain):
    for g, (d, r) in enumerate(zip(dims, rho)):
        assert tiles[15 * g:15 * g + 15] == _tiles(*d, r), d
        for s in range(15):
            c = _chunk(*d, s, grain)
            assert need[15 * g + s] == math.ceil(tiles[15 * g + s] / c), (d, s)
    assert len(items) == sum(need[15 * g + s] for g in range(len(dims)) for s in range(first, 15))
    pos0, pos1, covered = {}, {}, {}
    for pos, (g, s, t0, cnt) in enumerate(items):
        assert first <= s < 15 and 1 <= cnt <= 255 and t0 + cnt <= tiles[15 * g + s]
        covered.setdefault((g, s), []).append((t0, cnt))
        pos0.setdefault((g, s), pos)
        pos1[(g, s)] = pos
    # each stage's tiles covered exactly once, in runs
    for (g, s), runs in covered.items():
        t = 0
        for t0, cnt in sorted(runs):
            assert t0 == t
            t += cnt
        assert t == tiles[15 * g + s]
    # a grid's stage s - 1 is complete in the queue before its stage s begins
    for g in range(len(dims)):
        for s in range(first + 1, 15):
            if need[15 * g + s] and need[15 * g + s - 1]:
                assert pos1[(g, s - 1)] < pos0[(g, s)], (g, s)


@pytest.mark.parametrize("window,stagger", [(0, -1), (1, 100), (4, 2), (16, 3), (64, 0)])
@pytest.mark.parametrize("first", [0, 8])
@pytest.mark.parametrize("grain", [1, 65536, 1 << 20])
def test_batch_queue_of_the_uneven_batch(window, stagger, first, grain):
    dims = fields.batch_shapes(64, seed=3)
    rho = [g % 5 == 0 for g in range(64)]
    r = ppe.batch_schedule(dims, rho, window=window, stagger=stagger, first=first, grain=grain)
    assert r is not None
    items, need, tiles = r
    _check_queue(items, need, tiles, dims, rho, first, grain)


def test_window_and_stagger_orders():
    dims = [(32, 32, 32), (48, 64, 32), (64, 48, 96), (96, 32, 32)]
    rho = [False] * 4
    cells = [a * b * c for a, b, c in dims]
    # one window: stage-major (every grid's stage s before any stage s + 1),
    # larger grids first within a stage
    items = ppe.batch_schedule(dims, rho, window=0)[0]
    keys = [(s, -cells[g], g) for g, s, _, _ in items]
    assert keys == sorted(keys)
    # windows of one grid staggered by more than the stage count: grid after grid
    items = ppe.batch_schedule(dims, rho, window=1, stagger=1000)[0]
    gs = [g for g, _, _, _ in items]
    assert gs == sorted(gs)
    # windows of two grids, stagger 3: grid 2's stage s sits with grids 0-1's stage s + 3
    items = ppe.batch_schedule(dims, rho, window=2, stagger=3)[0]
    keys = [(s + 3 * (g // 2), -cells[g], g, s) for g, s, _, _ in items]
    assert keys == sorted(keys)


def test_lengths_and_first_stage_refused():
    assert ppe.batch_schedule([(16, 32, 32)], [False]) is None
    assert ppe.batch_schedule([(32, 32, 384)], [False]) is None
    assert ppe.batch_schedule([(32, 32, 32)], [False], first=3) is None
    assert ppe.batch_schedule([(32, 32, 32)], [False], grain=-1) is None
    for n in LENGTHS:
        assert ppe.batch_schedule([(n, 32, 48), (32, n, 48), (48, 32, n)], [True] * 3) is not None
