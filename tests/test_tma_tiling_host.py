"""Host check of the TMA step kernel's tiling arithmetic (no GPU), with the tile and stage
constants read from the kernel sources: every box starts on a 16-byte x boundary (the rule of
tiled bulk tensor copies), the box of plane i holds the pull source x - e_i of every site of
the tile at the column the kernel reads, the shared-memory reads stay inside their slots,
the slots and stages keep 128-byte alignment, a stage's byte count fits the mbarrier
transaction count, and three blocks fit one SM's shared memory."""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1611_03329_gb300", "csrc")


def _src(name):
    with open(os.path.join(CSRC, name)) as fh:
        return fh.read()


def _constants():
    hdr, tma = _src("lbm_internal.cuh"), _src("lbm_tma.cu")
    tx, ty = map(int, re.search(r"kTmaTileX = (\d+), kTmaTileY = (\d+)", hdr).groups())
    s16, s32 = map(int, re.search(r"kStages = sizeof\(T\) == 2 \? (\d+) : (\d+);", tma).groups())
    width = int(re.search(r"kW = (\d+);", tma).group(1))
    blocks = int(re.search(r"__launch_bounds__\(kTBlock, (\d+)\)", tma).group(1))
    return tx, ty, {2: s16, 4: s32}, width, blocks


def _box(x0, ex):
    """x start and width of the box of a plane with velocity component ex, and the column of
    site tx's source inside it (box_x, box_col of the kernel)."""
    start = x0 - 8 if ex == 1 else x0
    width = 64 if ex == 0 else 72
    col = 7 if ex == 1 else (1 if ex == -1 else 0)
    return start, width, col


@pytest.mark.parametrize("elem", [2, 4])
def test_tma_tiling_invariants(elem):
    tile_x, tile_y, stages, slot_w, blocks = _constants()
    assert tile_x == 64 and slot_w == 72
    for nx in (64, 128, 256, 1024):
        for x0 in range(0, nx, tile_x):
            for ex in (-1, 0, 1):
                start, width, col = _box(x0, ex)
                assert (start * elem) % 16 == 0          # x coordinate on a 16-byte boundary
                assert (width * elem) % 16 == 0          # inner box extent in whole 16 bytes
                assert width <= slot_w
                for t in range(tile_x):
                    assert start + t + col == x0 + t - ex  # the pull source x - e_x
                    assert 0 <= t + col < width            # inside the box row
    # shared-memory layout of one stage (the TmaCfg arithmetic)
    n_planes, n_t = 26, 7
    plane = (tile_y * slot_w * elem + 127) // 128 * 128
    tslot = (tile_y * slot_w * 4 + 127) // 128 * 128 if elem == 2 else 0
    stage = n_planes * plane + n_t * tslot
    assert plane % 128 == 0 and tslot % 128 == 0 and stage % 128 == 0
    assert tile_y * slot_w * elem <= plane and tile_y * slot_w * 4 <= (tslot or 1 << 30)
    # the last element a thread reads in a slot: row tile_y - 1, column 63 + 7
    assert ((tile_y - 1) * 72 + tile_x - 1 + 7) * elem < plane
    # bytes one stage expects on its mbarrier (10 of 19 f planes and 2 of 7 g planes are
    # x-shifted), below the transaction-count limit of 2^20 - 1
    f_bytes = tile_y * elem * (9 * 64 + 10 * 72)
    g_bytes = tile_y * (elem + (4 if elem == 2 else 0)) * (5 * 64 + 2 * 72)
    assert f_bytes + g_bytes < (1 << 20) - 1
    smem = stages[elem] * stage + 128
    assert blocks * (smem + 1024) <= 228 * 1024  # per-block reserve of 1 KB included
