"""Index maps of the tensor-core transforms (csrc/lsm_tc.cuh), restated on the host and checked for
every supported width: the natural-order positions (tc_xpos) and the frequency positions (tc_kpos) of
a warp's real matrix elements are each a bijection onto [0, N), and the per-warp buffer positions
(tc_phys) of all 8 NT columns, padding included, stay inside the 16 x LD buffer and are distinct.
For N = 16 R2 with R2 not a multiple of 8 the columns R2 .. 8 NT - 1 are zero padding and never
touch global memory.  (No GPU: this checks the arithmetic the kernel's loads and stores use.)
"""

import pytest

WIDTHS = [16, 32, 48, 64, 80, 96, 112, 128, 160, 192, 224, 256, 320, 384, 448, 512, 640, 768, 896, 1024]


def _shape(n):
    r2 = n // 16
    nt = (r2 + 7) // 8
    return r2, nt, r2 % 8 != 0, 8 * nt + 4


def _phys(row, col, ld):
    return row * ld + (col ^ ((row & 1) | (row & 4)))


@pytest.mark.parametrize("n", WIDTHS)
def test_tensor_core_index_maps(n):
    r2, nt, pad, ld = _shape(n)
    assert n == 16 * r2
    xs, ks, phys = [], [], set()
    for lane in range(32):
        g, tig = lane >> 2, lane & 3
        for j in range(nt):
            for e in range(4):
                col = 8 * j + 2 * tig + (e & 1)  # accumulator layout: row g + 8 (e / 2), column col
                row = g + 8 * (e >> 1)
                if not pad or col < r2:
                    xs.append(r2 * row + col)   # tc_xpos
                    ks.append(row + 16 * col)   # tc_kpos
                ph = _phys(row, col, ld)
                assert 0 <= ph < 16 * ld
                phys.add(ph)
    assert sorted(xs) == list(range(n))
    assert sorted(ks) == list(range(n))
    assert len(phys) == 16 * 8 * nt


@pytest.mark.parametrize("n", WIDTHS)
def test_buffer_base_plus_offset_forms(n):
    """tc_left reads and tc_store writes use a per-lane base plus a compile-time offset; that must
    equal tc_phys of the element it stands for (the XOR stays within each group of 8 columns)."""
    r2, nt, pad, ld = _shape(n)
    for lane in range(32):
        g, tig = lane >> 2, lane & 3
        for q in range(2):  # operand reads: rows 2 tig + 8 w + q, columns 8 j + g
            base = _phys(2 * tig + q, g, ld)
            for w in range(2):
                for j in range(nt):
                    assert base + 8 * w * ld + 8 * j == _phys(2 * tig + q + 8 * w, 8 * j + g, ld)
        for e0 in range(2):  # accumulator writes: rows g + 8 h, columns 8 j + 2 tig + e0
            base = _phys(g, 2 * tig + e0, ld)
            for h in range(2):
                for j in range(nt):
                    assert base + 8 * h * ld + 8 * j == _phys(g + 8 * h, 8 * j + 2 * tig + e0, ld)
