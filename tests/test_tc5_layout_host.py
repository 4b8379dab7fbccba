"""Index maps of the tcgen05 transforms (csrc/lsm_tc5.cuh), restated on the host and checked for every
width they exist for (nx = 16 R, R = 8, 16, 32, 64): in each of a depth step's four stages every
element of the shared-memory operand tiles is written exactly once and inside the operand buffer,
every TMEM column a thread reads or an MMA writes lies inside the CTA's allocation, each thread
reads only TMEM lanes its warp may access, and the adjoint's four image rows cover every column once.
The shared-memory size of the model is checked against the library's own launch-shape query.
(No GPU: this checks the arithmetic the kernel's stores and TMEM accesses use.)
"""

import os
import shutil

import pytest

WIDTHS = [128, 256, 512, 1024]


def _sw128(r, k):
    """Byte offset of 16-bit K element k of row r in a K-major 128-byte-swizzled block."""
    return (r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ r) & 7) << 4) + ((k & 7) << 1)


def _shape(n):
    R = n // 16
    items = 16 if R == 8 else 8
    groups = 2 if R == 64 else 1
    lt = items * R // 128
    rt = items * 16 // 128
    kb = (4 * R + 63) // 64
    ltile, rtile = 128 * 128, kb * 128 * 128
    brf = kb * 2 * R * 128
    off_a = (32 * 128 + brf + 1023) // 1024 * 1024
    a_bytes = max(lt * ltile, rt * rtile)
    off_stg = off_a + a_bytes + 2 * 16 * R * 8
    tm_l = 0
    tm_r = 0 if R == 64 else 64 * lt
    need = 64 * lt if R == 64 else 64 * lt + 4 * R * rt
    cols = next(c for c in (32, 64, 128, 256) if need <= c)
    return dict(R=R, items=items, groups=groups, threads=128 * groups, lt=lt, ltt=lt // groups, rt=rt,
                rcols=2 * R // groups, rch=min(32, 2 * R // groups), ltile=ltile, rtile=rtile, a_bytes=a_bytes,
                off_stg=off_stg, tm_l=tm_l, tm_r=tm_r, cols=cols)


@pytest.mark.parametrize("n", WIDTHS)
def test_tcgen05_operand_and_accumulator_maps(n):
    s = _shape(n)
    R, T = s["R"], s["threads"]
    assert s["items"] * R % 128 == 0 and s["items"] * 16 % 128 == 0 and (2 * R) % 16 == 0
    # TMEM: every left and right accumulator (FP16's second accumulator included) inside the allocation
    assert s["tm_l"] + 64 * s["lt"] <= s["cols"]
    assert s["tm_r"] + 4 * R * s["rt"] <= s["cols"]
    left1, right2, right3, left4, img = {}, {}, {}, {}, {}
    for tid in range(T):
        grp, r, warp, lane = tid >> 7, tid & 127, tid >> 5, tid & 31
        assert (warp & 3) * 32 <= r < (warp & 3) * 32 + 32  # the lane quarter of this warp
        n2, k1 = r % R, r % 16
        kb = grp * (R // s["groups"])
        for i in range(s["ltt"]):
            tau = grp * s["ltt"] + i
            item = (128 * tau + r) // R
            assert item < s["items"]
            # (1) left operand: row r of tile tau, K chunks of hi (0..31) and lo (32..63)
            for c in range(4):
                for k in (8 * c, 32 + 8 * c):
                    off = tau * s["ltile"] + _sw128(r, k)
                    assert off + 16 <= s["a_bytes"] and (tau, r, k) not in left1
                    left1[(tau, r, k)] = 1
            # (2) right operand rows (item, k1), K = 2 n2 (hi) and 2R + 2 n2 (lo)
            for kk in range(16):
                rho = item * 16 + kk
                sg, rr = rho >> 7, rho & 127
                assert sg < s["rt"]
                for e in (2 * n2, 2 * R + 2 * n2):
                    off = sg * s["rtile"] + (e // 64) * 16384 + _sw128(rr, e % 64)
                    assert off + 4 <= s["a_bytes"] and (sg, rr, e) not in right2
                    right2[(sg, rr, e)] = 1
            # (5) left accumulator columns read back
            assert s["tm_l"] + tau * 64 + 64 <= s["cols"]
        for sg in range(s["rt"]):
            item = (128 * sg + r) // 16
            assert item < s["items"]
            for h0 in range(s["rcols"] // s["rch"]):
                col = s["tm_r"] + sg * 4 * R + 2 * kb + h0 * s["rch"]
                assert col + s["rch"] + 2 * R <= s["cols"]  # both accumulators of the chunk
                # (3) inverse right operand, same row, K chunks of four complex columns
                for c in range(s["rch"] // 8):
                    k20 = kb + h0 * (s["rch"] // 2) + 4 * c
                    assert k1 + 16 * (k20 + 3) < n  # phase-shift table index
                    for e in (2 * k20, 2 * R + 2 * k20):
                        off = sg * s["rtile"] + (e // 64) * 16384 + _sw128(r, e % 64)
                        assert e % 8 == 0 and off + 16 <= s["a_bytes"] and (sg, r, e) not in right3
                        right3[(sg, r, e)] = 1
                # (4) inverse left operand rows (item, n2), K = 2 k1 (hi) and 32 + 2 k1 (lo)
                for q in range(s["rch"] // 2):
                    nn = kb + h0 * (s["rch"] // 2) + q
                    rho = item * R + nn
                    tile, row = rho >> 7, rho & 127
                    assert tile < s["lt"]
                    for e in (2 * k1, 32 + 2 * k1):
                        off = tile * s["ltile"] + _sw128(row, e)
                        assert off + 4 <= s["a_bytes"] and (tile, row, e) not in left4
                        left4[(tile, row, e)] = 1
        # adjoint image rows: after the sum over lanes of equal n2, lanes < R (or all) write
        islot = warp >> 1 if R == 64 else warp
        if R >= 32 or lane < R:
            for n1 in range(16):
                key = (islot, R * n1 + n2)
                assert key not in img
                img[key] = 1
    assert len(left1) == s["lt"] * 128 * 8
    assert len(right2) == s["rt"] * 128 * 2 * R
    assert len(right3) == s["rt"] * 128 * 2 * R // 4
    assert len(left4) == s["lt"] * 128 * 32
    assert len(img) == 4 * n and 4 * n * 4 <= s["a_bytes"]


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1801_00819_gb300 import build as B
    B.build()
    from paper_1801_00819_gb300 import lsm
    return lsm


@pytest.mark.parametrize("n", WIDTHS)
def test_tcgen05_shared_memory_model_matches_library(lib, n):
    """The model's shared-memory layout gives the library's size: base + staged slots + alignment."""
    s = _shape(n)
    for nshots, nw in ((16, 128), (4, 64), (3, 10)):
        sh = lib.lsm_tcgen05_shape(n, nshots, nw)
        assert sh["items"] == s["items"] and sh["threads"] == s["threads"]
        assert sh["smem_bytes"] == s["off_stg"] + sh["wslots"] * 2 * n * 8 + 1024
