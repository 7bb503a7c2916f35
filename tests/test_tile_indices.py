"""Host model of the paired-column D3Q19 forward's tile indexing (fwd3p_kernel).

compute-sanitizer is not available on the GPU pool, so the shared-memory and global
indices the kernel forms are checked here, on the CPU, for every lane, warp and
tile of many lattice shapes: the staged box reads (rows and columns, including the
one-sided differences on the faces), the exchange rows and columns written and
read, and the 8-byte alignment of every node pair.  The tile constants are read
from the CUDA source, so the model follows any change of the tiling.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2411_03090_gb300", "csrc", "lks_3d.cu")


def _constants():
    src = open(SRC).read()
    env = {}
    for name in ("CX3", "NYC3", "NYP3", "NXS3", "NCB3"):
        m = re.search(rf"\b{name} = ([0-9]+)", src)
        assert m, name
        env[name] = int(m.group(1))
    env["CBW3"] = env["CX3"] + 8          # constexpr CBW3 = CX3 + 8
    env["PBH3"] = env["NYP3"] + 4         # constexpr PBH3 = NYP3 + 4
    env["XW3"] = env["CX3"]               # constexpr XW3 = CX3
    env["NWP3"] = env["NYP3"] // 2 + 1    # constexpr NWP3 = NYP3 / 2 + 1
    for name, expr in (("CBW3", r"CBW3 = CX3 \+ 8"), ("PBH3", r"PBH3 = NYP3 \+ 4"), ("XW3", r"XW3 = CX3;"),
                       ("NWP3", r"NWP3 = NYP3 / 2 \+ 1")):
        assert re.search(expr, src), name  # the model's formulas are the source's
    return env


SHAPES = [(192, 192), (44, 21), (8, 5), (36, 20), (60, 10), (28, 8), (32, 9), (100, 33), (116, 40), (12, 6),
          (88, 9), (24, 16), (136, 13)]


@pytest.mark.parametrize("nx,ny", SHAPES)
def test_paired_forward_indices_stay_inside_their_buffers(nx, ny):
    k = _constants()
    CX3, NYP3, CBW3, PBH3, XW3, NWP3, NCB3 = (k[n] for n in ("CX3", "NYP3", "CBW3", "PBH3", "XW3", "NWP3", "NCB3"))
    assert 2 * NWP3 == NYP3 + 2 and CX3 % 2 == 0 and XW3 % 2 == 0 and CBW3 % 2 == 0
    if nx % 4:
        pytest.skip("the column kernels need nx % 4 == 0")
    for x0 in range(0, nx, CX3):
        for y0 in range(0, ny, NYP3):
            for warp in range(NWP3):
                for lane in range(32):
                    h, q = lane >> 4, lane & 15
                    t = 2 * warp + h
                    i0, j = x0 - 2 + 2 * q, y0 - 1 + t
                    bx, by, xl = 2 + 2 * q, 1 + t, 2 * q - 2
                    in_xy = 0 <= i0 < nx and 0 <= j < ny
                    out = 1 <= q <= 14 and i0 < nx and 1 <= t <= NYP3 and j < ny
                    assert bx % 2 == 0 and (by * CBW3 + bx) % 2 == 0  # 8-byte pair reads of the box
                    # interior reads: rows by - 1 .. by + 1, columns bx - 1 .. bx + 2
                    assert 0 <= by - 1 and by + 1 < PBH3
                    assert 0 <= bx - 1 and bx + 2 < CBW3
                    if in_xy:
                        # one-sided differences on the faces (two nodes inward)
                        if i0 == 0:
                            assert bx + 2 < CBW3
                        if i0 + 1 == nx - 1:
                            assert bx + 1 - 2 >= 0
                        if j in (0, ny - 1):
                            s = 1 if j == 0 else -1
                            assert 0 <= by + 2 * s < PBH3
                        # a pair never straddles the lattice's last column (nx is even)
                        assert i0 + 1 < nx
                    # exchange writes: destination row td in 1 .. NYP3, columns 0 .. XW3 - 1
                    td = t + 1 if h else t - 1
                    if 1 <= td <= NYP3:
                        for b in range(NCB3):
                            cx = 1 if b == 1 else (-1 if b == 2 else 0)
                            if cx == 0:
                                if 1 <= q <= 14:
                                    assert 0 <= xl and xl + 1 < XW3 and xl % 2 == 0
                            # shifted writes are guarded column by column in the kernel
                    if out:
                        assert 0 <= t - 1 < NYP3 and 0 <= xl and xl + 1 < XW3 and xl % 2 == 0
