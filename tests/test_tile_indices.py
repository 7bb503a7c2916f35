"""Host models of the D3Q19 column kernels' tile indexing (fwd3p_kernel, adj3c_kernel).

No memory checker runs over these kernels, so the shared-memory and global
indices the kernel forms are checked here, on the CPU, for every lane, warp and
tile of many lattice shapes: the staged box reads (rows and columns, including the
one-sided differences on the faces), the exchange rows and columns written and
read, and the 8-byte alignment of every node pair; for the adjoint, the routing of
every link through the shared exchange and the shuffle ring over a z chunk.  The
tile constants are read from the CUDA source, so the models follow any change of
the tiling.
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


def _links():
    src = open(SRC).read()
    body = re.search(r"constexpr int c\[19\]\[3\] = \{(.*?)\};", src, re.S).group(1)
    c = [tuple(int(v) for v in t.split(",")) for t in re.findall(r"\{([-0-9, ]+)\}", body)]
    assert len(c) == 19 and len(set(c)) == 19
    return c


def _nxs3():
    m = re.search(r"\bNXS3 = ([0-9]+)", open(SRC).read())
    return int(m.group(1))


ADJ_SHAPES = [(192, 192, 9), (44, 21, 7), (8, 5, 4), (36, 20, 6), (60, 10, 5), (32, 9, 8), (116, 40, 6)]


@pytest.mark.parametrize("nx,ny,nz", ADJ_SHAPES)
def test_column_adjoint_exchange_routes_every_link_from_its_source(nx, ny, nz):
    """adj3c_kernel: a lane routes P + c_k.V of its node to x - c_k.  Model the exchange
    writes (slot = destination plane mod NXS3, row, link, column) and the c_y = 0 links
    (shuffles along x, a ring of three destination planes along z) over the planes of
    a z chunk, and check that every value an output node gathers was written in this
    plane loop by the node x + c_k, that no write leaves its buffer, that no entry is
    written while a slower warp may still read it, and that the staged box reads (with
    the one-sided differences on the faces) stay inside it."""
    k = _constants()
    CX3, NYC3, CBW3, XW3 = k["CX3"], k["NYC3"], k["CBW3"], k["XW3"]
    CBH3, NWC3, NXS3, NXL3 = NYC3 + 4, NYC3 + 2, _nxs3(), 10
    NSLC3 = int(re.search(r"\bNSLC3 = ([0-9]+)", open(SRC).read()).group(1))
    c = _links()
    yslot = {q: sum(1 for p in range(q) if c[p][1] != 0) for q in range(19)}
    assert sorted(yslot[q] for q in range(19) if c[q][1] != 0) == list(range(NXL3))
    tx = sorted({0, CX3, ((nx - 1) // CX3) * CX3})
    ty = sorted({0, NYC3, ((ny - 1) // NYC3) * NYC3})
    for zc in (2, 3, nz):
        for x0 in [t for t in tx if t < nx]:
            for y0 in [t for t in ty if t < ny]:
                for z0 in range(0, nz, zc):
                    z1 = min(z0 + zc, nz)
                    ex = {}  # (slot, row, yslot, col) -> (destination plane, source node)
                    ring = {}  # (warp, lane, destination plane, link) -> source node
                    read_prev = set()  # exchange entries the gather of the previous plane reads
                    for z in range(z0 - 1, z1 + 1):
                        written = set()
                        for warp in range(NWC3):
                            for lane in range(32):
                                i, j = x0 - 2 + lane, y0 - 1 + warp
                                bx, by = lane + 2, warp + 1
                                assert 0 <= by - 1 and by + 1 < CBH3 and 0 <= bx - 1 and bx + 1 < CBW3
                                src = 0 <= i < nx and 0 <= j < ny and 0 <= z < nz
                                if src and i in (0, nx - 1):
                                    assert 0 <= bx - 2 and bx + 2 < CBW3
                                if src and j in (0, ny - 1):
                                    assert 0 <= by + (2 if j == 0 else -2) < CBH3
                                for q in range(19):
                                    cx, cy, cz = c[q]
                                    node = (i, j, z) if src else None  # outside: a routed zero
                                    dz = z - cz
                                    if cy != 0:
                                        row = warp + (-2 if cy > 0 else 0)
                                        ok_r = warp >= 2 if cy > 0 else warp < NYC3
                                        lo, hi = (3, CX3 + 2) if cx > 0 else ((2, CX3 + 1) if cx == 0 else (1, CX3))
                                        if ok_r and lo <= lane <= hi:
                                            col = lane - 2 - cx
                                            assert 0 <= row < NYC3 and 0 <= col < XW3
                                            ex[(dz % NXS3, row, yslot[q], col)] = (dz, node)
                                            written.add((dz % NXS3, row, yslot[q], col))
                                    else:
                                        # shuffle: the value arrives at lane - c_x of the same warp
                                        dl = lane - cx
                                        if 0 <= dl < 32:
                                            ring[(warp, dl, dz, q)] = node
                        # Between two barriers a warp may still gather plane z - 2 while
                        # another already routes plane z: no entry may be in both.
                        assert not (written & read_prev), (x0, y0, z)
                        read_prev = set()
                        # the staged planes the routing of z + 1 reads (z - 1 .. z + 3) never
                        # share a ring slot with the plane issued after this barrier (z + NSLC3 - 3)
                        assert (z + NSLC3 - 3) % NSLC3 not in {(z + 1 + d) % NSLC3 for d in range(-2, 3)}
                        # after the barrier: the gather of plane z - 1
                        zd = z - 1
                        if not (z0 <= zd < z1):
                            continue
                        for warp in range(1, NYC3 + 1):
                            for lane in range(2, 2 + CX3):
                                i, j = x0 - 2 + lane, y0 - 1 + warp
                                if i >= nx or j >= ny:
                                    continue
                                for q in range(19):
                                    cx, cy, cz = c[q]
                                    s = (i + cx, j + cy, zd + cz)
                                    want = s if (0 <= s[0] < nx and 0 <= s[1] < ny and 0 <= s[2] < nz) else None
                                    if cy != 0:
                                        read_prev.add((zd % NXS3, warp - 1, yslot[q], lane - 2))
                                        got = ex.get((zd % NXS3, warp - 1, yslot[q], lane - 2))
                                        assert got is not None and got[0] == zd, (x0, y0, zd, warp, lane, q)
                                        assert got[1] == want, (x0, y0, zd, warp, lane, q, got, want)
                                    else:
                                        assert ring.get((warp, lane, zd, q), "missing") == want, (x0, y0, zd, lane, q)
