"""CPU model of the halo-tiled dslash's index arithmetic (csrc/sq_dslash_tile.cu).

The tiled kernel stages, per source, the input spinors of a site tile and of
its y, z, t halo rows into a compact shared-memory buffer with one bulk copy
per contiguous row run, and every thread then reads its eight neighbours at
precomputed buffer positions. This module restates the kernel's host plan
(`tile_plan`), its segment slots (`tile_segment`) and its neighbour lookup in
plain Python and checks, for every tile of several lattices, that

* the copies fill every compact row exactly once, from the right global row,
  within the buffer, with 16-byte aligned addresses and sizes;
* every neighbour position lands on the staged copy of the true neighbour
  site (periodic wrap in every direction) and inside the buffer;
* the threads of all tiles cover every output site once.

No GPU and no oracle are involved: this is the kernel's addressing, checked
against the lattice geometry directly.
"""

import itertools

import pytest

MAX_THREADS = 256
MAX_SLOTS = 512


def plan(dims, prec, by, bz, bt, nbuf=2):
    X, Y, Z, T = dims
    X2 = X // 2
    if Y % by or Z % bz or T % bt:
        return None
    threads = X2 * by * bz * bt
    if threads > MAX_THREADS or threads % 32:
        return None
    if prec == "f16" and X2 % 4:
        return None
    hy, hz, ht = int(by < Y), int(bz < Z), int(bt < T)
    nyA = by + 2 * hy
    NA = bt * bz * nyA
    NB = 2 * bt * by if hz else 0
    NC = 2 * bz * by if ht else 0
    rows = NA + NB + NC
    S = rows * X2
    nslot = 3 * bt * bz + 2 * bt + 2 * bz
    if nslot > MAX_SLOTS or rows > 0xFFFF:
        return None
    buf = S * (52 if prec == "f16" else 96)
    smem = 64 + 8 * MAX_SLOTS + nbuf * buf
    if smem > 227 * 1024:
        return None
    return dict(X2=X2, Y=Y, Z=Z, T=T, X=X, by=by, bz=bz, bt=bt, hy=hy, hz=hz, ht=ht, nyA=nyA, NA=NA, NB=NB,
                rows=rows, S=S, nslot=nslot, threads=threads, buf=buf, nty=Y // by, ntz=Z // bz, ntt=T // bt)


def rowA(p, tr, zr, yy):
    return (tr * p["bz"] + zr) * p["nyA"] + yy + p["hy"]


def segment(p, y0, z0, t0, q):
    """(srow, nrows, grow) of slot q, as the kernel's tile_segment."""
    Y, Z, T = p["Y"], p["Z"], p["T"]
    nA = 3 * p["bt"] * p["bz"]
    if q < nA:
        pr, piece = divmod(q, 3)
        tr, zr = divmod(pr, p["bz"])
        z, t = z0 + zr, t0 + tr
        lo, hi = -p["hy"], p["by"] - 1 + p["hy"]
        k, yy = 0, lo
        while yy <= hi:
            gy = (y0 + yy + Y) % Y
            ln = 1
            while yy + ln <= hi and (y0 + yy + ln + Y) % Y == gy + ln:
                ln += 1
            if k == piece:
                return rowA(p, tr, zr, yy), ln, gy + Y * (z + Z * t)
            k += 1
            yy += ln
        return 0, 0, 0
    q -= nA
    if q < 2 * p["bt"]:
        if not p["hz"]:
            return 0, 0, 0
        tr, side = q >> 1, q & 1
        z = (z0 + p["bz"]) % Z if side else (z0 - 1 + Z) % Z
        return p["NA"] + (tr * 2 + side) * p["by"], p["by"], y0 + Y * (z + Z * (t0 + tr))
    q -= 2 * p["bt"]
    if q < 2 * p["bz"]:
        if not p["ht"]:
            return 0, 0, 0
        side, zr = divmod(q, p["bz"])
        t = (t0 + p["bt"]) % T if side else (t0 - 1 + T) % T
        return p["NA"] + p["NB"] + (side * p["bz"] + zr) * p["by"], p["by"], y0 + Y * (z0 + zr + Z * t)
    return 0, 0, 0


def neighbours(p, tid, y0, z0, t0, p_out):
    """(own cb, [8 staged positions]) of thread tid, as the kernel computes them."""
    X2, by, bz, bt = p["X2"], p["by"], p["bz"], p["bt"]
    xh = tid % X2
    r = tid // X2
    yr = r % by
    r //= by
    zr, tr = r % bz, r // bz
    y, z, t = y0 + yr, z0 + zr, t0 + tr
    cb = xh + X2 * (y + p["Y"] * (z + p["Z"] * t))
    bpar = (y + z + t + p_out) & 1
    own = rowA(p, tr, zr, yr)
    sn = [own * X2 + ((xh + 1) % X2 if bpar else xh), own * X2 + (xh if bpar else (xh - 1 + X2) % X2)]
    sn.append((rowA(p, tr, zr, yr + 1) if p["hy"] else rowA(p, tr, zr, (yr + 1) % by)) * X2 + xh)
    sn.append((rowA(p, tr, zr, yr - 1) if p["hy"] else rowA(p, tr, zr, (yr - 1 + by) % by)) * X2 + xh)
    if zr + 1 < bz:
        rz = rowA(p, tr, zr + 1, yr)
    elif p["hz"]:
        rz = p["NA"] + (tr * 2 + 1) * by + yr
    else:
        rz = rowA(p, tr, 0, yr)
    sn.append(rz * X2 + xh)
    if zr > 0:
        rz = rowA(p, tr, zr - 1, yr)
    elif p["hz"]:
        rz = p["NA"] + tr * 2 * by + yr
    else:
        rz = rowA(p, tr, bz - 1, yr)
    sn.append(rz * X2 + xh)
    if tr + 1 < bt:
        rt = rowA(p, tr + 1, zr, yr)
    elif p["ht"]:
        rt = p["NA"] + p["NB"] + (bz + zr) * by + yr
    else:
        rt = rowA(p, 0, zr, yr)
    sn.append(rt * X2 + xh)
    if tr > 0:
        rt = rowA(p, tr - 1, zr, yr)
    elif p["ht"]:
        rt = p["NA"] + p["NB"] + zr * by + yr
    else:
        rt = rowA(p, bt - 1, zr, yr)
    sn.append(rt * X2 + xh)
    return cb, (2 * xh + bpar, y, z, t), sn


def check_plan(dims, prec, by, bz, bt, tiles=None):
    p = plan(dims, prec, by, bz, bt)
    assert p is not None
    X, Y, Z, T = dims
    X2, S = p["X2"], p["S"]
    Vh = X2 * Y * Z * T
    ntiles = p["nty"] * p["ntz"] * p["ntt"]
    seen = set()
    for tile in (range(ntiles) if tiles is None else tiles):
        tt, rem = divmod(tile, p["nty"] * p["ntz"])
        tz, ty = divmod(rem, p["nty"])
        y0, z0, t0 = ty * by, tz * bz, tt * bt
        # the staged rows: compact row -> global row index y + Y (z + Z t)
        staged = {}
        for q in range(p["nslot"]):
            srow, nrows, grow = segment(p, y0, z0, t0, q)
            if nrows == 0:
                continue
            # a run is contiguous in the checkerboard order
            assert (grow % Y) + nrows <= Y
            for j in range(nrows):
                assert srow + j not in staged, "compact row staged twice"
                staged[srow + j] = grow + j
            # bulk-copy alignment and bounds (16-byte chunks, FP16 norms)
            assert (srow + nrows) * X2 <= S
            assert (grow * X2 * 16) % 16 == 0 and (nrows * X2 * 16) % 16 == 0
            if prec == "f16":
                assert (grow * X2 * 4) % 16 == 0 and (nrows * X2 * 4) % 16 == 0 and (srow * X2 * 4) % 16 == 0
        assert sorted(staged) == list(range(p["rows"])), "every compact row is staged"
        total = sum(segment(p, y0, z0, t0, q)[1] for q in range(p["nslot"])) * X2
        assert total * (52 if prec == "f16" else 96) == p["buf"]
        for p_out in (0, 1):
            for tid in range(p["threads"]):
                cb, (x, y, z, t), sn = neighbours(p, tid, y0, z0, t0, p_out)
                assert 0 <= cb < Vh
                if p_out == 0:
                    assert cb not in seen
                    seen.add(cb)
                want = [((x + 1) % X, y, z, t), ((x - 1) % X, y, z, t), (x, (y + 1) % Y, z, t),
                        (x, (y - 1) % Y, z, t), (x, y, (z + 1) % Z, t), (x, y, (z - 1) % Z, t),
                        (x, y, z, (t + 1) % T), (x, y, z, (t - 1) % T)]
                for pos, (nx, ny, nz, nt) in zip(sn, want):
                    assert 0 <= pos < S
                    row, xh = divmod(pos, X2)
                    g = staged[row]
                    assert g == ny + Y * (nz + Z * nt), "neighbour row"
                    assert xh == nx // 2, "neighbour x"
                    assert (nx + ny + nz + nt) % 2 == 1 - p_out
    if tiles is None:
        assert len(seen) == Vh


def shapes(dims, prec):
    X, Y, Z, T = dims
    out = []
    for by, bz, bt in itertools.product(range(1, Y + 1), range(1, Z + 1), range(1, T + 1)):
        p = plan(dims, prec, by, bz, bt)
        if p is not None:
            out.append((by, bz, bt))
    return out


@pytest.mark.parametrize("dims", [(8, 4, 4, 8), (8, 8, 4, 4), (4, 4, 4, 8), (8, 2, 2, 16), (16, 4, 2, 4)])
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_every_shape_every_tile_small(dims, prec):
    sh = shapes(dims, prec)
    if prec == "f16" and (dims[0] // 2) % 4:
        assert sh == []
        return
    assert sh, "some tile shape applies"
    for by, bz, bt in sh:
        check_plan(dims, prec, by, bz, bt)


@pytest.mark.parametrize("dims,prec", [((16, 16, 16, 32), "f32"), ((24, 24, 24, 48), "f16"), ((32, 32, 32, 64), "f16"),
                                       ((16, 16, 16, 32), "f16"), ((24, 24, 24, 48), "f32")])
def test_workload_shapes_boundary_tiles(dims, prec):
    """The benchmark lattices: every applicable shape, on the tiles at the
    lattice corners (all wraps) and one interior tile."""
    for by, bz, bt in shapes(dims, prec):
        p = plan(dims, prec, by, bz, bt)
        nty, ntz, ntt = p["nty"], p["ntz"], p["ntt"]
        corner = []
        for ty, tz, tt in itertools.product({0, nty - 1}, {0, ntz - 1}, {0, ntt - 1}):
            corner.append((tt * ntz + tz) * nty + ty)
        mid = ((ntt // 2) * ntz + ntz // 2) * nty + nty // 2
        check_plan(dims, prec, by, bz, bt, tiles=sorted(set(corner + [mid])))
