"""Host model of the TMA-staged sweep's plane schedule (pf_sweep_tma.cu).

The kernel marches a CTA along z over a 32 x TY column tile: in step s the
first-colour threads update plane s over the tile plus a one-cell ring from
the staged planes s - 1 .. s + 1, the second-colour threads update plane
s - 2 from the new first-colour values of planes s - 3 .. s - 1 and write both
colours of it. Planes of rho, f and x_in live in rings of RING slots: a tile
away from the periodic seams has them issued by the producer warp once every
compute warp has released the slot's previous plane (end of step q + 3 for
plane q); a tile across a seam copies plane s + RING - 4 itself in step s.

This model replays that schedule on the host with the kernel's constants and
thread-to-cell maps and checks that
  * every ring slot a step reads holds the plane the step expects, and that
    plane was issued and waited for before the read;
  * the 16-byte copy chunks of the seam tiles cover the staged plane exactly;
  * every global access is in bounds and every cell is written exactly once;
  * the result equals one plain red-black Gauss-Seidel sweep (the smoother's
    per-cell update with weights 1 / (rho_c + rho_q)), first colour first.
No GPU is involved; the GPU parity tests check the kernel itself.
"""
import itertools
from dataclasses import dataclass

import numpy as np
import pytest

TX, OX, RN = 32, 4, 4


@dataclass(frozen=True)
class Tile:
    ty: int      # tile height (8 or 16)
    cpt: int     # cells of a colour per thread and plane (1 or 2)
    ring: int = 8

    @property
    def hx(self):
        return TX + 2 * OX

    @property
    def hy(self):
        return self.ty + 4

    @property
    def rxh(self):
        return (TX + 2) // 2

    @property
    def npl(self):
        return (self.ty + 2) * self.rxh

    @property
    def w1(self):
        return ((self.npl + 32 * self.cpt - 1) // (32 * self.cpt)) * 32

    @property
    def w2(self):
        return (TX // 2) * self.ty // self.cpt

    @property
    def nc(self):
        return self.w1 + self.w2


def zc_of(t, nx, ny, nz):
    zc = 32
    cols = ((nx + TX - 1) // TX) * ((ny + t.ty - 1) // t.ty)
    while zc > 2 and cols * ((nz + zc - 1) // zc) < 8 * 152:
        zc >>= 1
    if zc == 32 and cols * ((nz + 63) // 64) >= 8 * 152:
        zc = 64
    return zc


def gs_sweep(rho, f, xin, fs, c0):
    """One red-black Gauss-Seidel sweep, colour c0 first (periodic box)."""
    nz, ny, nx = rho.shape
    x = np.zeros_like(f) if xin is None else xin.copy()
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    colour = (i + j + k) & 1
    shifts = [(2, 1), (2, -1), (1, 1), (1, -1), (0, 1), (0, -1)]
    w = [1.0 / (rho + np.roll(rho, sh, axis=ax)) for ax, sh in shifts]
    for c in (c0, 1 - c0):
        num = f * fs + sum(wq * np.roll(x, sh, axis=ax) for wq, (ax, sh) in zip(w, shifts))
        v = num / sum(w)
        x = np.where(colour == c, v, x)
    return x


def model_sweep(t, rho, f, xin, fs, c0, edge_ahead=None, zc=None):
    """The sweep as the kernel schedules it; edge_ahead: how many planes ahead
    a seam tile copies (the kernel: RING - 4); zc: planes per CTA (the
    kernel's choice for the grid when None; small grids get 2, so the tests
    pass larger chunks to make the rings wrap)."""
    if edge_ahead is None:
        edge_ahead = t.ring - 4
    nz, ny, nx = rho.shape
    hx, hy, rxh, npl, ring = t.hx, t.hy, t.rxh, t.npl, t.ring
    zero = xin is None
    zc = zc_of(t, nx, ny, nz) if zc is None else zc
    grid = ((nx + TX - 1) // TX, (ny + t.ty - 1) // t.ty, (nz + zc - 1) // zc)
    out = np.full(rho.size, np.nan)
    writes = np.zeros(rho.size, dtype=int)
    src = {"rho": rho.ravel(), "f": f.ravel(), "x": None if zero else xin.ravel()}
    sz = nx * ny
    for bz, by, bx in itertools.product(range(grid[2]), range(grid[1]), range(grid[0])):
        i0, j0, z0 = bx * TX, by * t.ty, bz * zc
        z1 = min(z0 + zc, nz)
        p0 = z0 - 2
        qmax = z1 + 1 - p0
        interior = i0 - OX >= 0 and i0 + TX + OX <= nx and j0 - 2 >= 0 and j0 + t.ty + 2 <= ny
        ringbuf = {a: np.full((ring, hy, hx), np.nan) for a in ("rho", "f", "x")}
        held = {a: [None] * ring for a in ("rho", "f", "x")}
        waited = -1
        nbuf = np.full((RN, npl), np.nan)
        nheld = [None] * RN

        def stage(q):
            if q > qmax:
                return
            slot, z = q % ring, (p0 + q) % nz
            for a in ("rho", "f") + (() if zero else ("x",)):
                for r in range(hy):
                    jj = (j0 - 2 + r) % ny
                    for c in range(0, hx, 4):   # 16-byte chunks, wrapped addresses
                        ii = (i0 - OX + c) % nx
                        assert ii % 4 == 0 and ii + 4 <= nx   # never straddles the seam
                        g = (z * ny + jj) * nx + ii
                        ringbuf[a][slot, r, c:c + 4] = src[a][g:g + 4]
                held[a][slot] = q

        def rd(a, q, r, c):
            assert held[a][q % ring] == q and q <= waited, (a, q, held[a][q % ring], waited)
            assert 0 <= r < hy and 0 <= c < hx
            return ringbuf[a][q % ring, r, c]

        def rdn(q, idx):
            assert nheld[q % RN] == q and 0 <= idx < npl
            return nbuf[q % RN, idx]

        # thread -> cell maps of the two colour groups
        cells = []
        for tid in range(t.nc):
            first = tid < t.w1
            for h in range(t.cpt):
                if first:
                    u = tid + h * t.w1
                    b1, m = divmod(u, rxh)
                    cells.append((True, u < npl, (b1 + 1) * hx + 2 * m + OX - 1, b1 * rxh + m,
                                  (c0 + b1 + z0) & 1, None))
                else:
                    tt = tid - t.w1 + h * t.w2
                    tb, m = tt >> 4, tt & 15
                    cells.append((False, j0 + tb < ny and i0 + 2 * m < nx,
                                  (tb + 2) * hx + 2 * m + OX, (tb + 1) * rxh + m,
                                  (1 + c0 + tb + z0) & 1, (j0 + tb) * nx + i0 + 2 * m))
        # prologue: the producer fills the ring (interior), or the compute
        # threads copy planes 0 .. ring - 4 (tiles across a seam)
        for q in range(ring if interior else edge_ahead + 1):
            stage(q)
        waited = 1
        for s in range(1, qmax + 1):
            if s + 1 <= qmax:
                waited = s + 1
            if not interior:
                stage(s + edge_ahead)   # the slot of plane s - 4, last read in step s - 1
            odd = s & 1
            newn = {}
            for first, act, ce, cn, e0, gcol in cells:
                if first and s + 1 <= qmax and act:
                    c = ce + (e0 ^ odd)
                    r, col = divmod(c, hx)
                    rc = rd("rho", s, r, col)
                    nb = [(s, r, col - 1), (s, r, col + 1), (s, r - 1, col), (s, r + 1, col),
                          (s - 1, r, col), (s + 1, r, col)]
                    w = [1.0 / (rc + rd("rho", *n)) for n in nb]
                    num = rd("f", s, r, col) * fs
                    if not zero:
                        num += sum(wq * rd("x", *n) for wq, n in zip(w, nb))
                    newn[cn] = num / sum(w)
                elif not first and s >= 4:
                    s2 = e0 ^ odd
                    c = ce + s2
                    r, col = divmod(c, hx)
                    b = s - 2
                    rc = rd("rho", b, r, col)
                    nb = [(b, r, col - 1), (b, r, col + 1), (b, r - 1, col), (b, r + 1, col),
                          (b - 1, r, col), (b + 1, r, col)]
                    w = [1.0 / (rc + rd("rho", *n)) for n in nb]
                    vals = [rdn(b, cn), rdn(b, cn + 1), rdn(b, cn + s2 - rxh),
                            rdn(b, cn + s2 + rxh), rdn(b - 1, cn + s2), rdn(b + 1, cn + s2)]
                    v2 = (rd("f", b, r, col) * fs + sum(wq * v for wq, v in zip(w, vals))) / sum(w)
                    other = rdn(b, cn + 1 - s2)
                    if act:
                        k = p0 + b
                        assert z0 <= k < z1
                        g = k * sz + gcol
                        assert 0 <= g and g + 1 < rho.size
                        out[g], out[g + 1] = (v2, other) if s2 == 0 else (other, v2)
                        writes[g] += 1
                        writes[g + 1] += 1
            if s + 1 <= qmax:
                nbuf[s % RN] = np.nan
                for idx, v in newn.items():
                    nbuf[s % RN, idx] = v
                nheld[s % RN] = s
            # end of step s: plane s - 3 released, the producer issues plane s - 3 + ring
            if s >= 3 and interior:
                stage(s - 3 + ring)
    return out.reshape(rho.shape), writes.reshape(rho.shape)


TILES = [Tile(8, 2), Tile(8, 1), Tile(16, 2), Tile(16, 1)]


@pytest.mark.parametrize("t", TILES, ids=lambda t: f"{t.ty}x{t.cpt}")
def test_thread_groups_and_copy_chunks(t):
    assert t.cpt * t.w1 >= t.npl and t.cpt * t.w2 == (TX // 2) * t.ty
    assert t.nc % 32 == 0
    cpr, nch = t.hx // 4, (t.hx // 4) * t.hy
    per = (nch + t.nc - 1) // t.nc
    cover = sorted(r * t.hx + 4 * (ch - r * cpr)
                   for tid in range(t.nc) for k in range(per)
                   for ch in [tid + k * t.nc] if ch < nch for r in [ch // cpr])
    assert cover == list(range(0, t.hy * t.hx, 4))
    # a staged plane starts on a 128-byte boundary in shared memory
    assert t.hx * t.hy * 4 % 128 == 0


@pytest.mark.parametrize("t", TILES, ids=lambda t: f"{t.ty}x{t.cpt}")
@pytest.mark.parametrize("n,zc", [((48, 16, 8), None), ((48, 16, 16), 16), ((96, 24, 20), 10),
                                  ((64, 40, 12), 12)])
def test_schedule_reproduces_one_red_black_sweep(t, n, zc):
    """The kernel's own chunking (two planes per CTA on these small grids) and
    chunks long enough for every ring to wrap several times."""
    nx, ny, nz = n
    if t.ty == 16 and ny < 20:
        pytest.skip("32 x 16 tiles need 20 rows")
    rng = np.random.default_rng(nx + ny + nz + t.ty)
    rho = rng.uniform(1.0, 10.0, (nz, ny, nx))
    f = rng.uniform(-1.0, 1.0, (nz, ny, nx))
    for zero, c0 in itertools.product((True, False), (0, 1)):
        xin = None if zero else rng.uniform(-1.0, 1.0, (nz, ny, nx))
        got, writes = model_sweep(t, rho, f, xin, 0.3, c0, zc=zc)
        assert np.all(writes == 1)
        np.testing.assert_allclose(got, gs_sweep(rho, f, xin, 0.3, c0), rtol=1e-13, atol=1e-14)


def test_copying_one_plane_further_ahead_is_caught():
    """The model fails if the seam tiles copied plane s + RING - 3 in step s:
    its slot then still holds plane s - 3, which the second colour reads in
    that step. So the slot checks are not vacuous."""
    t = Tile(8, 2)
    rng = np.random.default_rng(3)
    rho = rng.uniform(1.0, 10.0, (16, 16, 48))
    f = rng.uniform(-1.0, 1.0, (16, 16, 48))
    got, _ = model_sweep(t, rho, f, None, 0.3, 0, zc=16)
    np.testing.assert_allclose(got, gs_sweep(rho, f, None, 0.3, 0), rtol=1e-13, atol=1e-14)
    with pytest.raises(AssertionError):
        model_sweep(t, rho, f, None, 0.3, 0, edge_ahead=t.ring - 3, zc=16)
