"""The two in-place streaming maps of the step kernel, emulated location by location on
the host: the AA pattern and the esoteric twist (lbm_params.streaming 0 and 1).

A location is (cell, slot) of a single buffer of 7 slots per cell. Each map says, for
a step of a given parity, from which location a cell reads the incoming population of
direction i and into which location it writes the outgoing one. Pinned here, without
the GPU:
* the twist is the AA map composed with one fixed relabelling (slot 2, 4, 6 of a cell
  stored with the cell one step along +x, +y, +z), so its buffer is a permutation of
  the AA buffer after every step;
* each map is in place: at every parity the locations a cell reads are exactly the
  locations it writes, and the cells' sets partition the buffer (no two threads touch
  one location in a step);
* stepping in place with a nonlinear cell-local map and reading the buffer through the
  next step's read map equals two-buffer pull streaming f_i(x) <- f*_i(x - e_i).
"""
import itertools

import numpy as np
import pytest

OPP = (0, 2, 1, 4, 3, 6, 5)
E = ((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))
SHAPES = [(5, 4, 3), (1, 1, 1), (2, 1, 3), (32, 1, 1), (3, 2, 1), (4, 4, 4)]


class Grid:
    def __init__(self, nx, ny, nz):
        self.n = (nx, ny, nz)
        self.ncell = nx * ny * nz

    def xyz(self, c):
        nx, ny, _ = self.n
        return c % nx, (c // nx) % ny, c // (nx * ny)

    def cell(self, x, y, z):
        nx, ny, nz = self.n
        return (x % nx) + nx * ((y % ny) + ny * (z % nz))

    def nb(self, c, i):  # the cell one link along e_i (periodic)
        x, y, z = self.xyz(c)
        ex, ey, ez = E[i]
        return self.cell(x + ex, y + ey, z + ez)


def aa_read(g, c, i, odd):
    return (g.nb(c, OPP[i]), OPP[i]) if odd else (c, i)


def aa_write(g, c, i, odd):
    return (g.nb(c, i), i) if odd else (c, OPP[i])


def relabel(g, loc):
    """Twist storage of an AA location: slots 2, 4, 6 move one cell along +x, +y, +z."""
    cell, s = loc
    return (g.nb(cell, s - 1), s) if s in (2, 4, 6) else (cell, s)


def eso_read(g, c, i, odd):
    """The twist as the step kernel states it: -x, -y, -z come from x + e_x, x + e_y,
    x + e_z, the rest from the own cell; slot i on even steps, opp(i) on odd ones."""
    cell = g.nb(c, i - 1) if i in (2, 4, 6) else c
    return cell, (OPP[i] if odd else i)


def eso_write(g, c, i, odd):
    """+x, +y, +z go to x + e_x, x + e_y, x + e_z, the rest to the own cell; slot opp(i)
    on even steps, i on odd ones."""
    cell = g.nb(c, i) if i in (1, 3, 5) else c
    return cell, (i if odd else OPP[i])


MAPS = {"aa": (aa_read, aa_write), "eso": (eso_read, eso_write)}


@pytest.mark.parametrize("shape", SHAPES)
def test_twist_is_the_aa_map_under_one_relabelling(shape):
    g = Grid(*shape)
    for c, i, odd in itertools.product(range(g.ncell), range(7), (0, 1)):
        assert eso_read(g, c, i, odd) == relabel(g, aa_read(g, c, i, odd)), (c, i, odd)
        assert eso_write(g, c, i, odd) == relabel(g, aa_write(g, c, i, odd)), (c, i, odd)
    # the relabelling is a permutation of the locations
    locs = [(c, s) for c in range(g.ncell) for s in range(7)]
    assert sorted(relabel(g, loc) for loc in locs) == sorted(locs)


@pytest.mark.parametrize("kind", ["aa", "eso"])
@pytest.mark.parametrize("shape", SHAPES)
def test_maps_are_in_place(kind, shape):
    read, write = MAPS[kind]
    g = Grid(*shape)
    for odd in (0, 1):
        seen = set()
        for c in range(g.ncell):
            r = {read(g, c, i, odd) for i in range(7)}
            w = {write(g, c, i, odd) for i in range(7)}
            assert len(r) == 7 and r == w, (kind, c, odd)
            assert not (r & seen)
            seen |= r
        assert len(seen) == 7 * g.ncell


def test_twist_touches_the_same_cells_at_both_parities():
    g = Grid(5, 4, 3)
    for c in range(g.ncell):
        cells = [{eso_read(g, c, i, odd)[0] for i in range(7)} for odd in (0, 1)]
        assert cells[0] == cells[1] == {c, g.nb(c, 1), g.nb(c, 3), g.nb(c, 5)}


def _cell_map(f):
    s = f.sum(axis=0)
    return np.stack([f[i] + 0.3 * (s / 7 - f[i]) + 0.05 * np.sin((i + 1) * f[i] + s) for i in range(7)])


@pytest.mark.parametrize("kind", ["aa", "eso"])
@pytest.mark.parametrize("shape", SHAPES)
def test_in_place_stepping_equals_pull_streaming(kind, shape):
    read, write = MAPS[kind]
    g = Grid(*shape)
    rng = np.random.default_rng(11)
    f0 = rng.standard_normal((7, g.ncell))  # canonical: f_i of each cell
    buf = {}
    for c in range(g.ncell):  # the state before an even step, in this map's storage
        for i in range(7):
            buf[read(g, c, i, 0)] = f0[i, c]
    assert len(buf) == 7 * g.ncell
    ref = f0.copy()
    for step in range(6):
        odd = step & 1
        pre = np.array([[buf[read(g, c, i, odd)] for c in range(g.ncell)] for i in range(7)])
        post = _cell_map(pre)
        for c in range(g.ncell):
            for i in range(7):
                buf[write(g, c, i, odd)] = post[i, c]
        # two buffers, pull: f_i(x) <- f*_i(x - e_i)
        rpost = _cell_map(ref)
        ref = np.array([[rpost[i, g.nb(c, OPP[i])] for c in range(g.ncell)] for i in range(7)])
        nxt = 1 - odd
        got = np.array([[buf[read(g, c, i, nxt)] for c in range(g.ncell)] for i in range(7)])
        assert np.array_equal(got, ref), (kind, shape, step)
