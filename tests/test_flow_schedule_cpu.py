"""The flow schedule's dependency rule, checked on the host against the
stencil's geometry: an item (step s, x-chunk, y tile, z tile) waits only for
the 27 items of step s - 1 around it. That must cover every item that wrote a
u^s value it uses (its taps reach R planes/rows/columns past its own points)
and every item that still reads the u^{s-1} values it overwrites; both hold
when every x-chunk and tile but the last along its axis spans at least R
planes, rows or columns (the last may be shorter: nothing lies beyond it).
Checked for every tile shape the TMA kernel has, at each radius it is built
for, with x-chunks down to R, on grids with ragged last chunks and tiles, and on
domains thinner than R (one chunk or tile along an axis)."""
import itertools

import numpy as np
import pytest

# (tile_z, tile_y) of the FP32 TMA kernel: radius <= 8 and radius 9-12
TILES_LOW = [(32, 32), (64, 16), (128, 8), (32, 16), (64, 8)]
TILES_HIGH = [(32, 32), (32, 16)]


def _owner(n, size):
    """Item index along one axis of each node."""
    return np.arange(n) // size


def _check(N, R, tz, ty, xb):
    Nx, Ny, Nz = N
    ox, oy, oz = _owner(Nx, xb), _owner(Ny, ty), _owner(Nz, tz)
    nbx, nby, nbz = ox[-1] + 1, oy[-1] + 1, oz[-1] + 1
    for bx, by, bz in itertools.product(range(nbx), range(nby), range(nbz)):
        x0, x1 = bx * xb, min((bx + 1) * xb, Nx)
        y0, y1 = by * ty, min((by + 1) * ty, Ny)
        z0, z1 = bz * tz, min((bz + 1) * tz, Nz)
        # u^s values the item's points use: R past its points on every axis (inside the domain)
        xs = ox[max(x0 - R, 0):min(x1 + R, Nx)]
        ys = oy[max(y0 - R, 0):min(y1 + R, Ny)]
        zs = oz[max(z0 - R, 0):min(z1 + R, Nz)]
        # writers of those values (items of step s - 1) and, by the stencil's symmetry, the
        # readers of the item's own u^{s-1} values at step s - 1: within one item on each axis
        for own, touched in ((bx, xs), (by, ys), (bz, zs)):
            assert np.abs(touched - own).max() <= 1
    return nbx * nby * nbz


@pytest.mark.parametrize("R", list(range(1, 13)))
def test_dependency_neighbourhood_covers_the_stencil(R):
    rng = np.random.default_rng(R)
    tiles = TILES_LOW if R <= 8 else TILES_HIGH
    for tz, ty in tiles:
        for xb in sorted({R, R + 1, 2 * R + 3, 40}):
            N = tuple(int(v) for v in rng.integers(2 * R + 1, 150, size=3))
            assert _check(N, R, tz, ty, xb) >= 1


def test_a_shorter_chunk_breaks_the_rule():
    """x-chunks shorter than R would let an item read planes two chunks away:
    the host rejects them (x_block >= k/2)."""
    with pytest.raises(AssertionError):
        _check((60, 40, 70), 4, 32, 16, 3)


def test_dependencies_have_lower_item_numbers():
    """Items are numbered step-major (z fastest), so every dependency (step s - 1)
    precedes its dependent: the lowest unfinished item never waits."""
    nbz, nby, nbx, nt = 3, 4, 5, 6
    per_step = nbz * nby * nbx
    for s in range(1, nt):
        for j in range(per_step):
            item = s * per_step + j
            bx, r = divmod(j, nbz * nby)
            by, bz = divmod(r, nbz)
            for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3):
                nx, ny, nz = bx + dx, by + dy, bz + dz
                if 0 <= nx < nbx and 0 <= ny < nby and 0 <= nz < nbz:
                    dep = (s - 1) * per_step + (nx * nby + ny) * nbz + nz
                    assert dep < item


@pytest.mark.parametrize("R", [1, 2, 4, 8, 12])
def test_short_last_items_and_thin_domains(R):
    """A last chunk or tile shorter than R, after full ones, and a domain
    thinner than R along an axis (a single chunk or tile) keep the rule."""
    tz, ty = (32, 16)
    cases = [((1, 1, 1), 40), ((3, 2, 5), 40), ((R - 1 or 1, 40, 70), 40),
             ((3 * R + 1, 2 * ty + 1, 2 * tz + 1), R),      # last chunk, tile row and column: 1 wide
             ((2 * R + R // 2 + 1, ty + 1, 70), R)]
    for N, xb in cases:
        assert _check(N, R, tz, ty, max(xb, R)) >= 1
