"""The short-range search's cell geometry, checked on the host with the binning arithmetic the
sort uses (FP32): particles closer than r_c must land in rows at most R apart (R = cell rows per
cutoff, 1, 2 or 3, rows (1 + 4 slack) r_c / R wide) and in an x-cell inside the run window the walk
derives from the other particle's FP32 position. This is the argument that lets the walk visit
only the (2R + 1)^2 row block around a particle's row (eq. (summation_short): the particles
"close to" it), including at the largest extent the parameters allow (4092 cutoff lengths) and
for pairs just inside the cutoff across a row or cell boundary."""
import numpy as np
import pytest

RC = 2.3e-5      # r_c in metres (the bench sphere's scale)
LO = -1.1e-3     # mesh origin


def slack_for(ext):
    return max(1e-4, 1e-6 * ext)


def sort_cell(x, cw):
    """The sort's cell index along one axis: floor(fl32(x - lo) * fl32(1 / (cw r_c)))."""
    f = (x - LO).astype(np.float32)
    inv = np.float32(1.0 / (cw * RC))
    return np.floor((f * inv).astype(np.float32)).astype(np.int64)


def walk_window(x, cw, slack):
    """The walk's x-window of cells for a particle at x (distance 0 from the row): cells
    floor(fl32(px -+ w) * fl32(1 / cw)) with px the FP32 position in cutoff units and
    w = 1 + slack."""
    px = ((x - LO) / RC).astype(np.float32)
    w = np.float32(1.0 + slack)
    iw = np.float32(1.0 / cw)
    c0 = np.floor(((px - w).astype(np.float32) * iw).astype(np.float32)).astype(np.int64)
    c1 = np.floor(((px + w).astype(np.float32) * iw).astype(np.float32)).astype(np.int64)
    return c0, c1


def pairs_near_boundaries(rng, cw, ext, n):
    # a at a random boundary k cw (+- a few ulps of the coordinate), b within r_c of a, with a
    # share of the separations just under r_c
    k = rng.integers(1, int(ext / cw) - 2, size=n)
    xa = LO + (k * cw + rng.uniform(-1e-6, 1e-6, size=n)) * RC
    d = rng.uniform(-1.0, 1.0, size=n)
    edge = rng.random(n) < 0.3
    d[edge] = np.sign(d[edge]) * (1.0 - 1e-9)
    return xa, xa + d * RC


@pytest.mark.parametrize("rows", [1, 2, 3])
@pytest.mark.parametrize("ext", [10.0, 500.0, 4092.0])
def test_close_particles_sit_at_most_rows_apart(rows, ext):
    rng = np.random.default_rng(int(ext) + rows)
    s = slack_for(ext)
    cw = (1.0 + 4.0 * s) / rows
    xa, xb = pairs_near_boundaries(rng, cw, ext, 200_000)
    ra, rb = sort_cell(xa, cw), sort_cell(xb, cw)
    assert np.all(np.abs(ra - rb) <= rows)
    # and uniformly spread pairs
    xa = LO + rng.uniform(0.0, ext - 1.0, size=200_000) * RC
    xb = xa + rng.uniform(-1.0, 1.0, size=xa.size) * RC
    assert np.all(np.abs(sort_cell(xa, cw) - sort_cell(xb, cw)) <= rows)


@pytest.mark.parametrize("nsub", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("ext", [10.0, 500.0, 4092.0])
def test_partner_cell_inside_the_run_window(nsub, ext):
    rng = np.random.default_rng(int(ext) * 7 + nsub)
    s = slack_for(ext)
    cw = (1.0 + 1e-9) / nsub
    xa, xb = pairs_near_boundaries(rng, cw, ext, 200_000)
    c0, c1 = walk_window(xa, cw, s)
    cb = sort_cell(xb, cw)
    assert np.all((c0 <= cb) & (cb <= c1))


def test_rows_without_the_slack_would_fail():
    # the check above has teeth: with rows exactly r_c / 2 (no widening by the slack), the FP32
    # binning puts some pairs just under r_c apart three rows apart
    rng = np.random.default_rng(5)
    cw = 0.5
    xa, xb = pairs_near_boundaries(rng, cw, 500.0, 200_000)
    assert np.any(np.abs(sort_cell(xa, cw) - sort_cell(xb, cw)) > 2)
