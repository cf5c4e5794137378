"""The slab order of the FP32 correction sweep (option slab32) is a Gauss-Seidel
order equivalent to four whole colour stages (Sec. III.B: each colour's cells are
updated from the current values of the other colours).

Checked on the host, without a GPU: the order that libmg.so reports
(mg_slab_order) is replayed on a small periodic grid with a colour-stage update
that reads the 18 neighbours of Sec. III.B's stencil, and must give the same bits
as the four whole stages; every cell is updated exactly once per sweep; and a
schedule with a colour moved one plane too far ahead is caught by the replay."""
import numpy as np
import pytest

from paper_1303_0008_gb300 import mg

# the 18 neighbours of the 19-point stencil: 6 faces and 12 edges
OFFS = [o for o in np.ndindex(3, 3, 3)
        if 1 <= sum(abs(d - 1) for d in o) <= 2]
OFFS = [(a - 1, b - 1, c - 1) for a, b, c in OFFS]
assert len(OFFS) == 18


def colour_of(n):
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return ((i + k) & 1) + 2 * ((j + k) & 1)


def update(e, rhs, col, colour, planes):
    """One colour's cells on the given z planes: a nonlinear function of the 18
    neighbours (they are all of other colours) and the cell's own right-hand side."""
    n = e.shape[0]
    acc = np.zeros_like(e)
    for dk, dj, di in OFFS:
        acc += np.roll(e, shift=(-dk, -dj, -di), axis=(0, 1, 2)) * (1 + 0.01 * (dk + 2 * dj + 3 * di))
    new = np.tanh(acc / 18.0) + rhs
    mask = np.zeros_like(col, dtype=bool)
    mask[list(planes)] = True
    mask &= col == colour
    out = e.copy()
    out[mask] = new[mask]
    return out, mask


def whole_stages(e, rhs, col):
    n = e.shape[0]
    for c in range(4):
        e, _ = update(e, rhs, col, c, range(n))
    return e


def replay(e, rhs, col, order):
    n = e.shape[0]
    count = np.zeros(e.shape, dtype=int)
    for c, z0, nz in order:
        e, mask = update(e, rhs, col, c, [(z0 + t) % n for t in range(nz)])
        count += mask
    return e, count


@pytest.mark.parametrize("n,slab", [(16, 8), (32, 8), (32, 16), (48, 8), (64, 16), (64, 32)])
def test_slab_order_matches_whole_colour_stages(n, slab):
    rng = np.random.default_rng(n * 1000 + slab)
    e0 = rng.standard_normal((n, n, n))
    rhs = 0.1 * rng.standard_normal((n, n, n))
    col = colour_of(n)
    order = mg.mg_slab_order(n, slab)
    assert len(order) == 4 * (n // slab)
    assert [c for c, _, _ in order] == [0, 1, 2, 3] * (n // slab)
    ref = whole_stages(e0.copy(), rhs, col)
    got, count = replay(e0.copy(), rhs, col, order)
    assert (count == 1).all()
    assert np.array_equal(got, ref)


def test_a_colour_one_plane_too_early_is_caught():
    """Move colour 1's first slab one plane up (so it runs on a plane whose upper
    neighbour colour 0 has not reached yet): the replay no longer matches."""
    n, slab = 32, 8
    rng = np.random.default_rng(7)
    e0 = rng.standard_normal((n, n, n))
    rhs = 0.1 * rng.standard_normal((n, n, n))
    col = colour_of(n)
    order = mg.mg_slab_order(n, slab)
    bad = list(order)
    c, z0, nz = bad[1]
    assert c == 1
    c2, z2, nz2 = bad[5]
    bad[1] = (c, z0, nz + 1)
    bad[5] = (c2, z2 + 1, nz2 - 1)
    ref = whole_stages(e0.copy(), rhs, col)
    got, count = replay(e0.copy(), rhs, col, bad)
    assert (count == 1).all()
    assert not np.array_equal(got, ref)


@pytest.mark.parametrize("n,slab", [(32, 4), (32, 32), (40, 16), (8, 8)])
def test_slab_order_rejects_sizes_without_an_order(n, slab):
    with pytest.raises(mg.MGError) as e:
        mg.mg_slab_order(n, slab)
    assert e.value.status == mg.MG_EINVAL


@pytest.mark.parametrize("bad", [4, 12, 512, -8])
def test_slab_option_is_validated_without_gpu(bad):
    with pytest.raises(mg.MGError) as e:
        mg.mg_create_grid(64, mg.options(prec=mg.MG_MIXED, slab32=bad))
    assert e.value.status == mg.MG_EINVAL


@pytest.mark.parametrize("bad", [3, 16, -1])
def test_tile_option_is_validated_without_gpu(bad):
    with pytest.raises(mg.MGError) as e:
        mg.mg_create_grid(64, mg.options(prec=mg.MG_MIXED, tile32=bad))
    assert e.value.status == mg.MG_EINVAL
