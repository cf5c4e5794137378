"""Particles to mesh (TSC and CIC, Sec. VI) and the N_pc refinement criterion
(Sec. III.B) through the C-ABI, against the CPU oracle."""
import numpy as np
import pytest

from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1303_0008_gb300 import mg  # noqa: E402


def clustered_particles(count, seed):
    """Particles in a few Gaussian clumps plus a uniform background (box units)."""
    rng = np.random.default_rng(seed)
    k = count // 2
    centres = rng.random((4, 3))
    clump = centres[rng.integers(0, 4, k)] + 0.05 * rng.standard_normal((k, 3))
    pos = np.concatenate([clump, rng.random((count - k, 3))])
    return np.ascontiguousarray(np.mod(pos, 1.0).T)


def density(g, level, shape):
    out = np.empty(shape)
    mg.mg_get_density(g, level, -1, out)
    return out


@pytest.mark.parametrize("scheme", [mg.MG_CIC, mg.MG_TSC])
def test_domain_assignment_matches_the_oracle(scheme):
    n = 32
    pos = clustered_particles(40000, 11)
    mass = np.random.default_rng(12).random(pos.shape[1])
    mass /= mass.sum()
    want = O.assign_density(n, pos, mass, scheme)
    for on_device in (False, True):
        g = mg.mg_create_grid(n)
        try:
            if on_device:
                mg.mg_assign_density(g, 0, torch.from_numpy(pos).cuda(),
                                     torch.from_numpy(mass).cuda(), scheme)
            else:
                mg.mg_assign_density(g, 0, pos, mass, scheme)
            d = density(g, 0, (n,) * 3)
        finally:
            mg.mg_destroy_grid(g)
        assert np.abs(d - want).max() <= 1e-12 * np.abs(want).max()
        assert abs((d + 1.0).mean() - 1.0) < 1e-12


def test_nonfinite_particles_are_dropped_and_positions_fold():
    n = 16
    pos = clustered_particles(2000, 5)
    bad = pos.copy()
    bad[0, 7] = np.nan
    bad[2, 9] = np.inf
    shifted = pos + np.array([[2.0], [-3.0], [1.0]])   # whole periods: same density
    g = mg.mg_create_grid(n)
    try:
        mg.mg_assign_density(g, 0, np.ascontiguousarray(shifted))
        a = density(g, 0, (n,) * 3)
        mg.mg_assign_density(g, 0, np.ascontiguousarray(bad))
        b = density(g, 0, (n,) * 3)
    finally:
        mg.mg_destroy_grid(g)
    want = O.assign_density(n, pos)
    assert np.abs(a - want).max() <= 1e-12 * np.abs(want).max()
    keep = np.ones(pos.shape[1], bool)
    keep[[7, 9]] = False
    want_b = O.assign_density(n, pos[:, keep], np.full(keep.sum(), 1.0 / pos.shape[1]))
    assert np.abs(b - want_b).max() <= 1e-12 * np.abs(want_b).max()


def test_refinement_from_particles_end_to_end():
    """Particles -> domain density -> N_pc blocks -> level-1 patches -> density on
    the patches -> N_pc blocks again -> level-2 patches -> a converged solve."""
    n, count, npc = 32, 60000, 9.0
    pos = clustered_particles(count, 21)
    mp = 1.0 / count
    want0 = O.assign_density(n, pos)
    g = mg.mg_create_grid(n)
    try:
        mg.mg_assign_density(g, 0, pos)
        org1 = mg.mg_refine_blocks(g, 0, npc, mp)
        assert np.array_equal(org1, O.refine_blocks(want0, npc, mp))
        assert 0 < len(org1) < (n // 4) ** 3
        mg.mg_add_patches(g, 1, org1)
        mg.mg_assign_density(g, 1, pos)
        d1 = density(g, 1, (len(org1), 8, 8, 8))
        dense1 = O.assign_density(2 * n, pos)
        covered = np.zeros((2 * n,) * 3, bool)
        for q, o in enumerate(org1):
            want = dense1[o[2]:o[2] + 8, o[1]:o[1] + 8, o[0]:o[0] + 8]
            assert np.abs(d1[q] - want).max() <= 1e-11 * max(1.0, np.abs(want).max())
            covered[o[2]:o[2] + 8, o[1]:o[1] + 8, o[0]:o[0] + 8] = True
        org2 = mg.mg_refine_blocks(g, 1, npc, mp)
        assert np.array_equal(org2, O.refine_blocks(dense1, npc, mp, covered))
        # level-2 patches must nest in level 1 with a one-cell margin; keep those
        ok = [o for o in org2 if all(covered[(o[2] // 2 + dz) % (2 * n), (o[1] // 2 + dy) % (2 * n),
                                             (o[0] // 2 + dx) % (2 * n)]
                                     for dz in (-1, 4) for dy in (-1, 4) for dx in (-1, 4))]
        if ok:
            mg.mg_add_patches(g, 2, np.array(ok, dtype=np.int32))
            mg.mg_assign_density(g, 2, pos)
        st = mg.mg_solve(g, 0, 1e-3, 1.0, 1e-9)
        assert st["rc"] == mg.MG_OK
        for lvl in range(1, 3 if ok else 2):
            assert mg.mg_get_level_stats(g, lvl)["res"] < 1e-9
    finally:
        mg.mg_destroy_grid(g)


def test_assignment_and_refinement_errors():
    g = mg.mg_create_grid(16)
    try:
        pos = clustered_particles(100, 1)
        with pytest.raises(mg.MGError):
            mg.mg_assign_density(g, 0, pos, scheme=3)
        with pytest.raises(mg.MGError):
            mg.mg_assign_density(g, 1, pos)            # no level-1 patches
        with pytest.raises(mg.MGError):
            mg.mg_refine_blocks(g, 0, 9.0, 0.01)       # no density yet
    finally:
        mg.mg_destroy_grid(g)
