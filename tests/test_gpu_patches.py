"""GPU parity of the refinement levels (8^3 patches, coarse-to-fine Dirichlet fill,
FAS on the patch union) against the CPU oracle, through the C-ABI.

Each level is checked on its own: the oracle solves level l with its Dirichlet
values taken from the GPU's level l-1, so both sides solve the same system.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_0008_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1303_0008_gb300 import mg  # noqa: E402

ALPHA = I.alpha_kappa_for_rv(8.0)


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def solve_hierarchy(h, alpha=ALPHA, kappa=1.0, tol=1e-11, zero_start=False, **opt):
    n0 = h["delta0"].shape[0]
    g = mg.mg_create_grid(n0, mg.options(**opt))
    out = {"levels": []}
    try:
        mg.mg_set_density(g, 0, -1, h["delta0"])
        for lvl, L in enumerate(h["levels"], start=1):
            if len(L["origins"]) == 0:
                continue
            mg.mg_add_patches(g, lvl, L["origins"])
            mg.mg_set_density(g, lvl, -1, np.ascontiguousarray(L["delta"]))
            if zero_start:
                mg.mg_set_field(g, lvl, -1, np.zeros((len(L["origins"]), 8, 8, 8)))
        out["stats"] = mg.mg_solve(g, 0, alpha, kappa, tol, check=False)
        phi0 = np.empty_like(h["delta0"])
        mg.mg_get_field(g, 0, -1, phi0)
        out["phi0"] = phi0
        for lvl, L in enumerate(h["levels"], start=1):
            if len(L["origins"]) == 0:
                continue
            phi = np.empty((len(L["origins"]), 8, 8, 8))
            mg.mg_get_field(g, lvl, -1, phi)
            force = np.empty((3, len(L["origins"]), 8, 8, 8))
            mg.mg_get_force(g, lvl, -1, force)
            one = np.empty(512)
            mg.mg_get_field(g, lvl, 1, one)
            assert np.array_equal(one.reshape(8, 8, 8), phi[1])
            out["levels"].append({"phi": phi, "force": force})
    finally:
        mg.mg_destroy_grid(g)
    return out


@pytest.fixture(scope="module")
def small():
    return I.refined_hierarchy(16, 2.0, 5, thresholds=(15.0, 40.0))


@pytest.mark.parametrize("galerkin", [1, 0])
def test_refined_levels_match_oracle(small, galerkin):
    """Both coarse-grid corrections of the union (Galerkin, the default, and the
    rediscretised FAS) reach the oracle's solution of each level."""
    h = small
    res = solve_hierarchy(h, patch_galerkin=galerkin)
    assert res["stats"]["rc"] == mg.MG_OK, res["stats"]
    l1, l2 = h["levels"]
    # level 1 against the oracle, Dirichlet values from the GPU's domain solution
    ref1, st1 = O.patch_solve(16, 1, l1["origins"], l1["delta"], res["phi0"], ALPHA, 1.0,
                              tol=1e-12)
    assert st1["status"] == O.OK
    assert rel(res["levels"][0]["phi"], ref1) < 1e-10
    # level 2, Dirichlet values from the GPU's level 1
    ref2, st2 = O.patch_solve(16, 2, l2["origins"], l2["delta"], res["levels"][0]["phi"], ALPHA,
                              1.0, parent_org=l1["origins"], tol=1e-12)
    assert st2["status"] == O.OK
    assert rel(res["levels"][1]["phi"], ref2) < 1e-10
    # the oracle's residual of the GPU's level solutions
    d1, _ = O.patch_residual(16, 1, l1["origins"], res["levels"][0]["phi"], l1["delta"],
                             res["phi0"], ALPHA, 1.0)
    assert np.abs(d1).max() < 1e-11


def test_patch_force_uses_neighbours_and_dirichlet_values(small):
    h = small
    res = solve_hierarchy(h)
    l1 = h["levels"][0]
    phi = res["levels"][0]["phi"]
    ghosts = O.patch_ghosts(16, 1, l1["origins"], res["phi0"])
    org = l1["origins"]
    table = {tuple(o // 8): q for q, o in enumerate(org)}
    n1 = 32
    ref = np.empty((3,) + phi.shape)
    for q, o in enumerate(org):
        blk = ghosts[q].copy()
        blk[1:9, 1:9, 1:9] = phi[q]
        for k in range(-1, 9):
            for j in range(-1, 9):
                for i in range(-1, 9):
                    x, y, z = (o[0] + i) % n1, (o[1] + j) % n1, (o[2] + k) % n1
                    p = table.get((x // 8, y // 8, z // 8))
                    if p is not None and p != q:
                        blk[k + 1, j + 1, i + 1] = phi[p, z % 8, y % 8, x % 8]
        inv2h = n1 / 2.0
        ref[0, q] = -0.5 * inv2h * (blk[1:9, 1:9, 2:10] - blk[1:9, 1:9, 0:8])
        ref[1, q] = -0.5 * inv2h * (blk[1:9, 2:10, 1:9] - blk[1:9, 0:8, 1:9])
        ref[2, q] = -0.5 * inv2h * (blk[2:10, 1:9, 1:9] - blk[0:8, 1:9, 1:9])
    assert rel(res["levels"][0]["force"], ref) < 1e-12


def test_refinement_improves_on_the_domain_solution():
    """Sec. IV.D: a refinement over the top-hat, same density, agrees with a domain
    solve at the refined resolution much better than the interpolated coarse one."""
    n0 = 16
    delta0 = I.tophat(n0, 10.0, 2.0)
    org1 = np.array([[x, y, z] for z in (8, 16) for y in (8, 16) for x in (8, 16)], dtype=np.int32)
    fine = I.tophat(2 * n0, 10.0, 4.0)
    same = fine.copy()
    same[same != 10.0] = delta0[delta0 != 10.0][0]
    cut = lambda a: np.stack([a[o[2]:o[2] + 8, o[1]:o[1] + 8, o[0]:o[0] + 8] for o in org1])
    h = {"delta0": delta0, "levels": [{"origins": org1, "delta": cut(same)},
                                      {"origins": np.zeros((0, 3), np.int32), "delta": None}]}
    res = solve_hierarchy(h)
    assert res["stats"]["rc"] == mg.MG_OK
    ref_fine, _ = O.fas_solve(fine, ALPHA, 1.0, tol=1e-11)
    interp = O.prolong_add(res["phi0"], np.zeros((2 * n0,) * 3))
    e_ref = np.abs(res["levels"][0]["phi"] - cut(ref_fine)).max()
    e_int = np.abs(cut(interp) - cut(ref_fine)).max()
    assert e_ref < 0.3 * e_int


def test_patch_errors():
    g = mg.mg_create_grid(16)
    try:
        with pytest.raises(mg.MGError) as e:
            mg.mg_add_patches(g, 1, [[4, 0, 0]])              # not a multiple of 8
        assert e.value.status == mg.MG_EINVAL
        with pytest.raises(mg.MGError) as e:
            mg.mg_add_patches(g, 1, [[8, 8, 8], [8, 8, 8]])   # duplicate
        assert e.value.status == mg.MG_EINVAL
        with pytest.raises(mg.MGError) as e:
            mg.mg_add_patches(g, 2, [[0, 0, 0]])              # level 2 before level 1
        assert e.value.status == mg.MG_ESTATE
        # level 2 whose parents (dilated by one cell) leave level 1
        mg.mg_set_density(g, 0, -1, I.lognormal_delta(16, 1.0, 3))
        mg.mg_add_patches(g, 1, [[8, 8, 8]])
        mg.mg_set_density(g, 1, -1, np.zeros((1, 8, 8, 8)))
        mg.mg_add_patches(g, 2, [[24, 24, 24]])
        mg.mg_set_density(g, 2, -1, np.zeros((1, 8, 8, 8)))
        st = mg.mg_solve(g, 0, ALPHA, 1.0, 1e-8, check=False)
        assert st["rc"] == mg.MG_EINVAL and "nesting" in mg.mg_last_error()
    finally:
        mg.mg_destroy_grid(g)


def _levels_vs_oracle(h, res, alpha, tol_rel):
    n0 = h["delta0"].shape[0]
    l1, l2 = h["levels"]
    ref1, st1 = O.patch_solve(n0, 1, l1["origins"], l1["delta"], res["phi0"], alpha, 1.0,
                              tol=1e-12, max_sweeps=400000)
    assert st1["status"] == O.OK, st1
    assert rel(res["levels"][0]["phi"], ref1) < tol_rel
    if len(l2["origins"]):
        ref2, st2 = O.patch_solve(n0, 2, l2["origins"], l2["delta"], res["levels"][0]["phi"],
                                  alpha, 1.0, parent_org=l1["origins"], tol=1e-12,
                                  max_sweeps=400000)
        assert st2["status"] == O.OK, st2
        assert rel(res["levels"][1]["phi"], ref2) < tol_rel


def test_high_density_union_matches_oracle():
    """The refinement recipe at sigma 2 (patches over delta > 20, then > 80, 10 %
    cell-scale noise) with r_V = 8 cells (alpha*kappa = 0.3): the level-1 density
    reaches 138, alpha*kappa*delta ~ 41.  Both levels match the oracle's plain
    Newton-Gauss-Seidel solution of the same system."""
    h = I.refined_hierarchy(16, 2.0, 7)
    assert [len(L["origins"]) for L in h["levels"]] == [22, 2]
    alpha = I.alpha_kappa_for_rv(8.0)
    res = solve_hierarchy(h, alpha=alpha, tol=1e-11)
    assert res["stats"]["rc"] == mg.MG_OK, res["stats"]
    _levels_vs_oracle(h, res, alpha, 1e-10)


def test_union_where_the_rediscretised_correction_fails():
    """32^3 at sigma 2 (170 level-1 and 16 level-2 patches, level-1 delta up to 274)
    with alpha*kappa = 0.3.  From the default initial guess (the interpolation of
    the level below) the Galerkin correction converges to the oracle's solution of
    each level.  From a zero initial guess the FAS correction with the
    rediscretised coarse operator makes the union residual grow, while the
    Galerkin correction still converges."""
    h = I.refined_hierarchy(32, 2.0, 1303)
    l1, l2 = h["levels"]
    assert (len(l1["origins"]), len(l2["origins"])) == (170, 16)
    alpha = I.alpha_kappa_for_rv(8.0)
    tol = 1e-11
    res = solve_hierarchy(h, alpha=alpha, tol=tol)
    assert res["stats"]["rc"] == mg.MG_OK, (res["stats"], mg.mg_last_error())
    _levels_vs_oracle(h, res, alpha, 1e-10)
    d1, _ = O.patch_residual(32, 1, l1["origins"], res["levels"][0]["phi"], l1["delta"],
                             res["phi0"], alpha, 1.0)
    assert np.abs(d1).max() < tol
    d2, _ = O.patch_residual(32, 2, l2["origins"], res["levels"][1]["phi"], l2["delta"],
                             res["levels"][0]["phi"], alpha, 1.0, parent_org=l1["origins"])
    assert np.abs(d2).max() < tol
    gal0 = solve_hierarchy(h, alpha=alpha, tol=tol, zero_start=True)
    assert gal0["stats"]["rc"] == mg.MG_OK
    assert rel(gal0["levels"][0]["phi"], res["levels"][0]["phi"]) < 1e-10
    fas0 = solve_hierarchy(h, alpha=alpha, tol=tol, zero_start=True, patch_galerkin=0)
    assert fas0["stats"]["rc"] == mg.MG_ENOCONV


def test_level_initial_guess_and_reset(small):
    """A refinement level without an initial guess starts from the interpolation of
    the level below; after a solve its last iterate is kept, and passing NULL for
    the whole level (patch -1) resets it.  Every start reaches the same solution."""
    h = small
    n0 = h["delta0"].shape[0]
    g = mg.mg_create_grid(n0)
    try:
        mg.mg_set_density(g, 0, -1, h["delta0"])
        for lvl, L in enumerate(h["levels"], start=1):
            mg.mg_add_patches(g, lvl, L["origins"])
            mg.mg_set_density(g, lvl, -1, np.ascontiguousarray(L["delta"]))
        mg.mg_solve(g, 0, ALPHA, 1.0, 1e-11)
        first = mg.mg_get_level_stats(g, 1)
        a = np.empty((len(h["levels"][0]["origins"]), 8, 8, 8))
        mg.mg_get_field(g, 1, -1, a)
        mg.mg_solve(g, 0, ALPHA, 1.0, 1e-11)      # resumes from the converged field
        assert mg.mg_get_level_stats(g, 1)["cycles"] <= 1
        mg.mg_set_field(g, 1, -1, None)           # start over from the level below
        mg.mg_set_field(g, 2, -1, None)
        mg.mg_solve(g, 0, ALPHA, 1.0, 1e-11)
        again = mg.mg_get_level_stats(g, 1)
        assert again["hist"][0] == pytest.approx(first["hist"][0], rel=1e-6)
        b = np.empty_like(a)
        mg.mg_get_field(g, 1, -1, b)
        assert rel(b, a) < 1e-10
        mg.mg_set_field(g, 1, -1, np.zeros_like(a))   # an explicit (zero) initial guess
        mg.mg_solve(g, 0, ALPHA, 1.0, 1e-11)
        mg.mg_get_field(g, 1, -1, b)
        assert rel(b, a) < 1e-10
        with pytest.raises(mg.MGError) as e:
            mg.mg_set_field(g, 1, 0, None)            # NULL resets whole levels only
        assert e.value.status == mg.MG_EINVAL
    finally:
        mg.mg_destroy_grid(g)
