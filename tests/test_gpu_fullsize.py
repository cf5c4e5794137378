"""Full-size workloads against the CPU oracle by properties that hold at any size:
the oracle's own residual of the GPU fields (C3: 256^3 domain with two levels of
8^3 patches; C4: 512^3, mixed and FP64), and mixed against FP64."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1303_0008_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1303_0008_gb300 import mg  # noqa: E402

TOL = 1e-8


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("sigma,alpha,min_patches", [(2.0, 0.3, (60000, 4000)),
                                                     (1.0, 0.3, (3000,))])
def test_c3_refined_levels_full_size(sigma, alpha, min_patches):
    """256^3 domain with two refinement criteria (delta > 20, then > 80), r_V = 8
    cells (alpha*kappa = 0.3).

    sigma 2.0 gives 72,167 level-1 and 4,449 level-2 patches; the level-1 density
    reaches delta = 3382 with 10% noise at the cell scale, alpha*kappa*delta ~ 1000.
    The unions converge with the Galerkin coarse-grid correction (the default).
    sigma 1.0 gives 3,124 level-1 patches (no level 2)."""
    h = I.refined_hierarchy(256, sigma, 1303)
    levels = h["levels"]
    counts = [len(L["origins"]) for L in levels if len(L["origins"])]
    assert len(counts) == len(min_patches)
    assert all(c > m for c, m in zip(counts, min_patches))
    g = mg.mg_create_grid(256)
    phis = []
    try:
        mg.mg_set_density(g, 0, -1, h["delta0"])
        for lvl, L in enumerate(levels[:len(counts)], start=1):
            mg.mg_add_patches(g, lvl, L["origins"])
            mg.mg_set_density(g, lvl, -1, np.ascontiguousarray(L["delta"]))
        mg.mg_solve(g, 0, alpha, 1.0, TOL)
        phi0 = np.empty_like(h["delta0"])
        mg.mg_get_field(g, 0, -1, phi0)
        for lvl, L in enumerate(levels[:len(counts)], start=1):
            p = np.empty((len(L["origins"]), 8, 8, 8))
            mg.mg_get_field(g, lvl, -1, p)
            phis.append(p)
    finally:
        mg.mg_destroy_grid(g)
    d0, _ = O.residual(phi0, h["delta0"], alpha, 1.0)
    assert np.abs(d0 - d0.mean()).max() < TOL
    parent, parent_org = phi0, None
    for lvl, (L, p) in enumerate(zip(levels, phis), start=1):
        d, _ = O.patch_residual(256, lvl, L["origins"], p, L["delta"], parent, alpha, 1.0,
                                parent_org=parent_org)
        assert np.abs(d).max() < TOL, lvl
        parent, parent_org = p, L["origins"]


def test_c4_512_mixed_and_fp64():
    n = 512
    delta = I.lognormal_delta(n, 2.0, 1304)
    alpha = I.alpha_kappa_for_rv(16.0)
    out = {}
    for prec in (1, 0):
        g = mg.mg_create_grid(n, mg.options(prec=prec))
        try:
            d = torch.from_numpy(delta).cuda()
            mg.mg_set_density(g, 0, -1, d)
            st = mg.mg_solve(g, 0, alpha, 1.0, TOL if prec else 1e-10)
            phi = np.empty_like(delta)
            mg.mg_get_field(g, 0, -1, phi)
            out[prec] = (st, phi)
        finally:
            mg.mg_destroy_grid(g)
    fl, hits = O.density_floor(delta, alpha, 1.0)
    assert out[1][0]["guard_hits"] == hits == out[0][0]["guard_hits"]
    for prec, tol in ((1, TOL), (0, 1e-10)):
        d, g = O.residual(out[prec][1], fl, alpha, 1.0)
        assert np.abs(d - d.mean()).max() < 1.5 * tol and g == 0
    # the mixed answer is the FP64 system's solution to the bound of the target
    assert rel(out[1][1], out[0][1]) < 1e-7
    assert rel(O.force(out[1][1]), O.force(out[0][1])) < 1e-7


def test_c4_512_against_one_oracle_solve():
    """C4 at full size against one oracle solve of the same system: the oracle's
    four-colour OpenMP build (pinned to the lexicographic oracle's fixed point)
    solves the floored 512^3 system to 1e-10 on the host cores; the GPU's FP64
    solve to the same residual and its mixed-precision solve to 1e-8 are compared
    with it element by element, for phi and for the force -grad(phi)/2."""
    n = 512
    delta = I.lognormal_delta(n, 2.0, 1304)
    alpha = I.alpha_kappa_for_rv(16.0)
    fl, _ = O.density_floor(delta, alpha, 1.0)
    ref, rst = O.fas_solve_colour(fl, alpha, 1.0, tol=1e-10, max_cycles=100)
    assert rst["status"] == O.OK, rst
    ref_force = O.force(ref)
    # two solutions of the same system with residuals below 1e-10 differ by about
    # res / (4 pi^2) = 3e-12 absolute, i.e. 1e-9 of max|phi| (~3e-3); the mixed solve
    # stops at 1e-8, and its bound is the 1e-7 of the precision target
    for prec, tol, bound in ((0, 1e-10, 2e-9), (1, TOL, 1e-7)):
        g = mg.mg_create_grid(n, mg.options(prec=prec))
        try:
            mg.mg_set_density(g, 0, -1, torch.from_numpy(delta).cuda())
            st = mg.mg_solve(g, 0, alpha, 1.0, tol)
            phi = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
            mg.mg_get_field(g, 0, -1, phi)
            force = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
            mg.mg_get_force(g, 0, -1, force)
        finally:
            mg.mg_destroy_grid(g)
        assert st["rc"] == mg.MG_OK
        assert rel(phi.cpu().numpy(), ref) < bound, prec
        assert rel(force.cpu().numpy(), ref_force) < bound, prec
        del phi, force


@pytest.mark.parametrize("prec", [0, 1])
def test_largest_grid_1024_sampled_residual(prec):
    """n = 1024, the largest grid the library accepts (2^30 cells per array):
    a lognormal field drawn on the device, solved to 1e-8; the oracle evaluates
    the operator at 2048 sampled cells from their 3^3 neighbourhoods."""
    n = 1024
    delta = I.lognormal_delta_device(n, 1.0, 1306)
    alpha = I.alpha_kappa_for_rv(8.0)
    g = mg.mg_create_grid(n, mg.options(prec=prec))
    try:
        mg.mg_set_density(g, 0, -1, delta)
        st = mg.mg_solve(g, 0, alpha, 1.0, TOL)
        phi = torch.empty_like(delta)
        mg.mg_get_field(g, 0, -1, phi)
    finally:
        mg.mg_destroy_grid(g)
    assert st["rc"] == mg.MG_OK and st["res"] < TOL and st["guard_hits"] == 0
    rng = np.random.default_rng(1024 + prec)
    c = torch.from_numpy(rng.integers(0, n, size=(2048, 3))).cuda()
    o = torch.arange(-1, 2, device="cuda")
    K = (c[:, 2, None, None, None] + o[None, :, None, None]) % n
    J = (c[:, 1, None, None, None] + o[None, None, :, None]) % n
    Ii = (c[:, 0, None, None, None] + o[None, None, None, :]) % n
    pb = phi[K, J, Ii].cpu().numpy()
    db = delta[K, J, Ii].cpu().numpy()
    del phi, delta
    worst = 0.0
    for s in range(pb.shape[0]):
        d, gh = O.residual(pb[s], db[s], alpha, 1.0, h=1.0 / n)
        assert gh == 0
        worst = max(worst, abs(d[1, 1, 1] - st["lambda"]))
    assert worst <= st["res"] * (1 + 1e-6) + 1e-12
